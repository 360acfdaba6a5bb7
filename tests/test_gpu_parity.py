"""Parity of the CUDA path with the CPU oracle (bit-exact: all arithmetic is integer).

Theorems 3.3 and 3.4 say BiDS and BiD-A* return d(s,t) for any stepping
schedule, so every launch configuration (Delta, frontier representation, block
size, team size, layout, batch strategy) must give the oracle's answer exactly.
"""

import numpy as np
import pytest

import oracle
from oracle import potential as opot
from paper_2506_16488_gb300 import ppsp
from workloads import (clique_pairs, config_workload, grid_graph, near_mid_far_pairs, random_pairs,
                       rmat_graph, road_like_graph, star_pairs)
from workloads.graphs import csr_from_undirected

pytestmark = pytest.mark.gpu

INF = oracle.INF_INT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def cfg1():
    g = grid_graph(64, seed=1001)
    pairs = random_pairs(g, 100, seed=1002)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    G = ppsp.Graph.from_csr(g)
    yield g, pairs, want, G
    G.close()


def test_cfg1_bids_batch(cfg1):
    g, pairs, want, G = cfg1
    got, cnt = G.batch(pairs, mode="bids", return_counters=True)
    assert np.array_equal(got, want)
    assert cnt["groups"] > 0 and cnt["edges"] > 0


@pytest.mark.parametrize("mode", ["bids", "bidastar", "et", "astar"])
def test_cfg1_single_queries(cfg1, mode):
    g, pairs, want, G = cfg1
    for q in range(25):
        assert G.query(int(pairs[q, 0]), int(pairs[q, 1]), mode=mode) == int(want[q]), q


@pytest.mark.parametrize("strategy", ["multi", "plain_star", "plain"])
@pytest.mark.parametrize("mode", ["bids", "bidastar", "et", "astar"])
def test_cfg1_batch_strategies(cfg1, mode, strategy):
    g, pairs, want, G = cfg1
    assert np.array_equal(G.batch(pairs, mode=mode, strategy=strategy), want)


@pytest.mark.parametrize("delta", [1, 37, 0, 5000, 10 ** 7])
def test_delta_sweep(cfg1, delta):
    g, pairs, want, G = cfg1
    for mode in ("bids", "bidastar"):
        assert np.array_equal(G.batch(pairs, mode=mode, delta=delta), want)


@pytest.mark.parametrize("frontier,dense_den", [("sparse", 0), ("dense", 0), ("auto", 2), ("auto", 1000)])
def test_frontier_policies(cfg1, frontier, dense_den):
    g, pairs, want, G = cfg1
    for mode in ("bids", "bidastar", "et"):
        got = G.batch(pairs, mode=mode, frontier=frontier, dense_den=dense_den)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("block", [256, 512, 1024])
@pytest.mark.parametrize("team", [1, 2, 3])
def test_block_and_team_sizes(cfg1, block, team):
    g, pairs, want, G = cfg1
    got = G.batch(pairs, mode="bids", block_threads=block, team_ctas=team)
    assert np.array_equal(got, want)
    got = G.batch(pairs[:10], mode="bidastar", strategy="plain", block_threads=block, team_ctas=team)
    assert np.array_equal(got, want[:10])


def test_repeated_runs_are_stable(cfg1):
    g, pairs, want, G = cfg1
    for r in range(20):
        assert np.array_equal(G.batch(pairs, mode="bidastar" if r % 2 else "bids",
                                      delta=1 + 97 * r), want)


def test_u64_distances(cfg1):
    g, pairs, want, G = cfg1
    for mode in ("bids", "bidastar", "et"):
        assert np.array_equal(G.batch(pairs, mode=mode, dist_bits=64), want)


def _random_graph(rng, n, m, wmax, zero_frac):
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    w = rng.integers(1, wmax + 1, size=m)
    w[rng.random(m) < zero_frac] = 0
    keep = u != v
    # duplicates (parallel edges) are kept on purpose; the CSR builder needs
    # unique keys per direction, so build the directed lists by hand
    src = np.concatenate([u[keep], v[keep]])
    dst = np.concatenate([v[keep], u[keep]])
    ww = np.concatenate([w[keep], w[keep]])
    order = np.lexsort((ww, dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=off[1:])
    return off, dst.astype(np.uint32), ww.astype(np.uint32)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_graphs_vs_floyd_warshall(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 48))
    m = int(rng.integers(0, 3 * n + 1))
    off, tgt, w = _random_graph(rng, n, m, int(rng.choice([3, 100, 60000])), zero_frac=0.2)
    coords = rng.uniform(0, 10, size=(n, 2)).astype(np.float32)
    fw = oracle.floyd_warshall(off, tgt, w)
    pairs = np.array([(s, t) for s in range(n) for t in range(n)], dtype=np.uint32)
    want = fw[pairs[:, 0], pairs[:, 1]]
    with ppsp.Graph(off, tgt, w, coords) as G:
        for mode in ("bids", "bidastar", "et", "astar"):
            for strategy in ("multi", "plain_star"):
                got = G.batch(pairs, mode=mode, strategy=strategy, delta=int(rng.integers(1, 50)))
                assert np.array_equal(got, want), (mode, strategy)


def test_query_graph_patterns():
    g = road_like_graph(80, seed=31)
    G = ppsp.Graph.from_csr(g)
    batches = [star_pairs(g, 40, 1), clique_pairs(g, 12, 2), random_pairs(g, 50, 3)]
    mixed = np.concatenate(batches)
    # duplicates, reversed pairs and s == t queries collapse or short-cut
    mixed = np.concatenate([mixed, mixed[:20][:, ::-1], mixed[:5], np.stack([mixed[:3, 0]] * 2, axis=1)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, mixed)
    for mode in ("bids", "bidastar"):
        for layout in ("interleaved", "stacked"):
            got = G.batch(mixed, mode=mode, layout=layout)
            assert np.array_equal(got, want), (mode, layout)
        for team in (1, 2):
            got = G.batch(mixed, mode=mode, big_team_ctas=4, team_ctas=team)
            assert np.array_equal(got, want)
    G.close()


def test_star_equals_one_sssp():
    g = road_like_graph(64, seed=41)
    st = star_pairs(g, 64, 5)
    full = oracle.sssp(g.offsets, g.targets, g.weights, int(st[0, 0]))
    with ppsp.Graph.from_csr(g) as G:
        assert np.array_equal(G.batch(st, mode="bids"), full[st[:, 1]])


def test_edge_cases():
    off, tgt, w = csr_from_undirected(6, np.array([0, 1, 3]), np.array([1, 2, 4]),
                                      np.array([5, 7, 9], dtype=np.uint32))
    coords = np.arange(12, dtype=np.float32).reshape(6, 2)
    with ppsp.Graph(off, tgt, w, coords) as G:
        for mode in ("bids", "bidastar", "et", "astar"):
            assert G.query(2, 2, mode=mode) == 0
            assert G.query(0, 2, mode=mode) == 12
            assert G.query(0, 4, mode=mode) == INF  # disconnected
            assert G.query(5, 5, mode=mode) == 0  # isolated vertex, s == t
        assert G.batch(np.zeros((0, 2)), mode="bids").shape == (0,)
        st, _ = G.query_status(0, 6)
        assert st == ppsp.ERR_INVALID_ARG
        st, _ = G.batch_status(np.array([[0, 1], [9, 1]]))
        assert st == ppsp.ERR_INVALID_ARG
        st, _ = G.query_status(0, 1, delta=0, dist_bits=16)
        assert st == ppsp.ERR_INVALID_ARG
    with ppsp.Graph(off, tgt, w, None) as G:
        assert G.query_status(0, 1, mode="bidastar")[0] == ppsp.ERR_NO_COORDS
        assert G.query_status(0, 1, mode="astar")[0] == ppsp.ERR_NO_COORDS
        assert G.query(0, 1, mode="bids") == 5
    with ppsp.Graph(off, tgt, w, None, undirected=False) as G:
        # a directed graph searches backward from t over its transpose
        assert G.query(0, 1, mode="bids") == 5
        assert G.query(0, 2, mode="et") == 12
        assert G.query(0, 4, mode="bids") == INF
    one = np.zeros(2, dtype=np.uint64)
    with ppsp.Graph(one, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as G:
        assert G.query(0, 0) == 0


def test_overflow_is_reported():
    n = 6
    wt = np.full(n - 1, 2 ** 31, dtype=np.uint32)
    off, tgt, w = csr_from_undirected(n, np.arange(n - 1), np.arange(1, n), wt)
    with ppsp.Graph(off, tgt, w) as G:
        st, _ = G.query_status(0, n - 1, mode="bids", dist_bits=32)
        assert st == ppsp.ERR_OVERFLOW
        assert G.query(0, n - 1, mode="bids", dist_bits=64) == (n - 1) * 2 ** 31
        assert G.query(0, 1, mode="et", dist_bits=32) == 2 ** 31


def test_timeout_hook_returns_status_and_recovers(cfg1):
    g, pairs, want, G = cfg1
    st, _ = G.query_status(int(pairs[0, 0]), int(pairs[0, 1]), mode="bids", team_ctas=2,
                           spin_limit=2000, debug_flags=ppsp.DEBUG_BARRIER_NEVER_RELEASES)
    assert st == ppsp.ERR_TIMEOUT
    assert np.array_equal(G.batch(pairs, mode="bids"), want)
    assert G.query(int(pairs[1, 0]), int(pairs[1, 1])) == int(want[1])


def test_potential_matches_oracle():
    g = road_like_graph(96, seed=51)
    # the oracle chooses c, F and P by the creation rule on its own; nothing
    # is taken from the library
    c, F, P = opot.choose_scale(g.offsets, g.targets, g.weights, g.coords)
    assert 0.99 * 1000 < c <= 1000.0 and F >= 1
    with ppsp.Graph.from_csr(g) as G:
        info = G.info()
        assert info["potential_scale"] == c and info["potential_shift"] == F
        assert np.array_equal(G.potential_coords(), P)
        assert opot.certificate_ok(g.offsets, g.targets, g.weights, P, F).all()
        rng = np.random.default_rng(2)
        verts = rng.integers(0, g.n, size=2000).astype(np.uint32)
        for x in rng.integers(0, g.n, size=5):
            h_gpu = G.potential_eval(int(x), verts)
            h_ref = opot.h_all(P, int(x), F)
            assert np.array_equal(h_gpu, h_ref[verts])
            assert opot.consistent_for_anchor(g.offsets, g.targets, g.weights, h_ref)


def test_plan_writes_device_output(cfg1):
    torch = pytest.importorskip("torch")
    g, pairs, want, G = cfg1
    stream = torch.cuda.Stream()
    out = torch.zeros(pairs.shape[0], dtype=torch.int64, device="cuda")
    plan = G.plan(pairs, mode="bidastar", stream=stream.cuda_stream)
    for _ in range(3):
        out.zero_()
        torch.cuda.synchronize()
        plan.run(out.data_ptr())
        cnt = plan.sync()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
        # Multi-BiDS: one search per distinct endpoint of the query graph (Sec. 4.2)
        uniq = {(min(a, b), max(a, b)) for a, b in pairs.tolist() if a != b}
        assert cnt["searches"] == len({v for e in uniq for v in e})
    plan.close()


def test_road_small_near_mid_far():
    wl = config_workload(2, small=True)
    g, pairs = wl["graph"], wl["batches"]["nmf"]
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bidastar", "bids"):
            assert np.array_equal(G.batch(pairs, mode=mode), want)
        assert np.array_equal(G.batch(pairs[:40], mode="bidastar", strategy="plain"), want[:40])


def test_rmat_small_batches():
    wl = config_workload(3, small=True)
    g = wl["graph"]
    with ppsp.Graph.from_csr(g, with_coords=False) as G:
        for name, pairs in wl["batches"].items():
            want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
            for strategy in ("multi", "plain_star"):
                for team in (1, 4):
                    got = G.batch(pairs, mode="bids", strategy=strategy, team_ctas=team, big_team_ctas=8)
                    assert np.array_equal(got, want), (name, strategy, team)


def test_cfg4_small_mixed_clique():
    wl = config_workload(4, small=True)
    g, pairs = wl["graph"], wl["batches"]["mixed"]
    want = oracle.pairs_threaded(g.offsets, g.targets, g.weights, pairs, 8)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bidastar", "bids"):
            assert np.array_equal(G.batch(pairs, mode=mode), want)


def test_plan_replays_a_cuda_graph(cfg1):
    torch = pytest.importorskip("torch")
    g, pairs, want, G = cfg1
    stream = torch.cuda.Stream()
    out = torch.zeros(pairs.shape[0], dtype=torch.int64, device="cuda")
    out2 = torch.zeros(pairs.shape[0], dtype=torch.int64, device="cuda")
    plan = G.plan(pairs, mode="bidastar", stream=stream.cuda_stream, cuda_graph=True)
    for dst in (out, out, out2, out):
        dst.zero_()
        torch.cuda.synchronize()
        plan.run(dst.data_ptr())
        plan.sync()
        assert np.array_equal(dst.cpu().numpy().view(np.uint64), want)
        assert plan.uses_graph()
    plan.close()


@pytest.mark.parametrize("delta", [1, 3, 0, 5000, 10 ** 7])
def test_one_cta_bucket_frontier_delta_sweep(cfg1, delta):
    g, pairs, want, G = cfg1
    for mode in ("bids", "bidastar", "et", "astar"):
        for bits in (32, 64):
            got = G.batch(pairs, mode=mode, delta=delta, team_ctas=1, dist_bits=bits)
            assert np.array_equal(got, want), (mode, bits)


@pytest.mark.parametrize("delta", [1, 0, 10 ** 9])
def test_one_cta_far_list_and_spills(delta):
    # Delta = 1 sends most entries to the far list; a huge Delta puts whole
    # frontiers into one bucket, overflowing it into the spill bitmap.
    g = road_like_graph(160, seed=91)
    pairs = np.concatenate([random_pairs(g, 40, 92), clique_pairs(g, 5, 93)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bids", "bidastar"):
            for bits in (32, 64):
                got = G.batch(pairs, mode=mode, delta=delta, team_ctas=1, big_team_ctas=1, dist_bits=bits)
                assert np.array_equal(got, want), (mode, bits)


@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_graphs_one_cta(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(2, 40))
    off, tgt, w = _random_graph(rng, n, int(rng.integers(0, 3 * n + 1)), 1000, zero_frac=0.2)
    coords = rng.uniform(0, 10, size=(n, 2)).astype(np.float32)
    fw = oracle.floyd_warshall(off, tgt, w)
    pairs = np.array([(s, t) for s in range(n) for t in range(n)], dtype=np.uint32)
    want = fw[pairs[:, 0], pairs[:, 1]]
    with ppsp.Graph(off, tgt, w, coords) as G:
        for mode in ("bids", "bidastar", "et", "astar"):
            for strategy in ("multi", "plain_star"):
                got = G.batch(pairs, mode=mode, strategy=strategy, team_ctas=1, big_team_ctas=1,
                              delta=int(rng.integers(1, 3000)))
                assert np.array_equal(got, want), (mode, strategy)


@pytest.mark.parametrize("rho", [1, 64, 512, 10 ** 6])
@pytest.mark.parametrize("delta", [1, 0, 300, 10 ** 9])
def test_stepping_rho_merges_buckets(cfg1, rho, delta):
    # GetDist variants (Sec. 2): a step takes buckets until it holds >= rho
    # entries; rho = 10^6 with a huge Delta is Bellman-Ford.  Any schedule
    # returns d(s, t) (Theorems 3.3/3.4).
    g, pairs, want, G = cfg1
    for mode in ("bids", "bidastar", "et", "astar"):
        got = G.batch(pairs, mode=mode, team_ctas=1, big_team_ctas=1, stepping_rho=rho, delta=delta)
        assert np.array_equal(got, want), (mode, rho, delta)


@pytest.mark.parametrize("rho", [32, 4096])
def test_stepping_rho_road_far_list_and_spills(rho):
    g = road_like_graph(160, seed=77)
    pairs, _ = near_mid_far_pairs(g, 60, seed=78)
    pairs = np.concatenate([pairs, clique_pairs(g, 6, 79), star_pairs(g, 12, 80)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for delta in (1, 0, 10 ** 9):
            for strategy in ("multi", "auto"):
                got = G.batch(pairs, mode="bidastar", strategy=strategy, team_ctas=1, big_team_ctas=1,
                              stepping_rho=rho, delta=delta)
                assert np.array_equal(got, want), (delta, strategy)


def test_large_clique_uncached_partners_and_split():
    # a 50-clique has 2,450 partner entries (more than the shared-memory
    # partner cache holds) and a 70-clique more vertices than one Multi-BiDS
    # group takes (it is split into sub-groups)
    g = road_like_graph(72, seed=97)
    for size in (50, 70):
        pairs = clique_pairs(g, size, 98 + size)
        want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
        with ppsp.Graph.from_csr(g) as G:
            for team in (1, 4):
                got, cnt = G.batch(pairs, mode="bids", strategy="multi", big_team_ctas=team, team_ctas=team,
                                   return_counters=True)
                assert np.array_equal(got, want), (size, team)
            if size == 70:
                assert cnt["groups"] > 1


@pytest.mark.parametrize("team", [1, 4])
def test_multi_target_astar_cliques_and_stars(team):
    """Multi-BiDS with the multi-target A* potential (each shared search
    prunes with the smallest partner potential against mumax): exact on
    cliques, stars and mixed components, on the one-CTA (bucketed) and the
    multi-CTA (queue / bitmap) paths."""
    g = road_like_graph(120, seed=131)
    pairs = np.concatenate([clique_pairs(g, 16, 132), star_pairs(g, 20, 133), random_pairs(g, 30, 134)])
    # a component mixing a clique with pendant pairs
    pairs = np.concatenate([pairs, np.stack([pairs[:5, 0], random_pairs(g, 5, 135)[:, 1]], axis=1)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for delta in (0, 1, 10 ** 7):
            got, cnt_a = G.batch(pairs, mode="bidastar", strategy="multi", team_ctas=team, big_team_ctas=team,
                                 delta=delta, multi_potential=True, return_counters=True)
            assert np.array_equal(got, want), delta
        got = G.batch(pairs, mode="bidastar", strategy="multi", team_ctas=team, big_team_ctas=team)
        assert np.array_equal(got, want)  # the default: shared searches without a potential
        for frontier in ("sparse", "dense"):
            got = G.batch(pairs, mode="bidastar", strategy="multi", frontier=frontier, big_team_ctas=2,
                          multi_potential=True)
            assert np.array_equal(got, want), frontier


@pytest.mark.parametrize("team", [1, 3])
def test_memoized_potential(team):
    """Heuristic memoization (Sec. 5): the potential term of an entry is
    computed once per group and read back afterwards.  Answers are exact for
    every plug-in with a potential, on the one-CTA and the queue / bitmap
    paths, also when the same slots serve the next groups and batches (the
    memo is cleared with the touched entries)."""
    g = road_like_graph(140, seed=141)
    batches = [random_pairs(g, 60, 142), np.concatenate([clique_pairs(g, 9, 143), star_pairs(g, 15, 144)]),
               near_mid_far_pairs(g, 45, 145)[0]]
    wants = [oracle.pairs(g.offsets, g.targets, g.weights, b) for b in batches]
    with ppsp.Graph.from_csr(g) as G:
        for rep in range(2):
            for b, want in zip(batches, wants):
                for mode in ("bidastar", "astar"):
                    for delta in (0, 1):
                        got = G.batch(b, mode=mode, memo_potential=True, team_ctas=team, big_team_ctas=team,
                                      delta=delta)
                        assert np.array_equal(got, want), (rep, mode, delta)
        # tiny touched lists force the full reset of the slot (and its memo)
        for frontier in ("sparse", "dense"):
            got = G.batch(batches[0], mode="bidastar", memo_potential=True, frontier=frontier, team_ctas=2)
            assert np.array_equal(got, wants[0]), frontier


@pytest.mark.parametrize("team", [2, 8])
def test_pull_then_push(team):
    """Bidirectional relaxation (App. B): on the queue / bitmap path an
    extracted vertex first pulls the best distance over its neighbours, then
    pushes.  Exact for every plug-in and batch strategy; on a directed graph
    the option is ignored."""
    g = road_like_graph(100, seed=151)
    pairs = np.concatenate([random_pairs(g, 40, 152), clique_pairs(g, 7, 153), star_pairs(g, 10, 154)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bids", "bidastar", "et", "astar"):
            for strategy in ("multi", "plain_star", "vc" if mode in ("bids", "et") else "auto"):
                for delta in (0, 10 ** 7):
                    got, cnt = G.batch(pairs, mode=mode, strategy=strategy, pull_push=True, team_ctas=team,
                                       big_team_ctas=team, delta=delta, return_counters=True)
                    assert np.array_equal(got, want), (mode, strategy, delta)
        got = G.batch(pairs, mode="bidastar", pull_push=True, memo_potential=True, frontier="dense",
                      team_ctas=team)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("ring", [1, 7, 256])
def test_ring_entries(ring):
    """The one-CTA frontier's shared-memory entries per bucket only move
    entries between shared memory and the global overflow region: exact for
    a ring of 1 entry (almost everything overflows), an odd size, and the
    largest (256), with 32- and 64-bit distances and both block sizes."""
    g = road_like_graph(150, seed=161)
    pairs = np.concatenate([near_mid_far_pairs(g, 60, 162)[0], clique_pairs(g, 6, 163), star_pairs(g, 12, 164)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bidastar", "bids", "astar"):
            for bits in (32, 64):
                for block in (0, 256):
                    got = G.batch(pairs, mode=mode, ring_entries=ring, dist_bits=bits, block_threads=block,
                                  team_ctas=1, big_team_ctas=1, strategy="auto")
                    assert np.array_equal(got, want), (mode, bits, block)
        with pytest.raises(ppsp.PPSPError):
            G.batch(pairs, ring_entries=257)
