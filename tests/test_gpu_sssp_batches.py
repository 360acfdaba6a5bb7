"""SSSP-based batch strategies (Sec. 4.3) on the GPU against the oracle.

Plain-SSSP runs a full single-source search from every query source, VC-SSSP
from a vertex cover of the query graph; both read each answer from the final
distances of one search, so they must equal Dijkstra exactly, and the number
of searches the engine ran must equal the number of sources the host selected.
"""

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import ppsp
from workloads import clique_pairs, grid_graph, random_pairs, road_like_graph, star_pairs
from workloads.graphs import csr_from_undirected

pytestmark = pytest.mark.gpu

INF = oracle.INF_INT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def road():
    g = road_like_graph(80, seed=61)
    batches = [star_pairs(g, 40, 1), clique_pairs(g, 12, 2), random_pairs(g, 50, 3)]
    mixed = np.concatenate(batches)
    mixed = np.concatenate([mixed, mixed[:20][:, ::-1], mixed[:5], np.stack([mixed[:3, 0]] * 2, axis=1)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, mixed)
    G = ppsp.Graph.from_csr(g)
    yield g, mixed, want, G
    G.close()


@pytest.mark.parametrize("strategy", ["sssp", "vc"])
@pytest.mark.parametrize("mode", ["bids", "bidastar", "et", "astar"])
def test_mixed_patterns(road, strategy, mode):
    g, pairs, want, G = road
    got, cnt = G.batch(pairs, mode=mode, strategy=strategy, return_counters=True)
    assert np.array_equal(got, want)
    _, n_src = ppsp.batch_sources(pairs, strategy)
    assert cnt["searches"] == n_src and cnt["groups"] == n_src


@pytest.mark.parametrize("team", [1, 2, 4])
@pytest.mark.parametrize("delta", [0, 1, 50, 10 ** 6])
def test_team_sizes_and_delta(road, team, delta):
    g, pairs, want, G = road
    got = G.batch(pairs, mode="bids", strategy="vc", team_ctas=team, delta=delta)
    assert np.array_equal(got, want), (team, delta)


def test_star_and_clique_search_counts():
    g = grid_graph(48, seed=71)
    st = star_pairs(g, 30, 4)
    cl = clique_pairs(g, 11, 5)
    with ppsp.Graph.from_csr(g) as G:
        full = oracle.sssp(g.offsets, g.targets, g.weights, int(st[0, 0]))
        got, cnt = G.batch(st, strategy="vc", return_counters=True)
        assert np.array_equal(got, full[st[:, 1]]) and cnt["searches"] == 1
        want = oracle.pairs(g.offsets, g.targets, g.weights, cl)
        got, cnt = G.batch(cl, strategy="vc", return_counters=True)
        assert np.array_equal(got, want) and cnt["searches"] == 10
        got, cnt = G.batch(cl, strategy="sssp", return_counters=True)
        assert np.array_equal(got, want)


def test_u64_and_disconnected():
    # two components; heavy weights need 64-bit distances
    off, tgt, w = csr_from_undirected(7, np.array([0, 1, 2, 4, 5]), np.array([1, 2, 3, 5, 6]),
                                      np.array([2 ** 31, 2 ** 31, 7, 3, 4], dtype=np.uint32))
    pairs = np.array([(0, 3), (3, 0), (0, 6), (4, 6), (6, 4), (2, 2), (1, 5)], dtype=np.uint32)
    want = oracle.pairs(off, tgt, w, pairs)
    assert want[2] == INF and want[0] == 2 ** 32 + 7
    with ppsp.Graph(off, tgt, w) as G:
        for strategy in ("sssp", "vc"):
            assert np.array_equal(G.batch(pairs, strategy=strategy, dist_bits=64), want)
            st, _ = G.batch_status(pairs, strategy=strategy, dist_bits=32)
            assert st == ppsp.ERR_OVERFLOW


def test_directed_graph():
    # Plain-SSSP follows out-edges from each source; VC-SSSP covers the
    # bipartite query graph, a target in the cover searching in-edges
    off = np.array([0, 1, 2, 3, 3], dtype=np.uint64)
    tgt = np.array([1, 2, 3], dtype=np.uint32)
    w = np.array([4, 5, 6], dtype=np.uint32)
    pairs = np.array([(0, 3), (1, 3), (3, 0), (0, 2)], dtype=np.uint32)
    want = oracle.pairs(off, tgt, w, pairs)
    with ppsp.Graph(off, tgt, w, undirected=False) as G:
        assert np.array_equal(G.batch(pairs, mode="et", strategy="sssp"), want)
        got, cnt = G.batch(pairs, mode="et", strategy="vc", return_counters=True)
        assert np.array_equal(got, want)
        assert cnt["searches"] == ppsp.batch_sources(pairs, "vc", undirected=False)[1]


def test_paths_unsupported(road):
    g, pairs, want, G = road
    st = G.batch_paths(pairs[:4], 1024, strategy="vc")[0]
    assert st == ppsp.ERR_UNSUPPORTED


@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_graphs_vs_floyd_warshall(seed):
    from test_gpu_parity import _random_graph

    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 40))
    m = int(rng.integers(0, 3 * n + 1))
    off, tgt, w = _random_graph(rng, n, m, int(rng.choice([3, 100, 60000])), zero_frac=0.2)
    fw = oracle.floyd_warshall(off, tgt, w)
    pairs = np.array([(s, t) for s in range(n) for t in range(n)], dtype=np.uint32)
    want = fw[pairs[:, 0], pairs[:, 1]]
    with ppsp.Graph(off, tgt, w) as G:
        for strategy in ("sssp", "vc"):
            for team in (1, 2):
                got = G.batch(pairs, strategy=strategy, team_ctas=team, delta=int(rng.integers(1, 50)))
                assert np.array_equal(got, want), (strategy, team)


@pytest.mark.parametrize("team", [1, 4])
def test_search_stops_once_targets_are_settled(team):
    # a star whose leaves all lie within a few cells of its centre: the one
    # search of VC-SSSP must stop long before it has settled the whole grid
    side = 200
    g = grid_graph(side, seed=81)
    c = (side // 2) * side + side // 2
    leaves = [c + k for k in range(1, 4)] + [c - k * side for k in range(1, 4)]
    pairs = np.array([(c, x) for x in leaves], dtype=np.uint32)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for strategy in ("vc", "sssp"):
            got, cnt = G.batch(pairs, strategy=strategy, team_ctas=team, big_team_ctas=team,
                               return_counters=True)
            assert np.array_equal(got, want)
            assert cnt["extracted"] < g.n // 20, (strategy, cnt)


@pytest.mark.parametrize("mode", ["bids", "bidastar", "et", "astar"])
def test_auto_strategy_mixed_patterns(road, mode):
    g, pairs, want, G = road
    assert np.array_equal(G.batch(pairs, mode=mode, strategy="auto"), want)
    for team in (1, 4):
        got = G.batch(pairs, mode=mode, strategy="auto", team_ctas=team, big_team_ctas=team)
        assert np.array_equal(got, want), team


def test_auto_strategy_choices():
    # searches per pattern: with BiD-A* potentials a star is one SSSP search
    # and a clique runs as independent pairs; without them (BiDS) the star is
    # one SSSP search and the clique one Multi-BiDS group
    g = road_like_graph(64, seed=91)
    star = star_pairs(g, 20, 6)
    clique = clique_pairs(g, 8, 7)
    single = random_pairs(g, 1, 8)
    with ppsp.Graph.from_csr(g) as G:
        for pat, bidastar_searches, bids_searches in ((star, 1, 1), (clique, 2 * 28, 8), (single, 2, 2)):
            want = oracle.pairs(g.offsets, g.targets, g.weights, pat)
            got, cnt = G.batch(pat, mode="bidastar", strategy="auto", return_counters=True)
            assert np.array_equal(got, want) and cnt["searches"] == bidastar_searches
            got, cnt = G.batch(pat, mode="bids", strategy="auto", return_counters=True)
            assert np.array_equal(got, want) and cnt["searches"] == bids_searches
        # ET: a source with several targets is one multi-target search
        got, cnt = G.batch(star, mode="et", strategy="auto", return_counters=True)
        assert np.array_equal(got, oracle.pairs(g.offsets, g.targets, g.weights, star))
        assert cnt["searches"] == 1
        # paths: SSSP groups record none, so AUTO falls back to pair searches
        st, dist, paths, lens = G.batch_paths(star, 4096, mode="bidastar", strategy="auto")
        assert st == ppsp.OK and np.array_equal(dist, oracle.pairs(g.offsets, g.targets, g.weights, star))
        for (s, t), p in zip(star, paths):
            assert p is not None and p[0] == s and p[-1] == t


def test_auto_strategy_on_a_dense_graph():
    # average degree >= 8 (the social shape): every component, isolated pairs
    # too, runs as VC-SSSP single-source searches
    from workloads import rmat_graph

    g = rmat_graph(12, seed=93)
    assert g.m >= 8 * g.n
    pairs = np.concatenate([random_pairs(g, 20, 94), star_pairs(g, 10, 95), clique_pairs(g, 5, 96)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g, with_coords=False) as G:
        got, cnt = G.batch(pairs, mode="bids", strategy="auto", return_counters=True)
        assert np.array_equal(got, want)
        assert cnt["searches"] == ppsp.batch_sources(pairs, "vc")[1]
