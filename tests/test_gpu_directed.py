"""Directed graphs on the GPU against the oracle.

On a directed graph a query's source searches out-edges and its target
searches in-edges (a transposed CSR built at create); Multi-BiDS groups hold
(vertex, role) searches, so G_q is bipartite (Sec. 4.4).  Theorems 3.3/3.4
carry over unchanged (d(s, v) + d(v, t) over meeting vertices v), so every
strategy must equal Dijkstra on the directed CSR exactly.
"""

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import ppsp
from workloads import (clique_pairs, near_mid_far_pairs, one_way_graph, random_pairs, road_like_graph,
                       star_pairs)

pytestmark = pytest.mark.gpu

INF = oracle.INF_INT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _random_digraph(rng, n, m, wmax, zero_frac):
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    w = rng.integers(1, wmax + 1, size=m)
    w[rng.random(m) < zero_frac] = 0
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    order = np.lexsort((w, v, u))
    u, v, w = u[order], v[order], w[order]
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(u, minlength=n), out=off[1:])
    return off, v.astype(np.uint32), w.astype(np.uint32)


@pytest.mark.parametrize("seed", range(8))
def test_tiny_random_digraphs_vs_floyd_warshall(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(2, 40))
    m = int(rng.integers(0, 4 * n + 1))
    off, tgt, w = _random_digraph(rng, n, m, int(rng.choice([3, 100, 60000])), zero_frac=0.2)
    coords = rng.uniform(0, 10, size=(n, 2)).astype(np.float32)
    fw = oracle.floyd_warshall(off, tgt, w)
    pairs = np.array([(s, t) for s in range(n) for t in range(n)], dtype=np.uint32)
    want = fw[pairs[:, 0], pairs[:, 1]]
    with ppsp.Graph(off, tgt, w, coords, undirected=False) as G:
        for mode in ("bids", "bidastar", "et", "astar"):
            for strategy in ("multi", "plain_star", "auto", "vc"):
                for team in (1, 2):
                    got = G.batch(pairs, mode=mode, strategy=strategy, team_ctas=team, big_team_ctas=team,
                                  delta=int(rng.integers(1, 50)))
                    assert np.array_equal(got, want), (mode, strategy, team)
        assert np.array_equal(G.batch(pairs, mode="et", strategy="sssp"), want)
        for q in range(0, pairs.shape[0], max(1, pairs.shape[0] // 25)):
            assert G.query(int(pairs[q, 0]), int(pairs[q, 1]), mode="bidastar") == int(want[q])


@pytest.fixture(scope="module")
def one_way():
    g = one_way_graph(road_like_graph(96, seed=111), 0.3, 112)
    nmf, _ = near_mid_far_pairs(g, 60, seed=113)
    pairs = np.concatenate([nmf, star_pairs(g, 16, 114), clique_pairs(g, 8, 115), random_pairs(g, 30, 116)])
    pairs = np.concatenate([pairs, pairs[:20][:, ::-1]])  # reversed pairs differ on a directed graph
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    G = ppsp.Graph.from_csr(g, undirected=False)
    yield g, pairs, want, G
    G.close()


@pytest.mark.parametrize("strategy", ["multi", "plain_star", "plain", "auto"])
@pytest.mark.parametrize("mode", ["bids", "bidastar"])
def test_one_way_road_graph(one_way, mode, strategy):
    g, pairs, want, G = one_way
    assert np.array_equal(G.batch(pairs, mode=mode, strategy=strategy), want)
    for team in (1, 4):
        got = G.batch(pairs, mode=mode, strategy=strategy, team_ctas=team, big_team_ctas=team)
        assert np.array_equal(got, want), team


def test_one_way_forward_modes_and_frontiers(one_way):
    g, pairs, want, G = one_way
    for mode in ("et", "astar"):
        assert np.array_equal(G.batch(pairs, mode=mode, strategy="auto"), want)
    for frontier in ("sparse", "dense"):
        got = G.batch(pairs, mode="bidastar", frontier=frontier, team_ctas=2, big_team_ctas=2)
        assert np.array_equal(got, want), frontier
    # VC-SSSP: a minimum bipartite cover, targets in it searching backward
    for strategy in ("vc", "sssp"):
        got, cnt = G.batch(pairs, mode="bids", strategy=strategy, return_counters=True)
        assert np.array_equal(got, want), strategy
        _, n_src = ppsp.batch_sources(pairs, strategy, undirected=False)
        assert cnt["searches"] == n_src
    rstar = np.ascontiguousarray(star_pairs(g, 12, 117)[:, ::-1])
    got, cnt = G.batch(rstar, mode="bids", strategy="vc", return_counters=True)
    assert np.array_equal(got, oracle.pairs(g.offsets, g.targets, g.weights, rstar)) and cnt["searches"] == 1


def test_one_way_paths(one_way):
    g, pairs, want, G = one_way
    sub = pairs[:40]
    st, dist, paths, lens = G.batch_paths(sub, 1 << 14, mode="bidastar")
    assert st == ppsp.OK and np.array_equal(dist, want[:40])
    edge_w = {}
    for u in range(g.n):
        for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
            edge_w[(u, int(g.targets[e]))] = int(g.weights[e])
    for (s, t), d, p in zip(sub, dist, paths):
        if d == INF:
            continue
        assert p is not None and p[0] == s and p[-1] == t
        assert sum(edge_w[(int(a), int(b))] for a, b in zip(p[:-1], p[1:])) == d


def test_potential_is_consistent_on_directed_edges(one_way):
    from oracle import potential as opot

    g, pairs, want, G = one_way
    P = G.potential_coords()
    info = G.info()
    # the same creation rule, applied by the oracle to the directed CSR
    c, F, P_ref = opot.choose_scale(g.offsets, g.targets, g.weights, g.coords)
    assert (info["potential_scale"], info["potential_shift"]) == (c, F)
    assert np.array_equal(P, P_ref)
    rng = np.random.default_rng(5)
    for anchor in rng.choice(g.n, size=4, replace=False):
        h = opot.h_all(P, int(anchor), int(info["potential_shift"]))
        src = np.repeat(np.arange(g.n), np.diff(g.offsets).astype(np.int64))
        # h_x(u) - h_x(v) <= w(u, v) on every directed edge, both ways round
        assert np.all(h[src] - h[g.targets] <= g.weights.astype(np.int64))
        assert np.all(h[g.targets] - h[src] <= g.weights.astype(np.int64))
