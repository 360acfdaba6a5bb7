"""Pins for the CPU oracle (runs without a GPU).

The oracle is the plain definition of d(s,t) (binary-heap Dijkstra).  These
tests tie it to things other than itself: brute-force path enumeration,
Floyd-Warshall (itself pinned to enumeration), scipy's independent Dijkstra,
closed forms on grids and paths, BFS hop counts on unit weights, a hand-worked
example, and the metric properties (symmetry, triangle inequality).
"""

import itertools
import math
from collections import deque

import numpy as np
import pytest

import oracle
from workloads import grid_graph, road_like_graph
from workloads.graphs import csr_from_undirected

INF = oracle.INF_INT


def _csr_directed(n, edges):
    """Directed CSR from (u, v, w) triples, rows sorted by target."""
    edges = sorted(edges)
    off = np.zeros(n + 1, dtype=np.uint64)
    for u, _, _ in edges:
        off[u + 1] += 1
    off = np.cumsum(off).astype(np.uint64)
    tgt = np.array([v for _, v, _ in edges], dtype=np.uint32)
    w = np.array([x for _, _, x in edges], dtype=np.uint32)
    return off, tgt, w


def _random_graph(rng, n, m, wmax, undirected=True, zero_frac=0.1):
    edges = []
    for _ in range(m):
        u, v = int(rng.integers(0, n)), int(rng.integers(0, n))
        wt = 0 if rng.random() < zero_frac else int(rng.integers(1, wmax + 1))
        edges.append((u, v, wt))
        if undirected and u != v:
            edges.append((v, u, wt))
    return _csr_directed(n, edges)


def _enumerate_simple_paths(n, off, tgt, w, s, t):
    """Minimum weight over all simple s-t paths (exhaustive DFS)."""
    best = INF
    if s == t:
        return 0
    stack = [(s, 0, frozenset([s]))]
    while stack:
        u, d, seen = stack.pop()
        for e in range(int(off[u]), int(off[u + 1])):
            v = int(tgt[e])
            if v in seen:
                continue
            nd = d + int(w[e])
            if v == t:
                best = min(best, nd)
            else:
                stack.append((v, nd, seen | {v}))
    return best


def test_hand_worked_example():
    # 0 -(4)- 1 -(1)- 2 -(2)- 3,  0 -(7)- 2,  1 -(6)- 3,  4 isolated, undirected.
    # From 0: d1 = 4, d2 = min(7, 4+1) = 5, d3 = min(5+2, 4+6) = 7, d4 = inf.
    u = np.array([0, 1, 2, 0, 1])
    v = np.array([1, 2, 3, 2, 3])
    wt = np.array([4, 1, 2, 7, 6], dtype=np.uint32)
    off, tgt, w = csr_from_undirected(5, u, v, wt)
    assert [oracle.dijkstra_pair(off, tgt, w, 0, t) for t in range(5)] == [0, 4, 5, 7, INF]
    d, p = oracle.path(off, tgt, w, 0, 3)
    assert d == 7 and list(p) == [0, 1, 2, 3]


@pytest.mark.parametrize("seed", range(6))
def test_floyd_warshall_vs_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    n = 6
    off, tgt, w = _random_graph(rng, n, 9, 9, undirected=bool(seed % 2))
    fw = oracle.floyd_warshall(off, tgt, w)
    for s in range(n):
        for t in range(n):
            assert int(fw[s, t]) == _enumerate_simple_paths(n, off, tgt, w, s, t)


@pytest.mark.parametrize("seed", range(8))
def test_dijkstra_vs_floyd_warshall(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 60))
    m = int(rng.integers(0, 3 * n))
    off, tgt, w = _random_graph(rng, n, m, 50, undirected=bool(seed % 2), zero_frac=0.15)
    fw = oracle.floyd_warshall(off, tgt, w)
    for s in range(n):
        dist = oracle.sssp(off, tgt, w, s)
        assert np.array_equal(dist, fw[s])
        for t in rng.integers(0, n, size=5):
            assert oracle.dijkstra_pair(off, tgt, w, s, int(t)) == int(fw[s, t])


def test_dijkstra_vs_scipy():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra as sp_dijkstra

    g = road_like_graph(40, seed=7)
    a = csr_matrix((g.weights.astype(np.float64), g.targets.astype(np.int64),
                    g.offsets.astype(np.int64)), shape=(g.n, g.n))
    rng = np.random.default_rng(3)
    srcs = rng.integers(0, g.n, size=5)
    ref = sp_dijkstra(a, directed=True, indices=srcs)
    for row, s in zip(ref, srcs):
        dist = oracle.sssp(g.offsets, g.targets, g.weights, int(s))
        finite = np.isfinite(row)
        assert np.array_equal(dist[finite], row[finite].astype(np.uint64))
        assert np.all(dist[~finite] == oracle.INF)


def test_closed_form_uniform_grid():
    side, wt = 23, 7
    g = grid_graph(side, seed=1, jitter=0.0, uniform_weight=wt)
    rng = np.random.default_rng(5)
    for s, t in rng.integers(0, g.n, size=(40, 2)):
        sx, sy = int(s) % side, int(s) // side
        tx, ty = int(t) % side, int(t) // side
        assert oracle.dijkstra_pair(g.offsets, g.targets, g.weights, int(s), int(t)) == \
            wt * (abs(sx - tx) + abs(sy - ty))


def test_path_graph_prefix_sums():
    n = 50
    rng = np.random.default_rng(9)
    wt = rng.integers(0, 1000, size=n - 1).astype(np.uint32)
    off, tgt, w = csr_from_undirected(n, np.arange(n - 1), np.arange(1, n), wt)
    pre = np.concatenate([[0], np.cumsum(wt.astype(np.int64))])
    for s, t in rng.integers(0, n, size=(30, 2)):
        assert oracle.dijkstra_pair(off, tgt, w, int(s), int(t)) == abs(int(pre[t]) - int(pre[s]))


def _bfs(off, tgt, s):
    n = off.shape[0] - 1
    d = [INF] * n
    d[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for e in range(int(off[u]), int(off[u + 1])):
            v = int(tgt[e])
            if d[v] == INF:
                d[v] = d[u] + 1
                q.append(v)
    return d


def test_unit_weights_equal_bfs():
    g = road_like_graph(30, seed=11)
    ones = np.ones_like(g.weights)
    for s in [0, 17, g.n // 2, g.n - 1]:
        assert list(oracle.sssp(g.offsets, g.targets, ones, s)) == _bfs(g.offsets, g.targets, s)


def test_symmetry_triangle_and_paths():
    g = road_like_graph(48, seed=13)
    rng = np.random.default_rng(17)
    for s, t, mid in rng.integers(0, g.n, size=(25, 3)):
        s, t, mid = int(s), int(t), int(mid)
        dst = oracle.dijkstra_pair(g.offsets, g.targets, g.weights, s, t)
        assert dst == oracle.dijkstra_pair(g.offsets, g.targets, g.weights, t, s)
        dsm = oracle.dijkstra_pair(g.offsets, g.targets, g.weights, s, mid)
        dmt = oracle.dijkstra_pair(g.offsets, g.targets, g.weights, mid, t)
        assert dst <= dsm + dmt
        d, p = oracle.path(g.offsets, g.targets, g.weights, s, t)
        assert d == dst and p[0] == s and p[-1] == t
        assert oracle.path_weight(g.offsets, g.targets, g.weights, p) == d


def test_degenerate_cases():
    off, tgt, w = csr_from_undirected(4, np.array([0]), np.array([1]), np.array([5], dtype=np.uint32))
    assert oracle.dijkstra_pair(off, tgt, w, 2, 2) == 0
    assert oracle.dijkstra_pair(off, tgt, w, 0, 3) == INF
    d, p = oracle.path(off, tgt, w, 0, 3)
    assert d == INF and p.shape[0] == 0
    d, p = oracle.path(off, tgt, w, 1, 1)
    assert d == 0 and list(p) == [1]
    out = oracle.pairs(off, tgt, w, np.array([[0, 1], [1, 0], [0, 2]]))
    assert list(out) == [5, 5, INF]


def test_threaded_pairs_match_serial():
    g = road_like_graph(32, seed=19)
    pairs = np.random.default_rng(1).integers(0, g.n, size=(20, 2)).astype(np.uint32)
    assert np.array_equal(oracle.pairs_threaded(g.offsets, g.targets, g.weights, pairs, 4),
                          oracle.pairs(g.offsets, g.targets, g.weights, pairs))
