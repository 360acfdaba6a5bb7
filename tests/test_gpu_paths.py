"""Shortest paths returned with the distances.

Shortest paths need not be unique, so a returned path is checked for what is
unique: it starts at s, ends at t, consecutive vertices are CSR neighbours,
and its weight equals the oracle distance.
"""

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import ppsp
from workloads import clique_pairs, grid_graph, random_pairs, road_like_graph, star_pairs
from workloads.graphs import csr_from_undirected

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _check(g, s, t, d, path):
    if d == oracle.INF_INT:
        assert path is not None and len(path) == 0
        return
    assert path[0] == s and path[-1] == t
    assert oracle.path_weight(g.offsets, g.targets, g.weights, path) == d


@pytest.mark.parametrize("mode", ["bids", "bidastar", "et", "astar"])
def test_single_query_paths(mode):
    g = road_like_graph(64, seed=71)
    pairs = random_pairs(g, 15, 72)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for (s, t), w in zip(pairs.tolist(), want.tolist()):
            st, d, path, n = G.query_path(s, t, mode=mode)
            assert st == ppsp.OK and d == w
            _check(g, s, t, d, path)
        st, d, path, n = G.query_path(5, 5, mode=mode)
        assert st == ppsp.OK and d == 0 and list(path) == [5]


@pytest.mark.parametrize("strategy", ["multi", "plain_star"])
def test_batch_paths_with_shared_endpoints(strategy):
    g = road_like_graph(72, seed=73)
    pairs = np.concatenate([star_pairs(g, 10, 1), clique_pairs(g, 6, 2), random_pairs(g, 20, 3)])
    pairs = np.concatenate([pairs, pairs[:8, ::-1]])  # reversed pairs get reversed paths
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        for mode in ("bids", "bidastar"):
            st, d, paths, lens = G.batch_paths(pairs, 4096, mode=mode, strategy=strategy)
            assert st == ppsp.OK and np.array_equal(d, want)
            for (s, t), dd, p in zip(pairs.tolist(), d.tolist(), paths):
                _check(g, s, t, dd, p)


def test_path_buffer_too_small_reports_length():
    g = grid_graph(32, seed=74)
    with ppsp.Graph.from_csr(g) as G:
        st, d, path, n = G.query_path(0, g.n - 1, cap=5)
        assert st == ppsp.ERR_BUFFER_TOO_SMALL and n >= 63 and path is None
        assert d == oracle.dijkstra_pair(g.offsets, g.targets, g.weights, 0, g.n - 1)
        st, d, path, n2 = G.query_path(0, g.n - 1, cap=n)
        assert st == ppsp.OK and len(path) == n2 == n


def test_paths_disconnected_and_zero_weights():
    off, tgt, w = csr_from_undirected(5, np.array([0, 2]), np.array([1, 3]), np.array([4, 6], dtype=np.uint32))
    with ppsp.Graph(off, tgt, w) as G:
        st, d, path, n = G.query_path(0, 3)
        assert st == ppsp.OK and d == oracle.INF_INT and n == 0
    off, tgt, w = csr_from_undirected(3, np.array([0, 1]), np.array([1, 2]), np.array([0, 6], dtype=np.uint32))
    with ppsp.Graph(off, tgt, w) as G:
        st, d, path, n = G.query_path(0, 2)
        assert st == ppsp.ERR_UNSUPPORTED
        assert G.query(0, 2) == 6
