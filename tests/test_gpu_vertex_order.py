"""The device vertex order (a Hilbert curve over the coordinates) is internal:
every call takes and returns the caller's ids, and answers equal those of the
caller's order and of the oracle."""

import numpy as np
import pytest

import oracle
from oracle import potential as opot
from paper_2506_16488_gb300 import ppsp
from workloads import clique_pairs, near_mid_far_pairs, one_way_graph, random_pairs, road_like_graph, star_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_batches_paths_and_potentials_match_the_callers_order():
    g = road_like_graph(160, seed=171)
    pairs = np.concatenate([random_pairs(g, 60, 172), near_mid_far_pairs(g, 30, 173)[0], clique_pairs(g, 6, 174),
                            star_pairs(g, 8, 175), [[int(g.lcc[0]), int(g.lcc[0])]]]).astype(np.uint32)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    c, F, P = opot.choose_scale(g.offsets, g.targets, g.weights, g.coords)
    with ppsp.Graph.from_csr(g) as G, ppsp.Graph.from_csr(g, keep_order=True) as K:
        for mode in ("bids", "bidastar", "astar", "et"):
            for strategy in ("multi", "auto", "vc", "plain_star"):
                got = G.batch(pairs, mode=mode, strategy=strategy)
                assert np.array_equal(got, want), (mode, strategy)
                assert np.array_equal(K.batch(pairs, mode=mode, strategy=strategy), want), (mode, strategy)
        # potentials are reported per caller vertex and equal the oracle's
        assert np.array_equal(G.potential_coords(), P)
        assert np.array_equal(K.potential_coords(), P)
        verts = np.arange(0, g.n, 7, dtype=np.uint32)
        for x in (0, int(g.lcc[3]), g.n - 1):
            assert np.array_equal(G.potential_eval(x, verts), opot.h_all(P, x, F)[verts])
        # paths come back in caller ids and are shortest paths
        for s, t in pairs[:20].tolist():
            st, d, path, n = G.query_path(s, t, mode="bidastar")
            assert st == ppsp.OK and d == oracle.dijkstra_pair(g.offsets, g.targets, g.weights, s, t)
            if d != oracle.INF_INT:
                assert path[0] == s and path[-1] == t
                assert oracle.path_weight(g.offsets, g.targets, g.weights, path) == d


def test_directed_graph_in_device_order():
    g = one_way_graph(road_like_graph(96, seed=181), 0.3, seed=182)
    pairs = np.concatenate([random_pairs(g, 50, 183), clique_pairs(g, 5, 184)]).astype(np.uint32)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g, undirected=False) as G:
        for mode in ("bids", "bidastar"):
            for strategy in ("multi", "auto", "vc"):
                assert np.array_equal(G.batch(pairs, mode=mode, strategy=strategy), want), (mode, strategy)
        for q, (s, t) in enumerate(pairs[:10].tolist()):
            st, d, path, n = G.query_path(s, t, mode="bids")
            assert st == ppsp.OK and d == int(want[q])
            if d != oracle.INF_INT and s != t:
                assert path[0] == s and path[-1] == t
                assert oracle.path_weight(g.offsets, g.targets, g.weights, path) == d
