"""Shape checks for the seeded synthetic inputs (no method arithmetic here)."""

import numpy as np

from workloads import (clique_pairs, config_workload, grid_graph, near_mid_far_pairs, random_pairs,
                       rmat_graph, road_like_graph, star_pairs)


def _symmetric(g):
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.offsets).astype(np.int64))
    fwd = set(zip(src.tolist(), g.targets.tolist(), g.weights.tolist()))
    return all((v, u, w) in fwd for (u, v, w) in fwd)


def test_grid_config1_shape():
    g = grid_graph(64, seed=1001)
    assert g.n == 4096 and g.m == 2 * 8064
    assert _symmetric(g)
    assert g.weights.min() >= 400 and g.weights.max() <= 1600 + 100
    g2 = grid_graph(64, seed=1001)
    assert np.array_equal(g.weights, g2.weights)


def test_road_like_shape():
    g = road_like_graph(96, seed=5)
    assert 0.8 * 96 * 96 < g.n <= 96 * 96
    assert _symmetric(g)
    assert 3.0 < g.m / g.n < 4.0  # road-like average degree
    assert g.coords.shape == (g.n, 2) and g.grid_xy.shape == (g.n, 2)
    assert np.all(np.diff(g.offsets.astype(np.int64)) >= 0)
    pairs, lab = near_mid_far_pairs(g, 99, seed=6)
    assert pairs.shape == (99, 2) and np.bincount(lab).tolist() == [33, 33, 33]
    man = np.abs(g.grid_xy[pairs[:, 0]] - g.grid_xy[pairs[:, 1]]).sum(axis=1)
    assert man[lab == 0].max() <= man[lab == 2].min()


def test_rmat_small():
    g = rmat_graph(10, seed=3)
    assert g.n == 1024
    assert _symmetric(g)
    assert g.weights.min() >= 1 and g.weights.max() <= 65535
    deg = np.diff(g.offsets.astype(np.int64))
    assert deg.max() > 10 * max(1.0, np.median(deg))  # skewed degrees


def test_query_sets():
    g = grid_graph(16, seed=2)
    assert random_pairs(g, 10, 1).shape == (10, 2)
    st = star_pairs(g, 8, 1)
    assert len(set(st[:, 0].tolist())) == 1 and len(set(st[:, 1].tolist())) == 8
    cl = clique_pairs(g, 5, 1)
    assert cl.shape == (10, 2) and len(set(cl.ravel().tolist())) == 5


def test_config_workloads_small():
    for cfg in (1, 2, 3, 4, 5):
        wl = config_workload(cfg, small=True)
        assert wl["graph"].n > 0
        for pairs in wl["batches"].values():
            assert pairs.ndim == 2 and pairs.shape[1] == 2
            assert pairs.max() < wl["graph"].n
    assert config_workload(4, small=True)["batches"]["mixed"].shape == (2048, 2)


def test_one_way_graph_keeps_one_direction_of_every_edge():
    from workloads import one_way_graph, road_like_graph

    g = road_like_graph(40, seed=3)
    d = one_way_graph(g, 0.3, 4)
    und = {(int(u), int(v)): int(w) for u, v, w in zip(np.repeat(np.arange(g.n), np.diff(g.offsets).astype(np.int64)),
                                                        g.targets, g.weights)}
    dire = {(int(u), int(v)): int(w) for u, v, w in zip(np.repeat(np.arange(d.n), np.diff(d.offsets).astype(np.int64)),
                                                         d.targets, d.weights)}
    assert set(dire) <= set(und) and all(dire[e] == und[e] for e in dire)
    pairs = {(min(u, v), max(u, v)) for u, v in und}
    for a, b in pairs:
        assert (a, b) in dire or (b, a) in dire  # never both directions dropped
    one_way = sum(1 for a, b in pairs if ((a, b) in dire) != ((b, a) in dire))
    assert abs(one_way / len(pairs) - 0.3) < 0.05
    assert d.meta["directed"]
