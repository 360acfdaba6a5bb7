"""Seeded query sets: random pairs, near/mid/far terciles, stars and cliques.

The paper picks query endpoints from the largest connected component (Sec. 6
"Setup") and studies queries by distance percentile and by query-graph shape
(Sec. 6.3: stars, cliques, random pairs).  Pairs are returned as uint32
arrays of shape [k, 2] (source, target).
"""

from __future__ import annotations

import numpy as np

from .graphs import CSRGraph, grid_graph, road_like_graph, rmat_graph


def _pool(g: CSRGraph) -> np.ndarray:
    return g.lcc if g.lcc is not None else np.arange(g.n, dtype=np.uint32)


def random_pairs(g: CSRGraph, k: int, seed: int) -> np.ndarray:
    """k uniform random pairs of vertices of the largest component."""
    rng = np.random.default_rng(seed)
    pool = _pool(g)
    idx = rng.integers(0, pool.shape[0], size=(k, 2))
    return pool[idx].astype(np.uint32)


def near_mid_far_pairs(g: CSRGraph, k: int, seed: int, oversample: int = 30) -> tuple:
    """k pairs split into thirds by grid (Manhattan) distance terciles.

    Candidates are uniform random pairs from the largest component; their
    Manhattan distance on the original grid cells defines the terciles.
    Returns (pairs [k, 2], label [k] with 0 = near, 1 = mid, 2 = far).
    """
    assert g.grid_xy is not None, "near/mid/far needs grid cells"
    rng = np.random.default_rng(seed)
    pool = _pool(g)
    cand = pool[rng.integers(0, pool.shape[0], size=(oversample * k, 2))]
    dxy = np.abs(g.grid_xy[cand[:, 0]].astype(np.int64) - g.grid_xy[cand[:, 1]].astype(np.int64))
    man = dxy.sum(axis=1)
    q1, q2 = np.quantile(man, [1.0 / 3.0, 2.0 / 3.0])
    bins = [man <= q1, (man > q1) & (man <= q2), man > q2]
    sizes = [k // 3, k // 3, k - 2 * (k // 3)]
    out, lab = [], []
    for b, (mask, sz) in enumerate(zip(bins, sizes)):
        idx = np.nonzero(mask)[0]
        pick = rng.choice(idx, size=sz, replace=False)
        out.append(cand[pick])
        lab.append(np.full(sz, b, dtype=np.int32))
    return np.concatenate(out).astype(np.uint32), np.concatenate(lab)


def star_pairs(g: CSRGraph, leaves: int, seed: int) -> np.ndarray:
    """One centre and ``leaves`` distinct leaves: a star query graph."""
    rng = np.random.default_rng(seed)
    pool = _pool(g)
    pick = rng.choice(pool.shape[0], size=leaves + 1, replace=False)
    verts = pool[pick]
    return np.stack([np.full(leaves, verts[0]), verts[1:]], axis=1).astype(np.uint32)


def clique_pairs(g: CSRGraph, size: int, seed: int) -> np.ndarray:
    """All size*(size-1)/2 pairs among ``size`` distinct vertices."""
    rng = np.random.default_rng(seed)
    pool = _pool(g)
    verts = pool[rng.choice(pool.shape[0], size=size, replace=False)]
    ii, jj = np.triu_indices(size, k=1)
    return np.stack([verts[ii], verts[jj]], axis=1).astype(np.uint32)


def config_workload(cfg: int, small: bool = False) -> dict:
    """The five benchmark configurations as graph + query batches.

    Seeds are cfg * 1000 + j.  ``small`` shrinks the graph with the same
    recipe (used where a test only needs the shape, not the size).

    1: 64x64 jittered grid, 100 random pairs, BiDS.
    2: 1024^2 road-like grid, 1,000 near/mid/far pairs, BiD-A*.
    3: RMAT scale 22 (edge factor 16), batches of 64: random pairs, 64-leaf star,
       11-clique (55 pairs), BiDS.
    4: 2048^2 road-like grid, 1,552 random pairs + a 32-clique (496 pairs).
    5: 4096^2 road-like grid, uint64 distances (serving).
    """
    base = cfg * 1000
    if cfg == 1:
        g = grid_graph(64, seed=base + 1)
        return {"graph": g, "batches": {"random": random_pairs(g, 100, base + 2)}, "mode": "bids"}
    if cfg == 2:
        g = road_like_graph(128 if small else 1024, seed=base + 1)
        pairs, lab = near_mid_far_pairs(g, 1000, base + 2)
        return {"graph": g, "batches": {"nmf": pairs}, "labels": lab, "mode": "bidastar"}
    if cfg == 3:
        g = rmat_graph(14 if small else 22, seed=base + 1)
        return {
            "graph": g,
            "batches": {
                "random": random_pairs(g, 64, base + 2),
                "star": star_pairs(g, 64, base + 3),
                "clique": clique_pairs(g, 11, base + 4),
            },
            "mode": "bids",
        }
    if cfg == 4:
        g = road_like_graph(256 if small else 2048, seed=base + 1)
        pairs = np.concatenate([random_pairs(g, 1552, base + 2), clique_pairs(g, 32, base + 3)])
        lab = np.r_[np.zeros(1552, dtype=np.int32), np.ones(496, dtype=np.int32)]  # random pairs, clique
        return {"graph": g, "batches": {"mixed": pairs}, "labels": lab, "mode": "multi_astar"}
    if cfg == 5:
        g = road_like_graph(256 if small else 4096, seed=base + 1)
        return {"graph": g, "batches": {"random": random_pairs(g, 256, base + 2)}, "mode": "serving"}
    raise ValueError(f"unknown config {cfg}")
