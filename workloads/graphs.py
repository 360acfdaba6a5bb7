"""Seeded synthetic graph generators (CSR, undirected, uint32 weights).

Every generator returns a :class:`CSRGraph` whose adjacency lists are sorted
by target id and hold both directions of each undirected edge with the same
weight.  Vertex ids of grid graphs are row-major (``y * side + x``) after the
largest-component relabelling, which keeps grid neighbours close in memory.

Shapes (paper Sec. 6 "Setup" and its graph table): road graphs have average
degree about 2.5-2.7 and diameters in the thousands of hops; social graphs are
power-law with integer weights uniform in a range.  The paper's real datasets
are not available here, so these recipes stand in for their shapes only.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class CSRGraph:
    """A seeded synthetic graph in CSR form (an undirected edge is stored in
    both directions), with the vertex coordinates and grid cells of the
    grid-based recipes and the ids of the largest connected component."""

    n: int
    offsets: np.ndarray  # uint64 [n+1]
    targets: np.ndarray  # uint32 [m]
    weights: np.ndarray  # uint32 [m]
    coords: Optional[np.ndarray] = None  # float32 [n, 2] (cell units), or None
    grid_xy: Optional[np.ndarray] = None  # int32 [n, 2] original grid cell, or None
    lcc: Optional[np.ndarray] = None  # uint32 ids of the largest component
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.targets.shape[0])

    def degree(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def _components(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    a = coo_matrix((np.ones(u.shape[0], dtype=np.int8), (u, v)), shape=(n, n)).tocsr()
    _, labels = connected_components(a, directed=False)
    return labels


def csr_from_undirected(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray) -> tuple:
    """Build a symmetric CSR from unique undirected edges (u, v, w), u != v.

    Returns (offsets uint64[n+1], targets uint32[m], weights uint32[m]) with
    each row sorted by target id.  Repeated (u, v) pairs are kept, in input
    order within their row.
    """
    u = np.asarray(u).astype(np.int64)
    v = np.asarray(v).astype(np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w]).astype(np.uint32)
    from scipy.sparse import coo_matrix

    # distinct pairs: a counting sort by row, then each row sorted by target
    # (the same result as sorting the (row, target) keys)
    a = coo_matrix((ww, (src, dst)), shape=(n, n)).tocsr()
    a.sort_indices()
    if a.nnz == src.shape[0]:
        return a.indptr.astype(np.uint64), a.indices.astype(np.uint32), a.data.astype(np.uint32)
    # repeated pairs (merged by the conversion above): a stable sort of the
    # (row, target) keys keeps every copy, in input order
    key = (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)
    order = np.argsort(key, kind="stable")
    src = src[order]
    targets = dst[order].astype(np.uint32)
    weights = ww[order]
    counts = np.bincount(src, minlength=n)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    return offsets, targets, weights


def _dedup_undirected(u, v, w):
    """Drop self-loops and repeated undirected edges, keeping the first copy."""
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    lo = np.minimum(u, v).astype(np.uint64)
    hi = np.maximum(u, v).astype(np.uint64)
    key = (lo << np.uint64(32)) | hi
    # the first copy of each key is its smallest index: an unstable sort,
    # then the minimum index over each run of equal keys
    order = np.argsort(key)
    sk = key[order]
    starts = np.flatnonzero(np.r_[True, sk[1:] != sk[:-1]])
    first = np.minimum.reduceat(order, starts)
    first.sort()
    return lo[first], hi[first], w[first]


def _grid_edges(side: int):
    ids = np.arange(side * side, dtype=np.int64).reshape(side, side)  # [y, x]
    hu = ids[:, :-1].ravel()
    hv = ids[:, 1:].ravel()
    vu = ids[:-1, :].ravel()
    vv = ids[1:, :].ravel()
    return np.concatenate([hu, vu]), np.concatenate([hv, vv])


def _jittered_coords(side: int, jitter: float, rng: np.random.Generator) -> tuple:
    ys, xs = np.divmod(np.arange(side * side, dtype=np.int64), side)
    grid_xy = np.stack([xs, ys], axis=1).astype(np.int32)
    coords = grid_xy.astype(np.float64) + rng.uniform(-jitter, jitter, size=(side * side, 2))
    return coords, grid_xy


def _euclid(coords: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    d = coords[u] - coords[v]
    return np.sqrt((d * d).sum(axis=1))


def _finish(n, u, v, w, coords, grid_xy, name, meta, keep_lcc: bool) -> CSRGraph:
    labels = _components(n, u.astype(np.int64), v.astype(np.int64))
    big = np.bincount(labels).argmax()
    in_lcc = labels == big
    if keep_lcc:
        new_id = np.full(n, -1, dtype=np.int64)
        kept = np.nonzero(in_lcc)[0]
        new_id[kept] = np.arange(kept.shape[0])
        eu = new_id[u.astype(np.int64)]
        ev = new_id[v.astype(np.int64)]
        ok = (eu >= 0) & (ev >= 0)
        u, v, w = eu[ok], ev[ok], w[ok]
        n = int(kept.shape[0])
        if coords is not None:
            coords = coords[kept]
        if grid_xy is not None:
            grid_xy = grid_xy[kept]
        lcc = np.arange(n, dtype=np.uint32)
    else:
        lcc = np.nonzero(in_lcc)[0].astype(np.uint32)
    off, tgt, wgt = csr_from_undirected(n, u, v, w)
    return CSRGraph(
        n=n,
        offsets=off,
        targets=tgt,
        weights=wgt,
        coords=None if coords is None else coords.astype(np.float32),
        grid_xy=grid_xy,
        lcc=lcc,
        name=name,
        meta=meta,
    )


def grid_graph(side: int, seed: int, jitter: float = 0.3, noise_max: int = 100,
               uniform_weight: Optional[int] = None) -> CSRGraph:
    """4-neighbour side x side grid with jittered coordinates.

    Weight of an undirected edge = round(1000 * Euclidean length) + U{0..noise_max},
    drawn once per undirected edge.  ``uniform_weight`` replaces that with a
    constant (and ``jitter`` is then usually 0): the closed-form test case.
    """
    rng = np.random.default_rng(seed)
    n = side * side
    coords, grid_xy = _jittered_coords(side, jitter, rng)
    u, v = _grid_edges(side)
    if uniform_weight is not None:
        w = np.full(u.shape[0], uniform_weight, dtype=np.uint32)
    else:
        w = np.rint(1000.0 * _euclid(coords, u, v)).astype(np.int64)
        w = w + rng.integers(0, noise_max + 1, size=u.shape[0])
        w = np.maximum(w, 1).astype(np.uint32)
    meta = {"kind": "grid", "side": side, "seed": seed, "jitter": jitter}
    return _finish(n, u, v, w, coords, grid_xy, f"grid{side}", meta, keep_lcc=False)


def road_like_graph(side: int, seed: int, jitter: float = 0.3, delete_frac: float = 0.10,
                    shortcut_frac: float = 0.005, shortcut_radius: int = 20) -> CSRGraph:
    """Road-like graph: jittered side x side grid, a fraction of grid edges
    deleted at random, short random shortcuts added, largest component kept.

    * shortcut count = shortcut_frac * (grid edge count before deletion);
      each shortcut joins a uniform random vertex u to u + (dx, dy), with the
      integer offset uniform over lattice points of the disc of radius
      ``shortcut_radius`` cells, excluding (0, 0); offsets leaving the grid are
      redrawn;
    * weights = round(1000 * Euclidean length of the jittered coordinates);
    * the largest connected component is taken after deletion and shortcuts
      and relabelled in row-major order.
    """
    rng = np.random.default_rng(seed)
    n = side * side
    coords, grid_xy = _jittered_coords(side, jitter, rng)
    gu, gv = _grid_edges(side)
    e0 = gu.shape[0]
    n_del = int(round(delete_frac * e0))
    keep = np.ones(e0, dtype=bool)
    keep[rng.choice(e0, size=n_del, replace=False)] = False
    gu, gv = gu[keep], gv[keep]

    r = shortcut_radius
    lattice = np.array([(dx, dy) for dx in range(-r, r + 1) for dy in range(-r, r + 1)
                        if 0 < dx * dx + dy * dy <= r * r], dtype=np.int64)
    n_sc = int(round(shortcut_frac * e0))
    su = np.empty(0, dtype=np.int64)
    sv = np.empty(0, dtype=np.int64)
    while su.shape[0] < n_sc:
        need = n_sc - su.shape[0]
        cu = rng.integers(0, n, size=2 * need + 16)
        off = lattice[rng.integers(0, lattice.shape[0], size=cu.shape[0])]
        cx = cu % side + off[:, 0]
        cy = cu // side + off[:, 1]
        ok = (cx >= 0) & (cx < side) & (cy >= 0) & (cy < side)
        su = np.concatenate([su, cu[ok][:need]])
        sv = np.concatenate([sv, (cy * side + cx)[ok][:need]])

    u = np.concatenate([gu, su])
    v = np.concatenate([gv, sv])
    w = np.rint(1000.0 * _euclid(coords, u, v)).astype(np.int64)
    w = np.maximum(w, 1).astype(np.uint32)
    u, v, w = _dedup_undirected(u, v, w)
    meta = {"kind": "road_like", "side": side, "seed": seed, "jitter": jitter,
            "delete_frac": delete_frac, "shortcut_frac": shortcut_frac,
            "shortcut_radius": shortcut_radius, "shortcuts": n_sc, "deleted": n_del}
    return _finish(n, u, v, w, coords, grid_xy, f"road{side}", meta, keep_lcc=True)


def rmat_graph(scale: int, seed: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, wmin: int = 1, wmax: int = 65535, chunk: int = 1 << 23) -> CSRGraph:
    """Power-law RMAT graph: 2^scale vertices, edge_factor * 2^scale generated
    directed edges with quadrant probabilities (a, b, c, 1-a-b-c); self-loops
    dropped, symmetrised, duplicates removed; one uniform integer weight in
    [wmin, wmax] per undirected edge.  All vertices are kept (isolated ones
    included); ``lcc`` lists the largest component for query endpoints.
    """
    rng = np.random.default_rng(seed)
    n = 1 << scale
    total = edge_factor * n
    us, vs = [], []
    ab, abc = a + b, a + b + c
    for start in range(0, total, chunk):
        cnt = min(chunk, total - start)
        u = np.zeros(cnt, dtype=np.uint32)
        v = np.zeros(cnt, dtype=np.uint32)
        for level in range(scale):
            r = rng.random(cnt, dtype=np.float32)
            # quadrant: [0, a) top-left, [a, a+b) top-right, [a+b, a+b+c)
            # bottom-left, [a+b+c, 1) bottom-right
            down = r >= ab
            right = (r >= a) ^ down ^ (r >= abc)
            u |= down.view(np.uint8).astype(np.uint32) << np.uint32(level)
            v |= right.view(np.uint8).astype(np.uint32) << np.uint32(level)
        us.append(u)
        vs.append(v)
    u = np.concatenate(us)
    v = np.concatenate(vs)
    del us, vs
    w = rng.integers(wmin, wmax + 1, size=u.shape[0]).astype(np.uint32)
    u, v, w = _dedup_undirected(u, v, w)
    meta = {"kind": "rmat", "scale": scale, "edge_factor": edge_factor, "a": a, "b": b, "c": c,
            "seed": seed, "wmin": wmin, "wmax": wmax}
    return _finish(n, u, v, w, None, None, f"rmat{scale}", meta, keep_lcc=False)


def one_way_graph(g: CSRGraph, frac: float, seed: int) -> CSRGraph:
    """Directed variant of an undirected graph: for a seeded fraction of its
    undirected edges one direction (chosen at random) is dropped, the rest keep
    both (one-way streets on a road-like graph).  Coordinates are kept; the
    result is a directed CSR (rows sorted by target), ``meta["directed"]``."""
    rng = np.random.default_rng(seed)
    deg = np.diff(g.offsets).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.targets.astype(np.int64)
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    # one decision per undirected edge {lo, hi}: keep both, or only lo->hi / hi->lo
    key = lo * g.n + hi
    uniq, inv = np.unique(key, return_inverse=True)
    drop = rng.random(uniq.shape[0]) < frac
    keep_fwd = rng.random(uniq.shape[0]) < 0.5  # if dropping: keep lo->hi, else hi->lo
    d, kf = drop[inv], keep_fwd[inv]
    is_fwd = src == lo
    keep = ~d | (kf & is_fwd) | (~kf & ~is_fwd)
    src, dst, w = src[keep], dst[keep], g.weights[keep]
    off = np.zeros(g.n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(src, minlength=g.n), out=off[1:])
    meta = dict(g.meta)
    meta.update({"directed": True, "one_way_frac": frac, "one_way_seed": seed})
    return CSRGraph(n=g.n, offsets=off, targets=dst.astype(np.uint32), weights=w.astype(np.uint32),
                    coords=g.coords, grid_xy=g.grid_xy, lcc=g.lcc, name=g.name + f"-oneway{frac}", meta=meta)
