"""Integer A* potential, written out from its definition.  TEST INFRASTRUCTURE ONLY.

Paper Sec. 3.3: A* needs a heuristic h with h(u) <= w(u,v) + h(v) on every edge
(consistency, which with h(t) = 0 implies admissibility; Fact 3.1 then makes
the reduced weights non-negative).  The paper uses Euclidean distance for k-NN
graphs (Sec. 6 "Setup").  With integer weights w = round(1000 * length), the
literal floor(1000 * Euclid) is NOT always consistent (an edge of length 0.4004
has w = 400 but the floors of 1000 * distance can differ by 401), so the
library uses a scaled, fixed-point form whose consistency is certified edge by
edge:

* the graph's scale c (float64) is chosen at graph creation;
* a fixed-point shift F (default 4) and integer potential coordinates
  P(v) = floor(2^F * c * p(v) + 0.5), computed per component in float64 from
  the float32 input coordinates p(v) as ``floor(float64(p) * (2^F * c) + 0.5)``;
* h_x(v) = floor(|P(v) - P(x)| / 2^F) = isqrt(floor((dX^2 + dY^2) / 4^F)),
  exact in integers (floor(sqrt(floor(y))) = floor(sqrt(y)) for y >= 0);
* certificate: dX^2 + dY^2 <= (2^F * w)^2 on every edge (u, v).  Then
  h_x(u) - h_x(v) <= ceil(|P(u) - P(v)| / 2^F) <= w(u, v), i.e. h_x is
  consistent for every anchor x, and h_x(x) = 0.
"""

from __future__ import annotations

import math

import numpy as np


def potential_coords(coords: np.ndarray, c: float, shift: int = 4) -> np.ndarray:
    """P(v) = floor(float64(p(v)) * (2^F c) + 0.5) as int64 [n, 2]."""
    s = np.float64(1 << shift) * np.float64(c)
    p = np.asarray(coords, dtype=np.float32).astype(np.float64)
    return np.floor(p * s + 0.5).astype(np.int64)


def h_one(P: np.ndarray, x: int, v: int, shift: int = 4) -> int:
    """h_x(v) with Python integers and math.isqrt (the definition)."""
    dx = int(P[v, 0]) - int(P[x, 0])
    dy = int(P[v, 1]) - int(P[x, 1])
    return math.isqrt((dx * dx + dy * dy) >> (2 * shift))


def isqrt_array(d: np.ndarray) -> np.ndarray:
    """Exact floor(sqrt(d)) for int64 d >= 0: float estimate then integer fix-up."""
    d = np.asarray(d, dtype=np.int64)
    r = np.floor(np.sqrt(d.astype(np.float64))).astype(np.int64)
    for _ in range(4):
        over = r * r > d
        r = np.where(over, r - 1, r)
    for _ in range(4):
        under = (r + 1) * (r + 1) <= d
        r = np.where(under, r + 1, r)
    return r


def h_all(P: np.ndarray, x: int, shift: int = 4) -> np.ndarray:
    """h_x(v) for every v (int64 [n])."""
    d = P - P[x][None, :]
    return isqrt_array((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) >> (2 * shift))


def certificate_ok(off: np.ndarray, tgt: np.ndarray, w: np.ndarray, P: np.ndarray,
                   shift: int = 4) -> np.ndarray:
    """Per-edge certificate dX^2 + dY^2 <= (2^F w)^2 (bool [m])."""
    n = off.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off).astype(np.int64))
    d = P[src] - P[tgt.astype(np.int64)]
    lhs = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    rhs = ((1 << shift) * w.astype(np.int64)) ** 2
    return lhs <= rhs


def consistent_for_anchor(off: np.ndarray, tgt: np.ndarray, w: np.ndarray, h: np.ndarray) -> bool:
    """Fact 3.1 precondition: h(u) <= w(u,v) + h(v) on every CSR edge."""
    n = off.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off).astype(np.int64))
    return bool(np.all(h[src] <= w.astype(np.int64) + h[tgt.astype(np.int64)]))


MAX_SHIFT = 8          # at most 8 fixed-point bits
COORD_LIMIT = 2 ** 30  # |P(v)| stays below 2^30, so squared differences fit 63 bits
SHRINK_ATTEMPTS = 40   # the margin doubles at most this many times


def _edge_sources(off: np.ndarray) -> np.ndarray:
    n = off.shape[0] - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(off).astype(np.int64))


def certificate_ok_exact(off: np.ndarray, tgt: np.ndarray, w: np.ndarray, P: np.ndarray,
                         shift: int) -> bool:
    """The certificate dX^2 + dY^2 <= (2^F w)^2 on every edge, in exact
    unsigned 64-bit arithmetic (|P| < 2^30 keeps the left side below 2^63;
    a right side of 2^64 or more holds for any left side)."""
    src = _edge_sources(off)
    d = P[src] - P[tgt.astype(np.int64)]
    lhs = (d[:, 0] * d[:, 0]).astype(np.uint64) + (d[:, 1] * d[:, 1]).astype(np.uint64)
    sw = w.astype(np.uint64) << np.uint64(shift)
    big = sw >= np.uint64(1 << 32)
    rhs = np.where(big, np.uint64(0), sw * sw)
    return bool(np.all(big | (lhs <= rhs)))


def choose_scale(off: np.ndarray, tgt: np.ndarray, w: np.ndarray, coords: np.ndarray):
    """Scale c, shift F and coordinates P of the certified potential, by the
    rule the library states for graph creation (Sec. 3.3, Fact 3.1), written
    out step by step in float64:

    1. over the edges of positive Euclidean length l (float64 of the float32
       coordinates): c_max = min w / l and w_min = min w; a zero weight on
       such an edge admits no positive scale (c = 0: the potential is 0);
    2. F = the largest shift <= 8 with a_max * c_max * 2^F < 2^30, a_max the
       largest absolute coordinate (none: c = 0);
    3. margin e = 2 / (2^F w_min); try c = c_max (1 - e), P = floor(p 2^F c
       + 0.5), and double e until the certificate holds on every edge (at
       most 40 times; else c = 0).

    Returns (c, F, P int64 [n, 2]); c = 0 comes with F = 0 and P = 0.
    """
    off = np.asarray(off, dtype=np.uint64)
    tgt = np.asarray(tgt, dtype=np.uint32)
    w = np.asarray(w, dtype=np.uint32)
    p = np.asarray(coords, dtype=np.float32).astype(np.float64)
    n = p.shape[0]
    none = (0.0, 0, np.zeros((n, 2), dtype=np.int64))
    src = _edge_sources(off)
    d = p[src] - p[tgt.astype(np.int64)]
    ell = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    pos = ell > 0.0
    if not np.any(pos) or np.any(w[pos] == 0):
        return none
    c_max = float(np.min(w[pos].astype(np.float64) / ell[pos]))
    w_min = int(np.min(w[pos]))
    a_max = float(np.max(np.abs(p))) if n else 0.0
    if a_max == 0.0 or not np.isfinite(c_max) or c_max <= 0.0:
        return none
    F = MAX_SHIFT
    while F > 0 and a_max * c_max * float(2 ** F) >= float(COORD_LIMIT):
        F -= 1
    if a_max * c_max * float(2 ** F) >= float(COORD_LIMIT):
        return none
    e = 2.0 / (float(2 ** F) * float(max(1, w_min)))
    for _ in range(SHRINK_ATTEMPTS):
        c = c_max * (1.0 - e)
        if c <= 0.0:
            break
        P = np.floor(p * (float(2 ** F) * c) + 0.5).astype(np.int64)
        if certificate_ok_exact(off, tgt, w, P, F):
            return c, F, P
        e *= 2.0
    return none
