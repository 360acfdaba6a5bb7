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
