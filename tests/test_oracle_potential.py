"""Pins for the oracle's integer A* potential (runs without a GPU).

Definition (paper Sec. 3.3, Fact 3.1; the certified fixed-point form is spelled
out in oracle/potential.py): h_x(v) = isqrt(floor(|P(v) - P(x)|^2 / 256)).
"""

import math

import numpy as np

from oracle import potential as pot
from workloads import road_like_graph


def test_isqrt_array_matches_math_isqrt():
    rng = np.random.default_rng(0)
    vals = list(rng.integers(0, 1 << 53, size=2000)) + list(range(0, 300))
    for r in [1, 2, 3, 1000, 94906265, 67108863, 67108864]:
        vals += [r * r - 1, r * r, r * r + 1]
    d = np.array(vals, dtype=np.int64)
    got = pot.isqrt_array(d)
    assert all(int(g) == math.isqrt(int(v)) for g, v in zip(got, d))


def test_anchor_is_zero_and_pythagorean_triples():
    P = np.array([[0, 0], [16 * 3 * 7, 16 * 4 * 7], [-16 * 5, 16 * 12], [15, 0], [16, 0]],
                 dtype=np.int64)
    assert pot.h_one(P, 0, 0) == 0
    assert pot.h_one(P, 0, 1) == 35  # 3-4-5 triangle scaled by 7
    assert pot.h_one(P, 0, 2) == 13  # 5-12-13 triangle
    assert pot.h_one(P, 0, 3) == 0  # 15/16 of a unit floors to 0
    assert pot.h_one(P, 0, 4) == 1
    assert list(pot.h_all(P, 0)) == [0, 35, 13, 0, 1]
    assert pot.h_one(P, 1, 0) == 35  # symmetric


def test_literal_floor_1000_euclid_is_not_consistent():
    # Edge u=(0,0)-v=(0.4004,0): w = round(400.4) = 400.  Anchor x = (10, 0):
    # floor(1000|u-x|) - floor(1000|v-x|) = 10000 - 9599 = 401 > w.
    u, v, x = np.array([0.0, 0.0]), np.array([0.4004, 0.0]), np.array([10.0, 0.0])
    w = round(1000 * np.linalg.norm(u - v))
    hu = math.floor(1000 * np.linalg.norm(u - x))
    hv = math.floor(1000 * np.linalg.norm(v - x))
    assert hu - hv > w
    # The certified form: the same three points with a scale c for which the
    # certificate |P(u)-P(v)|^2 <= (16 w)^2 holds are consistent.
    coords = np.array([u, v, x], dtype=np.float32)
    c = 0.995 * w / np.linalg.norm(u - v)
    P = pot.potential_coords(coords, c)
    d = P[0] - P[1]
    assert int(d @ d) <= (16 * w) ** 2
    assert pot.h_one(P, 2, 0) - pot.h_one(P, 2, 1) <= w


def test_certified_potential_is_consistent_on_road_graph():
    g = road_like_graph(40, seed=23)
    n = g.n
    src = np.repeat(np.arange(n), np.diff(g.offsets).astype(np.int64))
    ell = np.linalg.norm(g.coords[src].astype(np.float64) - g.coords[g.targets].astype(np.float64), axis=1)
    c = 0.99 * float(np.min(g.weights / ell))
    P = pot.potential_coords(g.coords, c)
    assert pot.certificate_ok(g.offsets, g.targets, g.weights, P).all()
    rng = np.random.default_rng(4)
    for x in rng.integers(0, n, size=6):
        h = pot.h_all(P, int(x))
        assert h[int(x)] == 0
        assert pot.consistent_for_anchor(g.offsets, g.targets, g.weights, h)
    # Too large a scale breaks the certificate and consistency somewhere.
    Pbad = pot.potential_coords(g.coords, 1.5 * float(np.max(g.weights / ell)))
    assert not pot.certificate_ok(g.offsets, g.targets, g.weights, Pbad).all()
    bad = [pot.consistent_for_anchor(g.offsets, g.targets, g.weights, pot.h_all(Pbad, int(x)))
           for x in range(0, n, max(1, n // 20))]
    assert not all(bad)


def _csr(n, edges):
    from workloads.graphs import csr_from_undirected

    u = np.array([e[0] for e in edges], dtype=np.int64)
    v = np.array([e[1] for e in edges], dtype=np.int64)
    w = np.array([e[2] for e in edges], dtype=np.uint32)
    return csr_from_undirected(n, u, v, w)


def test_choose_scale_closed_form_on_a_uniform_grid():
    # Unit cells of weight 1000: c_max = 1000 / 1 exactly; a_max = 63, and
    # 63 * 1000 * 2^8 = 16,128,000 < 2^30, so F = 8; the margin is
    # e = 2 / (2^8 * 1000) = 2^-7 / 1000, so c = 1000 - 2^-7 = 999.9921875 and
    # 2^F c = 255,998: P(v) = 255,998 * (x, y), and the certificate holds at
    # once (|P(u) - P(v)| = 255,998 <= 256,000 = 2^F w).
    from workloads import grid_graph

    g = grid_graph(64, seed=1, jitter=0.0, uniform_weight=1000)
    c, F, P = pot.choose_scale(g.offsets, g.targets, g.weights, g.coords)
    assert F == 8
    assert c == 999.9921875
    assert np.array_equal(P, 255998 * g.grid_xy.astype(np.int64))


def test_choose_scale_shift_rule():
    # a_max * c_max * 2^F < 2^30 picks F: coordinates up to 5000 cells and
    # w / l = 1000 give 5e6 * 2^F < 1,073,741,824, i.e. 2^F <= 214: F = 7.
    off, tgt, w = _csr(2, [(0, 1, 1000)])
    coords = np.array([[4999.0, 0.0], [5000.0, 0.0]], dtype=np.float32)
    c, F, P = pot.choose_scale(off, tgt, w, coords)
    assert F == 7
    assert c == 1000.0 * (1.0 - 2.0 / (128 * 1000))
    # 2^F c = 127,998 per cell: P = floor(127,998 * x + 0.5)
    assert P.tolist() == [[127998 * 4999, 0], [127998 * 5000, 0]]
    # so large that even F = 0 overflows 2^30: no potential
    far = np.array([[2.0e6, 0.0], [2.0e6 + 1.0, 0.0]], dtype=np.float32)
    assert pot.choose_scale(off, tgt, w, far)[:2] == (0.0, 0)


def test_choose_scale_degenerate_inputs():
    # a zero weight on an edge of positive length admits no positive scale
    off, tgt, w = _csr(3, [(0, 1, 0), (1, 2, 700)])
    coords = np.array([[0, 0], [1, 0], [2, 0]], dtype=np.float32)
    c, F, P = pot.choose_scale(off, tgt, w, coords)
    assert (c, F) == (0.0, 0) and not P.any()
    # a zero weight between coincident points is fine: c from the other edge
    coords = np.array([[0, 0], [0, 0], [1, 0]], dtype=np.float32)
    c, F, P = pot.choose_scale(off, tgt, w, coords)
    assert F == 8 and c == 700.0 * (1.0 - 2.0 / (256 * 700))
    # every coordinate zero: nothing to scale
    c, F, _ = pot.choose_scale(off, tgt, w, np.zeros((3, 2), dtype=np.float32))
    assert (c, F) == (0.0, 0)


def test_choose_scale_is_certified_and_tight_on_a_road_graph():
    g = road_like_graph(64, seed=61)
    c, F, P = pot.choose_scale(g.offsets, g.targets, g.weights, g.coords)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets).astype(np.int64))
    ell = np.linalg.norm(g.coords[src].astype(np.float64) - g.coords[g.targets].astype(np.float64), axis=1)
    c_max = float(np.min(g.weights / ell))
    e0 = 2.0 / (2 ** F * float(g.weights.min()))
    # the first candidate of the rule is certified (rounding P moves an edge
    # by at most sqrt(2) fixed-point units, less than the margin of 2)
    assert c == c_max * (1.0 - e0) and 0.99 * 1000 < c < 1000
    assert pot.certificate_ok(g.offsets, g.targets, g.weights, P, F).all()
    assert pot.certificate_ok_exact(g.offsets, g.targets, g.weights, P, F)
    for x in (0, g.n // 2, g.n - 1):
        assert pot.consistent_for_anchor(g.offsets, g.targets, g.weights, pot.h_all(P, x, F))
    # without the margin the certificate fails on some edge
    Pn = pot.potential_coords(g.coords, c_max * (1.0 + 1e-4), F)
    assert not pot.certificate_ok_exact(g.offsets, g.targets, g.weights, Pn, F)
