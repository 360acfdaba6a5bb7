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
