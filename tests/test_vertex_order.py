"""The device vertex order of graphs with coordinates (host only, no GPU):
a Hilbert-curve order.  Pinned by the curve's defining properties on full
square lattices — every step moves to a lattice neighbour, every aligned
2^j x 2^j block is one contiguous stretch, the curve starts at the origin —
and by the 2 x 2 and 4 x 4 visiting orders written out by hand."""

import numpy as np
import pytest

import __graft_entry__
from paper_2506_16488_gb300 import ppsp


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()


def _lattice(side):
    x, y = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    return np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float32)


def _sequence(xy):
    perm = ppsp.vertex_order(xy)
    assert np.array_equal(np.sort(perm), np.arange(xy.shape[0]))  # a permutation
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.shape[0], dtype=np.uint32)
    return xy[inv].astype(np.int64)


def test_two_by_two_and_four_by_four_by_hand():
    # quadrants are visited lower-left, upper-left, upper-right, lower-right;
    # inside the lower-left quadrant the curve is reflected about the
    # diagonal, inside the lower-right one about the anti-diagonal
    assert _sequence(_lattice(2)).tolist() == [[0, 0], [0, 1], [1, 1], [1, 0]]
    assert _sequence(_lattice(4)).tolist() == [
        [0, 0], [1, 0], [1, 1], [0, 1],  # lower-left quadrant
        [0, 2], [0, 3], [1, 3], [1, 2],  # upper-left
        [2, 2], [2, 3], [3, 3], [3, 2],  # upper-right
        [3, 1], [2, 1], [2, 0], [3, 0],  # lower-right
    ]


@pytest.mark.parametrize("side", [8, 16, 64])
def test_unit_steps_contiguous_blocks_and_origin(side):
    seq = _sequence(_lattice(side))
    assert seq[0].tolist() == [0, 0]
    steps = np.abs(np.diff(seq, axis=0)).sum(axis=1)
    assert np.all(steps == 1)  # a continuous curve through every cell once
    for j in range(1, int(np.log2(side))):
        b = 1 << j
        block = (seq[:, 0] // b) * (side // b) + seq[:, 1] // b
        # each aligned b x b block occupies one stretch of b*b consecutive positions
        assert np.all(block.reshape(-1, b * b) == block[:: b * b][:, None])


def test_scale_and_translation_invariant_and_ties_by_id():
    xy = _lattice(16)
    base = ppsp.vertex_order(xy)
    assert np.array_equal(ppsp.vertex_order(xy * 37.5 - 1000.0), base)
    # duplicate points keep their ids' order
    dup = np.concatenate([xy, xy[:5]])
    p = ppsp.vertex_order(dup)
    for k in range(5):
        assert p[k] < p[xy.shape[0] + k] and abs(int(p[k]) - int(p[xy.shape[0] + k])) == 1


def test_random_points_are_ordered_locally():
    rng = np.random.default_rng(5)
    xy = rng.random((20000, 2)).astype(np.float32)
    perm = ppsp.vertex_order(xy)
    ordered = xy[np.argsort(perm)].astype(np.float64)  # points in device order
    hil = np.sqrt((np.diff(ordered, axis=0) ** 2).sum(1)).mean()
    rnd = np.sqrt((np.diff(xy.astype(np.float64), axis=0) ** 2).sum(1)).mean()
    assert hil < 0.05 * rnd  # consecutive device ids are near each other in the plane


def test_degenerate_inputs():
    assert ppsp.vertex_order(np.zeros((1, 2), dtype=np.float32)).tolist() == [0]
    same = ppsp.vertex_order(np.ones((6, 2), dtype=np.float32))
    assert same.tolist() == list(range(6))  # all points equal: ties by id
    bad = np.zeros((4, 2), dtype=np.float32)
    bad[2, 0] = np.nan
    with pytest.raises(ppsp.PPSPError):
        ppsp.vertex_order(bad)
