"""Host logic of the learned stepping increment (no GPU): labels from sweep
times, the regret measures and the margin choice.

The labels must be the smallest increment within 5% of a group's best time
(time rises steeply above the optimum), regret is zero exactly when every
prediction hits its group's best grid point, and the pessimistic regret
charges a prediction between two grid points the larger increment's time.
"""

import numpy as np

from paper_2506_16488_gb300 import learned_delta as ld
from paper_2506_16488_gb300.learned_delta import MARGINS, ceil_regret, default_regret, labels_from_times, regret

GRID = (-2, -1, 0, 1)


def test_labels_break_near_ties_towards_smaller_delta():
    t = np.array([[5.0, 3.0, 3.1, 9.0],      # -1 and 0 within 5%: -1
                  [np.inf, 2.0, 1.0, 1.02],  # 0 best, 1 within 5%: 0
                  [1.0, 2.0, 3.0, 4.0]])     # -2 strictly best
    assert labels_from_times(t, grid=GRID).tolist() == [-1.0, 0.0, -2.0]
    assert labels_from_times(t, grid=GRID, tie=0.0).tolist() == [-1.0, 0.0, -2.0]
    t2 = np.array([[1.0, 1.04, 1.2, 9.0]])
    assert labels_from_times(t2, grid=GRID, tie=0.0).tolist() == [-2.0]
    assert labels_from_times(t2[:, ::-1].copy(), grid=GRID).tolist() == [0.0]  # 1.04 within 5% of 1.0


def test_regret_measures():
    t = np.array([[4.0, 2.0, 3.0, 8.0],
                  [6.0, 5.0, 1.0, 2.0]])
    best = t.min(axis=1).sum()
    assert regret(t, np.array([-1.0, 0.0]), grid=GRID) == 0.0
    # nearest grid point vs the pessimistic (larger) one for predictions in between
    assert np.isclose(regret(t, np.array([-0.6, 0.4]), grid=GRID), (2.0 + 1.0) / best - 1.0)
    assert np.isclose(ceil_regret(t, np.array([-0.6, 0.4]), grid=GRID), (3.0 + 2.0) / best - 1.0)
    assert np.isclose(ceil_regret(t, np.array([-1.0, 0.0]), grid=GRID), 0.0)
    # predictions outside the grid are clipped to its ends
    assert np.isclose(ceil_regret(t, np.array([-9.0, 9.0]), grid=GRID), (4.0 + 2.0) / best - 1.0)
    assert np.isclose(default_regret(t, grid=GRID), (3.0 + 1.0) / best - 1.0)
    t[:, 2] = np.inf  # the default column never timed
    assert default_regret(t, grid=GRID) is None


def test_margins_start_at_zero_and_grow():
    m = np.asarray(MARGINS)
    assert m[0] == 0.0 and np.all(np.diff(m) > 0) and m[-1] <= 2.0


def test_doubling_rule_regret():
    # three groups, grid points -1, 0, 1 (the last one never swept)
    t = np.array([[2.0, 1.0, np.inf],
                  [1.0, 3.0, np.inf],
                  [4.0, 4.0, np.inf]])
    grid = (-1, 0, 1)
    # one increment for all: column totals 7 and 8, so -1 (7) against the
    # per-group best 1 + 1 + 4 = 6
    r, j = ld.doubling_regret(t, grid)
    assert j == -1 and abs(r - (7.0 / 6.0 - 1.0)) < 1e-12
    assert ld.doubling_regret(np.full((2, 3), np.inf), grid) == (None, None)
