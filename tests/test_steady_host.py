"""Host logic of the two-precision steady runner, on a fake solver whose
cases have prescribed residual histories (no GPU)."""
import math

import numpy as np

from paper_2506_00907_gb300 import steady as SD


class FakeSolver:
    """Case i's residual after its j-th interval is curves[i](j); frozen cases
    do not advance (their residual is 0, as lbm_check reports)."""

    def __init__(self, curves):
        self.curves = curves
        self.j = [0] * len(curves)
        self.active = [True] * len(curves)
        self.steps = 0
        self.log = []

    def check(self, raise_unstable=True):
        out = np.zeros((len(self.curves), 8))
        for i, f in enumerate(self.curves):
            r = f(self.j[i]) if self.active[i] and self.j[i] > 0 else 0.0
            out[i, 6], out[i, 7] = r * r, 1.0
        return out

    def step(self, n):
        self.steps += n
        for i in range(len(self.curves)):
            if self.active[i]:
                self.j[i] += 1

    def set_active(self, i, a):
        self.log.append((i, bool(a)))
        self.active[i] = bool(a)


def test_residuals_of_a_check_record():
    out = np.zeros((3, 8))
    out[:, 6] = [4.0, 0.0, 1.0]
    out[:, 7] = [16.0, 5.0, 0.0]
    assert np.allclose(SD.residuals(out), [0.5, 0.0, 0.0])


def _stop(c, w=20, ratio=0.9):
    """The first interval after which the mean of the last w residuals is
    above ratio times the mean of the w before (brute force)."""
    return next(j for j in range(2 * w, 10 ** 5)
                if np.mean([c(k) for k in range(j - w + 1, j + 1)]) >
                ratio * np.mean([c(k) for k in range(j - 2 * w + 1, j - w + 1)]))


def test_each_case_stops_at_its_own_plateau():
    # case 0 decays then levels off at 3e-3; case 1 decays more slowly
    c0 = lambda j: max(3e-3, 0.1 * math.exp(-0.1 * j))
    c1 = lambda j: max(3e-3, 0.1 * math.exp(-0.03 * j))
    s = FakeSolver([c0, c1])
    done, last = SD.run_to_plateau(s, 100000, interval=100)
    j0, j1 = _stop(c0), _stop(c1)
    assert j0 < j1 and s.j == [j0, j1]
    assert done == 100 * j1
    assert np.allclose(last, [c0(j0), c1(j1)])
    # both frozen when done and resumed before the return
    assert s.active == [True, True]
    assert s.log[-2:] == [(0, True), (1, True)] and (0, False) in s.log and (1, False) in s.log


def test_an_oscillating_residual_is_judged_by_window_means():
    """A residual that oscillates while it decays (period 12 intervals, as
    the warm-started pipes show) is not taken for a plateau at a trough: the
    means of 20-interval windows still fall until the floor."""
    c = lambda j: 3e-4 + 0.02 * math.exp(-0.04 * j) * (1.0 + 0.9 * math.cos(2 * math.pi * j / 12))
    s = FakeSolver([c])
    SD.run_to_plateau(s, 100000, interval=100)
    assert s.j[0] == _stop(c)
    assert 0.02 * math.exp(-0.04 * s.j[0]) < 0.25 * 3e-4 * 10     # within a few floors of the floor
    # a rule on single checks would have stopped at the first trough
    assert s.j[0] > 40


def test_tolerance_and_step_limit():
    s = FakeSolver([lambda j: 1e-7, lambda j: 1.0 / (j + 1)])
    done, last = SD.run_to_plateau(s, 1000, interval=100, window=10, ratio=0.9, tol=1e-6)
    assert s.j[0] == 1                       # below tol at its first check
    assert done == 1000 and s.j[1] == 10     # never level: stopped by the step limit
    assert last[0] == 1e-7 and math.isclose(last[1], 1.0 / 11)
    assert s.active == [True, True]
