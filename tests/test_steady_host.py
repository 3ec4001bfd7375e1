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


def test_each_case_stops_at_its_own_plateau():
    # case 0 decays then levels off at 3e-3 after 20 intervals; case 1 levels off after 50
    c0 = lambda j: max(3e-3, 0.1 * math.exp(-0.2 * j))
    c1 = lambda j: max(3e-3, 0.1 * math.exp(-0.07 * j))
    s = FakeSolver([c0, c1])
    done, last = SD.run_to_plateau(s, 100000, interval=100, window=10, ratio=0.9)
    # a plateau is declared once the last 10 intervals fell by less than 10 %
    # (monotone curves: the windows' minima are their last values)
    j0 = next(j for j in range(20, 999) if c0(j) > 0.9 * c0(j - 10))
    j1 = next(j for j in range(20, 999) if c1(j) > 0.9 * c1(j - 10))
    assert s.j == [j0, j1]
    assert done == 100 * max(j0, j1)
    assert np.allclose(last, [c0(j0), c1(j1)])
    # both frozen when done and resumed before the return
    assert s.active == [True, True]
    assert (0, False) in s.log and (1, False) in s.log and s.log[-2:] in ([(0, True), (1, True)],)


def test_an_oscillating_residual_is_judged_by_its_minima():
    """A residual that oscillates while it decays (a warm start's acoustic
    transient) is not taken for a plateau: its windows' minima still fall."""
    c = lambda j: max(3e-3, 0.05 * math.exp(-0.05 * j) * (1.5 + math.cos(1.3 * j)))
    s = FakeSolver([c])
    SD.run_to_plateau(s, 100000, interval=100, window=10, ratio=0.9)
    h = [c(j) for j in range(1, s.j[0] + 1)]
    assert min(h[-10:]) > 0.9 * min(h[-20:-10])
    assert all(min(h[:k][-10:]) <= 0.9 * min(h[:k][-20:-10]) for k in range(20, len(h)))
    assert c(s.j[0]) < 5e-3


def test_tolerance_and_step_limit():
    s = FakeSolver([lambda j: 1e-7, lambda j: 1.0 / (j + 1)])
    done, last = SD.run_to_plateau(s, 1000, interval=100, window=10, ratio=0.9, tol=1e-6)
    assert s.j[0] == 1                       # below tol at its first check
    assert done == 1000 and s.j[1] == 10     # never level: stopped by the step limit
    assert last[0] == 1e-7 and math.isclose(last[1], 1.0 / 11)
    assert s.active == [True, True]
