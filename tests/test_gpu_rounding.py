"""The stochastic rounding of 16-bit storage is unbiased, checked through the
step itself.

A fully periodic box at rest under a uniform body force has an exact
solution: every node stays alike, rho stays rho0, and the reported velocity
u = (sum e f + F/2) / rho grows by a per step, u(t) = (t + 1/2) a.  The force
is chosen so small that after ~2000 steps each step's change of a population
is below half the FP16 spacing of its (scaled) offset: storage that rounds to
nearest would stop following the solution there, while rounding stochastically
keeps the mean over the nodes on it, up to the random walk of the rounding
noise: about 0.3 of a spacing (2^-10 of an offset) per population and step,
as a random walk over 5000 steps averaged over 4096 nodes, is about 3e-4 of u
in FP16 and 8 times more in BF16 (the tolerances below).  Measured on GB300:
-1.2e-5 (FP16), -9.2e-4 (BF16); FP32, which rounds to nearest, -6.2e-5 (its
bias is the larger); FP64 -2.7e-13."""
import numpy as np
import pytest

from paper_2506_00907_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPE = (64, 64, 1)
A = 1e-8
STEPS = 5000


def _mean_u(prec):
    case = lbm.make_case(SHAPE, 0.8, 1.0, 1.0, (A, 0.0, 0.0))
    g = lbm.Solver(lbm.LBM_D2Q9, prec, lbm.LBM_FLOW, [case])
    g.set_graph(100)
    g.step(STEPS)
    m = g.moments(0)
    return m["u"][:, 0].mean(), np.abs(m["rho"] - 1.0).max()


@pytest.mark.parametrize("prec,tol", [(lbm.LBM_FP64, 1e-11), (lbm.LBM_FP32, 1e-4), (lbm.LBM_FP16S, 3e-4),
                                      (lbm.LBM_BF16S, 3e-3)])
def test_uniform_acceleration_follows_the_exact_solution(prec, tol):
    u, drho = _mean_u(prec)
    exact = (STEPS + 0.5) * A
    print("\nprec %d: mean u / exact - 1 = %.3g, max |rho - 1| = %.3g" % (prec, u / exact - 1.0, drho))
    assert abs(u - exact) <= tol * exact, (u, exact)
    assert drho <= 1e-3
