"""Oracle pins of a surface reaction nonlinear in the concentration (no GPU).
Sec. 4.2.2 evaluates the reaction flux F explicitly at C_X of Eq. 13 and adds
it to the bounced population, however nonlinear F is; here F is the rational
form (kappa0 + kappa1 C) / (1 + K C), which holds Michaelis-Menten and
Langmuir-Hinshelwood kinetics and is the Robin flux at K = 0."""
import numpy as np
import pytest

import oracle as O
from oracle import analytic as AN
from oracle import links as LK

D = 0.25 * (0.9 - 0.5)


def _channel(ny, d, bottom, C_top, steps, threads=1):
    walls = {1: (1 - d, ny - 2 + d)}
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(0.02, 0, 0)),
         (1, 0, O.H): bottom, (1, 1, O.H): dict(kind=O.GIVEN, phi_wall=C_top, u_wall=(0.02, 0, 0))}
    shape = (1, ny, 1)
    s = O.OracleSim(2, shape, LK.box_solid(shape, walls), 0.8, tau_D=0.9, has_h=True, threads=threads)
    s.set_links(LK.box_links(2, shape, walls, p, has_h=True))
    s.init(C0=1.0)
    s.step(steps)
    return s.moments()["C"][1:-1], walls[1]


def test_closed_form_balances_the_flux():
    """The wall value of the closed form satisfies the flux balance, and at
    K = 0 the closed form is the linear Robin one."""
    y0, y1, C_top = 0.5, 12.5, 3.0
    V, Km = 0.01, 0.8
    C = AN.reactive_channel_rational(np.array([y0, y1]), y0, y1, D, 0.0, -V / Km, 1 / Km, C_top)
    Cb = C[0]
    assert abs(C[1] - C_top) < 1e-14
    assert abs(D * (C_top - Cb) / (y1 - y0) - V * Cb / (Km + Cb)) < 1e-15
    y = np.linspace(y0, y1, 7)
    a = AN.reactive_channel_rational(y, y0, y1, D, 0.02, -0.02, 0.0, C_top)
    b = AN.reactive_channel(y, y0, y1, D, 0.02, -0.02, C_top)
    assert np.abs(a - b).max() < 1e-14


def test_rational_flux_at_zero_K_is_the_robin_wall():
    """With K = 0 the rational flux is k0 + k1 C_X, the same arithmetic as the
    linear flux wall: the trajectories agree bit for bit."""
    c1, _ = _channel(14, 0.3, dict(kind=O.FLUX, kappa0=0.02, kappa1=-0.02), 3.0, 500)
    c2, _ = _channel(14, 0.3, dict(kind=O.FLUX_RATIONAL, kappa0=0.02, kappa1=-0.02, phi_wall=0.0), 3.0, 500)
    assert np.array_equal(c1, c2)


@pytest.mark.parametrize("d", [0.5, 0.25, 1.0])
def test_michaelis_menten_wall(d):
    """A wall consuming C at the rate V C / (Km + C) under a shear flow along
    the wall: the steady profile is linear with the wall value of the flux
    balance.  Exact at d = 1/2 (C_X is exact for a linear profile and M = A);
    second-order close otherwise."""
    V, Km, C_top = 0.01, 0.8, 3.0
    bottom = dict(kind=O.FLUX_RATIONAL, kappa0=0.0, kappa1=-V / Km, phi_wall=1 / Km)
    C, (y0, y1) = _channel(14, d, bottom, C_top, 60000)
    Ca = AN.reactive_channel_rational(np.arange(14)[1:-1], y0, y1, D, 0.0, -V / Km, 1 / Km, C_top)
    tol = 1e-11 if d == 0.5 else 5e-3
    assert np.abs(C - Ca).max() / C_top < tol
