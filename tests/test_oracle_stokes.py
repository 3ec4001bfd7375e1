"""Oracle pins of the oscillating wall of Sec. 5.2 (Stokes' second problem,
Eq. 45), no GPU.  The wall at the top of a channel moves with U cos(omega t);
the bottom wall is at rest; the periodic state is compared with the closed
form of u_t = nu u_yy after the start-up transient has decayed."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import analytic as AN
from oracle import links as LK

WO_PAPER = 1e-3 * math.sqrt(2 * math.pi / 1e-6)     # H sqrt(omega / nu) of the tau = 0.8 case of Sec. 5.2


def _stokes_error(ny, d, Wo, periods, tau=0.8, U=1e-3, phase=0.0):
    walls = LK.channel_y(2, 1, ny, 1, d, d)
    y0, y1 = walls[1]
    nu = (tau - 0.5) / 3
    omega = Wo ** 2 * nu / (y1 - y0) ** 2
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0))}
    s = O.OracleSim(2, (1, ny, 1), LK.box_solid((1, ny, 1), walls), tau)
    s.set_links(LK.box_links(2, (1, ny, 1), walls, p))
    s.init()
    s.set_wall_motion(omega, phase)
    nT = int(round(2 * math.pi / omega))
    s.step(periods * nT)
    y = np.arange(ny)[1:-1]
    err = 0.0
    for _ in range(8):                                  # eight phases of one period
        t = O.lib().orc_steps(s._h)
        ua = AN.stokes_oscillating(y, t, y0, y1, U, omega, nu, phase)
        err = max(err, np.abs(s.moments()["u"][1:-1, 0] - ua).max() / U)
        s.step(nT // 8)
    return err


def test_closed_form_solves_the_diffusion_problem():
    """The closed form satisfies u_t = nu u_yy and both wall conditions
    (checked by differences on a fine grid)."""
    y0, y1, U, omega, nu = 0.5, 40.5, 1.0, 3e-3, 0.1
    y = np.linspace(y0, y1, 4001)
    h, dt = y[1] - y[0], 1e-3
    u = lambda t: AN.stokes_oscillating(y, t, y0, y1, U, omega, nu, 0.3)
    ut = (u(7.0 + dt) - u(7.0 - dt)) / (2 * dt)
    uyy = (u(7.0)[2:] - 2 * u(7.0)[1:-1] + u(7.0)[:-2]) / h ** 2
    assert np.abs(ut[1:-1] - nu * uyy).max() < 1e-6 * U * omega
    assert abs(u(7.0)[0]) < 1e-15 and abs(u(7.0)[-1] - U * math.cos(omega * 7.0 + 0.3)) < 1e-12


def test_stokes_second_problem_half_grid_second_order():
    """Half-grid walls (Eq. 41 at d = 1/2) at the paper's Womersley number: the
    periodic state is within 1e-4 U of the closed form at H = 40 and the error
    falls by about four when H doubles."""
    e1 = _stokes_error(42, 0.5, WO_PAPER, periods=3)
    e2 = _stokes_error(82, 0.5, WO_PAPER, periods=3)
    assert e1 < 1e-4
    assert e1 / e2 > 3.0


@pytest.mark.parametrize("d", [0.25, 1.0])
def test_stokes_second_problem_other_wall_distances(d):
    """Eq. 15/16 (d < 1/2) and Eq. 43 (d >= 1/2) with the oscillating wall: the
    periodic state is within 2e-3 U of the closed form at H ~ 40."""
    assert _stokes_error(42 if d < 0.5 else 41, d, WO_PAPER, periods=3, phase=0.7) < 2e-3


def test_wall_motion_refuses_moving_flux_walls():
    """The moving-wall term of a flux wall of h or g would need the same
    oscillation; such a link list is refused."""
    walls = LK.channel_y(2, 1, 10, 1, 0.5, 0.5)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(0.01, 0, 0)),
         (1, 0, O.H): dict(kind=O.GIVEN, phi_wall=1.0), (1, 1, O.H): dict(kind=O.FLUX, u_wall=(0.01, 0, 0))}
    s = O.OracleSim(2, (1, 10, 1), LK.box_solid((1, 10, 1), walls), 0.8, has_h=True)
    s.set_links(LK.box_links(2, (1, 10, 1), walls, p, has_h=True))
    with pytest.raises(ValueError):
        s.set_wall_motion(1e-3)
