"""Oracle pins of the open boundaries of Sec. 5.1 (no GPU): a given inlet
velocity (the velocity wall kind with a normal u, Eq. 41/43) and a given outlet
pressure (Eq. 42/44, with u at X extrapolated by Eq. 13)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import links as LK


def _open_x(shape, d, U, rho_out, walls_y=None, tau=0.8, threads=1):
    """Domain open along x: inlet of given velocity at the low x boundary,
    outlet of given density at the high one, both at distance d from the first
    and last fluid layers; optional static walls along y."""
    nx = shape[0]
    walls = {}
    if walls_y is not None:
        walls[1] = walls_y
    walls[0] = (1 - d, nx - 2 + d)
    p = {(0, 0, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0)),
         (0, 1, O.F): dict(kind=O.PRESSURE, phi_wall=rho_out)}
    if walls_y is not None:
        p[(1, 0, O.F)] = dict(kind=O.VELOCITY)
        p[(1, 1, O.F)] = dict(kind=O.VELOCITY)
    solid = LK.box_solid(shape, walls)
    links = LK.box_links(2, shape, walls, p)
    s = O.OracleSim(2, shape, solid, tau, threads=threads)
    return s, links, solid.reshape(-1) == 0, walls


@pytest.mark.parametrize("d", [0.25, 0.5, 0.75, 1.0])
def test_uniform_stream_is_a_fixed_point(d):
    """Uniform flow u = (U, 0) at the outlet density is an exact steady state
    of the open boundaries: the inlet increment f^eq_a - f^eq_a' and the outlet
    sum f^eq_a + f^eq_a' at the extrapolated u(X) (Eq. 13, exact for a uniform
    field) rebuild the equilibrium populations.  A wrong weight, sign or
    quadratic term in either scheme moves the state."""
    shape, U, rho_w = (16, 3, 1), 0.04, 1.02
    s, links, fl, _ = _open_x(shape, d, U, rho_w)
    s.set_links(links)
    N = shape[0] * shape[1]
    u = np.zeros((N, 3))
    u[:, 0] = U
    s.init(rho=np.full(N, rho_w), u=u)
    s.step(200)
    m = s.moments()
    assert np.abs(m["u"][fl, 0] - U).max() < 1e-13          # rounding over 200 steps
    assert np.abs(m["u"][fl, 1:]).max() < 1e-13
    assert np.abs(m["rho"][fl] - rho_w).max() < 1e-13


@pytest.mark.parametrize("d", [0.5, 1.0])
def test_open_domain_reaches_the_inlet_velocity_and_outlet_density(d):
    """Started at rest with density 1, the open domain settles to the inlet
    velocity and the outlet's given density (1.03): the outlet imposes the
    density itself, not an extrapolated one.  Eq. 44 at d = 1 is stable here."""
    shape, U, rho_w = (20, 3, 1), 0.03, 1.03
    s, links, fl, _ = _open_x(shape, d, U, rho_w)
    s.set_links(links)
    s.init()
    s.step(12000)
    m = s.moments()
    assert np.abs(m["u"][fl, 0] - U).max() < 1e-5
    assert np.abs(m["rho"][fl] - rho_w).max() < 1e-5


@pytest.mark.parametrize("d", [0.5, 1.0])
def test_open_poiseuille_channel(d):
    """Sec. 5.1's inlet/outlet pair on a plane channel (static half-grid walls,
    Eq. 43): a parabolic inlet profile, given outlet density.  Away from the
    outlet the profile stays the parabola (0.5 % of U at the channel middle)
    and the pressure gradient is the Poiseuille one, 8 rho nu U / (2H)^2, to
    the compressibility error of the lattice (3 %)."""
    nx, ny, U, tau = 48, 18, 0.02, 0.8
    y0, y1 = 0.5, ny - 1.5
    s, links, fl, walls = _open_x((nx, ny, 1), d, U, 1.0, walls_y=(y0, y1), tau=tau, threads=4)
    prof = lambda y: 4 * U * (y - y0) * (y1 - y) / (y1 - y0) ** 2
    e, _ = O.lattice(2)
    x, y = links["node"] % nx, links["node"] // nx
    inlet = (links["kind"] == O.VELOCITY) & (x == 1) & (links["u_wall"][:, 0] != 0)
    ey = np.array([e[a][1] for a in links["dir"]])
    links["u_wall"][inlet, 0] = prof(y[inlet] - links["d"][inlet] * ey[inlet])   # u at the wall point X
    s.set_links(links)
    s.init()
    s.step(20000)
    m = s.moments()
    u = m["u"][:, 0].reshape(ny, nx)
    rho = m["rho"].reshape(ny, nx)
    assert np.abs(u[1:-1, nx // 2] - prof(np.arange(1, ny - 1))).max() / U < 5e-3
    nu = (tau - 0.5) / 3
    grad = np.polyfit(np.arange(5, nx - 5), rho[ny // 2, 5:nx - 5] / 3.0, 1)[0]
    assert abs(-grad / (8 * nu * U / (y1 - y0) ** 2) - 1) < 0.03


@pytest.mark.parametrize("field", ["h", "g"])
def test_pressure_kind_is_refused_beside_other_fields(field):
    """The given-pressure kind belongs to flow-only cases (the paper's open
    channel): a case with a concentration or a magnetic field refuses it."""
    shape = (8, 3, 1)
    s, links, _, _ = _open_x(shape, 0.5, 0.01, 1.0)
    g = O.OracleSim(2, shape, LK.box_solid(shape, {0: (0.5, 6.5)}), 0.8,
                    has_h=(field == "h"), has_g=(field == "g"))
    with pytest.raises(ValueError):
        g.set_links(links)
