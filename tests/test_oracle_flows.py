"""Pins of the FP64 oracle on whole flows: closed-form steady solutions derived
from the governing equations, published exact results of the BGK lattice
Boltzmann scheme, the paper's printed values, and conservation invariants."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_bvp

import oracle as O
from oracle import analytic as AN
from oracle import links as LK
from tests.helpers import affine_fixed_point


def _channel(nx, ny, d_lo, d_hi, tau, accel=(0, 0, 0), U_hi=0.0, threads=1):
    walls = LK.channel_y(2, nx, ny, 1, d_lo, d_hi)
    solid = LK.box_solid((nx, ny, 1), walls)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U_hi, 0, 0))}
    s = O.OracleSim(2, (nx, ny, 1), solid, tau, accel=accel, threads=threads)
    s.set_links(LK.box_links(2, (nx, ny, 1), walls, p))
    s.init()
    return s, walls[1]


def test_poiseuille_exact_at_magic_tau():
    """BGK with halfway bounce-back gives the exact parabolic Poiseuille profile
    when (tau - 1/2)^2 = 3/16 (Ginzburg & d'Humieres 2003, a published property
    of the scheme, independent of this code); at other tau the profile is still
    an exact parabola of curvature -a/nu (He et al. 1997) shifted by a slip."""
    ny, a = 18, 1e-5
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    s, (y0, y1) = _channel(1, ny, 0.5, 0.5, tau, accel=(a, 0, 0))
    s.step(12000)
    u = s.moments()["u"][:, 0][1:-1]
    y = np.arange(ny)[1:-1]
    ua = AN.poiseuille(y, y0, y1, a, (tau - 0.5) / 3)
    assert np.abs(u - ua).max() / ua.max() < 1e-11
    s, (y0, y1) = _channel(1, ny, 0.5, 0.5, 0.8, accel=(a, 0, 0))
    s.step(12000)
    u = s.moments()["u"][:, 0][1:-1]
    c = np.polyfit(y, u, 2)
    assert np.abs(u - np.polyval(c, y)).max() / u.max() < 1e-11
    assert abs(2 * c[0] / (-a / 0.1) - 1) < 1e-9
    ua = AN.poiseuille(y, y0, y1, a, 0.1)
    assert 1e-5 < np.abs(u - ua).max() / ua.max() < 1e-2     # O(dx^2) slip away from the magic tau


@pytest.mark.parametrize("d", [0.25, 0.5, 0.75, 1.0])
def test_couette_linear_profile(d):
    """Moving-wall scheme (Eq. 15/16 and 43) reproduces plane Couette flow
    between walls at y = 1 - d and y = ny - 2 + d (linear interpolation is exact
    for a linear profile)."""
    ny, U = 12, 0.05
    s, (y0, y1) = _channel(1, ny, d, d, 0.8, U_hi=U)
    s.step(8000)
    u = s.moments()["u"][:, 0][1:-1]
    ua = AN.couette(np.arange(ny)[1:-1], y0, y1, 0.0, U)
    assert np.abs(u - ua).max() / U < 1e-10


def test_static_walls_conserve_mass_at_half_grid():
    """Halfway bounce-back conserves mass exactly; the tangential moving wall
    conserves it up to rounding (Sec. 4.1)."""
    s, _ = _channel(3, 10, 0.5, 0.5, 0.7, accel=(1e-5, 0, 0))
    m0 = s.sums()[0]
    s.step(500)
    assert abs(s.sums()[0] - m0) < 1e-12
    s, _ = _channel(3, 10, 0.5, 0.5, 0.7, U_hi=0.05)
    m0 = s.sums()[0]
    s.step(500)
    assert abs(s.sums()[0] - m0) < 500 * 1e-14


# ------------------------------------------------------------ Hartmann-Couette
def _hartmann_couette(ny, d, cw_top, Ha=5.0, U=1e-3, steps=15000, accel=0.0, cw_bot=0.0):
    tau, taue = 0.8, 0.9
    nu, eta = (tau - 0.5) / 3, (taue - 0.5) / 4
    walls = LK.channel_y(2, 1, ny, 1, d, d)
    y0, y1 = walls[1]
    H, yc = (y1 - y0) / 2, (y1 + y0) / 2
    B0 = Ha * math.sqrt(nu * eta) / H

    def b1(cw, uw):
        if cw == 0:
            return dict(kind=O.GIVEN, phi_wall=0.0, u_wall=uw)
        if cw == math.inf:
            return dict(kind=O.FLUX, u_wall=uw)
        return dict(kind=O.FLUX, u_wall=uw, kappa1=-eta / (cw * H))
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0)),
         (1, 0, O.G0): b1(cw_bot, (0, 0, 0)), (1, 1, O.G0): b1(cw_top, (U, 0, 0)),
         (1, 0, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0),
         (1, 1, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0, u_wall=(U, 0, 0))}
    solid = LK.box_solid((1, ny, 1), walls)
    s = O.OracleSim(2, (1, ny, 1), solid, tau, tau_eta=taue, accel=(accel, 0, 0), has_g=True)
    s.set_links(LK.box_links(2, (1, ny, 1), walls, p, has_g=True))
    s.init(B0=(0, B0, 0))
    s.step(steps)
    m = s.moments()
    y = np.arange(ny)[1:-1] - yc

    def wt(cw):
        return ("insulating",) if cw == 0 else ("conducting",) if cw == math.inf else ("shercliff", cw)
    ua, ba = AN.hartmann(y, H, B0, nu, eta, accel=accel, U_hi=U, wall_lo=wt(cw_bot), wall_hi=wt(cw_top))
    u, b = m["u"][1:-1, 0], m["B"][1:-1, 0]
    bscale = max(U, 1e-30) * math.sqrt(nu / eta)            # B1* normalisation of Eq. 46
    return np.abs(u - ua).max() / U, np.abs(b - ba).max() / bscale, m["B"][1:-1, 1], B0


def test_hartmann_closed_form_solves_the_ode():
    """The closed form used as reference agrees with an independent numerical
    BVP solve of the same ODEs and wall conditions."""
    H, B0, nu, eta, U, cw = 1.0, 2.0, 0.3, 0.2, 1.0, 0.3
    ua_fun = lambda y: AN.hartmann(y, H, B0, nu, eta, accel=0.5, U_hi=U,
                                   wall_lo=("insulating",), wall_hi=("shercliff", cw))

    def rhs(y, z):      # z = (u, u', b, b')
        return np.vstack([z[1], -(B0 * z[3] + 0.5) / nu, z[3], -B0 * z[1] / eta])

    def bc(za, zb):
        return np.array([za[0], zb[0] - U, za[2], zb[3] + zb[2] / (cw * H)])
    y = np.linspace(-H, H, 201)
    sol = solve_bvp(rhs, bc, y, np.zeros((4, y.size)), tol=1e-10, max_nodes=100000)
    assert sol.status == 0
    ua, ba = ua_fun(y)
    assert np.abs(sol.sol(y)[0] - ua).max() < 1e-7
    assert np.abs(sol.sol(y)[2] - ba).max() < 1e-7


@pytest.mark.parametrize("d,ny", [(0.5, 22), (1.0, 21)])
@pytest.mark.parametrize("cw", [0.0, 0.1, 1.0, 1e4, math.inf])
def test_hartmann_couette_vs_closed_form(d, ny, cw):
    """Sec. 5.4 (Fig. 8 and 9): Ha = 5, tau_nu = 0.8, tau_eta = 0.9, insulating
    bottom, moving top wall with Shercliff c_w; Eq. 31 (d = 0.5) / Eq. 32 (d = 1)
    for B1, Eq. 34/35 for B2 and the insulating B1.  At 2H = 20 the error is a
    few per cent (second order, see the refinement test); B2 stays B_ext,2."""
    eu, eb, B2, B0 = _hartmann_couette(ny, d, cw)
    tol = 0.03 if d == 0.5 else 0.08
    assert eu < tol and eb < tol
    assert np.abs(B2 - B0).max() < 1e-15


def test_hartmann_couette_second_order():
    """Halving dx divides the error by about four (both layouts, c_w = 0.1)."""
    for d, ny in ((0.5, 22), (1.0, 21)):
        e1 = _hartmann_couette(ny, d, 0.1, steps=12000)
        e2 = _hartmann_couette(2 * ny - 2 + (0 if d == 0.5 else 1), d, 0.1, steps=40000)
        assert e1[0] / e2[0] > 2.8 and e1[1] / e2[1] > 2.8


def test_hartmann_force_balance_sign():
    """Sec. 5.4: with c_w > 0 on the top wall the net Lorentz force
    (B_ext,2/mu)[B1] from -H to H is positive; with c_w = 0 on both walls B1 is
    symmetric and the net force vanishes.  Checked on the oracle's profiles."""
    for cw, positive in ((0.5, True), (0.0, False)):
        tau, taue, ny, U = 0.8, 0.9, 22, 1e-3
        walls = LK.channel_y(2, 1, ny, 1, 0.5, 0.5)
        H = (walls[1][1] - walls[1][0]) / 2
        B0 = 5 * math.sqrt(0.1 * 0.1) / H
        b1_top = dict(kind=O.GIVEN, phi_wall=0.0, u_wall=(U, 0, 0)) if cw == 0 else \
            dict(kind=O.FLUX, u_wall=(U, 0, 0), kappa1=-0.1 / (cw * H))
        p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0)),
             (1, 0, O.G0): dict(kind=O.GIVEN, phi_wall=0.0), (1, 1, O.G0): b1_top,
             (1, 0, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0),
             (1, 1, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0, u_wall=(U, 0, 0))}
        s = O.OracleSim(2, (1, ny, 1), LK.box_solid((1, ny, 1), walls), tau, tau_eta=taue, has_g=True)
        s.set_links(LK.box_links(2, (1, ny, 1), walls, p, has_g=True))
        s.init(B0=(0, B0, 0))
        s.step(15000)
        b = s.moments()["B"][:, 0]
        jump = B0 * ((1.5 * b[ny - 2] - 0.5 * b[ny - 3]) - (1.5 * b[1] - 0.5 * b[2]))   # B1 at X by Eq. 13
        scale = B0 * U
        if positive:
            assert jump > 0.1 * scale
        else:
            assert abs(jump) < 1e-6 * scale


# ------------------------------------------------------------ convection-diffusion
def _cd_box(shape, walls, params, threads):
    solid = LK.box_solid(shape, walls)
    s = O.OracleSim(2, shape, solid, 0.8, tau_D=0.9, has_h=True, threads=threads)
    s.set_links(LK.box_links(2, shape, walls, params, has_h=True))
    return s, solid


def _steady_C(s, shape):
    def step(h):
        s.set_populations(1, h)
        s.step(1)
        return s.populations(1)
    s.set_populations(1, affine_fixed_point(step, 5, shape))
    return s.moments()["C"]


@pytest.mark.parametrize("d", [0.5, 0.25, 1.0])
def test_reactive_channel_linear_profile(d, ncpu):
    """Steady diffusion between a Robin wall (M scheme, Eq. 25-27) at the bottom
    and a given-C wall (Eq. 19/20) at the top: C(y) is linear and its wall
    value follows from the flux balance -D dC/dn = k (C_eq - C)."""
    ny, k, Ceq, Ctop = 14, 0.02, 1.0, 3.0
    D = 0.25 * (0.9 - 0.5)
    walls = {1: (1 - d, ny - 2 + d)}
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY),
         (1, 0, O.H): dict(kind=O.FLUX, kappa0=k * Ceq, kappa1=-k),
         (1, 1, O.H): dict(kind=O.GIVEN, phi_wall=Ctop)}
    s, solid = _cd_box((1, ny, 1), walls, p, ncpu)
    s.init(C0=1.0)
    C = _steady_C(s, (1, ny, 1))[1:-1]
    Ca = AN.reactive_channel(np.arange(ny)[1:-1], walls[1][0], walls[1][1], D, k * Ceq, -k, Ctop)
    tol = 1e-12 if d == 0.5 else 5e-3
    assert np.abs(C - Ca).max() / Ctop < tol


def _x3(d, Da, scale, ncpu):
    nfx, nfy = 100 // scale, 80 // scale
    D = 0.1
    k = Da * D / nfy
    nx, ny = (nfx + 2, nfy + 2) if d == 0.5 else (nfx + 1, nfy + 1)
    walls = {0: (1 - d, nx - 2 + d), 1: (1 - d, ny - 2 + d)}
    p = {(ax, side, O.F): dict(kind=O.VELOCITY) for ax in (0, 1) for side in (0, 1)}
    p[(0, 0, O.H)] = dict(kind=O.GIVEN, phi_wall=10.0)
    p[(0, 1, O.H)] = dict(kind=O.NEUMANN_BFL)
    p[(1, 0, O.H)] = dict(kind=O.NEUMANN_BFL)
    p[(1, 1, O.H)] = dict(kind=O.FLUX, kappa0=k * 1.0, kappa1=-k)
    s, solid = _cd_box((nx, ny, 1), walls, p, ncpu)
    s.init(C0=1.0)
    C = _steady_C(s, (nx, ny, 1)).reshape(ny, nx)
    X, Y = np.meshgrid(np.arange(nx) - walls[0][0], np.arange(ny) - walls[1][0])
    Ca = AN.reaction_diffusion_series(X, Y, nfx, nfy, D, k, 10.0, 1.0)
    return C, Ca


@pytest.mark.parametrize("Da", [4.8, 48.0])
def test_reaction_diffusion_paper_values(Da, ncpu):
    """Sec. 5.3 at the paper's resolution (D = 1e-6, W = 0.01, L = 0.0125,
    dx = 1.25e-4, c = 0.08, tau_D = 0.9 -> 80 x 100 fluid cells, D = 0.1 in
    lattice units).  The paper prints, for the full-grid layout, an error of
    about 0.02 near the bottom wall (4.5 analytic vs 4.48 LBM); the half-grid
    layout agrees much better.  The analytic side is the separation-of-variables
    series of the Laplace problem."""
    C, Ca = _x3(1.0, Da, 1, ncpu)
    bottom = np.abs(C[1] - Ca[1])[1:-1]
    assert 0.01 < bottom.max() < 0.03
    j = np.argmax(bottom) + 1
    assert C[1, j] < Ca[1, j]                        # LBM below the analytic value, as printed
    C5, Ca5 = _x3(0.5, Da, 1, ncpu)
    assert np.abs(C5[1] - Ca5[1])[1:-1].max() < 0.1 * bottom.max()
    # away from the singular corner where the given-C and Robin walls meet
    assert np.abs(C5 - Ca5)[1:-1, 8:-1].max() < 0.03


def test_reaction_diffusion_refinement(ncpu):
    """The full-grid bottom-wall error of Sec. 5.3 halves with dx (it is the
    first-order error of Eq. 22 at d = 1 that the paper points out)."""
    e = []
    for scale in (4, 2):
        C, Ca = _x3(1.0, 48.0, scale, ncpu)
        e.append(np.abs(C[1] - Ca[1])[1:-1].max())
    assert 1.7 < e[0] / e[1] < 2.3


def test_flux_wall_adds_exactly_the_flux(ncpu):
    """Eq. 23: at d = 0.5 and a static wall each flux link adds exactly
    k0 + k1 C_X of solute per step, so sum C changes by the sum of increments."""
    nx, ny = 4, 8
    walls = {1: (0.5, ny - 1.5)}
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY),
         (1, 0, O.H): dict(kind=O.FLUX, kappa0=0.003, kappa1=-0.01),
         (1, 1, O.H): dict(kind=O.NEUMANN_BFL)}
    s, solid = _cd_box((nx, ny, 1), walls, p, ncpu)
    s.init(C0=2.0)
    for _ in range(5):
        m = s.moments()
        C = m["C"].reshape(ny, nx)
        CX = 1.5 * C[1] - 0.5 * C[2]
        expect = s.sums()[1] + np.sum(0.003 - 0.01 * CX)
        s.step(1)
        assert abs(s.sums()[1] - expect) < 1e-13
