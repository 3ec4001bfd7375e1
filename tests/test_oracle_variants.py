"""Oracle pins of the two comparison schemes the paper evaluates beside its
proposed ones (no GPU):

* Eq. 15 with Eq. 16 applied for every d (velocity walls), which Sec. 5.1
  replaces by Eq. 43 for d >= 1/2 because the extrapolation to Y is unstable;
* the simplified flux wall of Eq. 33 (flux and move increments added to the
  population bounced at X), which Sec. 5.4 (Fig. 12) shows to be inaccurate at
  small c_w on the full-grid layout, where the M scheme (Eq. 25-27) is not.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import analytic as AN
from oracle import links as LK


def _hartmann_couette_top(ny, d, cw, top_kind, steps, Ha=5.0, U=1e-3):
    """Hartmann-Couette channel of Sec. 5.4 (insulating bottom, moving top wall
    with Shercliff c_w imposed by ``top_kind``); returns the errors of u1 and B1
    against the closed form, normalised as in Eq. 46, and the final moments."""
    tau, taue = 0.8, 0.9
    nu, eta = (tau - 0.5) / 3, (taue - 0.5) / 4
    walls = LK.channel_y(2, 1, ny, 1, d, d)
    y0, y1 = walls[1]
    H, yc = (y1 - y0) / 2, (y1 + y0) / 2
    B0 = Ha * math.sqrt(nu * eta) / H
    top = dict(kind=top_kind, u_wall=(U, 0, 0))
    if cw != math.inf:
        top["kappa1"] = -eta / (cw * H)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0)),
         (1, 0, O.G0): dict(kind=O.GIVEN, phi_wall=0.0), (1, 1, O.G0): top,
         (1, 0, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0),
         (1, 1, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0, u_wall=(U, 0, 0))}
    s = O.OracleSim(2, (1, ny, 1), LK.box_solid((1, ny, 1), walls), tau, tau_eta=taue, has_g=True)
    s.set_links(LK.box_links(2, (1, ny, 1), walls, p, has_g=True))
    s.init(B0=(0, B0, 0))
    s.step(steps)
    m = s.moments()
    y = np.arange(ny)[1:-1] - yc
    wall_hi = ("conducting",) if cw == math.inf else ("shercliff", cw)
    ua, ba = AN.hartmann(y, H, B0, nu, eta, U_hi=U, wall_lo=("insulating",), wall_hi=wall_hi)
    u, b = m["u"][1:-1, 0], m["B"][1:-1, 0]
    return np.abs(u - ua).max() / U, np.abs(b - ba).max() / (U * math.sqrt(nu / eta)), m


def test_simplified_flux_is_the_m_scheme_at_half_grid():
    """At d = 1/2 both Eq. 25-27 and Eq. 33's construction reduce to Eq. 28
    (bounced population plus increments), so the two trajectories agree bit
    for bit."""
    _, _, m1 = _hartmann_couette_top(22, 0.5, 0.1, O.FLUX, 400)
    _, _, m2 = _hartmann_couette_top(22, 0.5, 0.1, O.FLUX_SIMPLIFIED, 400)
    for k in ("rho", "u", "B"):
        assert np.array_equal(m1[k], m2[k])


def test_simplified_flux_fails_at_small_cw_on_full_grid():
    """Sec. 5.4, Fig. 12: full-grid layout (d = 1, 2H = 100 with 101 nodes as in
    the paper, Ha = 5).  The M scheme stays within a few tenths of a per cent of
    the closed form for every c_w; the simplified scheme of Eq. 33 is an order
    of magnitude worse at c_w = 0.1 and 1, and the difference disappears for a
    perfectly conducting wall, where the flux term is zero."""
    for cw in (0.1, 1.0):
        eu_m, eb_m, _ = _hartmann_couette_top(101, 1.0, cw, O.FLUX, 40000)
        eu_s, eb_s, _ = _hartmann_couette_top(101, 1.0, cw, O.FLUX_SIMPLIFIED, 40000)
        assert eu_m < 0.006 and eb_m < 0.006
        assert eu_s > 10 * eu_m and eb_s > 10 * eb_m
    eu_m, eb_m, _ = _hartmann_couette_top(101, 1.0, math.inf, O.FLUX, 40000)
    eu_s, eb_s, _ = _hartmann_couette_top(101, 1.0, math.inf, O.FLUX_SIMPLIFIED, 40000)
    assert eu_m < 0.006 and abs(eu_s - eu_m) < 1e-5 and abs(eb_s - eb_m) < 1e-5


def _couette(d, kind, steps, ny=12, U=0.05, tau=0.8):
    walls = LK.channel_y(2, 1, ny, 1, d, d)
    p = {(1, 0, O.F): dict(kind=kind), (1, 1, O.F): dict(kind=kind, u_wall=(U, 0, 0))}
    s = O.OracleSim(2, (1, ny, 1), LK.box_solid((1, ny, 1), walls), tau)
    s.set_links(LK.box_links(2, (1, ny, 1), walls, p))
    s.init()
    s.step(steps)
    m = s.moments()
    ua = AN.couette(np.arange(ny)[1:-1], walls[1][0], walls[1][1], 0.0, U)
    return m, ua


@pytest.mark.parametrize("d", [0.2, 0.5])
def test_eq15_for_every_d_is_the_default_up_to_half(d):
    """For d < 1/2 the default velocity wall is Eq. 15/16 itself, and at d = 1/2
    Eq. 43 and Eq. 15/16 both give the halfway bounce-back plus the increment:
    the trajectories agree bit for bit, and Couette flow is exact."""
    m1, ua = _couette(d, O.VELOCITY, 3000)
    m2, _ = _couette(d, O.VELOCITY_EQ15, 3000)
    for k in ("rho", "u"):
        assert np.array_equal(m1[k], m2[k])
    m, ua = _couette(d, O.VELOCITY_EQ15, 8000)
    assert np.abs(m["u"][1:-1, 0] - ua).max() / 0.05 < 1e-10


@pytest.mark.parametrize("d", [0.6, 0.8, 1.0])
def test_eq15_extrapolated_beyond_half_diverges(d):
    """Sec. 5.1 finds Eq. 15/16 unstable on the full-grid layout because Y is
    extrapolated for d > 1/2, and replaces it by Eq. 43.  On a moving wall
    (tau = 0.8) the oracle's Eq. 15/16 diverges within 3000 steps for every d
    above 1/2 tried, while Eq. 43 gives the exact Couette line at the same d."""
    m, _ = _couette(d, O.VELOCITY_EQ15, 3000)
    u = m["u"][1:-1, 0]
    assert not np.all(np.isfinite(u)) or np.abs(u).max() > 1.0
    m, ua = _couette(d, O.VELOCITY, 8000)
    assert np.abs(m["u"][1:-1, 0] - ua).max() / 0.05 < 1e-10
