"""Case set-ups in lattice units (dx = dt = 1, rho0 = 1, mu = 1) built with the
product's wall-link builders.

Hartmann channels (Sec. 5.4), the MHD pipe (Sec. 6) and the convection-
diffusion channel with a moving wall and a reactive wall.  Conversions:
nu = (tau_nu - 1/2)/3, eta = (tau_eta - 1/2)/4, D = (tau_D - 1/2)/4,
Ha = B0 H / sqrt(rho nu eta) (Sec. 5.4 with sigma = 1/(mu eta)), Shercliff
flux F(B1) = -eta B1 / (c_w H) (Eq. 30).
"""
import math

import numpy as np

from . import lbm

# The explicit Shercliff flux of the M scheme (Eq. 25-27, 30) diverges once
# kappa = eta / (c_w H) passes a limit that falls with tau_eta = 1/2 + 4 eta and
# with the wall-to-node fraction q.  Limits measured on the FP64 reference step
# by bisection (6000 steps, Ha = 15): channel rows are q = 0, .25, .5, .7, .9,
# .97; the pipe (R = 16, every q on the curved wall) has one value per eta.
# The steady solution depends only on (Ha, c_w), so each case takes the
# largest tabulated eta whose kappa stays within KAPPA_MARGIN of its limit.
CHANNEL_Q = (0.0, 0.25, 0.5, 0.7, 0.9, 0.97)
CHANNEL_KAPPA_LIMIT = {
    0.0125: (0.0, 0.486, 0.424, 0.331, 0.207, 0.144),
    0.025: (1.046, 0.984, 0.797, 0.580, 0.393, 0.331),
    0.0375: (1.357, 1.295, 1.108, 1.046, 0.642, 0.517),
    0.05: (1.792, 1.668, 1.450, 1.264, 0.953, 0.735),
    0.075: (1.917, 1.855, 1.761, 1.668, 1.544, 1.481),
    0.1: (1.575, 1.512, 1.450, 1.326, 1.202, 1.139),
}
PIPE_KAPPA_LIMIT = {0.0125: 0.269, 0.025: 0.331, 0.0375: 0.455, 0.05: 0.611, 0.075: 0.735, 0.1: 0.580}
KAPPA_MARGIN = 0.8
ETA_DEFAULT = 0.1                       # tau_eta = 0.9, the paper's value


def channel_kappa_limit(eta, q):
    """Tabulated limit at eta for wall-to-node fraction q: the smaller of the
    two bracketing q rows (q beyond the last row takes the last row)."""
    row = CHANNEL_KAPPA_LIMIT[eta]
    for i in range(len(CHANNEL_Q) - 1):
        if q <= CHANNEL_Q[i + 1]:
            return min(row[i], row[i + 1])
    return row[-1]


def shercliff_eta(cw, H, limit):
    """Largest tabulated eta with eta / (c_w H) <= KAPPA_MARGIN * limit(eta),
    or None when no tabulated eta is stable for this c_w H."""
    best = None
    for eta in sorted(PIPE_KAPPA_LIMIT):
        if eta / (cw * H) <= KAPPA_MARGIN * limit(eta):
            best = eta
    return best


def hartmann_channel(W, Ha, q, cw, tau_nu=0.8, u_target=0.02, clamp_cw=False):
    """2D Hartmann channel, W fluid rows across and W nodes along x (periodic),
    walls at wall-to-node fraction q on both sides (d = 1 - q), Shercliff c_w
    on both walls for B1, given B2 = B_ext,2, static no-slip walls, body
    force along x.  eta is chosen per case by shercliff_eta (the steady
    solution depends only on Ha and c_w).  A c_w too small for any tabulated
    eta raises ValueError, or with clamp_cw is raised to the smallest stable
    value (info["cw_clamped"] is then True).

    Returns (lbm_case, solid, links, info)."""
    d = 1.0 - q
    nx, ny = W, W + 2
    H = (W - 1 + 2 * d) / 2.0
    nu = (tau_nu - 0.5) / 3.0
    limit = lambda e: channel_kappa_limit(e, q)
    eta = shercliff_eta(cw, H, limit)
    cw_in, clamped = cw, False
    if eta is None:
        if not clamp_cw:
            raise ValueError("c_w = %g is below the explicit Shercliff flux limit at H = %g, q = %g" % (cw, H, q))
        cw = min(e / (KAPPA_MARGIN * limit(e) * H) for e in PIPE_KAPPA_LIMIT if limit(e) > 0) * (1 + 1e-9)
        eta, clamped = shercliff_eta(cw, H, limit), True
    tau_eta = 0.5 + 4.0 * eta
    B0 = Ha * math.sqrt(nu * eta) / H
    accel = u_target * nu * (2.0 + Ha) / (H * H)
    kappa1 = -eta / (cw * H)
    f = lbm.wall_bc(lbm.LBM_W_VELOCITY)
    g0 = lbm.wall_bc(lbm.LBM_W_FLUX, kappa1=kappa1)
    g1 = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=B0)
    bc = [f, None, g0, g1, None]
    solid, links = lbm.lbm_build_channel(2, (nx, ny, 1), 1, d, d, lbm.LBM_FLOW | lbm.LBM_MHD, bc, bc)
    case = lbm.make_case((nx, ny, 1), tau_nu, 1.0, tau_eta, (accel, 0.0, 0.0), 1.0, 0.0, (0.0, B0, 0.0))
    info = dict(W=W, Ha=Ha, q=q, cw=cw, cw_drawn=cw_in, cw_clamped=clamped, H=H, nu=nu, eta=eta, B0=B0,
                accel=accel, kappa1=kappa1, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info


def pipe(shape, R, Ha, wall, tau_nu=0.8, tau_eta=None, u_target=0.02):
    """MHD pipe along x (Sec. 6): D3Q19 flow + D3Q7 vector B; static no-slip
    curved wall; B1 insulating ('insulating'), perfectly conducting
    ('conducting') or Shercliff (('shercliff', c_w)); B2 = B_ext,2 and B3 = 0
    given.  tau_eta defaults to 0.9 (the paper's value); Shercliff walls take
    shercliff_eta with the pipe limits (ValueError when c_w R is too small).
    Returns (lbm_case, solid, links, info)."""
    nu = (tau_nu - 0.5) / 3.0
    if tau_eta is None:
        eta = ETA_DEFAULT
        if wall not in ("insulating", "conducting"):
            eta = shercliff_eta(wall[1], R, PIPE_KAPPA_LIMIT.get)
            if eta is None:
                raise ValueError("c_w = %g is below the explicit Shercliff flux limit at R = %g" % (wall[1], R))
        tau_eta = 0.5 + 4.0 * eta
    eta = (tau_eta - 0.5) / 4.0
    B0 = Ha * math.sqrt(nu * eta) / R
    accel = u_target * nu * (2.0 + Ha) / (R * R)
    if wall == "insulating":
        g0 = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=0.0)
    elif wall == "conducting":
        g0 = lbm.wall_bc(lbm.LBM_W_FLUX)
    else:
        g0 = lbm.wall_bc(lbm.LBM_W_FLUX, kappa1=-eta / (wall[1] * R))
    bcs = [lbm.wall_bc(lbm.LBM_W_VELOCITY), None, g0, lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=B0),
           lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=0.0)]
    solid, links = lbm.lbm_build_pipe(shape, R, lbm.LBM_FLOW | lbm.LBM_MHD, bcs)
    case = lbm.make_case(shape, tau_nu, 1.0, tau_eta, (accel, 0.0, 0.0), 1.0, 0.0, (0.0, B0, 0.0))
    info = dict(R=R, Ha=Ha, wall=wall, nu=nu, eta=eta, B0=B0, accel=accel, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info


def reactive_channel(nx, ny, q, U, k, C_eq=1.0, C_top=2.0, tau_nu=0.8, tau_D=0.9):
    """2D flow + concentration: top wall moving at U (Couette) with given
    C = C_top, bottom static wall with the Robin reaction F(C) = k (C_eq - C)
    (M scheme), both at wall-to-node fraction q; periodic x."""
    d = 1.0 - q
    f_lo = lbm.wall_bc(lbm.LBM_W_VELOCITY)
    f_hi = lbm.wall_bc(lbm.LBM_W_VELOCITY, u_wall=(U, 0.0, 0.0))
    h_lo = lbm.wall_bc(lbm.LBM_W_FLUX, kappa0=k * C_eq, kappa1=-k)
    h_hi = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=C_top, u_wall=(U, 0.0, 0.0))
    solid, links = lbm.lbm_build_channel(2, (nx, ny, 1), 1, d, d, lbm.LBM_FLOW | lbm.LBM_CD,
                                         [f_lo, h_lo, None, None, None], [f_hi, h_hi, None, None, None])
    case = lbm.make_case((nx, ny, 1), tau_nu, tau_D, 1.0, (0.0, 0.0, 0.0), 1.0, C_eq, (0.0, 0.0, 0.0))
    info = dict(q=q, U=U, k=k, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info
