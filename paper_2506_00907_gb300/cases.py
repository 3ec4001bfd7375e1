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

# The explicit Shercliff flux of the M scheme diverges once the per-link
# coefficient eta/(c_w H) exceeds about 1.2 (measured); cases keep it below:
SHERCLIFF_KAPPA_MAX = 0.8
ETA_MIN, ETA_MAX = 0.0125, 0.1          # tau_eta in [0.55, 0.9]


def hartmann_channel(W, Ha, q, cw, tau_nu=0.8, u_target=0.02):
    """2D Hartmann channel, W fluid rows across and W nodes along x (periodic),
    walls at wall-to-node fraction q on both sides (d = 1 - q), Shercliff c_w
    on both walls for B1, given B2 = B_ext,2, static no-slip walls, body
    force along x.  eta is chosen per case so that eta/(c_w H) stays below
    SHERCLIFF_KAPPA_MAX (the steady solution depends only on Ha and c_w).

    Returns (lbm_case, solid, links, info)."""
    d = 1.0 - q
    nx, ny = W, W + 2
    H = (W - 1 + 2 * d) / 2.0
    nu = (tau_nu - 0.5) / 3.0
    eta = min(ETA_MAX, max(ETA_MIN, SHERCLIFF_KAPPA_MAX * cw * H))
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
    info = dict(W=W, Ha=Ha, q=q, cw=cw, H=H, nu=nu, eta=eta, B0=B0, accel=accel, kappa1=kappa1,
                fluid=int(np.sum(solid == 0)))
    return case, solid, links, info


def pipe(shape, R, Ha, wall, tau_nu=0.8, tau_eta=None, u_target=0.02):
    """MHD pipe along x (Sec. 6): D3Q19 flow + D3Q7 vector B; static no-slip
    curved wall; B1 insulating ('insulating'), perfectly conducting
    ('conducting') or Shercliff (('shercliff', c_w)); B2 = B_ext,2 and B3 = 0
    given.  tau_eta defaults to 0.9 (the paper's value), lowered for small
    Shercliff c_w so that eta/(c_w R) stays below SHERCLIFF_KAPPA_MAX.
    Returns (lbm_case, solid, links, info)."""
    nu = (tau_nu - 0.5) / 3.0
    if tau_eta is None:
        eta = ETA_MAX
        if wall not in ("insulating", "conducting"):
            eta = min(ETA_MAX, max(ETA_MIN, SHERCLIFF_KAPPA_MAX * wall[1] * R))
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
