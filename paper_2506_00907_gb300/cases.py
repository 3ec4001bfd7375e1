"""Case set-ups in lattice units (dx = dt = 1, rho0 = 1, mu = 1) built with the
product's wall-link builders.

Hartmann channels (Sec. 5.4), the MHD pipe (Sec. 6) and the convection-
diffusion channel with a moving wall and a reactive wall.  The lattice
parameters of each case (eta per case from the explicit-flux stability table,
B0 from Ha, the body force) come from the shared input recipe in
``inputs``; this module turns them into C-ABI case records and wall links.
"""
import numpy as np

from . import inputs as IN
from . import lbm

# re-exported for callers that read the stability table through this module
CHANNEL_Q = IN.CHANNEL_Q
CHANNEL_KAPPA_LIMIT = IN.CHANNEL_KAPPA_LIMIT
PIPE_KAPPA_LIMIT = IN.PIPE_KAPPA_LIMIT
KAPPA_MARGIN = IN.KAPPA_MARGIN
ETA_DEFAULT = IN.ETA_DEFAULT
channel_kappa_limit = IN.channel_kappa_limit
shercliff_eta = IN.shercliff_eta


def hartmann_channel(W, Ha, q, cw, tau_nu=0.8, u_target=0.02, clamp_cw=False):
    """2D Hartmann channel, W fluid rows across and W nodes along x (periodic),
    walls at wall-to-node fraction q on both sides (d = 1 - q), Shercliff c_w
    on both walls for B1, given B2 = B_ext,2, static no-slip walls, body
    force along x (parameters from ``inputs.hartmann_params``).

    Returns (lbm_case, solid, links, info)."""
    P = IN.hartmann_params(W, Ha, q, cw, tau_nu, u_target, clamp_cw)
    nx, ny, _ = P["shape"]
    f = lbm.wall_bc(lbm.LBM_W_VELOCITY)
    g0 = lbm.wall_bc(lbm.LBM_W_FLUX, kappa1=P["kappa1"])
    g1 = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=P["B0"])
    bc = [f, None, g0, g1, None]
    solid, links = lbm.lbm_build_channel(2, (nx, ny, 1), 1, P["d"], P["d"], lbm.LBM_FLOW | lbm.LBM_MHD, bc, bc)
    case = lbm.make_case((nx, ny, 1), tau_nu, 1.0, P["tau_eta"], (P["accel"], 0.0, 0.0), 1.0, 0.0,
                         (0.0, P["B0"], 0.0))
    info = dict(P, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info


def pipe(shape, R, Ha, wall, tau_nu=0.8, tau_eta=None, u_target=0.02):
    """MHD pipe along x (Sec. 6): D3Q19 flow + D3Q7 vector B; static no-slip
    curved wall; B1 insulating ('insulating'), perfectly conducting
    ('conducting') or Shercliff (('shercliff', c_w)); B2 = B_ext,2 and B3 = 0
    given (parameters from ``inputs.pipe_params``).
    Returns (lbm_case, solid, links, info)."""
    P = IN.pipe_params(R, Ha, wall, tau_nu, tau_eta, u_target)
    if wall == "insulating":
        g0 = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=0.0)
    elif wall == "conducting":
        g0 = lbm.wall_bc(lbm.LBM_W_FLUX)
    else:
        g0 = lbm.wall_bc(lbm.LBM_W_FLUX, kappa1=P["kappa1"])
    bcs = [lbm.wall_bc(lbm.LBM_W_VELOCITY), None, g0, lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=P["B0"]),
           lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=0.0)]
    solid, links = lbm.lbm_build_pipe(shape, R, lbm.LBM_FLOW | lbm.LBM_MHD, bcs)
    case = lbm.make_case(shape, tau_nu, 1.0, P["tau_eta"], (P["accel"], 0.0, 0.0), 1.0, 0.0, (0.0, P["B0"], 0.0))
    info = dict(P, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info


def reactive_channel(nx, ny, q, U, k, C_eq=1.0, C_top=2.0, tau_nu=0.8, tau_D=0.9):
    """2D flow + concentration: top wall moving at U (Couette) with given
    C = C_top, bottom static wall with the Robin reaction F(C) = k (C_eq - C)
    (M scheme), both at wall-to-node fraction q; periodic x (parameters from
    ``inputs.reactive_params``)."""
    P = IN.reactive_params(nx, ny, q, U, k, C_eq, C_top, tau_nu, tau_D)
    f_lo = lbm.wall_bc(lbm.LBM_W_VELOCITY)
    f_hi = lbm.wall_bc(lbm.LBM_W_VELOCITY, u_wall=(U, 0.0, 0.0))
    h_lo = lbm.wall_bc(lbm.LBM_W_FLUX, kappa0=P["kappa0"], kappa1=P["kappa1"])
    h_hi = lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=C_top, u_wall=(U, 0.0, 0.0))
    solid, links = lbm.lbm_build_channel(2, (nx, ny, 1), 1, P["d"], P["d"], lbm.LBM_FLOW | lbm.LBM_CD,
                                         [f_lo, h_lo, None, None, None], [f_hi, h_hi, None, None, None])
    case = lbm.make_case((nx, ny, 1), tau_nu, tau_D, 1.0, (0.0, 0.0, 0.0), 1.0, C_eq, (0.0, 0.0, 0.0))
    info = dict(P, fluid=int(np.sum(solid == 0)))
    return case, solid, links, info
