"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
side (parameter draws, random geometries, random initial fields, and the
recipe that turns a drawn case into lattice parameters).

This module holds no lattice-Boltzmann arithmetic: it draws numbers and
converts physical case parameters to lattice units.  Physical parameter sets
follow the paper's cases in lattice units (tau_nu = 0.8, tau_eta = 0.9,
tau_D = 0.9, rho0 = 1, B_ext along x2).  Conversions: nu = (tau_nu - 1/2)/3,
eta = (tau_eta - 1/2)/4, D = (tau_D - 1/2)/4, Ha = B0 H / sqrt(rho nu eta)
(Sec. 5.4 with sigma = 1/(mu eta)), Shercliff flux F(B1) = -eta B1 / (c_w H)
(Eq. 30).  Both the product's case set-up and the oracle's build their cases
from these parameters, each with its own wall-link builder.
"""
import math

import numpy as np

SEED = 2506


def rng(seed=SEED):
    return np.random.default_rng(seed)


def random_solid(r, shape, fill=0.15, blob=2):
    """uint8 solid mask (nz, ny, nx): random blobs of solid, at least half fluid."""
    nx, ny, nz = shape
    m = r.random((nz, ny, nx)) < fill / max(1, blob)
    out = m.copy()
    for _ in range(blob - 1):
        for ax in range(3 if nz > 1 else 2):
            out |= np.roll(m, 1, axis=2 - ax)
    if out.mean() > 0.5:
        out[:] = False
    return out.astype(np.uint8)


def random_fields(r, N, dim, du=0.02, dB=0.1, C=(0.5, 1.5), B0=(0.0, 0.0, 0.0)):
    """Initial fields near rest: rho ~ 1 +- 1 %, |u| <~ du, C in C, B ~ B0 +- dB."""
    rho = 1.0 + r.uniform(-0.01, 0.01, N)
    u = r.uniform(-du, du, (N, 3))
    Bf = np.asarray(B0, dtype=np.float64)[None, :] + r.uniform(-dB, dB, (N, 3))
    if dim == 2:
        u[:, 2] = 0.0
        Bf[:, 2] = 0.0
    Cf = r.uniform(C[0], C[1], N)
    return {"rho": rho, "u": u, "C": Cf, "B": Bf}


def hartmann_batch(n=64, seed=SEED, wmin=64, wmax=512):
    """Parameter draws of the batched 2D Hartmann channels: width W ~ U{wmin..wmax}
    nodes across the channel (also the periodic length), Ha ~ U[1, 30],
    wall-to-node fraction q ~ U[0, 1), wall conductance ratio c_w ~ log-U[1e-3, 1]."""
    r = rng(seed)
    W = r.integers(wmin, wmax + 1, n)
    Ha = r.uniform(1.0, 30.0, n)
    q = r.random(n)
    cw = 10.0 ** r.uniform(-3.0, 0.0, n)
    return [dict(W=int(W[i]), Ha=float(Ha[i]), q=float(q[i]), cw=float(cw[i])) for i in range(n)]


def pipe_draws(n, seed=SEED, Ha=(10.0, 50.0), cw=(1e-3, 1.0)):
    """Ha ~ U[Ha], c_w ~ log-U[cw] for MHD pipe cases."""
    r = rng(seed)
    h = r.uniform(Ha[0], Ha[1], n)
    c = 10.0 ** r.uniform(np.log10(cw[0]), np.log10(cw[1]), n)
    return [dict(Ha=float(h[i]), cw=float(c[i])) for i in range(n)]


def net_init(seed=SEED, dims=(4, 64, 64, 64, 2)):
    """Initial parameters of the warm-start network: Glorot-uniform weights,
    zero biases, in the flat layout W_1, b_1, W_2, b_2, ... (rows = outputs)."""
    r = rng(seed)
    out = []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        out.append(r.uniform(-lim, lim, fan_out * fan_in))
        out.append(np.zeros(fan_out))
    return np.concatenate(out).astype(np.float32)


# ----------------------------------------------------------------------------- case parameters
# The explicit Shercliff flux of the M scheme (Eq. 25-27, 30) diverges once
# kappa = eta / (c_w H) passes a limit that falls with tau_eta = 1/2 + 4 eta and
# with the wall-to-node fraction q.  Limits measured on the FP64 reference step
# by bisection (10 000 steps, Ha = 15, from rest plus a seeded perturbation of
# relative size 1e-3 on a domain several nodes long along the wall: fields
# uniform along the wall never excite the modes that grow first, and
# stochastically rounded storage does).  Channel rows are q = 0, .25, .5, .7,
# .9, .97; the pipe (R = 16, every q on the curved wall) has one value per
# eta.  A limit of 0 means that even the zero-flux wall diverges there.  The
# steady solution depends only on (Ha, c_w), so each case takes the largest
# tabulated eta whose kappa stays within KAPPA_MARGIN of its limit.
CHANNEL_Q = (0.0, 0.25, 0.5, 0.7, 0.9, 0.97)
CHANNEL_KAPPA_LIMIT = {
    0.0125: (0.0, 0.43, 0.383, 0.297, 0.195, 0.141),
    0.025: (0.789, 0.75, 0.633, 0.594, 0.398, 0.297),
    0.0375: (1.031, 0.961, 0.867, 0.758, 0.227, 0.0),
    0.05: (1.305, 1.219, 1.117, 0.523, 0.0, 0.0),
    0.075: (1.305, 1.125, 1.18, 0.336, 0.0, 0.0),
    0.1: (1.109, 1.016, 0.992, 0.0, 0.0, 0.0),
}
PIPE_KAPPA_LIMIT = {0.0125: 0.266, 0.025: 0.344, 0.0375: 0.453, 0.05: 0.602, 0.075: 0.477, 0.1: 0.383}
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


def hartmann_params(W, Ha, q, cw, tau_nu=0.8, u_target=0.02, clamp_cw=False):
    """Lattice parameters of a 2D Hartmann channel (Sec. 5.4): W fluid rows
    across and W nodes along x (periodic), solid rows y = 0 and y = W + 1,
    walls at wall-to-node fraction q on both sides (d = 1 - q, so the walls
    sit at y = 1 - d and y = W + d and 2H = W - 1 + 2d), body force along x
    with u_max ~ u_target, B_ext = (0, B0).  eta is chosen by shercliff_eta; a
    c_w too small for any tabulated eta raises ValueError, or with clamp_cw
    is raised to the smallest stable value ("cw_clamped")."""
    d = 1.0 - q
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
    B0 = Ha * math.sqrt(nu * eta) / H
    return dict(W=W, Ha=Ha, q=q, d=d, cw=cw, cw_drawn=cw_in, cw_clamped=clamped, shape=(W, W + 2, 1), H=H,
                tau_nu=tau_nu, tau_eta=0.5 + 4.0 * eta, nu=nu, eta=eta, B0=B0,
                accel=u_target * nu * (2.0 + Ha) / (H * H), kappa1=-eta / (cw * H))


def pipe_params(R, Ha, wall, tau_nu=0.8, tau_eta=None, u_target=0.02):
    """Lattice parameters of the MHD pipe along x (Sec. 6): radius R, wall
    'insulating', 'conducting' or ('shercliff', c_w); tau_eta defaults to the
    paper's 0.9, Shercliff walls take shercliff_eta with the pipe limits
    (ValueError when c_w R is too small).  B_ext = (0, B0), body force along x."""
    nu = (tau_nu - 0.5) / 3.0
    if tau_eta is None:
        eta = ETA_DEFAULT
        if wall not in ("insulating", "conducting"):
            eta = shercliff_eta(wall[1], R, PIPE_KAPPA_LIMIT.get)
            if eta is None:
                raise ValueError("c_w = %g is below the explicit Shercliff flux limit at R = %g" % (wall[1], R))
        tau_eta = 0.5 + 4.0 * eta
    eta = (tau_eta - 0.5) / 4.0
    kappa1 = None if wall in ("insulating", "conducting") else -eta / (wall[1] * R)
    return dict(R=R, Ha=Ha, wall=wall, tau_nu=tau_nu, tau_eta=tau_eta, nu=nu, eta=eta,
                B0=Ha * math.sqrt(nu * eta) / R, accel=u_target * nu * (2.0 + Ha) / (R * R), kappa1=kappa1)


def reactive_params(nx, ny, q, U, k, C_eq=1.0, C_top=2.0, tau_nu=0.8, tau_D=0.9):
    """Flow + concentration channel: periodic x, solid rows y = 0 and ny - 1,
    both walls at wall-to-node fraction q (d = 1 - q); the top wall moves at U
    with given C = C_top, the bottom wall is static and reacts with the Robin
    flux F(C) = k (C_eq - C) = kappa0 + kappa1 C."""
    return dict(shape=(nx, ny, 1), q=q, d=1.0 - q, U=U, k=k, C_eq=C_eq, C_top=C_top, tau_nu=tau_nu, tau_D=tau_D,
                kappa0=k * C_eq, kappa1=-k)


def reactive_grid(nx=512, ny=256):
    """The flow + concentration configuration set: q in {0, 1/4, 1/2, 3/4},
    k in {1e-3, 1e-2, 1e-1}, top wall U = 0.05."""
    return [reactive_params(nx, ny, q, 0.05, k) for q in (0.0, 0.25, 0.5, 0.75) for k in (1e-3, 1e-2, 1e-1)]
