"""Measures the stability limit of the explicit Shercliff flux wall on the
FP64 oracle and prints the tables the case builders use (test infrastructure:
run by hand, ``python -m oracle.stability_table``).

The M scheme (Eq. 25-27) with the flux F = -eta B1 / (c_w H) of Eq. 30,
evaluated explicitly at each link's own B1(X) (Eq. 13), diverges once
kappa = eta / (c_w H) passes a limit.  The limit depends on tau_eta and on
the wall-to-node fraction q, and it is lower for perturbations that vary
along the wall than for fields uniform along it: a run that starts exactly
uniform along the wall never excites those modes, so each run here starts
from rest plus a seeded perturbation of relative size 1e-3 in u and B, on a
domain of several nodes along the wall.  A run counts as stable when its
fields stay finite and |B1| < 10 for STEPS steps; the limit is found by
bisection on kappa (BISECT halvings of [0, 2 x start]).

Channels: W = 8 fluid rows, 8 nodes along x, Ha = 15, q on CHANNEL_Q.  Pipes:
R = 16 on a 36 x 36 cross-section, 4 nodes along the axis, Ha = 15, every q
of the curved wall at once.
"""
import math
import multiprocessing as mp

import numpy as np

import oracle as O
from oracle import links as LK

ETAS = (0.0125, 0.025, 0.0375, 0.05, 0.075, 0.1)
CHANNEL_Q = (0.0, 0.25, 0.5, 0.7, 0.9, 0.97)
STEPS = 10000
BISECT = 9
NOISE = 1e-3
START = 2.0          # upper end of the bisection interval is 2 x START


def _bounded(sim, fluid, steps):
    for _ in range(steps // 500):
        sim.step(500)
        m = sim.moments()
        if not np.all(np.isfinite(m["u"][fluid])) or np.abs(m["B"][fluid, 0]).max() > 10:
            return False
    return True


def _perturbed(N, B0, seed, dim):
    r = np.random.default_rng(seed)
    u = NOISE * 0.02 * r.standard_normal((N, 3))
    B = np.tile([0.0, B0, 0.0], (N, 1)) + NOISE * B0 * r.standard_normal((N, 3))
    if dim == 2:
        u[:, 2] = 0.0
        B[:, 2] = 0.0
    return u, B


def channel_stable(q, kappa, eta, steps=STEPS, W=8, nx=8, Ha=15.0, seed=1, threads=1):
    """One channel run (Sec. 5.4 layout: solid rows 0 and W + 1, walls at
    d = 1 - q): True when it stays bounded."""
    nu, d = 0.1, 1.0 - q
    ny = W + 2
    walls = LK.channel_y(2, nx, ny, 1, d, d)
    H = (walls[1][1] - walls[1][0]) / 2
    B0 = Ha * math.sqrt(nu * eta) / H
    p = {(1, s, O.F): dict(kind=O.VELOCITY) for s in (0, 1)}
    p.update({(1, s, O.G0): dict(kind=O.FLUX, kappa1=-kappa) for s in (0, 1)})
    p.update({(1, s, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0) for s in (0, 1)})
    shape = (nx, ny, 1)
    solid = LK.box_solid(shape, walls)
    sim = O.OracleSim(2, shape, solid, 0.8, 1.0, 0.5 + 4 * eta, (0.02 * nu * (2 + Ha) / H ** 2, 0, 0),
                      False, True, threads)
    sim.set_links(LK.box_links(2, shape, walls, p, has_g=True))
    u, B = _perturbed(nx * ny, B0, seed, 2)
    sim.init(u=u, B=B, B0=(0, B0, 0))
    return _bounded(sim, solid.reshape(-1) == 0, steps)


def pipe_stable(kappa, eta, steps=STEPS, R=16.0, n=36, nx=4, Ha=15.0, seed=1, threads=1):
    """One pipe run (Sec. 6: Shercliff B1, given B2 = B_ext and B3 = 0)."""
    nu = 0.1
    B0 = Ha * math.sqrt(nu * eta) / R
    params = {O.F: dict(kind=O.VELOCITY), O.G0: dict(kind=O.FLUX, kappa1=-kappa),
              O.G0 + 1: dict(kind=O.GIVEN, phi_wall=B0), O.G0 + 2: dict(kind=O.GIVEN, phi_wall=0.0)}
    shape = (nx, n, n)
    solid = LK.pipe_solid(shape, R)
    links, _ = LK.pipe_links(shape, R, params)
    sim = O.OracleSim(3, shape, solid, 0.8, 1.0, 0.5 + 4 * eta, (0.02 * nu * (2 + Ha) / R ** 2, 0, 0),
                      False, True, threads)
    sim.set_links(links)
    u, B = _perturbed(nx * n * n, B0, seed, 3)
    sim.init(u=u, B=B, B0=(0, B0, 0))
    return _bounded(sim, np.asarray(solid).reshape(-1) == 0, steps)


def bisect(stable, hi):
    """Largest kappa in [0, hi] found stable by BISECT halvings (0 when even
    the smallest tried is unstable)."""
    lo = 0.0
    for _ in range(BISECT):
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo


def _job(arg):
    kind, eta, q = arg
    if kind == "channel":
        return arg, bisect(lambda k: channel_stable(q, k, eta), 2 * START)
    return arg, bisect(lambda k: pipe_stable(k, eta), 2 * START)


def measure(processes=None):
    jobs = [("pipe", eta, None) for eta in ETAS] + [("channel", eta, q) for eta in ETAS for q in CHANNEL_Q]
    with mp.get_context("spawn").Pool(processes) as pool:
        res = dict(pool.map(_job, jobs, chunksize=1))
    channel = {eta: tuple(round(res[("channel", eta, q)], 3) for q in CHANNEL_Q) for eta in ETAS}
    pipe = {eta: round(res[("pipe", eta, None)], 3) for eta in ETAS}
    return channel, pipe


if __name__ == "__main__":
    ch, pi = measure()
    print("CHANNEL_KAPPA_LIMIT = {")
    for eta in ETAS:
        print("    %s: %s," % (eta, ch[eta]))
    print("}")
    print("PIPE_KAPPA_LIMIT = %s" % pi)
