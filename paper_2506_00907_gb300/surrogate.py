"""Warm start of steady MHD pipe runs by a small network (not part of the
paper's method; it only supplies initial fields).

The network maps (x2/R, x3/R, f_Ha, f_cw) of a cross-section point to the
dimensionless steady axial velocity u_hat = u nu / (a R^2) and induced field
b_hat = b eta nu / (B0 a R^3), functions of (Ha, c_w) and position only.  It is
trained on steady fields that the batched solver itself produces, with the
library's own forward, backward and Adam kernels, and used through
lbm_net_pipe_fields + lbm_init_equilibrium_device.  Outside the training range
of (Ha, c_w), or if the prediction is not finite, the run starts cold.
"""
import math

import numpy as np

from . import cases as CS
from . import inputs as IN
from . import lbm

HA_RANGE = (10.0, 50.0)
CW_RANGE = (1e-3, 1.0)
# lattice units keep the imposed field well below the lattice pressure: the
# magnetic stress makes f^eq along B proportional to rho - 3|B|^2, so runs
# need B0 = Ha sqrt(nu eta) / R <~ 0.2, i.e. R >= Ha / 2 at tau = 0.8 / 0.9
B0_MAX = 0.2


def f_ha(Ha):
    return (Ha - 30.0) / 20.0


def f_cw(cw):
    return (math.log10(cw) + 1.5) / 1.5


class Surrogate:
    """A trained network with the (Ha, c_w) range it was trained on and the
    per-output scale of its training targets (train() fits T / scale)."""

    def __init__(self, net, ha_range, cw_range, target_scale=None):
        self.net, self.ha_range, self.cw_range = net, tuple(ha_range), tuple(cw_range)
        if target_scale is None:
            target_scale = getattr(net, "target_scale", (1.0, 1.0))
        self.target_scale = tuple(float(v) for v in target_scale)

    def covers(self, Ha, cw):
        return self.ha_range[0] <= Ha <= self.ha_range[1] and self.cw_range[0] <= cw <= self.cw_range[1]


def scales(info, R):
    """(u_scale, b_scale): u = u_hat * u_scale, b = b_hat * b_scale."""
    us = info["accel"] * R * R / info["nu"]
    bs = info["B0"] * R * us / info["eta"]
    return us, bs


def pipe_cases(draws, n, R):
    """Cases of one-node-long pipes (the flow is axially invariant)."""
    out = []
    for d in draws:
        if d["Ha"] * math.sqrt(0.1 * 0.1) / R > B0_MAX:
            raise ValueError("Ha = %g needs R >= %g in lattice units" % (d["Ha"], d["Ha"] * 0.1 / B0_MAX))
        c, solid, links, info = CS.pipe((1, n, n), R, d["Ha"], ("shercliff", d["cw"]))
        out.append((c, solid, links, info))
    return out


def generate(draws, n=64, R=30.0, tol=1e-7, max_steps=400000, prec=lbm.LBM_FP32, batch=64, stream=None,
             per_case=None, seed=IN.SEED):
    """Steady fields of the drawn cases, solved in batches of `batch` cases
    (one launch per step each).  Returns (X [M, 4], T [M, 2], stats) with one
    sample per fluid node, or per_case nodes drawn at random per case."""
    Xs, Ts, stats = [], [], []
    r = IN.rng(seed + 3)
    for b0 in range(0, len(draws), batch):
        group = pipe_cases(draws[b0:b0 + batch], n, R)
        sol = lbm.Solver(lbm.LBM_D3Q19, prec, lbm.LBM_FLOW | lbm.LBM_MHD, [g[0] for g in group], stream=stream)
        for i, g in enumerate(group):
            sol.set_walls(i, g[1], g[2])
        sol.set_graph(100)
        steps, res = sol.run_to_steady(max_steps, 100, tol)
        stats.append(dict(cases=len(group), steps=steps, residual=res))
        c = (n - 1) / 2.0
        zz, yy = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
        for i, (case, solid, links, info) in enumerate(group):
            m = sol.moments(i)
            fl = np.asarray(solid).reshape(-1) == 0
            us, bs = scales(info, R)
            d = draws[b0 + i]
            X = np.stack([yy.ravel()[fl] / R, zz.ravel()[fl] / R, np.full(fl.sum(), f_ha(d["Ha"])),
                          np.full(fl.sum(), f_cw(d["cw"]))], axis=1)
            T = np.stack([m["u"][fl, 0] / us, m["B"][fl, 0] / bs], axis=1)
            if per_case and per_case < len(X):
                keep = r.choice(len(X), per_case, replace=False)
                X, T = X[keep], T[keep]
            Xs.append(X)
            Ts.append(T)
        sol.close()
    return np.concatenate(Xs).astype(np.float32), np.concatenate(Ts).astype(np.float32), stats


def train(X, T, epochs=30, batch=8192, lr=3e-3, seed=IN.SEED, stream=None, log=None, normalise=True):
    """Minibatch Adam on the GPU with the library's kernels; minibatches are
    a fixed host-side shuffle per epoch.  With normalise, each output is
    fitted as T / rms(T) so that both outputs weigh alike in the loss (the
    scale is kept as net.target_scale).  Returns (net, loss history)."""
    import torch
    net = lbm.Net(IN.net_init(seed), stream=stream)
    scale = np.sqrt(np.mean(np.asarray(T, dtype=np.float64) ** 2, axis=0)) if normalise else np.ones(T.shape[1])
    scale = np.where(scale > 0, scale, 1.0)
    net.target_scale = tuple(float(v) for v in scale)
    Tn = (np.asarray(T, dtype=np.float64) / scale).astype(np.float32)
    r = IN.rng(seed + 1)
    hist = []
    n = len(X)
    for ep in range(epochs):
        perm = r.permutation(n)
        Xd = torch.tensor(X[perm], device="cuda")
        Td = torch.tensor(Tn[perm], device="cuda")
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        tot = 0.0
        for b in range(0, n, batch):
            loss, _ = net.loss_grad(Xd[b:b + batch], Td[b:b + batch])
            net.adam(lr_ep)
            tot += loss * min(batch, n - b)
        hist.append(tot / n)
        if log:
            log(ep, hist[-1])
    return net, hist


def warm_start(sol, case_id, sur, info, shape, R, Ha, cw):
    """Initialise case `case_id` from the surrogate's prediction.  Returns
    True if the warm start was used, False if the case fell back to a cold
    start (outside the training range, or a non-finite prediction)."""
    import torch
    if sur is None or not sur.covers(Ha, cw):
        return False
    net = sur.net
    N = shape[0] * shape[1] * shape[2]
    u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    B = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    us, bs = scales(info, R)
    su, sb = sur.target_scale
    net.pipe_fields(shape, R, f_ha(Ha), f_cw(cw), us * su, bs * sb, info["B0"], u, B)
    torch.cuda.synchronize()              # the network's stream wrote u, B; the solver's stream reads them
    sol.init_equilibrium_device(case_id, u=u, B=B)
    out = sol.check(raise_unstable=False)
    if out[case_id, 5] != 0:
        sol.init_equilibrium(case_id)        # cold start
        return False
    return True
