"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
side (parameter draws, random geometries and random initial fields).

This module holds no lattice-Boltzmann arithmetic: it only draws numbers.
Physical parameter sets follow the paper's cases in lattice units
(tau_nu = 0.8, tau_eta = 0.9, tau_D = 0.9, rho0 = 1, B_ext along x2).
"""
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
