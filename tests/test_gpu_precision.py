"""Reduced-precision storage at the benchmark's own configurations, against
the FP64 oracle node by node and against the paper's closed forms.

Every workload here is invariant along x (periodic x, walls normal to y, or
the pipe axis along x) and starts from rest, so the oracle runs each case at
x length 1 and its rows are compared with every row of the GPU's full-width
run (``oracle.workloads``; the x-invariance itself is pinned on the CPU).

Errors are norm-relative per field over fluid nodes, max|gpu - ref| /
max|ref|, for u, b = B - B_ext and C, and absolute for the density (in units
of rho0 = 1; rho - 1 itself is of the order of the rounding).  Every bound is
the error measured on GB300 for these exact runs (the kernels and the oracle
are deterministic) times a margin of 1.5, so that a change in the arithmetic
of either side shows up; the measured values are listed in the design notes.
FP64 meets the 1e-12 parity target per step (``test_gpu_parity.py``); over
thousands of steps the two sides' different rounding orders accumulate over
the flow's relaxation time, to about 4e-12 after 2000 steps and 8e-12 at
steady state.  Both 16-bit storages round stochastically: the error has zero
mean, so the steady states are within 0.2 % (FP16, whose offsets are scaled
by 2^12 to stay out of its subnormal range) and 1.7 % (BF16, three significand
bits fewer) of the oracle's.  (Rounding to nearest, measured on the same runs
before, left errors of 10-26 % at steady state: the same rounding recurs every
step and acts as a fixed spurious source that the flow integrates over its
diffusion time.)  Rounding noise also excites every mode the geometry allows,
including modes that vary along a wall, which a start uniform along the wall
never excites in exact-order arithmetic: the Shercliff-flux limits the case
builders use are measured from perturbed starts for that reason.
"""
import concurrent.futures as cf
import os
import sys

import numpy as np
import pytest

from oracle import analytic as AN
from oracle import pipe_fd as FD
from oracle import workloads as WL
from paper_2506_00907_gb300 import inputs as IN
from paper_2506_00907_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

MARGIN = 1.5
# the launch shape the autotuner chose for the benchmark on GB300 (64-thread
# blocks, 3 nodes per thread, register budget of 5 blocks per SM); every other
# shape gives the same bits (checked below and in test_gpu_parity.py)
BENCH_LAUNCH = (0, 64, 0, 3, 2, 5)


def _workers():
    return max(1, min(16, os.cpu_count() or 1))


def _oracle_rows(spec, steps, which):
    """Oracle fields of every case of the spec at x length 1 after `steps`."""
    def one(P):
        if spec["kind"] == "hartmann":
            s, solid = WL.hartmann(P, nx=1, threads=1)
        elif spec["kind"] == "pipe":
            s, solid = WL.pipe(P, spec["shape"], nx=1, threads=_workers())
        else:
            s, solid = WL.reactive(P, nx=1, threads=1)
        s.step(steps)
        m = s.moments()
        fl = np.asarray(solid).reshape(-1) == 0
        out = {"u": m["u"][fl], "rho": m["rho"][fl] - 1.0, "y": np.flatnonzero(fl)}
        if "C" in which:
            out["C"] = m["C"][fl]
        if "b" in which:
            out["b"] = m["B"][fl] - np.array([0.0, P["B0"], 0.0])
        return out
    with cf.ThreadPoolExecutor(max_workers=1 if spec["kind"] == "pipe" else _workers()) as ex:
        return list(ex.map(one, spec["params"]))


def _gpu_run(spec, prec, steps, launch=BENCH_LAUNCH):
    stream = torch.cuda.current_stream()
    sol, geo, _ = bench.make_solver(dict(spec, prec=prec), stream, 0)
    sol.set_launch(*launch)
    sol.set_graph(100)
    sol.step(steps)
    fields = bench.gpu_fields(sol, spec, geo)
    blob = sol.get_state()
    sol.close()
    return fields, blob


def _nx(spec, P):
    return spec["shape"][0] if spec["kind"] == "pipe" else P["shape"][0]


def _errors(spec, gpu, ref, keys):
    """Max over cases of the per-case error, per field: norm-relative, except
    the density (absolute)."""
    out = {k: 0.0 for k in keys}
    for P, g, r in zip(spec["params"], gpu, ref):
        nx = _nx(spec, P)
        for k in keys:
            rr = WL.widen(r[k], nx)
            den = 1.0 if k == "rho" else np.abs(rr).max()
            out[k] = max(out[k], float(np.abs(g[k] - rr).max() / (den if den > 0 else 1.0)))
    return out


def _report(tag, errs):
    print("\n%s: %s" % (tag, "  ".join("%s %.3g" % kv for kv in sorted(errs.items()))))


def _assert_within(errs, bound):
    for k, v in errs.items():
        assert v <= bound[k], (k, v, bound[k])


# ----------------------------------------------------------------------------- the 64-case Hartmann batch
BATCH_STEPS = 2000
# errors measured on GB300 after 2000 steps from rest (all 64 cases, every fluid node)
BATCH_MEASURED = {
    "fp64": {"u": 4.53e-12, "b": 2.59e-12, "rho": 1.46e-13},
    "fp32": {"u": 5.39e-4, "b": 5.60e-5, "rho": 3.88e-7},
    "fp16s": {"u": 3.67e-3, "b": 1.93e-3, "rho": 3.97e-5},
    "bf16s": {"u": 2.60e-2, "b": 1.70e-2, "rho": 3.40e-4},
}


@pytest.fixture(scope="module")
def batch():
    spec = bench.workload_spec("hartmann_batch")
    return spec, _oracle_rows(spec, BATCH_STEPS, ("b",))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s", "bf16s"])
def test_hartmann_batch_against_oracle(batch, prec):
    """The benchmark's 64 channels (seed 2506, full widths 64..512), its
    launch shape, 2000 steps from rest, every fluid node against the oracle."""
    spec, ref = batch
    gpu, blob = _gpu_run(spec, prec, BATCH_STEPS)
    errs = _errors(spec, gpu, ref, ("u", "b", "rho"))
    _report("hartmann batch %s, %d steps" % (prec, BATCH_STEPS), errs)
    _assert_within(errs, {k: MARGIN * v for k, v in BATCH_MEASURED[prec].items()})
    if prec == "fp16s":
        # other launch shapes and the unwrapped-pull variant give the same bits
        for launch in ((0, 256, 0, 1, 2, 4), (2, 64, 0, 2, 2, 5)):
            _, other = _gpu_run(spec, prec, BATCH_STEPS, launch)
            assert np.array_equal(other[16:], blob[16:]), launch


# ----------------------------------------------------------------------------- Hartmann steady state
STEADY_DRAWS = (22, 57, 10)          # W = 100, 77, 150 of the batch draws
STEADY_STEPS = 140000
STEADY_MEASURED = {
    "fp64": {"u": 6.26e-12, "b": 8.39e-12},
    "fp32": {"u": 9.57e-5, "b": 1.14e-4},
    "fp16s": {"u": 1.51e-3, "b": 1.83e-3},
    "bf16s": {"u": 1.22e-2, "b": 1.74e-2},
}


@pytest.fixture(scope="module")
def hartmann_steady():
    draws = IN.hartmann_batch(64)
    params = [IN.hartmann_params(**draws[i], clamp_cw=True) for i in STEADY_DRAWS]
    spec = dict(bench.workload_spec("hartmann_batch"), params=params)
    ref = _oracle_rows(spec, STEADY_STEPS, ("b",))
    exact = []
    for P, r in zip(params, ref):
        y = r["y"] - (P["W"] + 1) / 2.0
        wall = ("shercliff", P["cw"])
        exact.append(AN.hartmann(y, P["H"], P["B0"], P["nu"], P["eta"], accel=P["accel"], wall_lo=wall,
                                 wall_hi=wall))
    return spec, ref, exact


def _closed_form_errors(spec, rows, exact, widen):
    out = {"u": 0.0, "b": 0.0}
    for P, r, (ua, ba) in zip(spec["params"], rows, exact):
        nx = _nx(spec, P) if widen else 1
        for k, a in (("u", ua), ("b", ba)):
            aw = WL.widen(a, nx)
            out[k] = max(out[k], float(np.abs(r[k][:, 0] - aw).max() / np.abs(aw).max()))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s", "bf16s"])
def test_hartmann_steady_state_against_closed_form(hartmann_steady, prec):
    """Three channels of the batch (W = 100, 77, 150; Ha 17, 21, 15; c_w
    0.0028, 0.0011 (raised from 0.00107 to the flux stability limit), 0.041)
    run to steady state (140 000 steps): each storage
    against the oracle's steady state node by node, and its error against the
    Hartmann closed form (Sec. 5.4) against the oracle's own."""
    spec, ref, exact = hartmann_steady
    gpu, _ = _gpu_run(spec, prec, STEADY_STEPS)
    errs = _errors(spec, gpu, ref, ("u", "b"))
    e_orc = _closed_form_errors(spec, ref, exact, False)
    e_gpu = _closed_form_errors(spec, gpu, exact, True)
    _report("hartmann steady %s vs oracle" % prec, errs)
    _report("hartmann steady %s vs closed form (oracle's own: u %.4g b %.4g)" % (prec, e_orc["u"], e_orc["b"]),
            e_gpu)
    bound = {k: MARGIN * v for k, v in STEADY_MEASURED[prec].items()}
    _assert_within(errs, bound)
    for k in ("u", "b"):
        assert e_gpu[k] <= e_orc[k] + bound[k], (k, e_gpu[k], e_orc[k])


# ----------------------------------------------------------------------------- flow + concentration channels
CD_STEPS = 2000
CD_MEASURED = {
    "fp64": {"u": 1.43e-13, "C": 1.66e-14, "rho": 1.13e-13},
    "fp32": {"u": 4.67e-6, "C": 1.11e-5, "rho": 1.13e-13},
    "fp16s": {"u": 1.03e-3, "C": 4.54e-4, "rho": 6.87e-5},
    "bf16s": {"u": 8.16e-3, "C": 3.79e-3, "rho": 5.72e-4},
}


@pytest.fixture(scope="module")
def cd_batch():
    spec = bench.workload_spec("cd")
    return spec, _oracle_rows(spec, CD_STEPS, ("C",))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s", "bf16s"])
def test_reactive_channels_against_oracle(cd_batch, prec):
    """The 12 flow + concentration channels of 512 x 256 (q in {0, 1/4, 1/2,
    3/4}, k in {1e-3, 1e-2, 1e-1}, top wall U = 0.05), 2000 steps from rest."""
    spec, ref = cd_batch
    gpu, _ = _gpu_run(spec, prec, CD_STEPS, (0, 128, 0, 2, 2, 1))
    errs = _errors(spec, gpu, ref, ("u", "C", "rho"))
    _report("reactive channels %s, %d steps" % (prec, CD_STEPS), errs)
    _assert_within(errs, {k: MARGIN * v for k, v in CD_MEASURED[prec].items()})


CD_STEADY_STEPS = 100000
CD_STEADY_MEASURED = {"fp32": {"u": 2.19e-4, "C": 1.40e-4}, "fp16s": {"u": 1.32e-3, "C": 6.14e-4},
                      "bf16s": {"u": 1.05e-2, "C": 4.23e-3}}


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "bf16s"])
def test_reactive_channels_steady_state_against_closed_form(prec):
    """The same 12 (q, k) channels at height 66 (2H = 63 + 2d), run to steady
    state (100 000 steps, ten diffusion times): the storage against the
    oracle's steady state node by node, and against the linear concentration
    profile of the Robin / given-C walls and the Couette velocity."""
    params = IN.reactive_grid(512, 66)
    spec = dict(bench.workload_spec("cd"), params=params)
    ref = _oracle_rows(spec, CD_STEADY_STEPS, ("C",))
    gpu, _ = _gpu_run(spec, prec, CD_STEADY_STEPS, (0, 128, 0, 2, 2, 1))
    errs = _errors(spec, gpu, ref, ("u", "C"))
    _report("reactive steady %s vs oracle" % prec, errs)
    _assert_within(errs, {k: MARGIN * v for k, v in CD_STEADY_MEASURED[prec].items()})
    e_orc = {"u": 0.0, "C": 0.0}
    e_gpu = {"u": 0.0, "C": 0.0}
    for P, r, g in zip(params, ref, gpu):
        ny = P["shape"][1]
        y = r["y"].astype(np.float64)
        y0, y1 = 1.0 - P["d"], ny - 2.0 + P["d"]
        Ca = AN.reactive_channel(y, y0, y1, 0.1, P["kappa0"], P["kappa1"], P["C_top"])
        ua = AN.couette(y, y0, y1, 0.0, P["U"])
        for k, a, fo, fg in (("C", Ca, r["C"], g["C"]), ("u", ua, r["u"][:, 0], g["u"][:, 0])):
            aw = WL.widen(a, P["shape"][0])
            e_orc[k] = max(e_orc[k], float(np.abs(fo - a).max() / np.abs(a).max()))
            e_gpu[k] = max(e_gpu[k], float(np.abs(fg - aw).max() / np.abs(aw).max()))
    _report("reactive steady %s vs closed form (oracle's own: u %.4g C %.4g)" % (prec, e_orc["u"], e_orc["C"]),
            e_gpu)
    for k in ("u", "C"):
        assert e_gpu[k] <= e_orc[k] + MARGIN * CD_STEADY_MEASURED[prec][k], (k, e_gpu[k], e_orc[k])


# ----------------------------------------------------------------------------- the MHD pipe, 32 x 128 x 128
PIPE_STEPS = 1000
PIPE_MEASURED = {"fp32": {"u": 2.24e-5, "b": 2.60e-5, "rho": 6.57e-8},
                 "fp16s": {"u": 5.88e-4, "b": 8.74e-4, "rho": 6.3e-6},
                 "bf16s": {"u": 4.96e-3, "b": 7.37e-3, "rho": 4.56e-5}}


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "bf16s"])
def test_pipe_against_oracle(prec):
    """The 3D pipe (R = 62, curved Shercliff wall, every q in (0, 1) on the
    circle), 1000 steps from rest, every fluid node against the oracle."""
    spec = bench.workload_spec("pipe")
    ref = _oracle_rows(spec, PIPE_STEPS, ("b",))
    gpu, _ = _gpu_run(spec, prec, PIPE_STEPS, (0, 128, 0, 1, 2, 1))
    errs = _errors(spec, gpu, ref, ("u", "b", "rho"))
    _report("pipe %s, %d steps" % (prec, PIPE_STEPS), errs)
    _assert_within(errs, {k: MARGIN * v for k, v in PIPE_MEASURED[prec].items()})


PIPE_STEADY_MEASURED = {"fp32": {"u": 1.11e-2, "b": 1.66e-2}, "fp16s": {"u": 1.13e-2, "b": 1.70e-2},
                        "bf16s": {"u": 1.18e-2, "b": 1.95e-2}}


def test_pipe_steady_state_against_finite_volume_solution():
    """The same pipe run towards steady state in FP32 (residual 1e-6, at most
    300 000 steps) and, for as many steps, in FP16 storage: axial velocity
    and induced field against the independent finite-volume solution of the
    pipe problem (Sec. 6)."""
    spec = bench.workload_spec("pipe")
    P = spec["params"][0]
    stream = torch.cuda.current_stream()
    r, th, uf, bf = FD.solve(P["R"], P["B0"], P["nu"], P["eta"], P["accel"], wall=P["wall"], nr=96, nt=192)
    out = {}
    steps = None
    for prec in ("fp32", "fp16s", "bf16s"):
        sol, geo, _ = bench.make_solver(dict(spec, prec=prec), stream, 0)
        sol.set_graph(100)
        if steps is None:
            steps, res = sol.run_to_steady(300000, 100, 1e-6)
            print("\npipe FP32: residual %.3g after %d steps" % (res, steps))
        else:
            sol.step(steps)
        nx, ny, nz = spec["shape"]
        fl = np.asarray(geo[0][0]).reshape(-1) == 0
        c = (ny - 1) / 2.0
        zz, yy, _ = np.meshgrid(np.arange(nz) - c, np.arange(ny) - c, np.arange(nx), indexing="ij")
        ua = FD.sample(r, th, uf, yy.ravel()[fl], zz.ravel()[fl])
        ba = FD.sample(r, th, bf, yy.ravel()[fl], zz.ravel()[fl])
        m = sol.moments(0)
        out[prec] = {"u": float(np.abs(m["u"][fl, 0] - ua).max() / np.abs(ua).max()),
                     "b": float(np.abs(m["B"][fl, 0] - ba).max() / np.abs(ba).max())}
        sol.close()
        _report("pipe steady %s vs finite volume (%d steps)" % (prec, steps), out[prec])
    for prec in out:
        for k in ("u", "b"):
            assert out[prec][k] <= MARGIN * PIPE_STEADY_MEASURED[prec][k], (prec, k, out[prec][k])
