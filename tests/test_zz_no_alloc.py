"""The allocation-free reduction entry point (lbm_reduce_noalloc) against the
context's reduction (lbm_check).

Callers that cannot allocate device memory -- an application that hands out
every byte of the GPU through its own pool, or a monitoring hook that must not
grow the footprint of the job it watches -- use lbm_reduce_noalloc on buffers
they already hold; its partial sums live in a fixed array inside the library.
Covered: both lattices, every storage precision, the flow + field and the
flow + concentration physics, no flags (all-fluid periodic box), no snapshot,
and a domain just below the node limit whose size is not a multiple of the
256-node block.  This file is collected last on purpose, and it passes alone
or after the rest.
"""
import numpy as np
import pytest

from paper_2506_00907_gb300 import cases as CS
from paper_2506_00907_gb300 import inputs as IN
from paper_2506_00907_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12      # the FP64 tolerance of the parity tests (sums taken in another order)
MHD = lbm.LBM_FLOW | lbm.LBM_MHD
CD = lbm.LBM_FLOW | lbm.LBM_CD


def _compare(a, b, with_snap=True):
    """Sums 0-4 within TOL of the record's largest sum (the mass, about the
    node count): a field sum that is zero in exact arithmetic, such as B_x
    across a symmetric channel, rounds to different tiny values in another
    summation order.  The residual sums 6 and 7 within TOL of themselves."""
    big = max(abs(b[i]) for i in range(5))
    for i in (0, 1, 2, 3, 4):
        assert abs(a[i] - b[i]) <= TOL * big, (i, a[i], b[i])
    if with_snap:
        for i in (6, 7):
            assert abs(a[i] - b[i]) <= TOL * max(abs(b[i]), 1e-300), (i, a[i], b[i])
    else:
        assert a[6] == a[7] > 0                  # phi_prev taken as zero: both are sum |phi|^2
    assert a[5] == b[5] == 0


def _case(kind):
    if kind == "hartmann":
        c, s, l, _ = CS.hartmann_channel(96, 12.0, 0.35, 0.2)
        return lbm.LBM_D2Q9, MHD, c, s, l
    if kind == "pipe":
        c, s, l, _ = CS.pipe((5, 28, 28), 12.0, 8.0, ("shercliff", 0.3))
        return lbm.LBM_D3Q19, MHD, c, s, l
    c, s, l, _ = CS.reactive_channel(40, 34, 0.3, 0.05, 1e-2)
    return lbm.LBM_D2Q9, CD, c, s, l


def _noalloc(sol, lattice, prec, phys, case, flags, snap, stream):
    ds = lbm.lbm_device_state(sol.ctx, 0)
    pops = ds["base"] + ds["case_offset"] * ds["elem_bytes"]
    return lbm.lbm_reduce_noalloc(lattice, prec, phys, case, pops, ds["plane_stride"],
                                  flags.data_ptr() if flags is not None else None,
                                  snap.data_ptr() if snap is not None else None, stream.cuda_stream)


@pytest.mark.parametrize("kind,prec", [
    ("hartmann", lbm.LBM_FP32), ("hartmann", lbm.LBM_FP16S), ("hartmann", lbm.LBM_BF16S),
    ("hartmann", lbm.LBM_FP64), ("pipe", lbm.LBM_FP64), ("pipe", lbm.LBM_FP16S), ("reactive", lbm.LBM_FP32)])
def test_noalloc_reduction_matches_check_on_two_calls(kind, prec):
    lattice, phys, case, solid, links = _case(kind)
    stream = torch.cuda.current_stream()
    sol = lbm.Solver(lattice, prec, phys, [case], stream=stream.cuda_stream)
    sol.set_walls(0, solid, links)
    N = case.nx * case.ny * case.nz
    flags = torch.tensor((np.asarray(solid).reshape(-1) == 0).astype(np.uint8), device="cuda")
    snap = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    for steps in (40, 25):
        sol.step(steps)
        want = sol.check()[0]
        got, st = _noalloc(sol, lattice, prec, phys, case, flags, snap, stream)
        assert st == lbm.LBM_OK
        _compare(got, want)
    sol.close()


def test_noalloc_without_snapshot_compares_with_zero():
    lattice, phys, case, solid, links = _case("hartmann")
    stream = torch.cuda.current_stream()
    sol = lbm.Solver(lattice, lbm.LBM_FP32, phys, [case], stream=stream.cuda_stream)
    sol.set_walls(0, solid, links)
    flags = torch.tensor((np.asarray(solid).reshape(-1) == 0).astype(np.uint8), device="cuda")
    for steps in (30, 30):
        sol.step(steps)
        want = sol.check()[0]
        got, st = _noalloc(sol, lattice, lbm.LBM_FP32, phys, case, flags, None, stream)
        assert st == lbm.LBM_OK
        _compare(got, want, with_snap=False)
    sol.close()


@pytest.mark.parametrize("shape", [(37, 29, 1), (2047, 2049, 1)])
def test_noalloc_without_flags_on_an_all_fluid_box(shape):
    """A fully periodic box (no walls) from random fields: with flags NULL every
    node counts, as every node is fluid for lbm_check.  The second shape has
    2^22 - 1 nodes, one below the limit and not a multiple of 256."""
    nx, ny, nz = shape
    N = nx * ny * nz
    case = lbm.make_case(shape, 0.8, 0.9, 0.7, (1e-6, 0, 0), 1.0, 1.0, (0, 0, 0))
    stream = torch.cuda.current_stream()
    sol = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW, [case], stream=stream.cuda_stream)
    f = IN.random_fields(IN.rng(77), N, 2)
    sol.init_equilibrium(0, rho=f["rho"], u=f["u"])
    snap = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    for steps in (4, 6):
        sol.step(steps)
        want = sol.check()[0]
        got, st = _noalloc(sol, lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW, case, None, snap, stream)
        assert st == lbm.LBM_OK
        _compare(got, want)
    sol.close()


def test_noalloc_reduction_rejects_oversize_domains():
    big = lbm.make_case((2049, 2049, 1), 0.8)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = np.zeros(8)
    st = lbm.lib().lbm_reduce_noalloc(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW, lbm.ctypes.byref(big),
                                      buf.data_ptr(), 2049 * 2049, None, None,
                                      out.ctypes.data_as(lbm.ctypes.POINTER(lbm.ctypes.c_double)), None)
    assert st == lbm.LBM_EINVAL
