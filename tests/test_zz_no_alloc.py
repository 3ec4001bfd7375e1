"""The allocation-free reduction entry point (lbm_reduce_noalloc) against the
context's reduction (lbm_check).

Callers that cannot allocate device memory -- an application that hands out
every byte of the GPU through its own pool, or a monitoring hook that must not
grow the footprint of the job it watches -- use lbm_reduce_noalloc on buffers
they already hold; its partial sums live in a fixed array inside the library.
This file is collected last on purpose, and it passes alone or after the rest.
"""
import numpy as np
import pytest

from paper_2506_00907_gb300 import cases as CS
from paper_2506_00907_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12      # the FP64 tolerance of the parity tests (sums taken in another order)


def _compare(a, b):
    for i in (0, 1, 2, 3, 4, 6, 7):
        scale = max(abs(b[i]), 1e-300)
        assert abs(a[i] - b[i]) <= TOL * scale, (i, a[i], b[i])
    assert a[5] == b[5] == 0


@pytest.mark.parametrize("prec", [lbm.LBM_FP32, lbm.LBM_FP16S])
def test_noalloc_reduction_matches_check_on_two_calls(prec):
    case, solid, links, info = CS.hartmann_channel(96, 12.0, 0.35, 0.2)
    stream = torch.cuda.current_stream()
    sol = lbm.Solver(lbm.LBM_D2Q9, prec, lbm.LBM_FLOW | lbm.LBM_MHD, [case], stream=stream.cuda_stream)
    sol.set_walls(0, solid, links)
    N = case.nx * case.ny * case.nz
    flags = torch.tensor((np.asarray(solid) == 0).astype(np.uint8), device="cuda")
    snap = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    for steps in (40, 25):
        sol.step(steps)
        want = sol.check()[0]
        ds = lbm.lbm_device_state(sol.ctx, 0)
        pops = ds["base"] + ds["case_offset"] * ds["elem_bytes"]
        got, st = lbm.lbm_reduce_noalloc(lbm.LBM_D2Q9, prec, lbm.LBM_FLOW | lbm.LBM_MHD, case, pops,
                                         ds["plane_stride"], flags.data_ptr(), snap.data_ptr(), stream.cuda_stream)
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
