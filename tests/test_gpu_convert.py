"""Changing the storage precision of a running state (lbm_convert_state):
FP64 -> FP32 keeps the FP32 parity bar against the FP64 oracle afterwards,
FP32 -> FP16 -> FP32 is exactly the element-wise rounding of the stored
values (FP16 storage holds them times 2^12, rounded to nearest on
conversion), and mismatched contexts are rejected."""
import numpy as np
import pytest

from paper_2506_00907_gb300 import lbm
from tests.helpers import norm_rel
from tests.test_gpu_parity import _random_pair

pytestmark = pytest.mark.gpu


def _twin(src, prec):
    """A context with the case and walls of the Pair `src` at another precision."""
    s = lbm.Solver(lbm.LBM_D2Q9 if src.dim == 2 else lbm.LBM_D3Q19, prec, src.gpu_phys, src.gpu.cases)
    s.set_walls(0, src.solid, src.abi_links)
    return s


def _pair(dim):
    p = _random_pair(dim, True, True, seed=300 + dim)
    p.gpu_phys = lbm.LBM_FLOW | lbm.LBM_CD | lbm.LBM_MHD
    return p


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_to_fp32_then_continue_against_oracle(dim):
    p = _pair(dim)
    p.step(30)
    t = _twin(p, lbm.LBM_FP32)
    t.convert_from(p.gpu)
    assert t.steps == p.gpu.steps == 30
    a, b = t.moments(0), p.orc.moments()
    fl = p.fluid
    for k in ("rho", "u", "C", "B"):
        assert norm_rel(a[k][fl], b[k][fl]) < 1e-6, k
    p.orc.step(30)
    t.step(30)
    a, b = t.moments(0), p.orc.moments()
    for k in ("rho", "u", "C", "B"):
        assert norm_rel(a[k][fl], b[k][fl]) < 1e-5, k


def test_fp32_fp16_fp32_round_trip_is_elementwise_rounding():
    p = _pair(2)
    f32 = _twin(p, lbm.LBM_FP32)
    f32.convert_from(p.gpu)
    f32.step(10)
    h = _twin(p, lbm.LBM_FP16S)
    h.convert_from(f32)
    back = _twin(p, lbm.LBM_FP32)
    back.convert_from(h)
    ds = lbm.lbm_device_state(f32.ctx, 0)
    stride, off, planes = ds["plane_stride"], ds["case_offset"], ds["planes"]
    N = p.N
    s0 = f32.get_state()[16:].view(np.float32)
    s1 = back.get_state()[16:].view(np.float32)
    for q in range(planes):
        a = s0[off + q * stride: off + q * stride + N]
        b = s1[off + q * stride: off + q * stride + N]
        want = (a * np.float32(4096)).astype(np.float16).astype(np.float32) / np.float32(4096)
        assert np.array_equal(want, b), q
    assert back.steps == f32.steps


def test_mismatched_contexts_are_rejected():
    p = _pair(2)
    other = lbm.make_case(p.shape, 0.81, 0.9, 0.7, (0.0, 0.0, 0.0), 1.0, 1.0, (0.0, 0.3, 0.0))
    s = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, p.gpu_phys, [other])
    with pytest.raises(lbm.LbmError):
        s.convert_from(p.gpu)
    with pytest.raises(lbm.LbmError):
        p.gpu.convert_from(p.gpu)
