"""Freezing cases of a batch (lbm_set_active) and running each case to its own
steady state (lbm_run_each_to_steady), on the GPU through the C ABI.

A frozen case keeps its state bit for bit while the others step exactly as
they step when nothing is frozen (no case reads another case's nodes); a
resumed case continues where it stopped.  Uneven Hartmann channels with wall
links on both walls, so both the bulk span list and the boundary-record list
lose the frozen case's entries."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import links as LK
from paper_2506_00907_gb300 import lbm
from tests.helpers import to_abi_links

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DRAWS = [dict(W=20, q=0.3, cw=0.05, Ha=4.0), dict(W=33, q=0.0, cw=1.0, Ha=12.0),
         dict(W=9, q=0.75, cw=0.5, Ha=1.5), dict(W=48, q=0.5, cw=0.2, Ha=25.0)]


def _channel(W, q, cw, Ha, tau=0.8, taue=0.9):
    nu, eta = (tau - 0.5) / 3, (taue - 0.5) / 4
    d = 1.0 - q
    ny = W + 2
    walls = LK.channel_y(2, W, ny, 1, d, d)
    H = (walls[1][1] - walls[1][0]) / 2
    B0 = Ha * math.sqrt(nu * eta) / H
    p = {(1, s, O.F): dict(kind=O.VELOCITY) for s in (0, 1)}
    p.update({(1, s, O.G0): dict(kind=O.FLUX, kappa1=-eta / (cw * H)) for s in (0, 1)})
    p.update({(1, s, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0) for s in (0, 1)})
    shape = (W, ny, 1)
    acc = (0.02 * 0.1 * (2 + Ha) / H ** 2, 0.0, 0.0)
    case = lbm.make_case(shape, tau, 1.0, taue, acc, 1.0, 0.0, (0, B0, 0))
    solid = LK.box_solid(shape, walls)
    return case, solid, to_abi_links(LK.box_links(2, shape, walls, p, has_g=True))


def _solver(prec=lbm.LBM_FP32, launch=None, graph=4, draws=DRAWS):
    geo = [_channel(**d) for d in draws]
    g = lbm.Solver(lbm.LBM_D2Q9, prec, lbm.LBM_FLOW | lbm.LBM_MHD, [c for c, _, _ in geo])
    for i, (_, solid, links) in enumerate(geo):
        g.set_walls(i, solid, links)
    if launch:
        g.set_launch(*launch)
    if graph:
        g.set_graph(graph)
    return g


def _case_bytes(g, blob, i):
    """Case i's populations inside a state blob (16-byte header, then the
    current buffer)."""
    ds = lbm.lbm_device_state(g.ctx, i)
    eb = ds["elem_bytes"]
    lo = 16 + ds["case_offset"] * eb
    return blob[lo:lo + ds["plane_stride"] * ds["planes"] * eb]


@pytest.mark.parametrize("prec,launch", [(lbm.LBM_FP32, (0, 128, 0, 1, 2, 1)), (lbm.LBM_FP32, (2, 64, 0, 2, 2, 5)),
                                         (lbm.LBM_FP16S, (0, 64, 0, 2, 2, 4))])
def test_frozen_case_is_unchanged_and_others_step_as_alone(prec, launch):
    a = _solver(prec, launch)
    a.step(40)
    at40 = a.get_state()
    a.set_active(1, False)
    a.step(61)                               # odd: the frozen state must sit in both buffers
    frozen = a.get_state()
    b = _solver(prec, launch)
    b.step(101)
    ref = b.get_state()
    for i in range(len(DRAWS)):
        if i == 1:
            assert np.array_equal(_case_bytes(a, frozen, i), _case_bytes(a, at40, i))
        else:
            assert np.array_equal(_case_bytes(a, frozen, i), _case_bytes(b, ref, i)), i
    out = a.check()
    a.step(8)
    out = a.check()
    assert out[1, 6] == 0.0 and out[0, 6] > 0.0      # no change of the frozen case since the last check
    # resumed, case 1 continues from step 40 (16-bit storage draws its rounding
    # bits from the context's step count, so there only FP32 compares bits)
    a.set_active(1, True)
    a.step(20)
    if prec == lbm.LBM_FP32:
        c = _solver(prec, launch)
        c.step(60)
        assert np.array_equal(_case_bytes(a, a.get_state(), 1), _case_bytes(c, c.get_state(), 1))


def test_state_written_into_a_frozen_case_is_kept():
    """A state blob loaded while a case is frozen is that case's state after
    any number of steps, odd or even."""
    a = _solver()
    a.step(30)
    blob = a.get_state()
    a.step(7)
    a.set_active(2, False)
    a.step(5)
    a.set_state(blob)
    for n in (3, 4):
        a.step(n)
        assert np.array_equal(_case_bytes(a, a.get_state(), 2), _case_bytes(a, blob, 2)), n
    # initialisation of the frozen case is kept the same way
    a.init_equilibrium(2)
    init = a.get_state()
    a.step(3)
    assert np.array_equal(_case_bytes(a, a.get_state(), 2), _case_bytes(a, init, 2))


def test_freezing_and_the_whole_case_variants_refuse_each_other():
    a = _solver(graph=0)
    a.set_active(0, False)
    with pytest.raises(lbm.LbmError):
        a.set_launch(1, 256, 0, 1, 2, 2)
    with pytest.raises(lbm.LbmError):
        a.set_launch(3, 256, 0, 2, 4, 2)
    with pytest.raises(lbm.LbmError):
        a.autotune(None, 2)
    a.set_active(0, True)
    a.set_launch(1, 256, 0, 1, 2, 2)
    with pytest.raises(lbm.LbmError):
        a.set_active(0, False)
    with pytest.raises(lbm.LbmError):
        a.set_active(len(DRAWS), False)
    with pytest.raises(lbm.LbmError):
        a.set_active(-1, True)


def test_run_each_to_steady_matches_run_to_steady():
    """Each case frozen at its own residual: the batch needs the slowest case's
    steps at most, every case ends below the residual, all cases are resumed, and the
    fields agree with a batch that ran every case to the slowest case's end
    (both converged: differences of the order of the residual)."""
    tol = 1e-6
    a = _solver(graph=100)
    k_a, r_a = a.run_each_to_steady(400000, 100, tol)
    assert r_a < tol
    a.set_launch(1, 256, 0, 1, 2, 2)          # accepted: no case is left frozen
    b = _solver(graph=100)
    k_b, r_b = b.run_to_steady(400000, 100, tol)
    assert r_b < tol and k_a <= k_b
    for i in range(len(DRAWS)):
        ua, ub = a.moments(i)["u"][:, 0], b.moments(i)["u"][:, 0]
        assert np.abs(ua - ub).max() <= 1e-4 * np.abs(ub).max(), i
    # a case frozen by the caller stays frozen through the call
    c = _solver(graph=100)
    c.step(200)
    keep = c.get_state()
    c.set_active(3, False)
    c.run_each_to_steady(400000, 100, tol)
    assert np.array_equal(_case_bytes(c, c.get_state(), 3), _case_bytes(c, keep, 3))
    with pytest.raises(lbm.LbmError):
        c.set_launch(1, 256, 0, 1, 2, 2)


@pytest.mark.parametrize("prec", [lbm.LBM_FP32, lbm.LBM_FP16S])
def test_frozen_pipe_with_link_kernel(prec):
    """3D cases evaluate their wall links in a kernel of their own (one thread
    per link, the links of frozen cases included): freezing one of three
    curved-wall pipes keeps its bits and leaves the others as they step
    alone."""
    from paper_2506_00907_gb300 import cases as CS
    geo = [CS.pipe((4, 36, 36), 16.0, 10.0, "insulating"), CS.pipe((6, 36, 36), 16.0, 15.0, ("shercliff", 0.5)),
           CS.pipe((3, 36, 36), 16.0, 5.0, "conducting")]

    def solver():
        g = lbm.Solver(lbm.LBM_D3Q19, prec, lbm.LBM_FLOW | lbm.LBM_MHD, [c for c, _, _, _ in geo])
        for i, (_, solid, links, _) in enumerate(geo):
            g.set_walls(i, solid, links)
        g.set_graph(10)
        return g
    a = solver()
    assert lbm.lib().lbm_launches_per_step(a.ctx) == 3          # bulk, links, boundary nodes
    a.step(30)
    at30 = a.get_state()
    a.set_active(1, False)
    a.step(41)
    b = solver()
    b.step(71)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(_case_bytes(a, sa, 1), _case_bytes(a, at30, 1))
    for i in (0, 2):
        assert np.array_equal(_case_bytes(a, sa, i), _case_bytes(b, sb, i)), i
