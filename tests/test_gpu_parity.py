"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 storage must match the oracle within 1e-12 norm-relative per field
(max|gpu - oracle| / max|oracle|).  FP32 and the 16-bit offset storages are
held to the tolerances stated in each test (their rounding, not the scheme,
sets them).  All inputs are seeded; links come from the oracle's builders."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import links as LK
from paper_2506_00907_gb300 import inputs as IN
from paper_2506_00907_gb300 import lbm
from tests.helpers import norm_rel, to_abi_links

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _phys(has_h, has_g):
    return lbm.LBM_FLOW | (lbm.LBM_CD if has_h else 0) | (lbm.LBM_MHD if has_g else 0)


class Pair:
    """The same case on the oracle and on the GPU."""

    def __init__(self, dim, shape, solid, links, prec=lbm.LBM_FP64, taus=(0.8, 0.9, 0.7),
                 accel=(0.0, 0.0, 0.0), has_h=False, has_g=False, fields=None, C0=1.0, B0=(0, 0, 0), threads=8):
        self.dim, self.shape = dim, shape
        self.N = shape[0] * shape[1] * shape[2]
        self.fluid = np.asarray(solid).reshape(-1) == 0
        self.orc = O.OracleSim(dim, shape, solid, taus[0], taus[1], taus[2], accel, has_h, has_g, threads)
        self.orc.set_links(links)
        f = fields or {}
        self.orc.init(rho=f.get("rho"), u=f.get("u"), C=f.get("C"), B=f.get("B"), rho0=1.0, C0=C0, B0=B0)
        case = lbm.make_case(shape, taus[0], taus[1], taus[2], accel, 1.0, C0, B0)
        self.gpu = lbm.Solver(lbm.LBM_D2Q9 if dim == 2 else lbm.LBM_D3Q19, prec, _phys(has_h, has_g), [case])
        self.solid, self.abi_links = solid, to_abi_links(links)
        self.gpu.set_walls(0, solid, self.abi_links)
        if fields:
            self.gpu.init_equilibrium(0, rho=f.get("rho"), u=f.get("u"), C=f.get("C"), B=f.get("B"))
        self.has_h, self.has_g = has_h, has_g

    def step(self, n):
        self.orc.step(n)
        self.gpu.step(n)

    def errors(self):
        a, b = self.gpu.moments(0), self.orc.moments()
        fl = self.fluid
        out = {"rho": norm_rel(a["rho"][fl], b["rho"][fl]), "u": norm_rel(a["u"][fl], b["u"][fl])}
        if self.has_h:
            out["C"] = norm_rel(a["C"][fl], b["C"][fl])
        if self.has_g:
            out["B"] = norm_rel(a["B"][fl], b["B"][fl])
        return out


def _random_pair(dim, has_h, has_g, seed, prec=lbm.LBM_FP64, shape=None, variants=False):
    r = IN.rng(seed)
    shape = shape or ((37, 29, 1) if dim == 2 else (13, 11, 9))
    solid = IN.random_solid(r, shape, fill=0.12)
    # given wall values near the bulk state (|B| well below the lattice pressure keeps the case stable)
    phi_range = {O.H: (0.5, 1.5), O.G0: (-0.05, 0.05), O.G0 + 1: (0.25, 0.35), O.G0 + 2: (-0.05, 0.05)}
    links = LK.random_links(dim, shape, solid, r, has_h, has_g, phi_range=phi_range, variants=variants)
    N = shape[0] * shape[1] * shape[2]
    fields = IN.random_fields(r, N, dim, B0=(0.0, 0.3, 0.0))
    accel = (1e-5, -2e-5, 5e-6 if dim == 3 else 0.0)
    return Pair(dim, shape, solid, links, prec=prec, accel=accel, has_h=has_h, has_g=has_g, fields=fields,
                C0=1.0, B0=(0.0, 0.3, 0.0))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("has_h,has_g", [(False, False), (True, False), (False, True), (True, True)])
def test_fp64_random_geometry_all_link_kinds(dim, has_h, has_g):
    """Random solids (ragged against the tile size, with E-solid links), every
    wall-link kind with random d in (0, 1], moving walls, fluxes, body force."""
    p = _random_pair(dim, has_h, has_g, seed=100 + 10 * dim + 2 * has_h + has_g)
    p.step(1)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)
    p.step(39)
    m = p.orc.moments()
    assert np.all(np.abs(m["rho"][p.fluid] - 1.0) < 0.5)          # the case stays well posed
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_comparison_schemes(dim):
    """The paper's comparison schemes (Eq. 15/16 for every d, the simplified
    flux wall of Eq. 33) drawn beside the default kinds on random geometry with
    every field: FP64 parity with the oracle.  Few steps, because Eq. 15/16
    beyond d = 1/2 is unstable by design."""
    p = _random_pair(dim, True, True, seed=300 + dim, variants=True)
    kinds = set(p.abi_links["kind"].tolist())
    assert {lbm.LBM_W_VELOCITY_EQ15, lbm.LBM_W_FLUX_SIMPLIFIED} <= kinds
    p.step(1)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)
    p.step(15)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)


def _open_channel_pair(dim, d, prec=lbm.LBM_FP64, has_h=False, steps_shape=None):
    """Channel open along x (Sec. 5.1): inlet of given velocity, outlet of
    given density (Eq. 42/44), static walls at random distances along y (and z),
    body force, and a concentration with a given inlet value and a zero-gradient
    outlet when has_h."""
    shape = steps_shape or ((45, 14, 1) if dim == 2 else (23, 9, 8))
    walls = {1: (0.3, shape[1] - 1.6)}
    if dim == 3:
        walls[2] = (0.55, shape[2] - 1.1)
    walls[0] = (1 - d, shape[0] - 2 + d)
    U = (0.03, 0.004, -0.002 if dim == 3 else 0.0)
    p = {(0, 0, O.F): dict(kind=O.VELOCITY, u_wall=U), (0, 1, O.F): dict(kind=O.PRESSURE, phi_wall=1.01)}
    for ax in walls:
        if ax != 0:
            p[(ax, 0, O.F)] = dict(kind=O.VELOCITY)
            p[(ax, 1, O.F)] = dict(kind=O.VELOCITY, u_wall=(0.01, 0, 0))
    if has_h:
        p[(0, 0, O.H)] = dict(kind=O.GIVEN, phi_wall=1.5, u_wall=U)
        p[(0, 1, O.H)] = dict(kind=O.NEUMANN_BFL)
        for ax in walls:
            if ax != 0:
                p[(ax, 0, O.H)] = dict(kind=O.FLUX, kappa0=0.002, kappa1=-0.01)
                p[(ax, 1, O.H)] = dict(kind=O.GIVEN, phi_wall=0.8)
    solid = LK.box_solid(shape, walls)
    links = LK.box_links(dim, shape, walls, p, has_h=has_h)
    r = IN.rng(400 + dim)
    N = shape[0] * shape[1] * shape[2]
    fields = IN.random_fields(r, N, dim, B0=(0.0, 0.0, 0.0))
    accel = (2e-5, 0.0, 0.0)
    return Pair(dim, shape, solid, links, prec=prec, accel=accel, has_h=has_h, fields=fields, C0=1.0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("d", [0.3, 0.5, 1.0])
def test_fp64_open_boundaries(dim, d):
    """Given inlet velocity and given outlet pressure (Sec. 5.1, Eq. 41-44):
    FP64 parity with the oracle over 200 steps from a random initial field."""
    p = _open_channel_pair(dim, d)
    assert np.any(p.abi_links["kind"] == lbm.LBM_W_PRESSURE)
    p.step(1)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)
    p.step(199)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)


@pytest.mark.parametrize("prec", [lbm.LBM_FP32, lbm.LBM_FP16S])
def test_open_boundaries_every_launch_variant(prec):
    """The pressure links' velocity extrapolation runs in every launch variant
    with the same arithmetic: variants 1, 2 and 3 (FP32; 16-bit storage, which
    rounds stochastically, has variants 0 and 2) equal variant 0 bit for bit on
    an open 2D channel."""
    ref = _open_channel_pair(2, 0.7, prec=prec).gpu
    ref.set_launch(0, 128, 0)
    ref.step(30)
    want = ref.get_state()
    variants = [(2, dict(nodes_per_thread=2, min_blocks=5))]
    if prec == lbm.LBM_FP32:
        variants += [(1, dict(min_blocks=2)), (3, dict(blocks_per_sm=1, stages=4, min_blocks=2))]
    for variant, kw in variants:
        g = _open_channel_pair(2, 0.7, prec=prec).gpu
        g.set_launch(variant, 256, **kw)
        g.step(30)
        assert np.array_equal(g.get_state(), want), variant


@pytest.mark.parametrize("phys", [lbm.LBM_FLOW | lbm.LBM_MHD, lbm.LBM_FLOW | lbm.LBM_CD])
def test_pressure_kind_is_refused_beside_other_fields(phys):
    """The C ABI refuses given-pressure links in a case with a magnetic field
    or a concentration (the kind belongs to flow-only cases)."""
    shape = (12, 10, 1)
    walls = {1: (0.5, 8.5), 0: (0.5, 10.5)}
    has_h, has_g = bool(phys & lbm.LBM_CD), bool(phys & lbm.LBM_MHD)
    p = {(0, 0, O.F): dict(kind=O.VELOCITY, u_wall=(0.01, 0, 0)), (0, 1, O.F): dict(kind=O.PRESSURE, phi_wall=1.0)}
    fields = [O.H] if has_h else [O.G0, O.G0 + 1]
    for side in (0, 1):
        p[(1, side, O.F)] = dict(kind=O.VELOCITY)
        for fld in fields:
            p[(0, side, fld)] = dict(kind=O.GIVEN, phi_wall=0.0)
            p[(1, side, fld)] = dict(kind=O.GIVEN, phi_wall=0.0)
    solid = LK.box_solid(shape, walls)
    links = to_abi_links(LK.box_links(2, shape, walls, p, has_h=has_h, has_g=has_g))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, phys,
                   [lbm.make_case(shape, 0.8, 0.9, 0.9, (0, 0, 0), 1.0, 1.0, (0, 0, 0))])
    with pytest.raises(lbm.LbmError) as ei:
        g.set_walls(0, solid, links)
    assert ei.value.status == lbm.LBM_EINVAL


def _stokes_geometry(nx, ny, d, U):
    walls = LK.channel_y(2, nx, ny, 1, d, d)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(U, 0, 0))}
    shape = (nx, ny, 1)
    return shape, LK.box_solid(shape, walls), LK.box_links(2, shape, walls, p)


@pytest.mark.parametrize("d", [0.25, 0.5, 1.0])
@pytest.mark.parametrize("graph", [0, 4])
def test_fp64_oscillating_wall(d, graph):
    """Stokes' second problem (Sec. 5.2, Eq. 45): the top wall moves with
    U cos(omega t + phase).  FP64 parity with the oracle over 600 steps (1.5
    periods), stepping eagerly or by graph replays that advance the device
    clock themselves."""
    shape, solid, links = _stokes_geometry(3, 22, d, 0.01)
    p = Pair(2, shape, solid, links)
    omega, phase = 2 * math.pi / 400, 0.4
    p.orc.set_wall_motion(omega, phase)
    p.gpu.set_wall_motion(0, omega, phase)
    if graph:
        p.gpu.set_graph(graph)
    for _ in range(6):
        p.step(100)
        for k, v in p.errors().items():
            assert v < FP64_TOL, (k, v)
    u = p.gpu.moments(0)["u"].reshape(shape[1], shape[0], 3)[1:-1, 0, 0]
    assert np.abs(u).max() > 1e-3                     # the wall did drive the flow


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_wall_motion_random_geometry(dim):
    """Random solids with randomly moving velocity walls (every direction of
    u_wall, both velocity kinds) and static scalar walls, under wall motion and
    graphs: FP64 parity with the oracle."""
    r = IN.rng(500 + dim)
    shape = (29, 23, 1) if dim == 2 else (13, 11, 9)
    solid = IN.random_solid(r, shape, fill=0.12)
    links = LK.random_links(dim, shape, solid, r, has_h=True, kinds=[O.GIVEN, O.NEUMANN_BFL],
                            phi_range={O.H: (0.5, 1.5)})
    links["kind"][(links["field"] == O.F) & (links["d"] < 0.5)] = O.VELOCITY_EQ15
    fields = IN.random_fields(r, shape[0] * shape[1] * shape[2], dim)
    p = Pair(dim, shape, solid, links, accel=(1e-5, 0, 0), has_h=True, fields=fields)
    p.orc.set_wall_motion(0.05, -1.0)
    p.gpu.set_wall_motion(0, 0.05, -1.0)
    p.gpu.set_graph(2)
    p.step(40)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)


def test_fp64_wall_motion_per_case():
    """One launch over three cases: two oscillate at different frequencies and
    phases, one keeps its steady moving wall.  Each matches its own oracle."""
    geo = [_stokes_geometry(2, ny, d, 0.01) for ny, d in ((14, 0.5), (19, 0.75), (11, 0.3))]
    motion = [(2 * math.pi / 150, 0.0), None, (2 * math.pi / 70, 1.2)]
    cases = [lbm.make_case(g[0], 0.8, 0.9, 0.7, (0, 0, 0), 1.0, 1.0, (0, 0, 0)) for g in geo]
    gpu = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW, cases)
    orcs = []
    for i, (shape, solid, links) in enumerate(geo):
        gpu.set_walls(i, solid, to_abi_links(links))
        o = O.OracleSim(2, shape, solid, 0.8)
        o.set_links(links)
        o.init()
        if motion[i]:
            o.set_wall_motion(*motion[i])
        orcs.append(o)
    for i, m in enumerate(motion):
        if m:
            gpu.set_wall_motion(i, *m)
    gpu.set_graph(4)
    gpu.step(300)
    for i, o in enumerate(orcs):
        o.step(300)
        fl = np.asarray(geo[i][1]).reshape(-1) == 0
        a, b = gpu.moments(i), o.moments()
        assert norm_rel(a["u"][fl], b["u"][fl]) < FP64_TOL
        assert norm_rel(a["rho"][fl], b["rho"][fl]) < FP64_TOL


def test_fp64_wall_motion_set_late_keeps_other_phases():
    """Case 0 oscillates from step 0; case 1's motion is set only after 70
    steps (its own t starts there).  Each matches an oracle whose motion was
    set at the same step: setting one case's motion leaves the other's phase
    alone."""
    geo = [_stokes_geometry(2, ny, d, 0.01) for ny, d in ((14, 0.5), (17, 0.8))]
    motion = [(2 * math.pi / 150, 0.3), (2 * math.pi / 90, -0.7)]
    cases = [lbm.make_case(g[0], 0.8, 0.9, 0.7, (0, 0, 0), 1.0, 1.0, (0, 0, 0)) for g in geo]
    gpu = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW, cases)
    orcs = []
    for i, (shape, solid, links) in enumerate(geo):
        gpu.set_walls(i, solid, to_abi_links(links))
        o = O.OracleSim(2, shape, solid, 0.8)
        o.set_links(links)
        o.init()
        orcs.append(o)
    orcs[0].set_wall_motion(*motion[0])
    gpu.set_wall_motion(0, *motion[0])
    gpu.set_graph(4)
    gpu.step(70)
    for o in orcs:
        o.step(70)
    orcs[1].set_wall_motion(*motion[1])
    gpu.set_wall_motion(1, *motion[1])
    gpu.step(200)
    for i, o in enumerate(orcs):
        o.step(200)
        fl = np.asarray(geo[i][1]).reshape(-1) == 0
        a, b = gpu.moments(i), o.moments()
        assert norm_rel(a["u"][fl], b["u"][fl]) < FP64_TOL, i


@pytest.mark.parametrize("graph", [0, 4])
def test_checkpoint_of_an_oscillating_wall_is_bitwise(graph):
    """A state blob taken mid-period and restored into a fresh context with the
    same walls (whose motion comes from the blob alone), then stepped, equals
    the run that never stopped, bit for bit (FP64), and so does a conversion
    into a second FP64 context."""
    shape, solid, links = _stokes_geometry(3, 22, 0.75, 0.01)
    omega, phase = 2 * math.pi / 130, 0.4

    def make():
        g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW,
                       [lbm.make_case(shape, 0.8, 0.9, 0.7, (1e-6, 0, 0), 1.0, 1.0, (0, 0, 0))])
        g.set_walls(0, solid, to_abi_links(links))
        if graph:
            g.set_graph(graph)
        return g
    a = make()
    a.step(12)                       # motion set at step 12: its t starts there
    a.set_wall_motion(0, omega, phase)
    a.step(52)
    blob = a.get_state()
    a.step(96)
    want = a.get_state()
    b = make()
    b.set_state(blob)
    b.step(96)
    assert b.steps == a.steps
    assert np.array_equal(b.get_state(), want)
    c = make()
    b2 = make()
    b2.set_state(blob)
    c.convert_from(b2)
    c.step(96)
    assert np.array_equal(c.get_state(), want)


def test_wall_motion_refuses_moving_flux_walls():
    """A case with a flux wall of h whose wall moves is refused, and so is a
    later link list with such a wall in a moving case."""
    walls = LK.channel_y(2, 1, 10, 1, 0.5, 0.5)
    shape = (1, 10, 1)
    solid = LK.box_solid(shape, walls)

    def links(u):
        p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(0.01, 0, 0)),
             (1, 0, O.H): dict(kind=O.GIVEN, phi_wall=1.0), (1, 1, O.H): dict(kind=O.FLUX, u_wall=(u, 0, 0))}
        return to_abi_links(LK.box_links(2, shape, walls, p, has_h=True))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW | lbm.LBM_CD,
                   [lbm.make_case(shape, 0.8, 0.9, 0.7, (0, 0, 0), 1.0, 1.0, (0, 0, 0))])
    g.set_walls(0, solid, links(0.01))
    with pytest.raises(lbm.LbmError) as ei:
        g.set_wall_motion(0, 1e-3)
    assert ei.value.status == lbm.LBM_EINVAL
    g.set_walls(0, solid, links(0.0))
    g.set_wall_motion(0, 1e-3)
    with pytest.raises(lbm.LbmError) as ei:
        g.set_walls(0, solid, links(0.01))
    assert ei.value.status == lbm.LBM_EINVAL


def test_fp64_poiseuille_64x32_5000_steps():
    """Body-force channel, 64 x 32 nodes, tau = 0.8, half-grid walls, 5000
    steps: the GPU matches the oracle and both match the analytic parabola to
    the scheme's O(dx^2) slip."""
    from oracle import analytic as AN
    nx, ny, a = 64, 32, 1e-5          # steady u_max = a (2H)^2 / (8 nu) ~ 0.011
    walls = LK.channel_y(2, nx, ny, 1, 0.5, 0.5)
    solid = LK.box_solid((nx, ny, 1), walls)
    links = LK.box_links(2, (nx, ny, 1), walls, {(1, 0, O.F): dict(kind=O.VELOCITY),
                                                  (1, 1, O.F): dict(kind=O.VELOCITY)})
    p = Pair(2, (nx, ny, 1), solid, links, accel=(a, 0, 0))
    p.step(5000)
    e = p.errors()
    assert e["u"] < FP64_TOL and e["rho"] < FP64_TOL
    u = p.gpu.moments(0)["u"][:, 0].reshape(ny, nx)[1:-1, 0]
    ua = AN.poiseuille(np.arange(ny)[1:-1], walls[1][0], walls[1][1], a, 0.1)
    # 5000 steps is about 0.5 H^2/nu: the profile is still developing; its shape is parabolic
    c = np.polyfit(np.arange(ny)[1:-1], u, 2)
    assert np.abs(u - np.polyval(c, np.arange(ny)[1:-1])).max() < 0.05 * u.max()
    assert 0.1 < u.max() / ua.max() < 1.0


def _hartmann_links(W, q, cw, Ha, tau=0.8, taue=0.9):
    nu, eta = (tau - 0.5) / 3, (taue - 0.5) / 4
    d = 1.0 - q
    ny = W + 2
    walls = LK.channel_y(2, W, ny, 1, d, d)
    H = (walls[1][1] - walls[1][0]) / 2
    B0 = Ha * math.sqrt(nu * eta) / H
    b1 = dict(kind=O.FLUX, kappa1=-eta / (cw * H))
    p = {(1, s, O.F): dict(kind=O.VELOCITY) for s in (0, 1)}
    p.update({(1, s, O.G0): b1 for s in (0, 1)})
    p.update({(1, s, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0) for s in (0, 1)})
    shape = (W, ny, 1)
    return shape, LK.box_solid(shape, walls), LK.box_links(2, shape, walls, p, has_g=True), B0


def test_fp64_batched_uneven_cases():
    """Several uneven Hartmann channels (different width, Ha, q, c_w) advanced
    by one launch per step; each matches its own oracle run."""
    draws = [dict(W=20, q=0.3, cw=0.05, Ha=4.0), dict(W=33, q=0.0, cw=1.0, Ha=12.0),
             dict(W=9, q=0.75, cw=0.5, Ha=1.5), dict(W=64, q=0.5, cw=0.2, Ha=25.0)]
    cases, orcs, geo = [], [], []
    for i, dr in enumerate(draws):
        shape, solid, links, B0 = _hartmann_links(dr["W"], dr["q"], dr["cw"], dr["Ha"])
        H = (dr["W"] - 1 + 2 * (1 - dr["q"])) / 2
        acc = (0.02 * 0.1 * (2 + dr["Ha"]) / H ** 2, 0.0, 0.0)      # u ~ 0.01 at steady state
        o = O.OracleSim(2, shape, solid, 0.8, 1.0, 0.9, acc, False, True, 4)
        o.set_links(links)
        o.init(B0=(0, B0, 0))
        orcs.append(o)
        cases.append(lbm.make_case(shape, 0.8, 1.0, 0.9, acc, 1.0, 0.0, (0, B0, 0)))
        geo.append((solid, links))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW | lbm.LBM_MHD, cases)
    for i, (solid, links) in enumerate(geo):
        g.set_walls(i, solid, to_abi_links(links))
    g.set_graph(4)
    g.step(60)
    for o in orcs:
        o.step(60)
    for i, o in enumerate(orcs):
        a, b = g.moments(i), o.moments()
        fl = geo[i][0].reshape(-1) == 0
        assert norm_rel(a["u"][fl], b["u"][fl]) < FP64_TOL
        assert norm_rel(a["B"][fl], b["B"][fl]) < FP64_TOL


def test_checkpoint_restore_and_graph_are_bitwise():
    """2N steps equal N + save + restore (fresh context) + N, and graph replay
    equals plain launches, bit for bit (FP32)."""
    def make():
        p = _random_pair(2, True, True, seed=7, prec=lbm.LBM_FP32)
        return p.gpu
    a = make()
    a.step(24)
    ref = a.get_state()
    b = make()
    b.step(12)
    blob = b.get_state()
    c = make()
    c.set_state(blob)
    c.step(12)
    assert np.array_equal(c.get_state()[16:], ref[16:])
    d = make()
    d.set_graph(4)
    d.step(24)
    assert np.array_equal(d.get_state()[16:], ref[16:])
    assert d.steps == 24


def test_fp64_reductions_match_oracle():
    """lbm_check: FP64 sums of rho, C and B over fluid nodes match the oracle;
    the residual numerator is the squared change of (u, C, B - B0)."""
    p = _random_pair(3, True, True, seed=31)
    p.gpu.check()
    p.step(5)
    out = p.gpu.check()[0]
    s = p.orc.sums()
    assert abs(out[0] - s[0]) < 1e-12 * abs(s[0])
    assert abs(out[1] - s[1]) < 1e-12 * abs(s[1])
    assert np.abs(out[2:5] - s[2:5]).max() < 1e-11 * max(1.0, np.abs(s[2:5]).max())
    assert out[5] == 0
    m0 = p.orc.moments()
    p.step(3)
    out = p.gpu.check()[0]
    m1 = p.orc.moments()
    fl = p.fluid
    phi0 = np.concatenate([m0["u"][fl], m0["C"][fl, None], m0["B"][fl] - [0, 0.3, 0]], axis=1)
    phi1 = np.concatenate([m1["u"][fl], m1["C"][fl, None], m1["B"][fl] - [0, 0.3, 0]], axis=1)
    assert abs(out[6] - np.sum((phi1 - phi0) ** 2)) < 1e-9 * np.sum((phi1 - phi0) ** 2)
    assert abs(out[7] - np.sum(phi1 ** 2)) < 1e-12 * np.sum(phi1 ** 2)


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_FP32])
def test_async_check_returns_the_check_record(prec):
    """lbm_check_async + lbm_check_wait give the record lbm_check gives for the
    same state, bit for bit, although more steps were enqueued behind the
    check before its result was collected; one check may be in flight."""
    a = _random_pair(2, True, True, seed=61, prec=prec).gpu
    b = _random_pair(2, True, True, seed=61, prec=prec).gpu
    a.step(20)
    b.step(20)
    want = a.check(raise_unstable=False)
    b.check_async()
    with pytest.raises(lbm.LbmError) as ei:
        b.check_async()
    assert ei.value.status == lbm.LBM_ESTATE
    with pytest.raises(lbm.LbmError) as ei:
        b.check()
    assert ei.value.status == lbm.LBM_ESTATE
    b.step(10)
    got = b.check_wait(raise_unstable=False)
    assert np.array_equal(got, want)
    with pytest.raises(lbm.LbmError) as ei:
        b.check_wait()
    assert ei.value.status == lbm.LBM_ESTATE
    a.step(10)
    assert np.array_equal(a.check(raise_unstable=False), b.check(raise_unstable=False))


def test_nonfinite_population_is_reported():
    """A NaN planted in the initial field is found by the FP64 check
    (LBM_EUNSTABLE) without any device fault."""
    shape, solid, links, B0 = _hartmann_links(16, 0.5, 0.5, 3.0)
    case = lbm.make_case(shape, 0.8, 1.0, 0.9, (0, 0, 0), 1.0, 0.0, (0, B0, 0))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, [case])
    g.set_walls(0, solid, to_abi_links(links))
    N = shape[0] * shape[1]
    rho = np.ones(N)
    rho[N // 2] = np.nan
    g.init_equilibrium(0, rho=rho)
    g.step(3)
    with pytest.raises(lbm.LbmError) as ei:
        g.check()
    assert ei.value.status == lbm.LBM_EUNSTABLE
    out = g.check(raise_unstable=False)
    assert out[0, 5] > 0


def test_invalid_link_lists_are_rejected():
    shape, solid, links, B0 = _hartmann_links(10, 0.5, 0.5, 3.0)
    case = lbm.make_case(shape, 0.8, 1.0, 0.9, (0, 0, 0), 1.0, 0.0, (0, B0, 0))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, [case])
    good = to_abi_links(links)
    bad = []
    x = good.copy(); x["d"][3] = 0.0; bad.append(x)                    # d outside (0, 1]
    x = good.copy(); x["d"][3] = 1.5; bad.append(x)
    bad.append(good[1:])                                                # missing link
    bad.append(np.concatenate([good, good[:1]]))                        # duplicate
    x = good.copy(); x["kind"][np.flatnonzero(good["field"] == 0)[0]] = lbm.LBM_W_GIVEN; bad.append(x)
    x = good.copy(); x["node"][0] = 0; bad.append(x)                    # node 0 is solid
    x = good.copy(); x["field"][0] = 1; bad.append(x)                   # CD not enabled
    for b in bad:
        with pytest.raises(lbm.LbmError) as ei:
            g.set_walls(0, solid, b)
        assert ei.value.status == lbm.LBM_EINVAL
    g.set_walls(0, solid, good)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW, [lbm.make_case((8, 8, 1), 0.5)])


def test_fully_periodic_domain_and_single_node_axes():
    """No walls at all (empty link list) and nx = 1 axes: the step reduces to
    the bulk update; FP64 parity with the oracle."""
    for shape in ((1, 17, 1), (5, 1, 1)):
        N = shape[0] * shape[1]
        r = IN.rng(5)
        solid = np.zeros(N, dtype=np.uint8)
        fields = IN.random_fields(r, N, 2)
        p = Pair(2, shape, solid, np.zeros(0, O.LINK_DTYPE), accel=(1e-5, 0, 0), has_h=True, fields=fields)
        p.step(25)
        for k, v in p.errors().items():
            assert v < FP64_TOL, (shape, k, v)


@pytest.mark.parametrize("dim,prec", [(2, lbm.LBM_FP32), (3, lbm.LBM_FP32)])
def test_bulk_copy_pipeline_is_bitwise_identical(dim, prec):
    """The shared-memory pipeline (variant 1: cp.async.bulk windows + mbarrier)
    computes exactly what the one-thread-per-node kernel computes, for several
    tile sizes that leave ragged tails and put periodic edges inside tiles."""
    shape = (53, 41, 1) if dim == 2 else (21, 13, 11)
    ref = _random_pair(dim, True, True, seed=77, prec=prec, shape=shape).gpu
    ref.set_launch(0, 128, 0)
    ref.step(15)
    want = ref.get_state()
    ran = 0
    for block, minb in ((128, 2), (256, 2), (256, 4), (512, 1), (512, 2)):
        g = _random_pair(dim, True, True, seed=77, prec=prec, shape=shape).gpu
        try:
            g.set_launch(1, block, min_blocks=minb)
        except lbm.LbmError as e:      # the tiles of this shape do not fit in shared memory
            assert e.status == lbm.LBM_EINVAL and "shared memory" in str(e)
            continue
        g.set_graph(4)
        g.step(15)
        assert np.array_equal(g.get_state(), want), (block, minb)
        g.check()
        ran += 1
    assert ran >= (1 if (dim == 3 and prec == lbm.LBM_FP32) else 3)   # 40 FP32 planes: only 128-node tiles fit


def test_bulk_copy_pipeline_batched_cases():
    """Variant 1 over many uneven cases equals variant 0 bit for bit (FP32:
    the variant rounds to nearest, 16-bit storage rounds stochastically)."""
    def make():
        cases, geo = [], []
        for i, (W, q) in enumerate(((20, 0.3), (33, 0.0), (9, 0.75), (64, 0.5), (130, 0.9))):
            shape, solid, links, B0 = _hartmann_links(W, q, 0.3, 5.0)
            cases.append(lbm.make_case(shape, 0.8, 1.0, 0.9, (2e-5, 0, 0), 1.0, 0.0, (0, B0, 0)))
            geo.append((solid, links))
        g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, cases)
        for i, (solid, links) in enumerate(geo):
            g.set_walls(i, solid, to_abi_links(links))
        return g
    a = make()
    a.set_launch(0, 256, 4)
    a.step(30)
    b = make()
    b.set_launch(1, 256, min_blocks=2)
    b.step(30)
    assert np.array_equal(a.get_state(), b.get_state())


def test_autotune_keeps_solution():
    p = _random_pair(3, False, True, seed=9, prec=lbm.LBM_FP32, shape=(24, 20, 18))
    p.gpu.step(3)
    before = p.gpu.get_state()
    lp, ms = p.gpu.autotune(None, iters=3)
    assert lp.variant in (0, 1, 2) and lp.block in (64, 128, 192, 256, 512) and ms > 0
    after = p.gpu.get_state()
    assert np.array_equal(before, after)
    p.gpu.step(2)   # still runs with the chosen launch shape


@pytest.mark.parametrize("launch", [(0, 128, 0, 1, 2, 1), (0, 256, 0, 4, 2, 1), (0, 128, 8, 2, 2, 1)])
def test_reductions_any_launch_shape(launch):
    """Every node of a tile enters the sums whatever the tile size (tiles of
    up to 1024 nodes are reduced by 256-thread blocks): FP32 storage against
    the FP64 oracle, sums at FP32 rounding of the per-node values."""
    p = _random_pair(2, True, True, seed=37, prec=lbm.LBM_FP32, shape=(61, 47, 1))
    p.gpu.set_launch(*launch)
    p.step(6)
    out = p.gpu.check()[0]
    s = p.orc.sums()
    assert abs(out[0] - s[0]) < 1e-6 * abs(s[0])
    assert abs(out[1] - s[1]) < 1e-6 * abs(s[1])
    assert np.abs(out[2:4] - s[2:4]).max() < 1e-5 * max(1.0, np.abs(s[2:4]).max())
    assert out[5] == 0
    m = p.orc.moments()
    fl = p.fluid
    phi = np.concatenate([m["u"][fl, :2], m["C"][fl, None], m["B"][fl, :2] - [0, 0.3]], axis=1)
    assert abs(out[7] - np.sum(phi ** 2)) < 1e-5 * np.sum(phi ** 2)


@pytest.mark.parametrize("dim", [2, 3])
def test_register_budgets_are_bitwise_identical(dim):
    """The step compiled for each register budget (launch min_blocks) gives
    the same state bit for bit."""
    from paper_2506_00907_gb300.lbm import lib  # noqa: F401  (library loaded)
    base = 4 if dim == 2 else 2
    states = []
    for mb in (base, base + 1, base + 2):
        p = _random_pair(dim, True, True, seed=53 + dim, prec=lbm.LBM_FP32)
        p.gpu.set_launch(0, 128, 0, 2, 2, mb)
        p.gpu.step(12)
        states.append(p.gpu.get_state()[16:])
    assert np.array_equal(states[0], states[1]) and np.array_equal(states[0], states[2])


@pytest.mark.parametrize("dim,prec,shape", [
    (2, lbm.LBM_FP16S, (53, 41, 1)), (2, lbm.LBM_BF16S, (52, 41, 1)), (2, lbm.LBM_FP32, (36, 30, 1)),
    (2, lbm.LBM_FP64, (31, 22, 1)), (3, lbm.LBM_FP16S, (21, 13, 11)), (3, lbm.LBM_BF16S, (20, 13, 11)),
    (3, lbm.LBM_FP32, (22, 14, 9))])
def test_unwrapped_pulls_are_bitwise_identical(dim, prec, shape):
    """Variant 2 (pulls read unwrapped from the node's own address plus a
    per-case constant, edge nodes reloading their wrapped planes, 16-bit
    values kept packed) computes exactly what variant 0 computes: ragged
    tails, periodic edges, solid blobs and every link kind, every register
    budget."""
    ref = _random_pair(dim, True, True, seed=91, prec=prec, shape=shape).gpu
    ref.set_launch(0, 128, 0)
    ref.step(15)
    want = ref.get_state()
    lo = 4 if dim == 2 else 2
    for block, npt, mb in ((128, 2, lo), (256, 4, lo + 1), (64, 8, lo + 2)):
        g = _random_pair(dim, True, True, seed=91, prec=prec, shape=shape).gpu
        g.set_launch(2, block, 0, npt, 2, mb)
        g.set_graph(4)
        g.step(15)
        assert np.array_equal(g.get_state(), want), (block, npt, mb)
        g.check()


@pytest.mark.parametrize("dim,prec,shape", [
    (2, lbm.LBM_FP16S, (1, 37, 1)), (2, lbm.LBM_FP16S, (3, 29, 1)), (2, lbm.LBM_BF16S, (40, 27, 1)),
    (2, lbm.LBM_FP16S, (65, 8, 1)), (3, lbm.LBM_FP16S, (1, 9, 11)), (3, lbm.LBM_FP16S, (7, 5, 6)),
    (3, lbm.LBM_BF16S, (12, 9, 7)), (2, lbm.LBM_FP32, (3, 29, 1)), (3, lbm.LBM_FP32, (7, 5, 6))])
def test_fully_periodic_boxes_every_variant_bitwise(dim, prec, shape):
    """A box without walls, periodic along every axis, from random fields:
    every bulk node wraps somewhere (x, y and z edges; odd and even nx; nx = 1,
    where a node pair straddles two rows).  Every launch variant gives the
    bits of the one-node step, which matches the FP64 oracle in FP64
    (test_fully_periodic_domain_and_single_node_axes)."""
    N = shape[0] * shape[1] * shape[2]
    phys = lbm.LBM_FLOW | lbm.LBM_CD | lbm.LBM_MHD
    lat = lbm.LBM_D2Q9 if dim == 2 else lbm.LBM_D3Q19
    f = IN.random_fields(IN.rng(41 + dim), N, dim, B0=(0.0, 0.3, 0.0))

    def run(launch):
        g = lbm.Solver(lat, prec, phys, [lbm.make_case(shape, 0.8, 0.9, 0.7, (1e-5, -2e-5, 0), 1.0, 1.0,
                                                       (0, 0.3, 0))])
        g.init_equilibrium(0, rho=f["rho"], u=f["u"], C=f["C"], B=f["B"])
        g.set_launch(*launch)
        g.step(9)
        return g.get_state()
    want = run((0, 128, 0, 1, 2, 1))
    lo = 4 if dim == 2 else 2
    launches = [(0, 64, 0, 3, 2, 1), (2, 128, 0, 2, 2, 1), (2, 64, 0, 8, 2, lo + 1)]
    if prec == lbm.LBM_FP32:                  # the bulk-copy variant rounds to nearest only
        launches.append((1, 256 if dim == 2 else 128, 0, 1, 2, 2))
    for launch in launches:
        assert np.array_equal(run(launch), want), launch


def test_unwrapped_pulls_batched_cases_and_flow_only():
    """Variant 2 over uneven batched cases (odd widths, empty-link cases) and
    for a flow-only D2Q9 lattice equals variant 0 bit for bit."""
    def make(phys):
        cases, geo = [], []
        for W, q in ((20, 0.3), (33, 0.0), (9, 0.75), (64, 0.5), (131, 0.9)):
            shape, solid, links, B0 = _hartmann_links(W, q, 0.3, 5.0)
            if not phys & lbm.LBM_MHD:
                links = links[links["field"] == O.F]
            cases.append(lbm.make_case(shape, 0.8, 1.0, 0.9, (2e-5, 0, 0), 1.0, 0.0, (0, B0, 0)))
            geo.append((solid, links))
        g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_BF16S, phys, cases)
        for i, (solid, links) in enumerate(geo):
            g.set_walls(i, solid, to_abi_links(links))
        return g
    for phys in (lbm.LBM_FLOW | lbm.LBM_MHD, lbm.LBM_FLOW):
        a = make(phys)
        a.set_launch(0, 256, 4)
        a.step(30)
        b = make(phys)
        b.set_launch(2, 128, 0, 3, 2, 5)
        b.step(30)
        assert np.array_equal(a.get_state(), b.get_state()), phys


def test_unwrapped_pulls_reject_bad_shapes():
    q = _random_pair(2, False, False, seed=5, prec=lbm.LBM_FP16S)
    for bad in ((2, 128, 0, 3, 2, 3), (2, 128, 0, 9, 2, 4), (2, 96 + 1, 0, 2, 2, 4), (2, 128, 65, 2, 2, 4)):
        with pytest.raises(lbm.LbmError):
            q.gpu.set_launch(*bad)


def _random_gpu(dim, shape, prec, seed, phys=lbm.LBM_FLOW | lbm.LBM_CD | lbm.LBM_MHD):
    """A GPU solver on a random geometry with every link kind (no oracle:
    for bitwise comparisons between launch variants at larger sizes)."""
    r = IN.rng(seed)
    has_h, has_g = bool(phys & lbm.LBM_CD), bool(phys & lbm.LBM_MHD)
    solid = IN.random_solid(r, shape, fill=0.12)
    phi_range = {O.H: (0.5, 1.5), O.G0: (-0.05, 0.05), O.G0 + 1: (0.25, 0.35), O.G0 + 2: (-0.05, 0.05)}
    links = LK.random_links(dim, shape, solid, r, has_h, has_g, phi_range=phi_range)
    N = shape[0] * shape[1] * shape[2]
    f = IN.random_fields(r, N, dim, B0=(0.0, 0.3, 0.0))
    case = lbm.make_case(shape, 0.8, 0.9, 0.7, (1e-5, -2e-5, 5e-6 if dim == 3 else 0.0), 1.0, 1.0, (0.0, 0.3, 0.0))
    g = lbm.Solver(lbm.LBM_D2Q9 if dim == 2 else lbm.LBM_D3Q19, prec, phys, [case])
    g.set_walls(0, solid, to_abi_links(links))
    g.init_equilibrium(0, rho=f.get("rho"), u=f.get("u"), C=f.get("C") if has_h else None,
                       B=f.get("B") if has_g else None)
    return g


def _ring_runs(make, steps, want):
    ran = 0
    for ns, bps in ((2, 1), (3, 0), (4, 1), (8, 0)):
        g = make()
        try:
            g.set_launch(3, 256, bps, 1, ns, 2)
        except lbm.LbmError as e:      # these stages do not fit in shared memory
            assert e.status == lbm.LBM_EINVAL and "shared memory" in str(e)
            continue
        g.set_graph(4)
        g.step(steps)
        assert np.array_equal(g.get_state(), want), (ns, bps)
        g.check()
        ran += 1
    return ran


@pytest.mark.parametrize("dim,prec,shape", [
    (2, lbm.LBM_FP32, (53, 41, 1)), (2, lbm.LBM_FP32, (52, 41, 1)), (2, lbm.LBM_FP32, (37, 30, 1)),
    (3, lbm.LBM_FP32, (21, 13, 11)), (3, lbm.LBM_FP32, (22, 14, 9))])
def test_ring_pipeline_is_bitwise_identical(dim, prec, shape):
    """Variant 3 (producer warp filling a ring of shared-memory stages with
    cp.async.bulk windows, consumer warps relaxing from it; packed node pairs
    in 2D) computes exactly what one thread per node computes: odd and even
    nx, ragged tails, periodic edges, every link kind, 2..8 stages."""
    ref = _random_pair(dim, True, True, seed=93, prec=prec, shape=shape).gpu
    ref.set_launch(0, 128, 0)
    ref.step(15)
    want = ref.get_state()
    ran = _ring_runs(lambda: _random_pair(dim, True, True, seed=93, prec=prec, shape=shape).gpu, 15, want)
    assert ran >= (1 if prec == lbm.LBM_FP32 else 2)     # FP32 tiles of 24-47 planes fit few stages


@pytest.mark.parametrize("dim,prec,shape,phys", [
    (2, lbm.LBM_FP32, (701, 523, 1), lbm.LBM_FLOW | lbm.LBM_MHD),
    (2, lbm.LBM_FP32, (640, 480, 1), lbm.LBM_FLOW),
    (3, lbm.LBM_FP32, (97, 61, 53), lbm.LBM_FLOW | lbm.LBM_CD | lbm.LBM_MHD),
    (3, lbm.LBM_FP32, (64, 48, 40), lbm.LBM_FLOW | lbm.LBM_MHD)])
def test_ring_pipeline_wraps_many_tiles(dim, prec, shape, phys):
    """Many more tiles than resident blocks: each block's ring of stages
    wraps many times (mbarrier phases flip), still bit for bit."""
    ref = _random_gpu(dim, shape, prec, 17, phys)
    ref.set_launch(0, 128, 0)
    ref.step(6)
    want = ref.get_state()
    assert _ring_runs(lambda: _random_gpu(dim, shape, prec, 17, phys), 6, want) >= (1 if prec == lbm.LBM_FP32 else 2)


def test_ring_pipeline_batched_cases():
    """Variant 3 over uneven batched Hartmann channels (tiles of one block in
    different cases) equals variant 0 bit for bit."""
    def make():
        cases, geo = [], []
        for W, q in ((20, 0.3), (33, 0.0), (9, 0.75), (64, 0.5), (131, 0.9), (300, 0.2)):
            shape, solid, links, B0 = _hartmann_links(W, q, 0.3, 5.0)
            cases.append(lbm.make_case(shape, 0.8, 1.0, 0.9, (2e-5, 0, 0), 1.0, 0.0, (0, B0, 0)))
            geo.append((solid, links))
        g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, cases)
        for i, (solid, links) in enumerate(geo):
            g.set_walls(i, solid, to_abi_links(links))
        return g
    a = make()
    a.set_launch(0, 256, 4)
    a.step(30)
    want = a.get_state()
    assert _ring_runs(make, 30, want) >= 1


def test_ring_rejects_fp64_16bit_and_bad_stages():
    p = _random_pair(2, False, False, seed=5)
    with pytest.raises(lbm.LbmError):
        p.gpu.set_launch(3, 256, 0, 1, 3, 2)       # FP64 storage
    q = _random_pair(2, False, False, seed=5, prec=lbm.LBM_FP32)
    for bad in ((3, 256, 0, 1, 1, 2), (3, 256, 0, 1, 9, 2)):
        with pytest.raises(lbm.LbmError):
            q.gpu.set_launch(*bad)
    for prec in (lbm.LBM_BF16S, lbm.LBM_FP16S):    # 16-bit storage rounds stochastically: variants 0 and 2
        r = _random_pair(2, False, False, seed=5, prec=prec)
        for bad in ((3, 256, 0, 1, 3, 2), (1, 256, 0, 1, 2, 2)):
            with pytest.raises(lbm.LbmError):
                r.gpu.set_launch(*bad)
