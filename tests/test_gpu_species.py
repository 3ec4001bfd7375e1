"""Several concentration species with surface reactions between them, on the
GPU through the C ABI, against the FP64 oracle (Sec. 4.2.2, text after
Eq. 23: each species' C_i(X) by Eq. 13, the reaction fluxes F_i(C_1, C_2, ..)
evaluated explicitly and added to their own species by the M scheme).

FP64 storage must match the oracle within 1e-12 norm-relative per field; the
other storages run the same kernels' arithmetic and are compared bit for bit
across launch shapes.  Links come from the oracle's builder."""
import numpy as np
import pytest

import oracle as O
from oracle import analytic as AN
from oracle import links as LK
from paper_2506_00907_gb300 import inputs as IN
from paper_2506_00907_gb300 import lbm
from tests.helpers import norm_rel, to_abi_links

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
CD = lbm.LBM_FLOW | lbm.LBM_CD
TAUS = (0.9, 0.7, 1.1)
C0S = (1.0, 0.6, 0.3)


def _network(r, nc):
    """A random mass-action network: 2 or 3 reactions, orders 0..2, moderate
    rates so that the fluxes stay small against the populations."""
    out = []
    for _ in range(int(r.integers(2, 4))):
        order = [int(v) for v in r.integers(0, 3, nc)]
        stoich = [float(v) for v in r.uniform(-1.0, 1.0, nc)]
        out.append(dict(rate=float(r.uniform(0.002, 0.02)), order=order, stoich=stoich))
    return out


class SpeciesPair:
    """The same multi-species case on the oracle and on the GPU."""

    def __init__(self, dim, nc, seed, prec=lbm.LBM_FP64, shape=None, launch=None):
        r = IN.rng(seed)
        self.shape = shape or ((33, 27, 1) if dim == 2 else (12, 11, 9))
        N = self.shape[0] * self.shape[1] * self.shape[2]
        solid = IN.random_solid(r, self.shape, fill=0.12)
        phi_range = {O.species_field(k): (0.4, 1.4) for k in range(nc)}
        links = LK.random_links(dim, self.shape, solid, r, has_h=True, phi_range=phi_range, nspecies=nc,
                                reaction=True)
        net = _network(r, nc)
        fields = IN.random_fields(r, N, dim)
        accel = (1e-5, -2e-5, 5e-6 if dim == 3 else 0.0)
        self.nc, self.fluid = nc, np.asarray(solid).reshape(-1) == 0
        self.orc = O.OracleSim(dim, self.shape, solid, 0.8, TAUS[0], 1.0, accel, True, False, 8)
        self.orc.set_species(list(TAUS[:nc]), list(C0S[:nc]))
        self.orc.set_network(net)
        self.orc.set_links(links)
        self.orc.init(rho=fields["rho"], u=fields["u"], C=fields["C"], C0=C0S[0])
        case = lbm.make_case(self.shape, 0.8, TAUS[0], 1.0, accel, 1.0, C0S[0], (0, 0, 0), tau_Dk=TAUS[1:],
                             C0k=C0S[1:])
        self.gpu = lbm.Solver(lbm.LBM_D2Q9 if dim == 2 else lbm.LBM_D3Q19, prec, CD, [case], nspecies=nc)
        self.links = to_abi_links(links)
        self.gpu.set_walls(0, solid, self.links)
        self.gpu.set_reactions(0, net)
        if launch:
            self.gpu.set_launch(*launch)
        self.gpu.init_equilibrium(0, rho=fields["rho"], u=fields["u"], C=fields["C"])

    def step(self, n):
        self.orc.step(n)
        self.gpu.step(n)

    def errors(self):
        fl = self.fluid
        a, b = self.gpu.moments(0), self.orc.moments()
        out = {"rho": norm_rel(a["rho"][fl], b["rho"][fl]), "u": norm_rel(a["u"][fl], b["u"][fl])}
        for k in range(self.nc):
            out["C%d" % k] = norm_rel(self.gpu.species(k)[fl], self.orc.species(k)[fl])
        return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("nc", [2, 3])
def test_fp64_species_random_geometry(dim, nc):
    """Random solids, every concentration link kind with random d in (0, 1]
    including reaction links of a random network (orders 0..2), moving walls,
    body force, random initial fields: FP64 parity with the oracle for every
    species."""
    p = SpeciesPair(dim, nc, seed=700 + 10 * dim + nc)
    assert np.any(p.links["kind"] == lbm.LBM_W_REACTION)
    p.step(1)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)
    p.step(39)
    for k, v in p.errors().items():
        assert v < FP64_TOL, (k, v)


def test_fp64_species_sums_in_the_check_record():
    """lbm_check with several species: slot 1 is sum C_0 and slots 2-3 the
    sums of the further species, equal to the oracle's sums."""
    p = SpeciesPair(2, 3, seed=9)
    p.step(25)
    out = p.gpu.check()[0]
    fl = p.fluid
    for k, slot in ((0, 1), (1, 2), (2, 3)):
        want = p.orc.species(k)[fl].sum()
        assert abs(out[slot] - want) <= 1e-12 * abs(want), (k, out[slot], want)
    assert out[5] == 0


@pytest.mark.parametrize("prec", [lbm.LBM_FP32, lbm.LBM_FP16S, lbm.LBM_BF16S])
def test_species_launch_variants_bitwise(prec):
    """Variants 0 and 2 and every register budget give the same bits with
    several species (the bulk-copy and ring variants serve one species)."""
    def run(launch):
        p = SpeciesPair(2, 2, seed=31, prec=prec, launch=launch)
        p.gpu.step(20)
        return p.gpu.get_state()
    want = run((0, 128, 0, 1, 2, 1))
    for launch in ((0, 64, 0, 3, 2, 5), (2, 128, 0, 2, 2, 4), (2, 64, 0, 4, 2, 6)):
        assert np.array_equal(run(launch), want), launch
    p = SpeciesPair(2, 2, seed=31, prec=prec)
    for bad in ((1, 256, 0, 1, 2, 2), (3, 256, 0, 2, 4, 2)):
        with pytest.raises(lbm.LbmError):
            p.gpu.set_launch(*bad)


def test_second_order_wall_reaction_on_the_gpu():
    """A + B -> products at the bottom wall (k C_A C_B), given C at the top,
    d = 1/2, shear flow along the walls: the GPU's FP64 steady state is the
    linear closed form (exact at d = 1/2, Sec. 4.2.2)."""
    ny, k, A_top, B_top = 14, 0.05, 3.0, 2.0
    walls = {1: (0.5, ny - 1.5)}
    shape = (3, ny, 1)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(0.02, 0, 0)),
         (1, 0, O.H): dict(kind=O.REACTION, kappa1=1.0), (1, 0, O.species_field(1)): dict(kind=O.REACTION, kappa1=1.0),
         (1, 1, O.H): dict(kind=O.GIVEN, phi_wall=A_top),
         (1, 1, O.species_field(1)): dict(kind=O.GIVEN, phi_wall=B_top)}
    solid = LK.box_solid(shape, walls)
    links = to_abi_links(LK.box_links(2, shape, walls, p, has_h=True, nspecies=2))
    case = lbm.make_case(shape, 0.8, 0.9, 1.0, (0, 0, 0), 1.0, 1.0, (0, 0, 0), tau_Dk=(0.7,), C0k=(1.0,))
    g = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, CD, [case], nspecies=2)
    g.set_walls(0, solid, links)
    g.set_reactions(0, [dict(rate=k, order=[1, 1], stoich=[-1, -1])])
    g.set_graph(100)
    g.step(60000)
    y = np.arange(ny)[1:-1]
    Aa, Ba = AN.reactive_channel_two_species(y, walls[1][0], walls[1][1], 0.1, 0.05, k, A_top, B_top)
    CA = g.species(0).reshape(ny, 3)[1:-1]
    CB = g.species(1).reshape(ny, 3)[1:-1]
    assert np.abs(CA - Aa[:, None]).max() / A_top < 1e-11
    assert np.abs(CB - Ba[:, None]).max() / B_top < 1e-11


def test_species_configurations_are_refused():
    case = lbm.make_case((8, 8, 1), 0.8, 0.9, 0.9, tau_Dk=(0.7, 0.7))
    with pytest.raises(lbm.LbmError):                        # several species with the magnetic field
        lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, CD | lbm.LBM_MHD, [case], nspecies=2)
    with pytest.raises(lbm.LbmError):                        # more species than compiled
        lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, CD, [case], nspecies=4)
    with pytest.raises(lbm.LbmError):                        # species without LBM_CD
        lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, lbm.LBM_FLOW, [case], nspecies=2)
    one = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, CD, [case])
    with pytest.raises(lbm.LbmError):                        # a network needs several species
        one.set_reactions(0, [dict(rate=0.1, order=[1, 0], stoich=[-1, 0])])
    two = lbm.Solver(lbm.LBM_D2Q9, lbm.LBM_FP64, CD, [case], nspecies=2)
    with pytest.raises(lbm.LbmError):                        # order outside 0..2
        two.set_reactions(0, [dict(rate=0.1, order=[3, 0], stoich=[-1, 0])])
    with pytest.raises(lbm.LbmError):                        # a species the context does not have
        two.set_reactions(0, [dict(rate=0.1, order=[1, 0, 1], stoich=[-1, 0, 0])])
    with pytest.raises(lbm.LbmError):
        two.species(2)
