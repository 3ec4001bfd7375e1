"""Oracle pins of several concentration species with surface reactions
between them (no GPU).  Sec. 4.2.2 (text after Eq. 23): each species' C_i(X)
comes from Eq. 13, the reaction fluxes F_i(C_1, C_2, ...) are evaluated
explicitly from them and each is added to its own species by the M scheme
(Eq. 23-27); no coupled solve.  The fluxes here come from a mass-action
network: reaction j runs at rate_j prod_m C_m^order[j][m] and produces
species i at stoich[j][i] times that rate."""
import numpy as np
import pytest

import oracle as O
from oracle import analytic as AN
from oracle import links as LK

DA, DB = 0.25 * (0.9 - 0.5), 0.25 * (0.7 - 0.5)
A, B = O.H, O.species_field(1)


def _sim(ny, d, bottom, top, steps, taus=(0.9, 0.7), C0=(1.0, 1.0), network=(), nx=1, u_top=0.02, threads=1):
    """Channel (periodic x) with a shear flow along the walls; species A and B
    with the given bottom / top wall parameters per field."""
    walls = {1: (1 - d, ny - 2 + d)}
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(u_top, 0, 0))}
    for f in (A, B):
        p[(1, 0, f)] = bottom[f]
        p[(1, 1, f)] = top[f]
    shape = (nx, ny, 1)
    s = O.OracleSim(2, shape, LK.box_solid(shape, walls), 0.8, tau_D=taus[0], has_h=True, threads=threads)
    s.set_species(list(taus), list(C0))
    s.set_network(list(network))
    s.set_links(LK.box_links(2, shape, walls, p, has_h=True, nspecies=2))
    s.init(C0=C0[0])
    if steps:
        s.step(steps)
    return s, walls[1]


def test_network_rate_is_the_mass_action_polynomial():
    rng = np.random.default_rng(3)
    s, _ = _sim(6, 0.5, {A: dict(kind=O.NEUMANN_BFL), B: dict(kind=O.NEUMANN_BFL)},
                {A: dict(kind=O.NEUMANN_BFL), B: dict(kind=O.NEUMANN_BFL)}, 0)
    for _ in range(20):
        net = [dict(rate=rng.uniform(0.1, 2), order=list(rng.integers(0, 3, 2)),
                    stoich=list(rng.uniform(-2, 2, 2))) for _ in range(rng.integers(1, 5))]
        s.set_network(net)
        C = rng.uniform(0.1, 3.0, 2)
        for i in range(2):
            want = sum(r["stoich"][i] * r["rate"] * C[0] ** r["order"][0] * C[1] ** r["order"][1] for r in net)
            assert abs(s.network_rate(i, C) - want) <= 1e-14 * max(1.0, abs(want))


def test_two_identical_species_evolve_as_one():
    """Two species with the same relaxation time, walls and initial state and
    no reaction coupling evolve bit for bit alike, and like the one-species run."""
    bottom = {A: dict(kind=O.FLUX, kappa0=0.003, kappa1=-0.01), B: dict(kind=O.FLUX, kappa0=0.003, kappa1=-0.01)}
    top = {A: dict(kind=O.GIVEN, phi_wall=2.0), B: dict(kind=O.GIVEN, phi_wall=2.0)}
    s, _ = _sim(16, 0.3, bottom, top, 400, taus=(0.9, 0.9), C0=(1.0, 1.0), nx=3)
    one = O.OracleSim(2, (3, 16, 1), LK.box_solid((3, 16, 1), {1: (0.7, 14.3)}), 0.8, tau_D=0.9, has_h=True)
    p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(0.02, 0, 0)),
         (1, 0, O.H): bottom[A], (1, 1, O.H): top[A]}
    one.set_links(LK.box_links(2, (3, 16, 1), {1: (0.7, 14.3)}, p, has_h=True))
    one.init(C0=1.0)
    one.step(400)
    assert np.array_equal(s.species(0), s.species(1))
    assert np.array_equal(s.species(0), one.species(0))
    assert np.array_equal(s.moments()["u"], one.moments()["u"])


def test_linear_network_is_the_robin_wall():
    """A first-order network (rate k C_A, stoich -1) on a reaction link with
    k1 = 1 is the linear flux wall with kappa1 = -k: bit for bit."""
    top = {A: dict(kind=O.GIVEN, phi_wall=3.0), B: dict(kind=O.GIVEN, phi_wall=1.0)}
    s1, _ = _sim(14, 0.3, {A: dict(kind=O.FLUX, kappa0=0.004, kappa1=-0.02), B: dict(kind=O.NEUMANN_BFL)}, top, 500)
    s2, _ = _sim(14, 0.3, {A: dict(kind=O.REACTION, kappa0=0.004, kappa1=1.0), B: dict(kind=O.NEUMANN_BFL)}, top,
                 500, network=[dict(rate=0.02, order=[1, 0], stoich=[-1, 0])])
    assert np.array_equal(s1.species(0), s2.species(0))
    assert np.array_equal(s1.species(1), s2.species(1))


@pytest.mark.parametrize("d", [0.5, 0.25, 1.0])
def test_second_order_two_species_wall(d):
    """A + B -> products at the bottom wall at the rate k C_A C_B, given C_A and
    C_B at the top wall, shear flow along the walls: the steady profiles are
    the linear closed form whose wall values balance both species' fluxes.
    Exact at d = 1/2; second-order close otherwise."""
    k, A_top, B_top = 0.05, 3.0, 2.0
    net = [dict(rate=k, order=[1, 1], stoich=[-1, -1])]
    bottom = {A: dict(kind=O.REACTION, kappa1=1.0), B: dict(kind=O.REACTION, kappa1=1.0)}
    top = {A: dict(kind=O.GIVEN, phi_wall=A_top), B: dict(kind=O.GIVEN, phi_wall=B_top)}
    s, (y0, y1) = _sim(14, d, bottom, top, 60000, network=net)
    y = np.arange(14)[1:-1]
    Aa, Ba = AN.reactive_channel_two_species(y, y0, y1, DA, DB, k, A_top, B_top)
    tol = 1e-11 if d == 0.5 else 5e-3
    assert np.abs(s.species(0)[1:-1] - Aa).max() / A_top < tol
    assert np.abs(s.species(1)[1:-1] - Ba).max() / B_top < tol
    assert Aa[0] < 0.9 * A_top and Ba[0] < 0.9 * B_top          # the reaction matters


def test_reaction_fluxes_enter_each_species_exactly():
    """2 A -> B at the bottom wall (rate k C_A^2; stoich -2 for A, +1 for B),
    zero-flux top wall, fluid at rest, d = 1/2: every step each species gains
    exactly the sum of its links' flux increments R_i(C_X), with C_X = 1.5 C(A)
    - 0.5 C(E) (Eq. 13 at d = 1/2), and C_A + 2 C_B is conserved."""
    k = 0.03
    net = [dict(rate=k, order=[2, 0], stoich=[-2, 1])]
    bottom = {A: dict(kind=O.REACTION, kappa1=1.0), B: dict(kind=O.REACTION, kappa1=1.0)}
    top = {A: dict(kind=O.NEUMANN_BFL), B: dict(kind=O.NEUMANN_BFL)}
    nx, ny = 4, 9
    s, _ = _sim(ny, 0.5, bottom, top, 0, C0=(2.0, 0.5), network=net, nx=nx, u_top=0.0)
    total0 = s.species(0).sum() + 2 * s.species(1).sum()
    for _ in range(6):
        CA = s.species(0).reshape(ny, nx)
        CB = s.species(1).reshape(ny, nx)
        CAX = 1.5 * CA[1] - 0.5 * CA[2]
        expect_A = CA.sum() + np.sum(-2 * k * CAX ** 2)
        expect_B = CB.sum() + np.sum(k * CAX ** 2)
        s.step(1)
        assert abs(s.species(0).sum() - expect_A) < 1e-13
        assert abs(s.species(1).sum() - expect_B) < 1e-13
    s.step(200)
    total = s.species(0).sum() + 2 * s.species(1).sum()
    assert abs(total - total0) < 1e-12 * total0
    assert s.species(1).sum() > 0.5 * nx * (ny - 2) + 1.0            # B was produced
