"""Pins of the FP64 oracle: lattices, equilibria, forcing and the wall-link
formulas, against what the paper and the mathematics fix independently of the
oracle's own code (identities, printed parameter sets, printed special cases)."""
import itertools

import numpy as np
import pytest

import oracle as O

DIMS = (2, 3)


# ---------------------------------------------------------------- lattices
@pytest.mark.parametrize("dim,scalar", list(itertools.product(DIMS, (False, True))))
def test_lattice_isotropy(dim, scalar):
    """sum w = 1, sum w e = 0, sum w e e = c^2 I (Sec. 2.2, 2.3; Qian 1992);
    4th-order isotropy for the flow lattices (needed by Eq. 8)."""
    e, w = O.lattice(dim, scalar)
    c2 = 0.25 if scalar else 1.0 / 3.0
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    second = np.einsum("a,ai,aj->ij", w, e, e)
    expect = np.diag([c2] * dim + [0.0] * (3 - dim))
    assert np.abs(second - expect).max() < 1e-15
    if not scalar:
        fourth = np.einsum("a,ai,aj,ak,al->ijkl", w, e, e, e, e)
        d = np.eye(3)
        d[dim:, dim:] = 0
        iso = c2 * c2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                         + np.einsum("il,jk->ijkl", d, d))
        assert np.abs(fourth - iso).max() < 1e-15
    # opposite directions exist and weights are symmetric
    for a in range(len(e)):
        b = O.opposite(e, a)
        assert w[a] == w[b]


def test_scalar_lattice_weights_reproduce_printed_parameters():
    """The D2Q5/D3Q7 weights are not printed; every parameter set of the paper
    fixes c_h^2 = c_g^2 = c^2/4 through D = dt c_h^2 (tau_D - 1/2) (Eq. 3) and
    eta = dt c_g^2 (tau_eta - 1/2) (Eq. 5), and c_s^2 = c^2/3 (Eq. 1)."""
    # Sec. 5.3: D = 1e-6, dx = 1.25e-4, c = 0.08, tau_D = 0.9
    ch2_x3 = 1e-6 / ((1.25e-4 / 0.08) * 0.08 ** 2 * (0.9 - 0.5))
    # Sec. 5.4: sigma = 1e6, mu = 1 -> eta = 1e-6; dx = 1e-5, c = 1, tau_eta = 0.9
    ch2_x4 = 1e-6 / ((1e-5 / 1.0) * 1.0 ** 2 * (0.9 - 0.5))
    # Sec. 6: eta = 1, dx = 0.04, c = 250, tau_eta = 0.9
    ch2_x6 = 1.0 / ((0.04 / 250) * 250.0 ** 2 * (0.9 - 0.5))
    # Sec. 5.2: nu = 1e-6, dx = 1e-5, tau 0.8 with dt 1e-5 and 0.53 with dt 1e-6
    cs2_a = 1e-6 / (1e-5 * (1e-5 / 1e-5) ** 2 * (0.8 - 0.5))
    cs2_b = 1e-6 / (1e-6 * (1e-5 / 1e-6) ** 2 * (0.53 - 0.5))
    for dim in DIMS:
        e, w = O.lattice(dim, scalar=True)
        ch2 = (w * e[:, 0] ** 2).sum()
        for v in (ch2_x3, ch2_x4, ch2_x6):
            assert abs(v - ch2) < 1e-12
        e, w = O.lattice(dim, scalar=False)
        cs2 = (w * e[:, 0] ** 2).sum()
        for v in (cs2_a, cs2_b):
            assert abs(v - cs2) < 1e-12


# ---------------------------------------------------------------- equilibria
@pytest.mark.parametrize("dim", DIMS)
def test_equilibrium_moments(dim):
    """Eq. 8-10 and the conservation statements after them, with the magnetic
    stress 1/2|B|^2 I - BB (mu = 1) in the second moment of f^eq."""
    rng = np.random.default_rng(7)
    e, w = O.lattice(dim)
    em, wm = O.lattice(dim, scalar=True)
    for _ in range(5):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        B = rng.uniform(-0.2, 0.2, 3)
        C = rng.uniform(0.1, 5)
        if dim == 2:
            u[2] = B[2] = 0.0
        f = np.array([O.feq(dim, a, rho, u, B) for a in range(len(e))])
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(e.T @ f - rho * u).max() < 1e-14
        Pi = np.einsum("a,ai,aj->ij", f, e, e)
        I = np.diag([1.0] * dim + [0.0] * (3 - dim))
        expect = rho * np.outer(u, u) + rho / 3 * I + 0.5 * (B @ B) * I - np.outer(B, B)
        assert np.abs(Pi - expect).max() < 1e-14
        h = np.array([O.heq(dim, a, C, u) for a in range(len(em))])
        assert abs(h.sum() - C) < 1e-14
        assert np.abs(em.T @ h - C * u).max() < 1e-14                 # Eq. 9
        g = np.array([[O.geq(dim, a, k, B, u) for k in range(3)] for a in range(len(em))])
        assert np.abs(g.sum(0) - B).max() < 1e-15
        Pg = np.einsum("aj,ak->jk", em, g)                              # sum e_j g_k
        assert np.abs(Pg - (np.outer(u, B) - np.outer(B, u))).max() < 1e-15   # Eq. 10


@pytest.mark.parametrize("dim", DIMS)
def test_guo_source_moments(dim):
    """Guo-Zheng-Shi forcing (reading of Sec. 2.4): the source carries no mass,
    momentum (1 - 1/(2 tau)) F and momentum flux (1 - 1/(2 tau)) (uF + Fu)."""
    rng = np.random.default_rng(3)
    e, w = O.lattice(dim)
    tau = 0.8
    u = rng.uniform(-0.1, 0.1, 3)
    F = rng.uniform(-1e-3, 1e-3, 3)
    if dim == 2:
        u[2] = F[2] = 0
    S = np.array([O.guo(dim, a, tau, u, F) for a in range(len(e))])
    k = 1 - 1 / (2 * tau)
    assert abs(S.sum()) < 1e-18
    assert np.abs(e.T @ S - k * F).max() < 1e-18
    assert np.abs(np.einsum("a,ai,aj->ij", S, e, e) - k * (np.outer(u, F) + np.outer(F, u))).max() < 1e-18


@pytest.mark.parametrize("dim", DIMS)
def test_moving_wall_increment_identities(dim):
    """Sec. 4.1 (after Eq. 16) and Sec. 4.2.2 (after Eq. 24):
    f^eq_a - f^eq_a' = 2 rho w_a (e_a.u)/c_s^2 = f^eq_a'(-u) - f^eq_a(-u),
    also with a magnetic field (its stress is even in e)."""
    rng = np.random.default_rng(11)
    e, w = O.lattice(dim)
    rho = 1.03
    u = rng.uniform(-0.05, 0.05, 3)
    B = rng.uniform(-0.1, 0.1, 3)
    if dim == 2:
        u[2] = B[2] = 0
    for a in range(1, len(e)):
        ap = O.opposite(e, a)
        inc = O.feq(dim, a, rho, u) - O.feq(dim, ap, rho, u)
        assert abs(inc - 2 * rho * w[a] * (e[a] @ u) * 3.0) < 1e-15
        assert abs(inc - (O.feq(dim, ap, rho, -u) - O.feq(dim, a, rho, -u))) < 1e-15
        incB = O.feq(dim, a, rho, u, B) - O.feq(dim, ap, rho, u, B)
        assert abs(incB - inc) < 1e-15


@pytest.mark.parametrize("dim", DIMS)
def test_tangential_wall_conserves_mass(dim):
    """Sec. 4.1: increments at a flat wall moving tangentially sum to zero; a
    normal velocity gives the mass flux (sum of increments = rho u.n)."""
    e, w = O.lattice(dim)
    n = np.array([0.0, 1.0, 0.0])               # wall below, fluid above
    unknown = [a for a in range(1, len(e)) if e[a] @ n > 0]
    ut = np.array([0.03, 0.0, 0.02 if dim == 3 else 0.0])
    tot = sum(O.feq(dim, a, 1.0, ut) - O.feq(dim, O.opposite(e, a), 1.0, ut) for a in unknown)
    assert abs(tot) < 1e-16
    un = np.array([0.0, 0.01, 0.0])
    tot = sum(O.feq(dim, a, 1.0, un) - O.feq(dim, O.opposite(e, a), 1.0, un) for a in unknown)
    assert abs(tot - 1.0 * 0.01) < 1e-16


# ---------------------------------------------------------------- link formulas
def _rand_inputs(rng):
    return dict(p_a_A=rng.uniform(0.01, 0.2), p_ap_A=rng.uniform(0.01, 0.2),
                p_ap_E=rng.uniform(0.01, 0.2), phi_A=rng.uniform(0.5, 2), phi_E=rng.uniform(0.5, 2),
                B_A=tuple(rng.uniform(-1, 1, 3)), B_E=tuple(rng.uniform(-1, 1, 3)))


def _flow_dirs(dim):
    e, _ = O.lattice(dim)
    return e, range(1, len(e))


@pytest.mark.parametrize("dim", DIMS)
def test_velocity_scheme_special_cases(dim):
    """Eq. 15/16 (d < 0.5) and Eq. 43 (d >= 0.5):
    - static wall: Eq. 11 for d < 0.5 and Eq. 12 for d >= 0.5 (Sec. 5.1 and 6);
    - d = 0.5: halfway bounce-back (remark after Eq. 12) and, moving, Eq. 41;
    - the two branches meet at d = 0.5."""
    rng = np.random.default_rng(5)
    e, dirs = _flow_dirs(dim)
    for a in dirs:
        ap = O.opposite(e, a)
        x = _rand_inputs(rng)
        for d in (0.1, 0.3, 0.49):
            v = O.eval_link(dim, dict(field=O.F, dir=a, kind=O.VELOCITY, d=d), **x)
            assert abs(v - ((1 - 2 * d) * x["p_ap_E"] + 2 * d * x["p_ap_A"])) < 1e-15     # Eq. 11
        for d in (0.5, 0.7, 1.0):
            v = O.eval_link(dim, dict(field=O.F, dir=a, kind=O.VELOCITY, d=d), **x)
            assert abs(v - ((2 * d - 1) * x["p_a_A"] + x["p_ap_A"]) / (2 * d)) < 1e-15  # Eq. 12
        v = O.eval_link(dim, dict(field=O.F, dir=a, kind=O.VELOCITY, d=0.5), **x)
        assert abs(v - x["p_ap_A"]) < 1e-16
        uw = rng.uniform(-0.05, 0.05, 3)
        if dim == 2:
            uw[2] = 0
        rhoX = 1.5 * x["phi_A"] - 0.5 * x["phi_E"]                                      # Eq. 13, d = 0.5
        eq41 = x["p_ap_A"] + O.feq(dim, a, rhoX, uw) - O.feq(dim, ap, rhoX, uw)
        v = O.eval_link(dim, dict(field=O.F, dir=a, kind=O.VELOCITY, d=0.5, u_wall=uw), **x)
        assert abs(v - eq41) < 1e-15
        lo = O.eval_link(dim, dict(field=O.F, dir=a, kind=O.VELOCITY, d=0.5 - 1e-12, u_wall=uw), **x)
        assert abs(lo - v) < 1e-11


@pytest.mark.parametrize("dim", DIMS)
def test_flux_scheme_reduces_to_eq28_eq29(dim):
    """M scheme (Eq. 25-27) reduces to Eq. 28 at d = 0.5 and to Eq. 29 at d = 1."""
    rng = np.random.default_rng(9)
    em, _ = O.lattice(dim, scalar=True)
    for field in (O.H, O.G0, O.G0 + 1):
        for a in range(1, len(em)):
            ap = O.opposite(em, a)
            x = _rand_inputs(rng)
            uw = rng.uniform(-0.05, 0.05, 3)
            if dim == 2:
                uw[2] = 0
            lk = dict(field=field, dir=a, kind=O.FLUX, u_wall=uw, k0=rng.uniform(-0.01, 0.01),
                      k1=rng.uniform(-0.1, 0))

            def increments(d):
                phiX = -d * x["phi_E"] + (d + 1) * x["phi_A"]
                dflux = lk["k0"] + lk["k1"] * phiX
                if field == O.H:
                    dmove = O.heq(dim, ap, phiX, -uw) - O.heq(dim, a, phiX, -uw)
                else:
                    k = field - O.G0
                    BX = -d * np.array(x["B_E"]) + (d + 1) * np.array(x["B_A"])
                    dmove = O.geq(dim, ap, k, BX, -uw) - O.geq(dim, a, k, BX, -uw)
                return dflux, dmove
            fl, mv = increments(0.5)
            v = O.eval_link(dim, dict(lk, d=0.5), **x)
            assert abs(v - (x["p_ap_A"] + fl + mv)) < 1e-15                             # Eq. 28
            fl, mv = increments(1.0)
            v = O.eval_link(dim, dict(lk, d=1.0), **x)
            eq29 = (0.5 * x["p_a_A"] - 0.5 * x["p_ap_E"] + 1.5 * x["p_ap_A"] + fl + mv) / 1.5
            assert abs(v - eq29) < 1e-15                                                # Eq. 29


def test_mhd_special_cases_eq36_eq37_eq38():
    """Sec. 4.3.1: at d = 0.5 with U = (U1, 0) on a wall normal to x2 (D2Q5):
    conducting (Eq. 31 with zero flux) -> Eq. 36; insulating B1 = 0 -> Eq. 37;
    given B2 = B_ext,2 -> Eq. 38."""
    rng = np.random.default_rng(21)
    em, wm = O.lattice(2, scalar=True)
    U1 = 0.01
    for a in (2, 4):                      # links normal to the wall: e_a . U = 0
        x = _rand_inputs(rng)
        BX = 1.5 * np.array(x["B_A"]) - 0.5 * np.array(x["B_E"])
        v = O.eval_link(2, dict(field=O.G0, dir=a, kind=O.FLUX, d=0.5, u_wall=(U1, 0, 0)), **x)
        eq36 = x["p_ap_A"] - 2 * wm[a] * (em[a] @ BX) * U1 / 0.25
        assert abs(v - eq36) < 1e-15
        v = O.eval_link(2, dict(field=O.G0, dir=a, kind=O.GIVEN, d=0.5, phi_wall=0.0, u_wall=(U1, 0, 0)), **x)
        assert abs(v - (-x["p_ap_A"])) < 1e-15                                          # Eq. 37
        Bext2 = 0.37
        v = O.eval_link(2, dict(field=O.G0 + 1, dir=a, kind=O.GIVEN, d=0.5, phi_wall=Bext2, u_wall=(U1, 0, 0)), **x)
        assert abs(v - (2 * wm[a] * Bext2 - x["p_ap_A"])) < 1e-15                        # Eq. 38


@pytest.mark.parametrize("dim", DIMS)
def test_given_and_neumann_special_cases(dim):
    """Given C (Eq. 19/20) at d = 0.5: anti-bounce-back 2 w C - h_rel,a'(A)
    (the concentration analogue of Eq. 42); zero gradient (Eq. 21/22) at
    d = 0.5: halfway bounce-back; Eq. 21 and 22 meet at d = 0.5; the M scheme
    without flux or motion equals Eq. 22 at d = 0.5."""
    rng = np.random.default_rng(13)
    em, wm = O.lattice(dim, scalar=True)
    for a in range(1, len(em)):
        x = _rand_inputs(rng)
        v = O.eval_link(dim, dict(field=O.H, dir=a, kind=O.GIVEN, d=0.5, phi_wall=2.5,
                                  u_wall=(0.02, -0.01, 0.0)), **x)
        assert abs(v - (2 * wm[a] * 2.5 - x["p_ap_A"])) < 1e-15
        v = O.eval_link(dim, dict(field=O.H, dir=a, kind=O.NEUMANN_BFL, d=0.5), **x)
        assert abs(v - x["p_ap_A"]) < 1e-16
        lo = O.eval_link(dim, dict(field=O.H, dir=a, kind=O.NEUMANN_BFL, d=0.5 - 1e-12), **x)
        assert abs(lo - v) < 1e-12
        m = O.eval_link(dim, dict(field=O.H, dir=a, kind=O.FLUX, d=0.5), **x)
        assert abs(m - v) < 1e-16
        # given C for any d: the sum of equilibria at X is 2 w C for any wall velocity
        for d in (0.2, 0.8, 1.0):
            v = O.eval_link(dim, dict(field=O.H, dir=a, kind=O.GIVEN, d=d, phi_wall=1.7,
                                      u_wall=(0.03, 0.01, 0.0)), **x)
            pY = (1 - 2 * d) * x["p_ap_E"] + 2 * d * x["p_ap_A"]
            assert abs(v - (2 * wm[a] * 1.7 - pY)) < 1e-15
