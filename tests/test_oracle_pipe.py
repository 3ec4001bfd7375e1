"""Pins of the oracle's curved-wall path (Sec. 6): the wall-link builder
(d per direction, surface segmentation, flux splitting), the independent
finite-volume reference, and the MHD pipe flows of Fig. 10-12."""
import math

import numpy as np
import pytest
import sympy as sy

import oracle as O
from oracle import links as LK
from oracle import pipe_fd as FD

TAU, TAUE = 0.8, 0.9
NU, ETA = (TAU - 0.5) / 3, (TAUE - 0.5) / 4


def test_fd_solver_hagen_poiseuille():
    """B0 -> 0: u = a (R^2 - r^2) / (4 nu)."""
    R, a = 1.0, 1.0
    r, th, u, b = FD.solve(R, 1e-12, 1.0, 1.0, a, nr=40, nt=64)
    exact = a * (R * R - r ** 2) / 4.0
    assert np.abs(u - exact[:, None]).max() / exact.max() < 1e-3


@pytest.mark.parametrize("wall", [("insulating",), ("conducting",), ("shercliff", 0.3)])
def test_fd_solver_manufactured_second_order(wall):
    """Manufactured solution with the coupling terms and the wall condition
    satisfied exactly; the error must fall about 4x per refinement."""
    y, z = sy.symbols("y z")
    R, B0, nu, eta, a = 1.0, 3.0, 0.7, 0.4, 0.0
    r2 = y ** 2 + z ** 2
    um = (R ** 2 - r2) * (1 + 0.3 * y + 0.2 * z ** 2)
    if wall[0] == "insulating":
        bm = (R ** 2 - r2) * (0.5 * z + 0.4 * y * z)
    elif wall[0] == "conducting":
        bm = (r2 - R ** 2) ** 2 * (0.5 + 0.4 * y) + 0.3
    else:   # db/dr + b/(cw R) = 0 at r = R: b = (1 + beta (R^2 - r^2)) f with beta from the condition
        cw = wall[1]
        beta = 1.0 / (2 * R * cw * R)          # d/dr[(R^2 - r^2)] = -2R at r = R
        bm = (1 + beta * (R ** 2 - r2)) * 0.7
    lap = lambda f: sy.diff(f, y, 2) + sy.diff(f, z, 2)
    su = -(nu * lap(um) + B0 * sy.diff(bm, y) + a)
    sb = -(eta * lap(bm) + B0 * sy.diff(um, y))
    fsu, fsb = sy.lambdify((y, z), su, "numpy"), sy.lambdify((y, z), sb, "numpy")
    fum, fbm = sy.lambdify((y, z), um, "numpy"), sy.lambdify((y, z), bm, "numpy")
    errs = []
    for nr in (16, 32):
        r, th, u, b = FD.solve(R, B0, nu, eta, a, wall=wall, nr=nr, nt=2 * nr,
                               src=lambda yy, zz: (float(fsu(yy, zz)), float(fsb(yy, zz))))
        Y, Z = r[:, None] * np.cos(th)[None, :], r[:, None] * np.sin(th)[None, :]
        bex = fbm(Y, Z) * np.ones_like(Y)
        if wall[0] == "conducting":           # b is defined up to a constant: compare without the mean
            w = r[:, None] * np.ones_like(Y)
            b = b - np.sum(b * w) / np.sum(w)
            bex = bex - np.sum(bex * w) / np.sum(w)
        errs.append(max(np.abs(u - fum(Y, Z)).max(), np.abs(b - bex).max()))
    assert errs[1] < 1e-2
    assert errs[0] / errs[1] > 3.0


def test_pipe_link_builder_invariants():
    """Sec. 6: d in (0, 1] per node and direction; sum of S_i = 2 pi R per axial
    slice (the segmentation keeps the area); split weights of Eq. 48 sum to one
    per outer-layer solid point; every required link present."""
    shape, R = (2, 40, 40), 17.3
    params = {O.F: dict(kind=O.VELOCITY), O.G0: dict(kind=O.FLUX, kappa1=-1.0),
              O.G0 + 1: dict(kind=O.GIVEN, phi_wall=0.1), O.G0 + 2: dict(kind=O.GIVEN)}
    links, info = LK.pipe_links(shape, R, params)
    assert np.all(links["d"] > 0) and np.all(links["d"] <= 1)
    segs = info["segments"]
    for x in range(shape[0]):
        tot = sum(S for n, (S, _) in segs.items() if n % shape[0] == x)
        assert abs(tot - 2 * math.pi * R) < 1e-10
    flux = links[links["field"] == O.G0]
    # k1 per link = kappa1 * S_B * w; summing over links of each solid point gives -S_B
    nx, ny = shape[0], shape[1]
    e7, _ = O.lattice(3, scalar=True)
    per_B = {}
    for lk in flux:
        A = lk["node"]
        x, y, z = A % nx, (A // nx) % ny, A // (nx * ny)
        e = e7[lk["dir"]]
        Bn = (x - e[0]) % nx + nx * ((y - e[1]) % ny + ny * ((z - e[2]) % shape[2]))
        per_B[Bn] = per_B.get(Bn, 0.0) + lk["k1"]
    for Bn, k1 in per_B.items():
        assert abs(k1 + segs[Bn][0]) < 1e-12
    assert info["e_solid_links"] == 0          # no link needs the E-solid reading on this pipe
    s = O.OracleSim(3, shape, LK.pipe_solid(shape, R), TAU, tau_eta=TAUE, has_g=True)
    s.set_links(links)          # completeness and uniqueness are checked by the oracle


def _pipe_case(wall, ncpu, R=25.0, n=54, Ha=10.0, accel=2e-6, steps=16000):
    """Sec. 6 set-up in lattice units: 54 x 54 cross-section, R = 25 dx
    (dx = 0.04, R = 1), tau_nu = 0.8, tau_eta = 0.9, Ha = 10, B_ext along x2;
    one axial node (the flow is axially invariant)."""
    B0 = Ha * math.sqrt(NU * ETA) / R
    shape = (1, n, n)
    if wall[0] == "insulating":
        g0 = dict(kind=O.GIVEN, phi_wall=0.0)
    elif wall[0] == "conducting":
        g0 = dict(kind=O.FLUX)
    else:
        g0 = dict(kind=O.FLUX, kappa1=-ETA / (wall[1] * R))
    params = {O.F: dict(kind=O.VELOCITY), O.G0: g0, O.G0 + 1: dict(kind=O.GIVEN, phi_wall=B0),
              O.G0 + 2: dict(kind=O.GIVEN, phi_wall=0.0)}
    links, info = LK.pipe_links(shape, R, params)
    solid = LK.pipe_solid(shape, R)
    s = O.OracleSim(3, shape, solid, TAU, tau_eta=TAUE, accel=(accel, 0, 0), has_g=True, threads=ncpu)
    s.set_links(links)
    s.init(B0=(0, B0, 0))
    s.step(steps)
    fl = solid.reshape(-1) == 0
    c = (n - 1) / 2.0
    zz, yy = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
    yy, zz = yy.ravel()[fl], zz.ravel()[fl]
    r, th, uf, bf = FD.solve(R, B0, NU, ETA, accel, wall=wall, nr=128, nt=256)
    Um = FD.mean_velocity(r, th, uf)
    m = s.moments()
    return dict(u=m["u"][fl, 0] / Um, b=m["B"][fl, 0] / Um, B2=m["B"][fl, 1], B0=B0,
                ua=FD.sample(r, th, uf, yy, zz) / Um, ba=FD.sample(r, th, bf, yy, zz) / Um,
                r=np.hypot(yy, zz), R=R)


@pytest.mark.parametrize("wall", [("insulating",), ("shercliff", 0.1)])
def test_pipe_insulating_and_thin_wall(wall, ncpu):
    """Fig. 10 and 12: "excellent agreement" away from the jagged wall."""
    c = _pipe_case(wall, ncpu)
    inner = c["r"] < c["R"] - 3
    assert np.abs(c["u"] - c["ua"])[inner].max() < 0.01
    assert np.abs(c["b"] - c["ba"])[inner].max() < 0.02 * np.abs(c["ba"]).max() + 0.005
    assert np.abs(c["u"] - c["ua"]).max() < 0.04
    assert np.abs(c["B2"] - c["B0"]).max() < 1e-6 * c["B0"]       # B2 = B_ext,2 up to lattice error (Sec. 6)


def test_pipe_conducting_printed_value(ncpu):
    """Fig. 11: the perfectly conducting wall (M scheme without flux) carries a
    small error that the paper prints near the u* = 1.3 contour: 1.314 analytic
    against 1.301 LBM, LBM below.  Same size and sign here."""
    c = _pipe_case(("conducting",), ncpu)
    sel = np.abs(c["ua"] - 1.3) < 0.03
    diff = c["u"][sel] - c["ua"][sel]
    i = np.argmax(np.abs(diff))
    assert 0.004 < abs(diff[i]) < 0.03
    assert diff[i] < 0
