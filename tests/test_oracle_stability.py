"""The explicit Shercliff flux of the M scheme (Eq. 25-27 with F = -eta B1 /
(c_w H), Eq. 30) has a stability limit on kappa = eta / (c_w H).  The case
builders choose eta from tabulated limits; these tests re-measure points of
those tables on the FP64 reference step: kappa at the builders' margin below
the limit stays bounded, kappa a quarter above it diverges."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import links as LK
from paper_2506_00907_gb300 import cases as CS


def _bounded(sim, fluid, steps):
    for _ in range(steps // 500):
        sim.step(500)
        m = sim.moments()
        if not np.all(np.isfinite(m["u"][fluid])) or np.abs(m["B"][fluid, 0]).max() > 10:
            return False
    return True


def _channel(q, kappa, eta, steps=6000, W=8, Ha=15.0):
    nu, d = 0.1, 1.0 - q
    ny = W + 2
    walls = LK.channel_y(2, W, ny, 1, d, d)
    H = (walls[1][1] - walls[1][0]) / 2
    B0 = Ha * math.sqrt(nu * eta) / H
    p = {(1, s, O.F): dict(kind=O.VELOCITY) for s in (0, 1)}
    p.update({(1, s, O.G0): dict(kind=O.FLUX, kappa1=-kappa) for s in (0, 1)})
    p.update({(1, s, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=B0) for s in (0, 1)})
    shape = (W, ny, 1)
    solid = LK.box_solid(shape, walls)
    sim = O.OracleSim(2, shape, solid, 0.8, 1.0, 0.5 + 4 * eta, (0.02 * nu * (2 + Ha) / H ** 2, 0, 0),
                      False, True, 2)
    sim.set_links(LK.box_links(2, shape, walls, p, has_g=True))
    sim.init(B0=(0, B0, 0))
    return _bounded(sim, solid.reshape(-1) == 0, steps)


def _pipe(kappa, eta, steps=6000, R=16.0, n=36, Ha=15.0):
    nu = 0.1
    B0 = Ha * math.sqrt(nu * eta) / R
    params = {O.F: dict(kind=O.VELOCITY), O.G0: dict(kind=O.FLUX, kappa1=-kappa),
              O.G0 + 1: dict(kind=O.GIVEN, phi_wall=B0), O.G0 + 2: dict(kind=O.GIVEN, phi_wall=0.0)}
    shape = (1, n, n)
    solid = LK.pipe_solid(shape, R)
    links, _ = LK.pipe_links(shape, R, params)
    sim = O.OracleSim(3, shape, solid, 0.8, 1.0, 0.5 + 4 * eta, (0.02 * nu * (2 + Ha) / R ** 2, 0, 0),
                      False, True, 4)
    sim.set_links(links)
    sim.init(B0=(0, B0, 0))
    return _bounded(sim, np.asarray(solid).reshape(-1) == 0, steps)


@pytest.mark.parametrize("eta,qi", [(0.075, 2), (0.025, 4), (0.1, 0)])
def test_channel_limit(eta, qi):
    q = CS.CHANNEL_Q[qi]
    lim = CS.CHANNEL_KAPPA_LIMIT[eta][qi]
    assert _channel(q, CS.KAPPA_MARGIN * lim, eta)
    assert not _channel(q, 1.25 * lim, eta)


@pytest.mark.parametrize("eta", [0.0125, 0.05])
def test_pipe_limit(eta):
    lim = CS.PIPE_KAPPA_LIMIT[eta]
    assert _pipe(CS.KAPPA_MARGIN * lim, eta)
    assert not _pipe(1.25 * lim, eta)


def test_builders_respect_the_limits():
    for q in (0.0, 0.3, 0.8, 0.99):
        for cw in (1e-3, 0.01, 0.3):
            H = 40.0
            eta = CS.shercliff_eta(cw, H, lambda e: CS.channel_kappa_limit(e, q))
            if eta is None:
                continue
            assert eta / (cw * H) <= CS.KAPPA_MARGIN * CS.channel_kappa_limit(eta, q) + 1e-12
    c, s, l, info = CS.hartmann_channel(77, 21.0, 0.2087, 1.0652e-3)
    assert not info["cw_clamped"] and info["kappa1"] < 0
    with pytest.raises(ValueError):
        CS.hartmann_channel(64, 10.0, 0.99, 1e-3)
    c, s, l, info = CS.hartmann_channel(64, 10.0, 0.99, 1e-3, clamp_cw=True)
    assert info["cw_clamped"] and info["cw"] > 1e-3
    with pytest.raises(ValueError):
        CS.pipe((1, 36, 36), 16.0, 15.0, ("shercliff", 1e-3))
