"""The product's wall-link builders (C++, host side of the C ABI) agree with
the oracle's independently written builders (no GPU needed)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import links as LK
from paper_2506_00907_gb300 import lbm
from tests.helpers import sort_links, to_abi_links

PHYS_ALL = lbm.LBM_FLOW | lbm.LBM_CD | lbm.LBM_MHD


def _compare(prod, orc):
    a, b = sort_links(prod), sort_links(to_abi_links(orc))
    assert len(a) == len(b)
    for k in ("node", "field", "dir", "kind"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("d", "u_wall", "phi_wall"):
        assert np.abs(a[k] - b[k]).max() < 1e-14, k
    for k in ("k0", "k1"):
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(1.0, np.abs(b[k]).max()), k


@pytest.mark.parametrize("dim,shape,axis", [(2, (12, 10, 1), 1), (2, (9, 7, 1), 0), (3, (5, 6, 8), 2)])
@pytest.mark.parametrize("d_lo,d_hi", [(0.5, 0.5), (0.3, 0.8), (1.0, 0.05)])
def test_channel_builder_matches_oracle(dim, shape, axis, d_lo, d_hi):
    n_axis = shape[axis]
    walls = {axis: (1.0 - d_lo, n_axis - 2.0 + d_hi)}
    bc = {
        (0, 0): dict(kind=O.VELOCITY, u_wall=(0.0, 0.0, 0.0)),
        (1, 0): dict(kind=O.VELOCITY, u_wall=(0.05, 0.01, 0.0)),
        (0, 1): dict(kind=O.FLUX, kappa0=0.002, kappa1=-0.01),
        (1, 1): dict(kind=O.GIVEN, phi_wall=3.0, u_wall=(0.05, 0.01, 0.0)),
        (0, 2): dict(kind=O.GIVEN, phi_wall=0.0),
        (1, 2): dict(kind=O.FLUX, kappa1=-0.3, u_wall=(0.05, 0.01, 0.0)),
        (0, 3): dict(kind=O.GIVEN, phi_wall=0.2),
        (1, 3): dict(kind=O.GIVEN, phi_wall=0.2),
        (0, 4): dict(kind=O.NEUMANN_BFL),
        (1, 4): dict(kind=O.NEUMANN_BFL),
    }
    params = {(axis, side, field): p for (side, field), p in bc.items()}
    orc = LK.box_links(dim, shape, walls, params, has_h=True, has_g=True)

    def abi(side):
        out = []
        for field in range(5):
            p = bc[(side, field)]
            out.append(lbm.wall_bc(p["kind"], p.get("u_wall", (0, 0, 0)), p.get("phi_wall", 0.0),
                                   p.get("kappa0", 0.0), p.get("kappa1", 0.0)))
        return out
    solid, prod = lbm.lbm_build_channel(dim, shape, axis, d_lo, d_hi, PHYS_ALL, abi(0), abi(1))
    assert np.array_equal(solid, LK.box_solid(shape, walls).reshape(-1))
    _compare(prod, orc)


@pytest.mark.parametrize("R,shape", [(17.3, (2, 40, 40)), (12.0, (1, 27, 26))])
@pytest.mark.parametrize("b1", ["insulating", "conducting", "shercliff", "shercliff_simplified"])
def test_pipe_builder_matches_oracle(R, shape, b1):
    """Product and oracle pipe builders give the same links (the simplified
    case also takes the comparison velocity scheme, Eq. 15/16 for every d)."""
    eta = 0.1
    fkind = O.VELOCITY_EQ15 if b1 == "shercliff_simplified" else O.VELOCITY
    if b1 == "insulating":
        g0 = dict(kind=O.GIVEN, phi_wall=0.0)
    elif b1 == "conducting":
        g0 = dict(kind=O.FLUX)
    else:
        g0 = dict(kind=O.FLUX if b1 == "shercliff" else O.FLUX_SIMPLIFIED, kappa1=-eta / (0.1 * R))
    params = {O.F: dict(kind=fkind), O.G0: g0, O.G0 + 1: dict(kind=O.GIVEN, phi_wall=0.04),
              O.G0 + 2: dict(kind=O.GIVEN, phi_wall=0.0)}
    orc, info = LK.pipe_links(shape, R, params)
    bcs = [lbm.wall_bc(fkind), None,
           lbm.wall_bc(g0["kind"], phi_wall=g0.get("phi_wall", 0.0), kappa1=g0.get("kappa1", 0.0)),
           lbm.wall_bc(lbm.LBM_W_GIVEN, phi_wall=0.04), lbm.wall_bc(lbm.LBM_W_GIVEN)]
    solid, prod = lbm.lbm_build_pipe(shape, R, lbm.LBM_FLOW | lbm.LBM_MHD, bcs)
    assert np.array_equal(solid, LK.pipe_solid(shape, R).reshape(-1))
    _compare(prod, orc)
    if b1.startswith("shercliff"):
        # conservative splitting: the flux coefficients of a slice add up to kappa1 * 2 pi R
        fl = prod[prod["field"] == 2]
        for x in range(shape[0]):
            tot = fl["k1"][fl["node"] % shape[0] == x].sum()
            assert abs(tot - g0["kappa1"] * 2 * math.pi * R) < 1e-10


@pytest.mark.parametrize("dim,shape", [(2, (14, 5, 1)), (3, (9, 4, 3))])
@pytest.mark.parametrize("d", [0.5, 0.3, 1.0])
def test_open_channel_builder_matches_oracle(dim, shape, d):
    """A domain open along x (Sec. 5.1): inlet of given velocity (the velocity
    kind with a normal u) and outlet of given density, built by the product's
    channel builder, equals the oracle's links."""
    walls = {0: (1.0 - d, shape[0] - 2.0 + d)}
    U = (0.03, 0.002, 0.0)
    params = {(0, 0, O.F): dict(kind=O.VELOCITY, u_wall=U), (0, 1, O.F): dict(kind=O.PRESSURE, phi_wall=1.01)}
    orc = LK.box_links(dim, shape, walls, params)
    lo = [lbm.wall_bc(lbm.LBM_W_VELOCITY, u_wall=U), None, None, None, None]
    hi = [lbm.wall_bc(lbm.LBM_W_PRESSURE, phi_wall=1.01), None, None, None, None]
    solid, prod = lbm.lbm_build_channel(dim, shape, 0, d, d, lbm.LBM_FLOW, lo, hi)
    assert np.array_equal(solid, LK.box_solid(shape, walls).reshape(-1))
    assert np.any(prod["kind"] == lbm.LBM_W_PRESSURE)
    _compare(prod, orc)
