"""The explicit Shercliff flux of the M scheme (Eq. 25-27 with F = -eta B1 /
(c_w H), Eq. 30) has a stability limit on kappa = eta / (c_w H).  The case
builders choose eta from tabulated limits (written by oracle/stability_table.py);
these tests re-measure points of those tables on the FP64 reference step, from
the same perturbed start: kappa at the builders' margin below the limit stays
bounded, kappa a quarter above it diverges."""
import pytest

from oracle import stability_table as ST
from paper_2506_00907_gb300 import cases as CS


@pytest.mark.parametrize("eta,qi", [(0.075, 2), (0.025, 4), (0.1, 0)])
def test_channel_limit(eta, qi):
    q = CS.CHANNEL_Q[qi]
    lim = CS.CHANNEL_KAPPA_LIMIT[eta][qi]
    assert ST.channel_stable(q, CS.KAPPA_MARGIN * lim, eta)
    assert not ST.channel_stable(q, 1.25 * lim, eta)


def test_channel_zero_limit_and_the_uniform_start():
    """Where the table holds 0 (q = 0.7 at tau_eta = 0.9) even a weak flux
    diverges from a perturbed start; started exactly uniform along the wall
    the same run stays bounded (the modes that grow vary along the wall)."""
    assert CS.CHANNEL_KAPPA_LIMIT[0.1][3] == 0.0
    assert not ST.channel_stable(0.7, 0.05, 0.1)
    saved = ST.NOISE
    try:
        ST.NOISE = 0.0
        assert ST.channel_stable(0.7, 0.05, 0.1)
    finally:
        ST.NOISE = saved


@pytest.mark.parametrize("eta", [0.075])
def test_pipe_limit(eta):
    lim = CS.PIPE_KAPPA_LIMIT[eta]
    assert ST.pipe_stable(CS.KAPPA_MARGIN * lim, eta, threads=8)
    assert not ST.pipe_stable(1.25 * lim, eta, threads=8)


def test_builders_respect_the_limits():
    for q in (0.0, 0.3, 0.8, 0.99):
        for cw in (1e-3, 0.01, 0.3):
            H = 40.0
            eta = CS.shercliff_eta(cw, H, lambda e: CS.channel_kappa_limit(e, q))
            if eta is None:
                continue
            assert eta / (cw * H) <= CS.KAPPA_MARGIN * CS.channel_kappa_limit(eta, q) + 1e-12
    c, s, l, info = CS.hartmann_channel(77, 21.0, 0.2087, 1.2e-3)
    assert not info["cw_clamped"] and info["kappa1"] < 0
    with pytest.raises(ValueError):
        CS.hartmann_channel(64, 10.0, 0.99, 1e-3)
    c, s, l, info = CS.hartmann_channel(64, 10.0, 0.99, 1e-3, clamp_cw=True)
    assert info["cw_clamped"] and info["cw"] > 1e-3
    with pytest.raises(ValueError):
        CS.pipe((1, 36, 36), 16.0, 15.0, ("shercliff", 1e-3))
