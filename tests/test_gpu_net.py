"""The warm-start network on the GPU: forward, gradient and Adam through the C
ABI against the FP64 reference (which uses the same FP16-rounded weights the
GPU passes read), and what the trained network gains: steady MHD pipe runs
started from its prediction reach the residual in fewer steps than cold
starts, and out-of-range cases fall back to cold starts."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2506_00907_gb300 import inputs as IN
from paper_2506_00907_gb300 import lbm
from paper_2506_00907_gb300 import steady as SD
from paper_2506_00907_gb300 import surrogate as SG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = list(lbm.NET_DIMS)


def _rounded(p):
    return np.asarray(p, dtype=np.float32).astype(np.float16).astype(np.float64)


def _data(seed, n):
    r = np.random.default_rng(seed)
    X = r.uniform(-1, 1, (n, 4)).astype(np.float32)
    T = np.stack([np.cos(2 * X[:, 0]) * (1 - X[:, 1] ** 2) + 0.3 * X[:, 2], np.sin(3 * X[:, 1]) * X[:, 3]],
                 axis=1).astype(np.float32)
    return X, T


def test_forward_matches_reference():
    p = IN.net_init(11)
    net = lbm.Net(p)
    X, _ = _data(1, 1000)
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty((1000, 2), dtype=torch.float32, device="cuda")
    net.forward(Xd, Yd)
    torch.cuda.synchronize()
    Yr, _ = M.forward(_rounded(p), DIMS, X.astype(np.float64))
    assert np.abs(Yd.cpu().numpy() - Yr).max() <= 1e-5 * max(1.0, np.abs(Yr).max())


def test_gradient_matches_reference():
    """FP32 accumulation of the loss gradient against the FP64 backpropagation
    (itself pinned by finite differences): within 1e-3 relative."""
    p = IN.net_init(12)
    net = lbm.Net(p)
    X, T = _data(2, 3000)
    loss, g = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), want_grad=True)
    Lr, gr = M.loss_grad(_rounded(p), DIMS, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - Lr) <= 1e-5 * Lr
    assert np.abs(g - gr).max() <= 1e-3 * np.abs(gr).max()


def test_adam_step_matches_reference():
    p = IN.net_init(13)
    net = lbm.Net(p)
    X, T = _data(3, 500)
    _, g = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), want_grad=True)
    net.adam(1e-3)
    p1 = net.get_params()
    pr, _, _ = M.adam(p.astype(np.float64), g.astype(np.float64), np.zeros(p.size), np.zeros(p.size), 1, 1e-3)
    assert np.abs(p1 - pr).max() <= 1e-7


def test_training_fits_a_smooth_function():
    X, T = _data(4, 20000)
    net, hist = SG.train(X, T, epochs=25, batch=2048, lr=3e-3, seed=5)
    assert hist[-1] < 0.05 * hist[0]


N_PIPE, R_PIPE = 36, 16.0
HA, CW = (10.0, 25.0), (0.01, 1.0)        # smaller c_w R is beyond the explicit Shercliff flux limit
PHYS = lbm.LBM_FLOW | lbm.LBM_MHD


@pytest.fixture(scope="module")
def trained():
    """A network trained on 48 steady pipes (R = 16, Ha in [10, 25], c_w in
    [0.01, 1]) that the batched solver itself produced."""
    draws = IN.pipe_draws(48, seed=2506, Ha=HA, cw=CW)
    X, T, stats = SG.generate(draws, n=N_PIPE, R=R_PIPE, tol=1e-5, batch=48, max_steps=100000)
    net, hist = SG.train(X, T, epochs=300, batch=1024, lr=3e-3, seed=7)
    return SG.Surrogate(net, HA, CW), hist


def _fluid(solid):
    return np.asarray(solid).reshape(-1) == 0


def _cold(group, prec=lbm.LBM_FP32, tol=1e-5):
    """Each case alone from rest; returns (steps, [(u1, b1) per case])."""
    steps, fields = [], []
    for case, solid, links, info in group:
        sol = lbm.Solver(lbm.LBM_D3Q19, prec, PHYS, [case])
        sol.set_walls(0, solid, links)
        sol.set_graph(100)
        k, res = sol.run_to_steady(100000, 100, tol)
        assert res < tol
        m = sol.moments(0)
        fl = _fluid(solid)
        steps.append(k)
        fields.append((m["u"][fl, 0], m["B"][fl, 0]))
        sol.close()
    return steps, fields


def test_training_reduces_the_normalised_loss(trained):
    sur, hist = trained
    assert hist[-1] < 2e-3 * hist[0], (hist[0], hist[-1])


def test_prediction_of_held_out_steady_fields(trained):
    """Held-out (Ha, c_w): the predicted axial velocity and induced field
    against the solver's own steady fields."""
    sur, _ = trained
    held = IN.pipe_draws(4, seed=2507, Ha=HA, cw=CW)
    group = SG.pipe_cases(held, N_PIPE, R_PIPE)
    _, fields = _cold(group)
    N = N_PIPE * N_PIPE
    for (case, solid, links, info), h, (u_ref, b_ref) in zip(group, held, fields):
        u = torch.empty(3 * N, device="cuda")
        B = torch.empty(3 * N, device="cuda")
        us, bs = SG.scales(info, R_PIPE)
        su, sb = sur.target_scale
        sur.net.pipe_fields((1, N_PIPE, N_PIPE), R_PIPE, SG.f_ha(h["Ha"]), SG.f_cw(h["cw"]), us * su, bs * sb,
                            info["B0"], u, B)
        fl = _fluid(solid)
        up = u.cpu().numpy().reshape(N, 3)[fl, 0]
        bp = B.cpu().numpy().reshape(N, 3)[fl, 0]
        eu = np.abs(up - u_ref).max() / np.abs(u_ref).max()
        eb = np.abs(bp - b_ref).max() / np.abs(b_ref).max()
        print("held-out Ha %.1f c_w %.3g: max error u %.3f, b %.3f" % (h["Ha"], h["cw"], eu, eb))
        assert eu < 0.1 and eb < 0.2, (eu, eb)


def test_warm_start_gains_over_cold_start(trained):
    """Held-out cases started from the network reach the residual in fewer
    steps than cold starts.  The interpolated bounce-back of the curved wall
    leaks mass (about 2.5e-8 of the total per step at R = 16) and through the
    Lorentz force the MHD velocity follows it, so the residual levels off near
    2e-6: the comparison stops at 1e-5."""
    sur, _ = trained
    held = IN.pipe_draws(6, seed=2507, Ha=HA, cw=CW)
    group = SG.pipe_cases(held, N_PIPE, R_PIPE)
    steps = {}
    for mode in ("cold", "warm"):
        sol = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, PHYS, [g[0] for g in group])
        for i, g in enumerate(group):
            sol.set_walls(i, g[1], g[2])
            if mode == "warm":
                assert SG.warm_start(sol, i, sur, g[3], (1, N_PIPE, N_PIPE), R_PIPE, held[i]["Ha"], held[i]["cw"])
        sol.set_graph(100)
        steps[mode], res = sol.run_to_steady(100000, 100, 1e-5)
        assert res < 1e-5
        sol.close()
    print(steps)
    assert steps["warm"] < 0.8 * steps["cold"], steps


def test_out_of_range_case_starts_cold(trained):
    sur, _ = trained
    c, solid, links, info = SG.pipe_cases([dict(Ha=30.0, cw=0.1)], N_PIPE, R_PIPE)[0]
    sol = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, PHYS, [c])
    sol.set_walls(0, solid, links)
    assert not SG.warm_start(sol, 0, sur, info, (1, N_PIPE, N_PIPE), R_PIPE, 30.0, 0.1)


def test_combined_form_reaches_the_plain_accuracy(trained):
    """Warm start + one launch for all cases + FP16 storage (stochastic
    rounding) until each case's residual levels off, then FP32, against the plain form (FP32, one case at a
    time, cold): both against the independent finite-volume solution of the
    pipe (the oracle), the combined error within 5 % of the plain one."""
    from oracle import pipe_fd as FD
    sur, _ = trained
    held = IN.pipe_draws(3, seed=2508, Ha=HA, cw=CW)
    group = SG.pipe_cases(held, N_PIPE, R_PIPE)
    _, plain = _cold(group)
    slo = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP16S, PHYS, [g[0] for g in group])
    s32 = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, PHYS, [g[0] for g in group])
    for i, g in enumerate(group):
        slo.set_walls(i, g[1], g[2])
        s32.set_walls(i, g[1], g[2])
        assert SG.warm_start(slo, i, sur, g[3], (1, N_PIPE, N_PIPE), R_PIPE, held[i]["Ha"], held[i]["cw"])
    slo.set_graph(100)
    s32.set_graph(100)
    rec = SD.two_precision_steady(slo, s32, 1e-5, 100000, 100)
    assert rec["lo_steps"] > 0 and rec["hi_residual"] < 1e-5
    c = (N_PIPE - 1) / 2.0
    zz, yy = np.meshgrid(np.arange(N_PIPE) - c, np.arange(N_PIPE) - c, indexing="ij")
    for i, ((case, solid, links, info), h) in enumerate(zip(group, held)):
        fl = _fluid(solid)
        r, th, uf, bf = FD.solve(R_PIPE, info["B0"], info["nu"], info["eta"], info["accel"],
                                 wall=("shercliff", h["cw"]), nr=64, nt=128)
        ua = FD.sample(r, th, uf, yy.ravel()[fl], zz.ravel()[fl])
        m = s32.moments(i)
        e_comb = np.abs(m["u"][fl, 0] - ua).max() / np.abs(ua).max()
        e_plain = np.abs(plain[i][0] - ua).max() / np.abs(ua).max()
        print("Ha %.1f c_w %.3g: error vs FV plain %.4f combined %.4f" % (h["Ha"], h["cw"], e_plain, e_comb))
        assert e_comb <= 1.05 * e_plain, (e_plain, e_comb)
