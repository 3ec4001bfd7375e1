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


def test_warm_start_gains_over_cold_start():
    """Train on steady pipes solved by the batched solver itself (R = 16,
    Ha in [10, 25], c_w in [1e-3, 1]); held-out cases started from the network
    reach the same residual in fewer steps; an out-of-range case starts cold."""
    n, R = 36, 16.0
    ha = (10.0, 25.0)
    draws = IN.pipe_draws(48, seed=2506, Ha=ha)
    X, T, stats = SG.generate(draws, n=n, R=R, tol=1e-7, batch=48)
    net, hist = SG.train(X, T, epochs=60, batch=4096, lr=3e-3, seed=7)
    assert hist[-1] < 0.02 * hist[0]
    net = SG.Surrogate(net, ha, SG.CW_RANGE)
    held = IN.pipe_draws(6, seed=2507, Ha=ha)
    group = SG.pipe_cases(held, n, R)
    steps = {}
    for mode in ("cold", "warm"):
        sol = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, [g[0] for g in group])
        for i, g in enumerate(group):
            sol.set_walls(i, g[1], g[2])
            if mode == "warm":
                assert SG.warm_start(sol, i, net, g[3], (1, n, n), R, held[i]["Ha"], held[i]["cw"])
        sol.set_graph(100)
        steps[mode], res = sol.run_to_steady(400000, 100, 1e-6)
        assert res < 1e-6
        sol.close()
    assert steps["warm"] < 0.8 * steps["cold"], steps
    # outside the training range: cold start
    c, solid, links, info = SG.pipe_cases([dict(Ha=30.0, cw=0.1)], n, R)[0]
    sol = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, lbm.LBM_FLOW | lbm.LBM_MHD, [c])
    sol.set_walls(0, solid, links)
    assert not SG.warm_start(sol, 0, net, info, (1, n, n), R, 30.0, 0.1)
