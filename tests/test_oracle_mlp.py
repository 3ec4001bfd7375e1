"""Pins of the FP64 network reference: backpropagation against central finite
differences, and Adam against its closed-form first steps."""
import numpy as np

from oracle import mlp as M

DIMS = [4, 16, 16, 16, 2]


def _setup(seed=3):
    r = np.random.default_rng(seed)
    p = r.normal(0, 0.4, M.n_params(DIMS))
    X = r.uniform(-1, 1, (37, 4))
    T = r.uniform(-1, 1, (37, 2))
    return p, X, T


def test_param_count_and_layout():
    assert M.n_params([4, 64, 64, 64, 2]) == 64 * 4 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    p, X, T = _setup()
    layers = M.unpack(p, DIMS)
    assert [W.shape for W, _ in layers] == [(16, 4), (16, 16), (16, 16), (2, 16)]
    # the first row of the first layer acts on x alone: z = W[0] . x + b[0]
    _, acts = M.forward(p, DIMS, X)
    W1, b1 = layers[0]
    assert np.allclose(acts[1][:, 0], np.tanh(X @ W1[0] + b1[0]), atol=1e-15)


def test_backprop_matches_central_differences():
    p, X, T = _setup()
    L, g = M.loss_grad(p, DIMS, X, T)
    assert abs(L - M.loss(p, DIMS, X, T)) < 1e-15
    r = np.random.default_rng(5)
    idx = r.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss(p + e, DIMS, X, T) - M.loss(p - e, DIMS, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_a_sign_step():
    """With bias correction the first Adam step moves every parameter by
    lr * g / (|g| + eps) ~ lr * sign(g)."""
    p, X, T = _setup()
    _, g = M.loss_grad(p, DIMS, X, T)
    p1, m, v = M.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    assert np.allclose(p - p1, 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_training_reduces_the_loss():
    p, X, T = _setup()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = M.loss(p, DIMS, X, T)
    for s in range(1, 301):
        _, g = M.loss_grad(p, DIMS, X, T)
        p, m, v = M.adam(p, g, m, v, s, 1e-2)
    assert M.loss(p, DIMS, X, T) < 0.1 * L0
