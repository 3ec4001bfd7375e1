"""FP64 reference of the warm-start network (test infrastructure only).

The network (not part of the paper's method; it only supplies initial
fields): layers l = 1..L with z_l = W_l a_{l-1} + b_l, a_l = tanh(z_l) for the
hidden layers and a linear output y = z_L.  Parameters are one flat vector,
layer by layer: W_l (rows = outputs, row-major) then b_l.  Loss: mean squared
error over all samples and outputs, L = (1/(n m)) sum_i sum_k (y_ik - t_ik)^2.
Adam (Kingma & Ba 2015) with bias correction.

Pinned by central finite differences of the loss (tests/test_oracle_mlp.py).
"""
import numpy as np


def n_params(dims):
    return sum(dims[i + 1] * dims[i] + dims[i + 1] for i in range(len(dims) - 1))


def unpack(params, dims):
    out, o = [], 0
    for i in range(len(dims) - 1):
        m, k = dims[i + 1], dims[i]
        W = params[o:o + m * k].reshape(m, k)
        o += m * k
        b = params[o:o + m]
        o += m
        out.append((W, b))
    return out


def forward(params, dims, X):
    """X: (n, dims[0]) -> (Y (n, dims[-1]), activations list)."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    a = np.asarray(X, dtype=np.float64)
    acts = [a]
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.tanh(z) if li < len(layers) - 1 else z
        acts.append(a)
    return a, acts


def loss(params, dims, X, T):
    Y, _ = forward(params, dims, X)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def loss_grad(params, dims, X, T):
    """(loss, gradient with the layout of params) by backpropagation."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    Y, acts = forward(params, dims, X)
    T = np.asarray(T, dtype=np.float64)
    n, m = Y.shape
    L = float(np.mean((Y - T) ** 2))
    delta = 2.0 * (Y - T) / (n * m)            # dL/dz of the linear output layer
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a_prev = acts[li]
        gW = delta.T @ a_prev
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            delta = (delta @ W) * (1.0 - acts[li] ** 2)    # through tanh of the layer below
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat


def adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; returns (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
