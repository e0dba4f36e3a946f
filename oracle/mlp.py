"""Plain FP64 reference of the chemistry-surrogate MLP (numpy).

TEST INFRASTRUCTURE ONLY (used by the tests and the smoke check).  The
network maps the normalised state (T, Y_1..Y_6, P0) to the normalised species
change over one step: 8 -> 64 -> 64 -> 64 -> 6, tanh on the hidden layers,
linear output, loss = mean squared error over all outputs.  Parameters are a
flat float vector in the order W1 (8x64, input-major), b1, W2 (64x64), b2, W3,
b3, W4 (64x6), b4; y = x W + b per layer.  Parity pin: the backpropagated
gradient against central finite differences (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

DIMS = [8, 64, 64, 64, 6]


def n_params(dims=DIMS):
    return sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))


def unpack(theta, dims=DIMS):
    out, o = [], 0
    for i in range(len(dims) - 1):
        a, b = dims[i], dims[i + 1]
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def init(seed, dims=DIMS):
    """Seeded Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(dims) - 1):
        a, b = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / (a + b))
        parts += [rng.uniform(-lim, lim, a * b), np.zeros(b)]
    return np.concatenate(parts)


def forward(theta, X, dims=DIMS):
    layers = unpack(theta, dims)
    hs = [np.asarray(X, dtype=np.float64)]
    for i, (W, b) in enumerate(layers):
        z = hs[-1] @ W + b
        hs.append(np.tanh(z) if i < len(layers) - 1 else z)
    return hs[-1], hs


def loss(theta, X, Y, dims=DIMS):
    out, _ = forward(theta, X, dims)
    return float(np.mean((out - Y) ** 2))


def gradient(theta, X, Y, dims=DIMS):
    """Backpropagation of the mean squared error; returns (loss, flat grad)."""
    layers = unpack(theta, dims)
    out, hs = forward(theta, X, dims)
    n = out.size
    d = 2.0 * (out - Y) / n
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        h_in = hs[i]
        grads.append((h_in.T @ d, d.sum(axis=0)))
        if i > 0:
            d = (d @ W.T) * (1.0 - hs[i] ** 2)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return float(np.mean((out - Y) ** 2)), flat


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
