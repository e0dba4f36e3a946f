"""Pins of the FP64 reference MLP: backprop against central finite
differences, and plain facts of the architecture."""
import numpy as np

from oracle import mlp as M


def test_parameter_count():
    assert M.n_params() == 8 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 6 + 6 == 9286


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = M.init(1) + rng.normal(0, 0.01, M.n_params())
    X = rng.normal(0, 1, (37, 8))
    Y = rng.normal(0, 1, (37, 6))
    L, g = M.gradient(theta, X, Y)
    idx = rng.choice(M.n_params(), 300, replace=False)
    idx = np.concatenate([idx, [0, 511, 575, 9285, 9280, 4000]])
    h = 1e-6
    fd = np.array([(M.loss(theta + h * np.eye(1, M.n_params(), i)[0], X, Y) -
                    M.loss(theta - h * np.eye(1, M.n_params(), i)[0], X, Y)) / (2 * h)
                   for i in idx])
    assert np.max(np.abs(fd - g[idx])) <= 1e-6 * max(np.max(np.abs(g[idx])), 1e-12) + 1e-11
    assert abs(L - M.loss(theta, X, Y)) < 1e-15


def test_linear_output_layer_gradient_closed_form():
    """With zero hidden weights the hidden activations are tanh(b) constants,
    so the output-bias gradient is the mean residual times 2: a closed form."""
    theta = np.zeros(M.n_params())
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (11, 8))
    Y = rng.normal(0, 1, (11, 6))
    L, g = M.gradient(theta, X, Y)
    gb4 = g[-6:]
    assert np.allclose(gb4, -2.0 * Y.sum(axis=0) / Y.size, atol=1e-15)


def test_adam_reduces_the_loss():
    rng = np.random.default_rng(3)
    X = rng.normal(0, 1, (256, 8))
    Y = np.tanh(X[:, :6] * 0.7) + 0.1 * X[:, 2:8]
    theta = M.init(4)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = M.loss(theta, X, Y)
    for t in range(1, 201):
        _, g = M.gradient(theta, X, Y)
        theta, m, v = M.adam(theta, g, m, v, t, 3e-3)
    assert M.loss(theta, X, Y) < 0.2 * L0


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step (Kingma & Ba, Sec. 3), so each step moves theta by
    -lr g / (|g| + eps): after t steps theta_t = theta_0 - t lr g / (|g| + eps).
    A missing or wrong bias correction changes every step but the limit."""
    rng = np.random.default_rng(6)
    theta0 = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50) * np.logspace(-6, 2, 50)
    lr, eps = 1e-2, 1e-8
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        theta, m, v = M.adam(theta, g, m, v, t, lr, eps=eps)
        ref = theta0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(theta, ref, rtol=0, atol=1e-13), t


def test_adam_second_step_with_new_gradient():
    """Two steps with gradients g1 then g2 (b1, b2 as in the library): the
    bias-corrected moments are (b1 g1 + g2)/(1 + b1) and
    (b2 g1^2 + g2^2)/(1 + b2), written out from the recursions by hand."""
    rng = np.random.default_rng(7)
    theta0 = rng.normal(0, 1, 20)
    g1, g2 = rng.normal(0, 1, 20), rng.normal(0, 1, 20)
    b1, b2, lr, eps = 0.9, 0.999, 1e-3, 1e-8
    th, m, v = M.adam(theta0, g1, np.zeros(20), np.zeros(20), 1, lr)
    th, m, v = M.adam(th, g2, m, v, 2, lr)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    ref = theta0 - lr * g1 / (np.abs(g1) + eps) - lr * mh / (np.sqrt(vh) + eps)
    assert np.allclose(th, ref, rtol=0, atol=1e-14)
