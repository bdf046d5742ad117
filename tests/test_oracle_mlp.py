"""Pins of the cost-model network reference (oracle/mlp.py) to facts that do
not come from it: central finite differences, a closed form in the linear
regime, the constant-output special case, and the bias-correction property of
Adam."""

import numpy as np
import pytest

from oracle import mlp

D = 7


def random_case(B=23, d=D, seed=0, margin=1e-3):
    """Parameters and inputs whose pre-activations all stay at least `margin`
    away from the ReLU kink, so that finite differences are valid."""
    rng = np.random.default_rng(seed)
    while True:
        theta = mlp.init(d, seed) + 0.05 * rng.standard_normal(mlp.param_count(d))
        X = rng.standard_normal((B, d))
        W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, d)
        z1 = X @ W1.T + b1
        z2 = np.maximum(z1, 0) @ W2.T + b2
        if np.abs(z1).min() > margin and np.abs(z2).min() > margin:
            return theta, X, rng.standard_normal(B)
        seed += 1


def test_param_count_and_unpack_cover_vector():
    d = 5
    P = mlp.param_count(d)
    theta = np.arange(P, dtype=np.float64)
    parts = mlp.unpack(theta, d)
    flat = np.concatenate([np.ravel(x) for x in parts])
    assert P == 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1
    assert np.array_equal(flat, theta)


def test_gradient_matches_central_differences():
    theta, X, t = random_case()
    loss, g = mlp.loss_and_grad(theta, X, t)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(mlp.param_count(D), 300, replace=False), [mlp.param_count(D) - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, t)[0] - mlp.loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i
    assert loss == pytest.approx(np.mean((mlp.forward(theta, X) - t) ** 2), rel=1e-15)


def test_linear_regime_closed_form():
    # With nonnegative weights, biases and inputs no ReLU is active, so the
    # network is the affine map x -> W3 W2 W1 x + (W3 W2 b1 + W3 b2 + b3).
    rng = np.random.default_rng(1)
    d = 4
    theta = np.abs(rng.standard_normal(mlp.param_count(d)))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, d)
    X = np.abs(rng.standard_normal((9, d)))
    M = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1) + W3 @ b2 + b3
    assert np.allclose(mlp.forward(theta, X), X @ M + c, rtol=1e-13)
    # and the gradient w.r.t. b3 is 2 * mean residual
    t = rng.standard_normal(9)
    _, g = mlp.loss_and_grad(theta, X, t)
    assert g[-1] == pytest.approx(2 * np.mean(X @ M + c - t), rel=1e-12)


def test_zero_weights_constant_output():
    d = 3
    theta = np.zeros(mlp.param_count(d))
    theta[-1] = 0.75
    X = np.random.default_rng(2).standard_normal((11, d))
    t = np.linspace(-1, 1, 11)
    loss, g = mlp.loss_and_grad(theta, X, t)
    assert np.all(mlp.forward(theta, X) == 0.75)
    assert loss == pytest.approx(np.mean((0.75 - t) ** 2))
    assert g[-1] == pytest.approx(2 * np.mean(0.75 - t))
    # every other parameter sits behind a zero weight or an inactive unit
    assert np.all(g[:-1] == 0)


def test_dead_units_have_zero_gradient():
    # A hidden unit of layer 1 with a very negative bias never activates:
    # its row of W1 and its bias receive no gradient.
    theta, X, t = random_case(seed=3)
    W1, b1, *_ = mlp.unpack(theta, D)
    b1[5] = -1e6
    _, g = mlp.loss_and_grad(theta, X, t)
    gW1 = g[:64 * D].reshape(64, D)
    gb1 = g[64 * D:64 * D + 64]
    assert np.all(gW1[5] == 0) and gb1[5] == 0
    assert np.any(gW1[4] != 0)


def test_adam_bias_correction():
    # With a constant gradient the bias-corrected moments equal g and g^2
    # exactly, so every step moves each parameter by lr * g / (|g| + eps).
    rng = np.random.default_rng(4)
    g = rng.standard_normal(50)
    theta = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 0.01, 1e-8
    cur = theta.copy()
    for step in range(1, 6):
        nxt, m, v = mlp.adam_step(cur, g, m, v, step, lr=lr, eps=eps)
        assert np.allclose(cur - nxt, lr * g / (np.abs(g) + eps), rtol=1e-10, atol=0)
        cur = nxt
    # zero gradient after a nonzero one keeps moving (momentum) with decaying size
    nxt, m2, v2 = mlp.adam_step(cur, np.zeros(50), m, v, 6, lr=lr, eps=eps)
    assert np.all(np.sign(cur - nxt) == np.sign(g))
