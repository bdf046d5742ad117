"""Reference for the cost model's network: a 3-layer perceptron
in -> 64 -> 64 -> 1 with ReLU, mean-squared-error loss, FP64.

Part of the test oracle (see ``oracle/__init__.py``).  The paper has no
learned component; this module exists to check the library's CUDA forward
and backward kernels.  Parameters are one flat vector in the library's order:
W1 (64 x in, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).
"""

import numpy as np

H = 64


def param_count(d):
    return H * d + H + H * H + H + H + 1


def unpack(theta, d):
    o = 0
    W1 = theta[o:o + H * d].reshape(H, d)
    o += H * d
    b1 = theta[o:o + H]
    o += H
    W2 = theta[o:o + H * H].reshape(H, H)
    o += H * H
    b2 = theta[o:o + H]
    o += H
    W3 = theta[o:o + H]
    o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def forward(theta, X):
    """Predictions for the rows of X (B x d)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), X.shape[1])
    a1 = np.maximum(X @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return a2 @ W3 + b3


def loss_and_grad(theta, X, t):
    """Mean squared error (1/B) sum (y - t)^2 and its gradient (chain rule)."""
    theta = np.asarray(theta, dtype=np.float64)
    B, d = X.shape
    W1, b1, W2, b2, W3, b3 = unpack(theta, d)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3 + b3
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    gW3 = a2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def init(d, seed=0):
    """He-style initialization (the library's Python side uses the same recipe)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, d)) * np.sqrt(2.0 / d)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0]])


def adam_step(theta, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1): exponential moving
    averages of the gradient and its square, bias-corrected by 1 - beta^step.
    Returns (theta, m, v) as new arrays."""
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return np.asarray(theta, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
