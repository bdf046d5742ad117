"""Accuracy of the Newton-iteration reflector scalars used by the GPU kernels
(rsqrt and reciprocal from FP32 seeds, two Newton steps each), emulated on the
CPU with seeds perturbed by the FP32 approximation error: beta, tau and scale
stay within a few ulp of the exactly computed values, as the quadratic
convergence of Newton's method predicts."""

import numpy as np


def newton_scalars(alpha, sig, seed_err):
    s = np.fma(alpha, alpha, sig) if hasattr(np, "fma") else alpha * alpha + sig
    h = 0.5 * s
    r = float(np.float32(1.0 / np.sqrt(np.float32(s)))) * (1.0 + seed_err)
    r = r * (1.5 - h * (r * r))
    r = r * (1.5 - h * (r * r))
    nrm = s * r
    b = -nrm if alpha >= 0 else nrm
    rb = -r if alpha >= 0 else r
    d = alpha - b
    q = float(np.float32(1.0 / np.float32(d))) * (1.0 - seed_err)
    q = q + q * (1.0 - d * q)
    q = q + q * (1.0 - d * q)
    return b, (b - alpha) * rb, q


def test_newton_scalars_within_a_few_ulp():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(20000):
        e = rng.uniform(-13, 13)
        alpha = rng.standard_normal() * 10.0 ** e
        sig = abs(rng.standard_normal()) * 10.0 ** rng.uniform(-13, 13)
        s = alpha * alpha + sig
        if not (1e-30 < s < 1e30):
            continue                                  # the kernels use IEEE sqrt / division there
        b, tau, scale = newton_scalars(alpha, sig, rng.uniform(-2.0 ** -21, 2.0 ** -21))
        nrm = np.sqrt(s)
        bx = -nrm if alpha >= 0 else nrm
        for got, want in ((b, bx), (tau, (bx - alpha) / bx), (scale, 1.0 / (alpha - bx))):
            worst = max(worst, abs(got - want) / abs(want))
    assert worst < 8 * 2.0 ** -53, worst
