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


def dot_f32_compensated(a, b):
    """The low-precision panel's Gram entry, emulated in numpy float32: exact
    products (p + pe, pe from one FMA) summed with TwoSum's error terms."""
    s, err = np.float32(0.0), np.float32(0.0)
    for x, y in zip(a, b):
        p = np.float32(x * y)
        pe = np.float32(np.float64(x) * np.float64(y) - np.float64(p))     # fmaf(x, y, -p): exact
        t = np.float32(s + p)
        bv = np.float32(t - s)
        e = np.float32(np.float32(s - np.float32(t - bv)) + np.float32(p - bv))
        err = np.float32(err + np.float32(e + pe))
        s = t
    return float(s) + float(err)


def test_compensated_f32_dot_is_exact_to_fp64_level():
    """Columns of FP32 reflector blocks (unit diagonal, random tails of mixed
    sign, lengths up to 256): the compensated FP32 dot product matches the
    exact dot product of the FP32 values to ~1e-12 relative, where a plain
    FP32 sum is off by ~1e-7."""
    rng = np.random.default_rng(4)
    worst, worst_plain = 0.0, 0.0
    for n in (8, 31, 128, 256):
        for _ in range(40):
            a = rng.standard_normal(n).astype(np.float32) * np.float32(0.1)
            b = rng.standard_normal(n).astype(np.float32) * np.float32(0.1)
            a[0] = np.float32(1.0)
            exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))     # products exact in FP64
            scale = float(np.dot(np.abs(a).astype(np.float64), np.abs(b).astype(np.float64)))
            worst = max(worst, abs(dot_f32_compensated(a, b) - exact) / scale)
            plain = np.float32(0.0)
            for x, y in zip(a, b):
                plain = np.float32(plain + np.float32(x * y))
            worst_plain = max(worst_plain, abs(float(plain) - exact) / scale)
    assert worst <= 1e-12, worst
    assert worst_plain >= 1e-9                       # the compensation is doing the work


def test_fp32_scalars_from_rsqrt_within_a_few_ulp():
    """The one-column kernel's FP32 reflector scalars: r = rsqrtf(s) (2 ulp),
    sqrt(s) = s r, 1/beta = -sign(alpha) r, scale = the correctly rounded
    reciprocal of alpha - beta.  Emulated in float32 with r perturbed by 2 ulp:
    beta, tau and scale stay within 8 ulp of the values computed in FP64."""
    rng = np.random.default_rng(1)
    f = np.float32
    eps = float(np.finfo(np.float32).eps)
    worst = 0.0
    for _ in range(20000):
        alpha = f(rng.standard_normal() * 10.0 ** rng.uniform(-6, 6))
        sig = f(abs(rng.standard_normal()) * 10.0 ** rng.uniform(-6, 6))
        s = f(np.float32(alpha) * alpha + sig)                 # fmaf(alpha, alpha, sig) up to 1 ulp
        if not (1e-30 < s < 1e30):
            continue
        r = f(f(1.0 / np.sqrt(np.float64(s))) * f(1.0 + rng.uniform(-2, 2) * eps))
        nrm = f(s * r)
        b = -nrm if alpha >= 0 else nrm
        rb = -r if alpha >= 0 else r
        tau = f(f(b - alpha) * rb)
        scale = f(1.0 / np.float64(f(alpha - b)))               # __frcp_rn: correctly rounded
        s64 = np.float64(alpha) ** 2 + np.float64(sig)
        bx = -np.sqrt(s64) if alpha >= 0 else np.sqrt(s64)
        for got, want in ((b, bx), (tau, (bx - alpha) / bx), (scale, 1.0 / (alpha - bx))):
            worst = max(worst, abs(float(got) - want) / abs(want))
    assert worst <= 8 * eps, worst / eps
