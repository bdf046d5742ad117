"""Seeded synthetic inputs for tiled QR.

This module holds input generators only (no arithmetic of the method); the
CUDA path's tests, the bench and the CPU oracle's checks all draw their
matrices from here so that both sides see the same numbers.

Workloads (entries are iid, generated on the host with numpy's PCG64):
* ``gaussian(m, n, seed)``  -- N(0,1) entries, column-major float64;
* ``uniform(m, n, seed)``   -- U[-0.5, 0.5] entries;
* ``rhs(m, nrhs, seed)``    -- N(0,1) right-hand sides.
"""

import numpy as np


def gaussian(m, n, seed=0):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)))


def uniform(m, n, seed=1):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-0.5, 0.5, (m, n)))


def rhs(m, nrhs=1, seed=2):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, nrhs)))


def small_config(seed=0):
    """1024 x 256, nb 64, ib 16 (16 x 4 tiles), Greedy, N(0,1) entries and an
    N(0,1) right-hand side drawn from the same stream."""
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((1024, 256)))
    b = rng.standard_normal(1024)
    return A, b


def haar(m, n, rng):
    """An m x n matrix with orthonormal columns, Haar distributed: the Q factor
    of a Gaussian matrix with the signs of diag(R) made positive (numpy's QR
    is used only to draw the input)."""
    Z = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))


def ls_problem(m, n, kappa, seed=3, noise=1e-10):
    """Least-squares test problem: A = U diag(sigma) V^T with Haar U (m x n) and
    V (n x n), sigma log-spaced from 1 down to 1/kappa; x_true ~ N(0,1);
    b = A x_true + noise * N(0,1).  Returns (A (Fortran order), b, x_true)."""
    rng = np.random.default_rng(seed)
    U = haar(m, n, rng)
    V = haar(n, n, rng)
    sigma = np.logspace(0.0, -np.log10(kappa), n)
    A = np.asfortranarray((U * sigma) @ V.T)
    x = rng.standard_normal(n)
    b = A @ x + noise * rng.standard_normal(m)
    return A, b, x


def ls_problem_device(m, n, kappa, seed=3, noise=1e-10, device="cuda"):
    """ls_problem drawn and assembled on the GPU with torch (for sizes where
    the host would take minutes): same recipe, torch's generator and QR.
    Returns CUDA tensors (A column-major, b, x_true)."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)

    def haar_t(r, c):
        Z = torch.randn(r, c, generator=g, dtype=torch.float64, device=device)
        Q, R = torch.linalg.qr(Z)
        return Q * torch.sign(torch.diagonal(R))

    U = haar_t(m, n)
    V = haar_t(n, n)
    sigma = torch.logspace(0.0, -float(np.log10(kappa)), n, dtype=torch.float64, device=device)
    A = (U * sigma) @ V.T
    del U
    x = torch.randn(n, generator=g, dtype=torch.float64, device=device)
    b = A @ x + noise * torch.randn(m, generator=g, dtype=torch.float64, device=device)
    Acm = A.T.contiguous().T          # column-major copy
    return Acm, b, x


def sweep_config(q, seed=1):
    """m = 16384 (64 tile rows of nb = 256), n = 256 q, U[-0.5, 0.5] entries."""
    return uniform(16384, 256 * q, seed)
