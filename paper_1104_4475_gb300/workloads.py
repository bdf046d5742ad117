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


def sweep_config(q, seed=1):
    """m = 16384 (64 tile rows of nb = 256), n = 256 q, U[-0.5, 0.5] entries."""
    return uniform(16384, 256 * q, seed)
