"""FP64 tiled Householder QR run sequentially in elimination-list order.

Part of the test oracle (see ``oracle/__init__.py``).  The factorization is
the paper's generic tiled algorithm (Section 2): the elimination list of a
tree is expanded into TS or TT kernel tasks (``oracle.dag.expand``) and the
kernels of ``oracle.kernels`` are run one after the other in that program
order.  Any order that respects the dependencies gives the same numbers,
because every kernel reads only what its predecessors wrote.

A matrix whose sizes are not multiples of nb is treated as if zero-padded to
full tiles (the paper assumes full tiles, Section 3.2 remarks): R and the
reflectors are unchanged by the padding, and only the m x n part is returned.

Tile (i,k) of the paper (1-based) is block ``[(i-1)*nb:i*nb, (k-1)*nb:k*nb]``.
"""

import numpy as np

from . import dag
from . import kernels
from . import trees


class Factors:
    """Result of :func:`factor`: A overwritten by R and V, plus the T arrays.

    ``Tge[i-1, k-1]`` is the ib x nb T of GEQRT(i,k); ``Tel[i-1, k-1]`` is the
    T of the TTQRT/TSQRT that zeroed tile (i,k).  Entries of tasks that did
    not run are zero.
    """

    def __init__(self, A, m, n, nb, ib, p, q, elims, tasks, ts, Tge, Tel, done):
        self.A, self.m, self.n, self.nb, self.ib = A, m, n, nb, ib
        self.p, self.q, self.elims, self.tasks, self.ts = p, q, elims, tasks, ts
        self.Tge, self.Tel, self.done = Tge, Tel, done

    def r(self):
        """The n x n upper-triangular R."""
        return np.triu(self.A[: self.n, : self.n])


def _tile(M, nb, i, k):
    return M[(i - 1) * nb: i * nb, (k - 1) * nb: k * nb]


def task_flops(task, nb):
    """Work of one task in flops, from its Table 1 weight (unit nb^3/3)."""
    return dag.WEIGHT[task[0]] * nb ** 3 / 3.0


def factor(A, nb, ib, tree, BS=1, elims=None, max_tasks=None):
    """Tiled QR of the m x n matrix A (m >= n) with the given tree.

    ``elims`` (1-based triplets) replaces the tree's list when given.
    ``max_tasks`` runs only that many tasks of the program order (a bounded
    sample of the work); ``Factors.done`` says how many ran.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        raise ValueError("need m >= n")
    if nb % ib:
        raise ValueError("ib must divide nb")
    p, q = -(-m // nb), -(-n // nb)
    if elims is None:
        elims = trees.elimination_list(p, q, tree, BS)
    ts = trees.ts_flags(tree, BS, elims)
    tasks = dag.expand(p, q, elims, ts)
    W = np.zeros((p * nb, q * nb))
    W[:m, :n] = A
    Tge = np.zeros((p, q, ib, nb))
    Tel = np.zeros((p, q, ib, nb))
    limit = len(tasks) if max_tasks is None else min(max_tasks, len(tasks))
    for t in range(limit):
        kind, i, piv, k, j = tasks[t]
        if kind == dag.GEQRT:
            out, T = kernels.geqrt(_tile(W, nb, i, k), ib)
            _tile(W, nb, i, k)[:] = out
            Tge[i - 1, k - 1] = T
        elif kind == dag.UNMQR:
            _tile(W, nb, i, j)[:] = kernels.unmqr(_tile(W, nb, i, k), Tge[i - 1, k - 1],
                                                  _tile(W, nb, i, j))
        elif kind in (dag.TTQRT, dag.TSQRT):
            fn = kernels.ttqrt if kind == dag.TTQRT else kernels.tsqrt
            r1, r2, T = fn(_tile(W, nb, piv, k), _tile(W, nb, i, k), ib)
            _tile(W, nb, piv, k)[:] = r1
            _tile(W, nb, i, k)[:] = r2
            Tel[i - 1, k - 1] = T
        else:
            fn = kernels.ttmqr if kind == dag.TTMQR else kernels.tsmqr
            c1, c2 = fn(_tile(W, nb, i, k), Tel[i - 1, k - 1],
                        _tile(W, nb, piv, j), _tile(W, nb, i, j))
            _tile(W, nb, piv, j)[:] = c1
            _tile(W, nb, i, j)[:] = c2
    return Factors(W[:m, :n].copy(), m, n, nb, ib, p, q, elims, tasks, ts, Tge, Tel, limit)


def _apply(F, B, trans):
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    if B.shape[0] != F.m:
        raise ValueError("B must have m rows")
    nb = F.nb
    W = np.zeros((F.p * nb, F.q * nb))
    W[: F.m, : F.n] = F.A
    X = np.zeros((F.p * nb, B.shape[1]))
    X[: F.m] = B

    def rows(i):
        return X[(i - 1) * nb: i * nb]

    panels = [t for t in F.tasks[: F.done] if t[0] in (dag.GEQRT, dag.TTQRT, dag.TSQRT)]
    if not trans:
        panels = panels[::-1]
    for kind, i, piv, k, _ in panels:
        if kind == dag.GEQRT:
            rows(i)[:] = kernels.unmqr(_tile(W, nb, i, k), F.Tge[i - 1, k - 1], rows(i), trans)
        else:
            fn = kernels.ttmqr if kind == dag.TTQRT else kernels.tsmqr
            c1, c2 = fn(_tile(W, nb, i, k), F.Tel[i - 1, k - 1], rows(piv), rows(i), trans)
            rows(piv)[:] = c1
            rows(i)[:] = c2
    out = X[: F.m]
    return out[:, 0].copy() if vec else out.copy()


def apply_qt(F, B):
    """Q^T B: the factorization's transformations replayed on B (m x nrhs)."""
    return _apply(F, B, True)


def apply_q(F, B):
    """Q B: the transposed transformations replayed in reverse order."""
    return _apply(F, B, False)


def explicit_q(F):
    """The m x n orthonormal factor Q1 = Q [I_n; 0]."""
    E = np.zeros((F.m, F.n))
    E[: F.n, : F.n] = np.eye(F.n)
    return apply_q(F, E)


def lstsq(F, b):
    """Least-squares solution of min ||A x - b|| from the factors:
    x = R^{-1} (Q^T b)[:n], by back substitution."""
    c = apply_qt(F, b)[: F.n]
    R = F.r()
    x = np.zeros(F.n)
    for r in range(F.n - 1, -1, -1):
        x[r] = (c[r] - R[r, r + 1:] @ x[r + 1:]) / R[r, r]
    return x
