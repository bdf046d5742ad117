"""The six FP64 tile kernels of tiled QR, one Householder reflector at a time.

Part of the test oracle (see ``oracle/__init__.py``).  Kernels and their
costs are those of Section 2.1 (Table 1); their arithmetic is the textbook
Householder QR that the paper defers to (LAPACK-style kernels, compact WY
representation with inner blocking ib, Section 1).  0-based indices inside a
tile.  Nothing here is blocked or reordered: every reflector is generated
and applied in turn, exactly as its definition reads.

Reflector convention (the LAPACK one): for a vector (alpha, x),
  beta = -sign(alpha) * ||(alpha, x)||_2   with sign(0) = +1,
  tau  = (beta - alpha) / beta,   v = (1, x / (alpha - beta)),
so that (I - tau v v^T) (alpha, x) = (beta, 0).  When x = 0 the reflector is
the identity: tau = 0, beta = alpha.

Storage (PLASMA / LAPACK layout):
* GEQRT leaves R in the upper triangle of the tile and the reflector tails
  in the strict lower triangle (unit diagonal implied);
* TTQRT leaves the updated R in the upper triangle of the top tile and the
  reflector tails in the upper triangle (with diagonal) of the bottom tile;
* TSQRT leaves them in the whole bottom tile;
* T is an ib x nb array; columns b*ib..(b+1)*ib-1 hold the ib x ib upper
  triangular factor of reflector block b, with Q_b = I - V_b T_b V_b^T and
  Q = Q_0 Q_1 ... .  The diagonal of T holds the tau of every reflector.
"""

import math

import numpy as np


def reflector(alpha, x):
    """Householder reflector that maps (alpha, x) to (beta, 0).

    Returns (beta, tau, vtail) with the convention of the module docstring.
    """
    xnorm = math.sqrt(float(np.dot(x, x))) if x.size else 0.0
    if xnorm == 0.0:
        return alpha, 0.0, np.zeros_like(x)
    norm = math.sqrt(alpha * alpha + xnorm * xnorm)
    beta = -norm if alpha >= 0.0 else norm
    tau = (beta - alpha) / beta
    return beta, tau, x / (alpha - beta)


def form_t(V, tau, ib):
    """Compact-WY factor T (ib x nb) of the reflectors in the columns of V.

    ``V`` holds each full reflector vector (unit entry included) as a column.
    For every block of ib reflectors, T is built column by column (forward
    accumulation of a product of reflectors, Schreiber and Van Loan):
        T[:c, c] = -tau_c * T[:c, :c] @ (V[:, :c]^T v_c),   T[c, c] = tau_c.
    """
    nb = len(tau)
    T = np.zeros((ib, nb))
    for b0 in range(0, nb, ib):
        for c in range(ib):
            j = b0 + c
            T[c, j] = tau[j]
            if c == 0:
                continue
            g = V[:, b0:j].T @ V[:, j]
            T[:c, j] = -tau[j] * (T[:c, b0:j] @ g)
    return T


def tau_of(T):
    """The tau of every reflector: the diagonals of the ib x ib blocks of T."""
    ib, nb = T.shape
    return np.array([T[j % ib, j] for j in range(nb)])


# --------------------------------------------------------------------------
# GEQRT / UNMQR: factor a square tile; apply its Q^T (or Q) to another tile.
# --------------------------------------------------------------------------
def geqrt(A, ib):
    """Householder QR of one tile.  Returns (A_out, T): R and V in A_out."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    tau = np.zeros(n)
    Vfull = np.zeros((m, n))
    for j in range(n):
        if j >= m:
            continue
        beta, tau[j], v = reflector(A[j, j], A[j + 1:, j])
        A[j, j] = beta
        A[j + 1:, j] = v
        # H_j = I - tau u u^T with u = (1, v) acting on rows j..m-1.
        w = A[j, j + 1:] + v @ A[j + 1:, j + 1:]
        A[j, j + 1:] -= tau[j] * w
        A[j + 1:, j + 1:] -= tau[j] * np.outer(v, w)
        Vfull[j, j] = 1.0
        Vfull[j + 1:, j] = v
    return A, form_t(Vfull, tau, ib)


def unmqr(V, T, C, trans=True):
    """C <- Q^T C (trans) or Q C, Q = H_0 H_1 ... from a GEQRT tile V."""
    C = np.array(C, dtype=np.float64, copy=True)
    m, n = V.shape
    tau = tau_of(T)
    order = range(n) if trans else range(n - 1, -1, -1)
    for j in order:
        if j >= m or tau[j] == 0.0:
            continue
        v = V[j + 1:, j]
        w = C[j, :] + v @ C[j + 1:, :]
        C[j, :] -= tau[j] * w
        C[j + 1:, :] -= tau[j] * np.outer(v, w)
    return C


# --------------------------------------------------------------------------
# TTQRT / TTMQR: triangle on top of triangle.
# --------------------------------------------------------------------------
def ttqrt(R1, R2, ib):
    """QR of [R1; R2] with R1, R2 upper triangular (only their upper
    triangles are read).  Returns (R1_out, R2_out, T); reflector tails go to
    the upper triangle of R2_out, its strict lower triangle is left as is."""
    R1 = np.array(R1, dtype=np.float64, copy=True)
    R2 = np.array(R2, dtype=np.float64, copy=True)
    m2, n = R2.shape
    tau = np.zeros(n)
    Vfull = np.zeros((n + m2, n))     # rows 0..n-1: top tile, then bottom
    for j in range(n):
        top = min(j + 1, m2)          # rows 0..j of the bottom triangle
        beta, tau[j], v = reflector(R1[j, j], R2[:top, j])
        R1[j, j] = beta
        R2[:top, j] = v
        w = R1[j, j + 1:] + v @ R2[:top, j + 1:]
        R1[j, j + 1:] -= tau[j] * w
        R2[:top, j + 1:] -= tau[j] * np.outer(v, w)
        Vfull[j, j] = 1.0
        Vfull[n:n + top, j] = v
    return R1, R2, form_t(Vfull, tau, ib)


def ttmqr(V2, T, C1, C2, trans=True):
    """[C1; C2] <- Q^T [C1; C2] (trans) or Q [...] for a TTQRT Q."""
    C1 = np.array(C1, dtype=np.float64, copy=True)
    C2 = np.array(C2, dtype=np.float64, copy=True)
    m2, n = V2.shape
    tau = tau_of(T)
    order = range(n) if trans else range(n - 1, -1, -1)
    for j in order:
        if tau[j] == 0.0:
            continue
        top = min(j + 1, m2)
        v = V2[:top, j]
        w = C1[j, :] + v @ C2[:top, :]
        C1[j, :] -= tau[j] * w
        C2[:top, :] -= tau[j] * np.outer(v, w)
    return C1, C2


# --------------------------------------------------------------------------
# TSQRT / TSMQR: triangle on top of square.
# --------------------------------------------------------------------------
def tsqrt(R1, A2, ib):
    """QR of [R1; A2] with R1 upper triangular and A2 full.  Reflector tails
    overwrite A2."""
    R1 = np.array(R1, dtype=np.float64, copy=True)
    A2 = np.array(A2, dtype=np.float64, copy=True)
    m2, n = A2.shape
    tau = np.zeros(n)
    Vfull = np.zeros((n + m2, n))     # rows 0..n-1: top tile, then bottom
    for j in range(n):
        beta, tau[j], v = reflector(R1[j, j], A2[:, j])
        R1[j, j] = beta
        A2[:, j] = v
        w = R1[j, j + 1:] + v @ A2[:, j + 1:]
        R1[j, j + 1:] -= tau[j] * w
        A2[:, j + 1:] -= tau[j] * np.outer(v, w)
        Vfull[j, j] = 1.0
        Vfull[n:, j] = v
    return R1, A2, form_t(Vfull, tau, ib)


def tsmqr(V2, T, C1, C2, trans=True):
    """[C1; C2] <- Q^T [C1; C2] (trans) or Q [...] for a TSQRT Q."""
    C1 = np.array(C1, dtype=np.float64, copy=True)
    C2 = np.array(C2, dtype=np.float64, copy=True)
    m2, n = V2.shape
    tau = tau_of(T)
    order = range(n) if trans else range(n - 1, -1, -1)
    for j in order:
        if tau[j] == 0.0:
            continue
        v = V2[:, j]
        w = C1[j, :] + v @ C2
        C1[j, :] -= tau[j] * w
        C2 -= tau[j] * np.outer(v, w)
    return C1, C2
