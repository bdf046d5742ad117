"""Pins of the oracle's FP64 side.

The six tile kernels are checked against LAPACK's own tile-QR routines
(dgeqrt, dgemqrt, dtpqrt, dtpmqrt: the same kernels written independently),
the reflector against its defining identities, and the whole tiled
factorization against LAPACK's unblocked-equivalent QR (numpy) and the
invariants every QR factorization satisfies.
"""

import numpy as np
import pytest

from oracle import (BINARY, FIBONACCI, FLAT_TS, FLAT_TT, GREEDY, PLASMA,
                    PLASMA_TS, SAMEH_KUCK)
from oracle import kernels as K
from oracle import tiled_qr as tq

lapack = pytest.importorskip("scipy.linalg.lapack")

SIZES = [(8, 2), (16, 4), (16, 16), (24, 8), (32, 8)]


def rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def test_reflector_identities():
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 40):
        for alpha in (rng.standard_normal(), 0.0, -3.0):
            x = rng.standard_normal(n)
            beta, tau, v = K.reflector(alpha, x)
            u = np.concatenate([[1.0], v])
            H = np.eye(n + 1) - tau * np.outer(u, u)
            y = H @ np.concatenate([[alpha], x])
            assert abs(y[0] - beta) < 1e-13 * abs(beta)
            assert np.abs(y[1:]).max() < 1e-13 * abs(beta)
            assert np.abs(H @ H.T - np.eye(n + 1)).max() < 1e-14
            assert 1.0 <= tau <= 2.0
            assert abs(tau * (u @ u) - 2.0) < 1e-13          # orthogonality of H
            assert beta * alpha <= 0.0                         # -sign(alpha), sign(0)=+1
    beta, tau, v = K.reflector(2.5, np.zeros(3))
    assert (beta, tau) == (2.5, 0.0) and not v.any()


@pytest.mark.parametrize("nb,ib", SIZES)
def test_geqrt_unmqr_vs_lapack(nb, ib):
    rng = np.random.default_rng(nb * 100 + ib)
    A = rng.standard_normal((nb, nb))
    Ao, T = K.geqrt(A, ib)
    Al, Tl, info = lapack.dgeqrt(ib, A)
    assert info == 0
    assert rel(Ao, Al) < 1e-13 and rel(T, Tl) < 1e-13
    C = rng.standard_normal((nb, 5))
    for trans in ("T", "N"):
        Cl, info = lapack.dgemqrt(Al, Tl, C, side="L", trans=trans)
        assert rel(K.unmqr(Ao, T, C, trans=(trans == "T")), Cl) < 1e-13


@pytest.mark.parametrize("nb,ib", SIZES)
def test_ttqrt_ttmqr_vs_lapack(nb, ib):
    rng = np.random.default_rng(nb * 101 + ib)
    R1 = np.triu(rng.standard_normal((nb, nb)))
    B = rng.standard_normal((nb, nb))                  # lower part must be left alone
    r1, r2, T = K.ttqrt(R1, B, ib)
    a, b, Tl, info = lapack.dtpqrt(nb, ib, R1, np.triu(B))
    assert info == 0
    assert rel(np.triu(r1), np.triu(a)) < 1e-13
    assert rel(np.triu(r2), np.triu(b)) < 1e-13
    assert np.array_equal(np.tril(r2, -1), np.tril(B, -1))
    assert np.array_equal(np.tril(r1, -1), np.tril(R1, -1))
    assert rel(T, Tl) < 1e-13
    C1, C2 = rng.standard_normal((nb, 3)), rng.standard_normal((nb, 3))
    for trans in ("T", "N"):
        a_, b_, info = lapack.dtpmqrt(nb, np.triu(b), Tl, C1, C2, side="L", trans=trans)
        c1, c2 = K.ttmqr(r2, T, C1, C2, trans=(trans == "T"))
        assert rel(c1, a_) < 1e-13 and rel(c2, b_) < 1e-13


@pytest.mark.parametrize("nb,ib", SIZES)
def test_tsqrt_tsmqr_vs_lapack(nb, ib):
    rng = np.random.default_rng(nb * 103 + ib)
    R1 = np.triu(rng.standard_normal((nb, nb)))
    A2 = rng.standard_normal((nb, nb))
    r1, r2, T = K.tsqrt(R1, A2, ib)
    a, b, Tl, info = lapack.dtpqrt(0, ib, R1, A2)
    assert info == 0
    assert rel(np.triu(r1), np.triu(a)) < 1e-13 and rel(r2, b) < 1e-13 and rel(T, Tl) < 1e-13
    C1, C2 = rng.standard_normal((nb, 4)), rng.standard_normal((nb, 4))
    for trans in ("T", "N"):
        a_, b_, info = lapack.dtpmqrt(0, b, Tl, C1, C2, side="L", trans=trans)
        c1, c2 = K.tsmqr(r2, T, C1, C2, trans=(trans == "T"))
        assert rel(c1, a_) < 1e-13 and rel(c2, b_) < 1e-13


def test_geqrt_single_tile_equals_lapack_geqrf():
    """p = q = 1: the tiled algorithm is one GEQRT = LAPACK's Householder QR."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((32, 32))
    F = tq.factor(A, 32, 8, GREEDY)
    qr, tau, work, info = lapack.dgeqrf(A)
    assert rel(F.A, qr) < 1e-13
    assert rel(K.tau_of(F.Tge[0, 0]), tau) < 1e-13


TREES = [(FLAT_TS, 1), (FLAT_TT, 1), (SAMEH_KUCK, 1), (BINARY, 1), (FIBONACCI, 1), (GREEDY, 1),
         (PLASMA, 2), (PLASMA, 3), (PLASMA_TS, 2), (PLASMA_TS, 3)]


@pytest.mark.parametrize("tree,BS", TREES)
@pytest.mark.parametrize("m,n,nb,ib", [(96, 48, 16, 4), (100, 45, 16, 8), (64, 64, 16, 4),
                                       (70, 13, 8, 4), (16, 16, 16, 16)])
def test_tiled_qr_invariants(tree, BS, m, n, nb, ib):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n))
    F = tq.factor(A, nb, ib, tree, BS)
    R = F.r()
    Rl = np.linalg.qr(A, mode="r")
    D = np.sign(np.diag(R)) * np.sign(np.diag(Rl))
    assert rel(D[:, None] * R, Rl) < 1e-12
    assert np.allclose(R.T @ R, A.T @ A, rtol=0, atol=1e-12 * np.linalg.norm(A) ** 2)
    Q = tq.explicit_q(F)
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) < 1e-13
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) < 1e-13
    b = rng.standard_normal(m)
    qtb = tq.apply_qt(F, b)
    assert abs(np.linalg.norm(qtb) - np.linalg.norm(b)) < 1e-13 * np.linalg.norm(b)
    xl, res, *_ = np.linalg.lstsq(A, b, rcond=None)
    assert abs(np.linalg.norm(qtb[n:]) - np.linalg.norm(A @ xl - b)) < 1e-12 * np.linalg.norm(b)
    assert np.abs(tq.lstsq(F, b) - xl).max() < 1e-10
    assert np.allclose(tq.apply_q(F, qtb), b, atol=1e-13 * np.linalg.norm(b))


def test_trees_agree_on_r():
    rng = np.random.default_rng(11)
    A = rng.uniform(-0.5, 0.5, (80, 40))
    Rs = [tq.factor(A, 8, 4, t, bs).r() for t, bs in TREES]
    for R in Rs[1:]:
        D = np.sign(np.diag(R)) * np.sign(np.diag(Rs[0]))
        assert rel(D[:, None] * R, Rs[0]) < 1e-12


def test_zero_padding_is_exact():
    """A ragged matrix factors like its zero-padded full-tile version."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((37, 21))
    F = tq.factor(A, 8, 4, GREEDY)
    P = np.zeros((40, 24))
    P[:37, :21] = A
    G = tq.factor(P, 8, 4, GREEDY)
    assert rel(F.A, G.A[:37, :21]) < 1e-15
    assert np.abs(G.A[37:, :]).max() == 0.0


# ---------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Each plausible slip in the oracle makes a LAPACK pin fail."""
    rng = np.random.default_rng(3)
    nb, ib = 8, 4
    A = rng.standard_normal((nb, nb))
    Al, Tl, _ = lapack.dgeqrt(ib, A)
    good = K.reflector

    def wrong_sign(alpha, x):
        beta, tau, v = good(alpha, x)
        return -beta, (-beta - alpha) / -beta, x / (alpha + beta)

    monkeypatch.setattr(K, "reflector", wrong_sign)
    Ao, T = K.geqrt(A, ib)
    assert rel(Ao, Al) > 1e-3
    monkeypatch.setattr(K, "reflector", good)

    # dropped T off-diagonal term
    Ao, T = K.geqrt(A, ib)
    Tbad = T.copy()
    Tbad[0, 1] = 0.0
    assert rel(Tbad, Tl) > 1e-3
    # wrong order of reflectors in the update
    C = rng.standard_normal((nb, 3))
    Cl, _ = lapack.dgemqrt(Al, Tl, C, side="L", trans="T")
    assert rel(K.unmqr(Ao, T, C, trans=False), Cl) > 1e-3
    # TT kernel reading the full bottom tile instead of its triangle
    R1 = np.triu(rng.standard_normal((nb, nb)))
    B = rng.standard_normal((nb, nb))
    a, b, _, _ = lapack.dtpqrt(nb, ib, R1, np.triu(B))
    r1, _, _ = K.tsqrt(R1, B, ib)
    assert rel(np.triu(r1), np.triu(a)) > 1e-3
