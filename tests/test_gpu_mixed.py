"""Mixed precision: FP64 panels with split-TF32 / TF32 tensor-core updates, and
the least-squares solver that refines such a factorization in FP64.

Tolerances.  A split-TF32 product carries about 21 bits (hi*hi + hi*lo +
lo*hi of 11-bit halves) and accumulates in FP32, so one update perturbs C by
about u_s = 2^-21 relative; a TF32 product keeps 11 bits, u_t = 2^-11.  The
factorization's backward error ||A - Q R~|| / ||A|| then grows like u * sqrt of
the number of updates a tile receives (q): the tests allow 16 u sqrt(q).  The
reflectors themselves are exact Householder transformations applied in FP64,
so Q stays orthogonal to FP64 accuracy.  Least squares must reach the FP64
path's backward error (times 2) when kappa(A) u_s < 1.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tiled_qr as otq
import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import workloads

pytestmark = pytest.mark.gpu

U_SPLIT, U_TF32 = 2.0 ** -21, 2.0 ** -11


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()


def explicit_q(f, m, n):
    E = np.zeros((m, n))
    E[:n, :n] = np.eye(n)
    Et = tqr.colmajor(E)
    tqr.tqr_apply_q(f, Et)
    tqr.tqr_sync(f)
    return tqr.to_numpy(Et)


@pytest.mark.parametrize("prec,u", [(tqr.TQR_SPLIT_TF32, U_SPLIT), (tqr.TQR_TF32, U_TF32)])
@pytest.mark.parametrize("m,n,nb,ib,tree", [
    (1024, 256, 64, 16, tqr.GREEDY),
    (1000, 300, 64, 32, tqr.FLAT_TS),
    (2048, 512, 256, 32, tqr.GREEDY),
    (1536, 768, 128, 32, tqr.FIBONACCI),
])
def test_mixed_factorization(prec, u, m, n, nb, ib, tree):
    A = workloads.gaussian(m, n, seed=11)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor_ex(At, nb, ib, tree, 1, prec)
    tqr.tqr_sync(f)
    Aout = tqr.to_numpy(At)
    R = np.triu(Aout[:n, :n])
    Q = explicit_q(f, m, n)
    q = -(-n // nb)
    back = np.linalg.norm(A - Q @ R) / np.linalg.norm(A)
    orth = np.linalg.norm(np.eye(n) - Q.T @ Q)
    assert orth <= 1e-13, orth
    assert back <= 16 * u * np.sqrt(q), (back, 16 * u * np.sqrt(q))
    # R~ is close to the FP64 oracle's R element-wise, up to row signs (R is
    # unique up to the signs of its rows; at TF32 accuracy a pivot near zero
    # can take the other sign).
    F = otq.factor(A, nb, ib, tree)
    kappa = np.linalg.cond(A)
    D = np.sign(np.diag(R)) * np.sign(np.diag(F.r()))
    err = np.abs(D[:, None] * R - F.r()).max() / np.abs(F.r()).max()
    assert err <= 16 * u * np.sqrt(q) * kappa, err
    # The FP64 path on the same handle afterwards is unaffected.
    At2 = tqr.colmajor(A)
    g = tqr.tqr_factor(At2, nb, ib, tree)
    tqr.tqr_sync(g)
    assert np.abs(tqr.to_numpy(At2) - F.A).max() / np.abs(F.r()).max() <= 1e-12
    f.free()
    g.free()


def solve(A, b, nb, ib, prec, tol=0.0, maxit=60):
    At = tqr.colmajor(A)
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.zeros(A.shape[1], dtype=torch.float64, device="cuda")
    info = tqr.tqr_lstsq(At, bt, xt, nb, ib, tqr.GREEDY, 1, prec, tol, maxit)
    return xt.cpu().numpy(), info, tqr.to_numpy(At)


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_lstsq_reaches_fp64_backward_error(kappa):
    m, n, nb, ib = 4096, 512, 128, 32
    A, b, x_true = workloads.ls_problem(m, n, kappa, seed=4)
    x64, info64, Aafter = solve(A, b, nb, ib, tqr.TQR_FP64)
    assert np.array_equal(Aafter, A)                      # A is left unchanged
    assert info64["converged"] == 1 and info64["status"] == 0
    xnp = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x64 - xnp) / np.linalg.norm(xnp) <= kappa * 1e-13
    # With the small residual of these problems (noise 1e-10), this backward
    # error measure is dominated by x's forward error: the bar is the FP64 path's.
    eta64 = info64["backward_error"]
    xs, infos, _ = solve(A, b, nb, ib, tqr.TQR_SPLIT_TF32, tol=2 * eta64)
    assert infos["converged"] == 1, infos
    assert infos["backward_error"] <= 2 * eta64
    assert np.linalg.norm(xs - xnp) / np.linalg.norm(xnp) <= kappa * 1e-13
    if kappa <= 1e2:
        xt_, infot, _ = solve(A, b, nb, ib, tqr.TQR_TF32, tol=2 * eta64)
        assert infot["converged"] == 1, infot
        assert np.linalg.norm(xt_ - xnp) / np.linalg.norm(xnp) <= kappa * 1e-13


def backward_error(A, b, x):
    r = b - A @ x
    return np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r))


@pytest.mark.parametrize("n,nb", [(300, 64), (512, 128)])
def test_lstsq_fp64_backward_error_matches_lapack(n, nb):
    """The FP64 path solves R x = Q^T b by back substitution, so its backward
    error stays within a small factor of LAPACK's (numpy lstsq) at kappa = 1e6,
    also when n is not a multiple of the substitution's 64-row blocks."""
    m, ib, kappa = 4096, 16, 1e6
    A, b, _ = workloads.ls_problem(m, n, kappa, seed=7)
    x64, info64, _ = solve(A, b, nb, ib, tqr.TQR_FP64)
    xnp = np.linalg.lstsq(A, b, rcond=None)[0]
    eta_np = backward_error(A, b, xnp)
    eta_gpu = backward_error(A, b, x64)
    assert info64["converged"] == 1 and info64["status"] == 0
    assert abs(info64["backward_error"] - eta_gpu) <= 0.1 * eta_gpu      # the reported eta is this eta
    assert eta_gpu <= 4 * eta_np, (eta_gpu, eta_np)
    assert np.linalg.norm(x64 - xnp) / np.linalg.norm(xnp) <= kappa * 1e-13
    # With a target, FP64 reports whether its backward error met it.
    _, info_t, _ = solve(A, b, nb, ib, tqr.TQR_FP64, tol=eta_gpu / 1e3)
    assert info_t["converged"] == 0


def test_lstsq_reuses_its_workspace():
    """The workspace kept for the next call gives the same solution on
    repeated calls, also after a call of another shape replaced it and after
    tqr_release_plans freed it.  (The refinement's dot products sum block
    partials in arrival order, so agreement is to rounding, not bitwise; a
    stale workspace would be far off.)"""
    A, b, _ = workloads.ls_problem(2048, 256, 1e4, seed=8)
    A2, b2, _ = workloads.ls_problem(1500, 200, 1e3, seed=9)
    same = lambda u, v: np.linalg.norm(u - v) <= 1e-12 * np.linalg.norm(u)
    tol = 2 * solve(A, b, 128, 32, tqr.TQR_FP64)[1]["backward_error"]
    x1, i1, _ = solve(A, b, 128, 32, tqr.TQR_SPLIT_TF32, tol=tol)
    x2, i2, _ = solve(A, b, 128, 32, tqr.TQR_SPLIT_TF32, tol=tol)
    assert same(x1, x2) and i1["converged"] == i2["converged"] == 1
    y1, _, _ = solve(A2, b2, 64, 16, tqr.TQR_FP64)
    x3, _, _ = solve(A, b, 128, 32, tqr.TQR_SPLIT_TF32, tol=tol)
    assert same(x1, x3)
    assert tqr.tqr_release_plans() >= 0
    x4, _, _ = solve(A, b, 128, 32, tqr.TQR_SPLIT_TF32, tol=tol)
    assert same(x1, x4)
    y2, _, _ = solve(A2, b2, 64, 16, tqr.TQR_FP64)
    assert same(y1, y2)
    xnp = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x1 - xnp) <= 1e4 * 1e-13 * np.linalg.norm(xnp)


def test_lstsq_ill_conditioned_reports_honestly():
    """kappa = 1e10 with split-TF32: kappa * u_s >> 1, plain refinement cannot
    contract; the solver hands over to preconditioned CGLS and reports whether
    it reached the target.  Its backward error never ends above the first
    solution's."""
    m, n, nb, ib = 2048, 256, 64, 16
    A, b, _ = workloads.ls_problem(m, n, 1e10, seed=5)
    x64, info64, _ = solve(A, b, nb, ib, tqr.TQR_FP64)
    _, info0, _ = solve(A, b, nb, ib, tqr.TQR_SPLIT_TF32, tol=1.0, maxit=0)
    xs, infos, _ = solve(A, b, nb, ib, tqr.TQR_SPLIT_TF32, tol=2 * info64["backward_error"], maxit=200)
    assert infos["backward_error"] <= info0["backward_error"]
    assert infos["converged"] in (0, 1)
    if infos["converged"]:
        assert infos["backward_error"] <= 2 * info64["backward_error"]


def test_lstsq_binding_rejects_wrong_vectors_before_the_call():
    """b and x must be contiguous float64 CUDA tensors of m and n elements:
    a short b, a float32 b and a strided x are refused before the library
    is called."""
    A = tqr.colmajor(workloads.gaussian(64, 32, seed=5))
    x = torch.zeros(32, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        tqr.tqr_lstsq(A, torch.zeros(63, dtype=torch.float64, device="cuda"), x, 32, 8, tqr.GREEDY)
    with pytest.raises(TypeError):
        tqr.tqr_lstsq(A, torch.zeros(64, dtype=torch.float32, device="cuda"), x, 32, 8, tqr.GREEDY)
    with pytest.raises(TypeError):
        tqr.tqr_lstsq(A, torch.zeros(64, dtype=torch.float64, device="cuda"),
                      torch.zeros(64, dtype=torch.float64, device="cuda")[::2], 32, 8, tqr.GREEDY)


def test_low_precision_refuses_layouts_not_checked_on_the_gpu():
    """Low-precision updates run only with nb >= 64 (64-column strips) and
    ib in {16, 32}; other configurations are refused, not run unchecked."""
    for nb, ib in ((32, 16), (48, 16), (64, 64)):
        A = tqr.colmajor(workloads.gaussian(256, 128, seed=6))
        with pytest.raises(tqr.TqrError) as e:
            tqr.tqr_factor_ex(A, nb, ib, tqr.GREEDY, 1, tqr.TQR_SPLIT_TF32)
        assert e.value.code == tqr.TQR_ERR_UNSUPPORTED
