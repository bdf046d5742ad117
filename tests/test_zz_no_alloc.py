"""tqr_factor_noalloc, the factorization for callers that cannot allocate
(stream capture, fixed memory budgets, real-time loops): through the C ABI,
its output must match tqr_factor's on two calls in a row, and problems beyond
its fixed 4 MiB scratch must be refused without a launch.

This file is collected last on purpose (pytest orders files by name).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def tol_for(A):
    """The parity suite's element-wise tolerance: 8 kappa(A) m u, floor 1e-13."""
    return max(1e-13, 8 * np.linalg.cond(A) * A.shape[0] * U)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()


def reference_factor(A, nb, ib, tree):
    """R, V and tau from the allocating entry point tqr_factor."""
    m, n = A.shape
    p, q = -(-m // nb), -(-n // nb)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, nb, ib, tree)
    Tge = torch.zeros(p * q * ib * nb, dtype=torch.float64, device="cuda")
    Tel = torch.zeros_like(Tge)
    tqr.tqr_form_t(f, Tge, Tel)
    tqr.tqr_sync(f)
    f.free()

    def taus(T):   # diagonal of each ib x ib block = tau of every reflector
        T = T.cpu().numpy().reshape(q, p, nb, ib)
        return np.array([[[T[k, i, r, r % ib] for r in range(nb)] for i in range(p)] for k in range(q)])

    return tqr.to_numpy(At), taus(Tge), taus(Tel)


@pytest.mark.parametrize("m,n,nb,ib,tree", [(1024, 256, 64, 16, tqr.GREEDY), (700, 300, 48, 16, tqr.FLAT_TS)])
def test_noalloc_matches_tqr_factor_on_two_calls(m, n, nb, ib, tree):
    p, q = -(-m // nb), -(-n // nb)
    elims = tqr.tqr_elimination_list(p, q, tree)
    tau_ge = torch.zeros(p * q * nb, dtype=torch.float64, device="cuda")
    tau_el = torch.zeros_like(tau_ge)
    status = torch.full((1,), -999, dtype=torch.int32, device="cuda")
    for call in range(2):                                  # two calls in a row, new input each time
        A = workloads.gaussian(m, n, seed=100 + call)
        ref, ref_tau_ge, ref_tau_el = reference_factor(A, nb, ib, tree)
        At = tqr.colmajor(A)
        rc = tqr.tqr_factor_noalloc(At, nb, ib, elims, tau_ge, tau_el, status, ts=(tree == tqr.FLAT_TS))
        assert rc == 0, tqr.tqr_strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        tol = tol_for(A)
        scale = np.abs(np.triu(ref[:n, :n])).max()
        assert np.abs(tqr.to_numpy(At) - ref).max() / scale <= tol
        got_ge = tau_ge.cpu().numpy().reshape(q, p, nb)
        got_el = tau_el.cpu().numpy().reshape(q, p, nb)
        assert np.abs(got_ge - ref_tau_ge).max() <= tol
        assert np.abs(got_el - ref_tau_el).max() <= tol


@pytest.mark.parametrize("m,n,nb,ib,tree", [(1024, 256, 64, 16, tqr.GREEDY), (700, 300, 48, 16, tqr.FLAT_TS),
                                           (600, 250, 64, 8, tqr.BINARY)])
def test_noalloc_matches_the_oracle(m, n, nb, ib, tree):
    """R, V and every tau element-wise against the CPU oracle's factorization
    with the same tree (not only against tqr_factor)."""
    from oracle import tiled_qr as otq
    p, q = -(-m // nb), -(-n // nb)
    A = workloads.gaussian(m, n, seed=130)
    F = otq.factor(A, nb, ib, tree)
    At = tqr.colmajor(A)
    tau_ge = torch.zeros(p * q * nb, dtype=torch.float64, device="cuda")
    tau_el = torch.zeros_like(tau_ge)
    status = torch.full((1,), -999, dtype=torch.int32, device="cuda")
    rc = tqr.tqr_factor_noalloc(At, nb, ib, tqr.tqr_elimination_list(p, q, tree), tau_ge, tau_el, status,
                                ts=(tree == tqr.FLAT_TS))
    assert rc == 0, tqr.tqr_strerror(rc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    tol = tol_for(A)
    scale = np.abs(F.r()).max()
    assert np.abs(tqr.to_numpy(At) - F.A).max() / scale <= tol

    def taus(T):   # the oracle's T blocks carry tau on their diagonal
        return np.array([[[T[i, k][r % ib, r] for r in range(nb)] for i in range(p)] for k in range(q)])

    assert np.abs(tau_ge.cpu().numpy().reshape(q, p, nb) - taus(F.Tge)).max() <= tol
    assert np.abs(tau_el.cpu().numpy().reshape(q, p, nb) - taus(F.Tel)).max() <= tol


def test_noalloc_refuses_problems_beyond_its_scratch():
    A = tqr.colmajor(np.zeros((8, 8)))
    tau = torch.zeros(8, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = tqr.lib()
    ct = tqr.tqr.ctypes
    dummy = np.zeros(3, dtype=np.int32)
    ptr = dummy.ctypes.data_as(ct.POINTER(ct.c_int32))
    s = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    a = ct.c_void_p(A.data_ptr())
    t = ct.c_void_p(tau.data_ptr())
    st = ct.c_void_p(status.data_ptr())
    # 65 x 64 tiles: more tiles than the scratch holds.
    assert L.tqr_factor_noalloc(a, 65 * 256, 64 * 256, 256, 32, ptr, 1, 0, t, t, st, s) == tqr.TQR_ERR_TOO_LARGE
    # 64 x 32 tiles at nb 256: the strip task graph exceeds the task limit.
    elims = tqr.tqr_elimination_list(64, 32, tqr.GREEDY)
    eptr = elims.ctypes.data_as(ct.POINTER(ct.c_int32))
    assert L.tqr_factor_noalloc(a, 64 * 256, 32 * 256, 256, 32, eptr, elims.shape[0], 0, t, t, st,
                                s) == tqr.TQR_ERR_TOO_LARGE
    assert "scratch" in tqr.tqr_strerror(tqr.TQR_ERR_TOO_LARGE)


def test_noalloc_rejects_ts_on_triangle_tile():
    """A BinaryTree list eliminates earlier pivots, whose tiles are triangles:
    invalid with TS kernels, before anything is launched."""
    p, q, nb, ib = 8, 2, 32, 8
    A = tqr.colmajor(workloads.gaussian(p * nb, q * nb, seed=13))
    elims = tqr.tqr_elimination_list(p, q, tqr.BINARY)
    tau = torch.zeros(p * q * nb, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = tqr.tqr_factor_noalloc(A, nb, ib, elims, tau, tau.clone(), status, ts=True)
    assert rc == tqr.TQR_ERR_INVALID_LIST


def test_noalloc_captured_in_cuda_graph_replays_tqr_factor():
    """Captured into a CUDA graph (after a first call outside the capture, as
    documented), each replay factors the matrix in place exactly as the
    uncaptured call does, also after an uncaptured call for another problem
    has rewritten the library's static graph arrays in between."""
    m, n, nb, ib, tree = 1024, 256, 64, 16, tqr.GREEDY
    p, q = -(-m // nb), -(-n // nb)
    elims = tqr.tqr_elimination_list(p, q, tree)
    A = workloads.gaussian(m, n, seed=120)
    tau_ge = torch.zeros(p * q * nb, dtype=torch.float64, device="cuda")
    tau_el = torch.zeros_like(tau_ge)
    status = torch.full((1,), -999, dtype=torch.int32, device="cuda")
    want = tqr.colmajor(A)                                  # the uncaptured call's result
    assert tqr.tqr_factor_noalloc(want, nb, ib, elims, tau_ge, tau_el, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    want = tqr.to_numpy(want)
    want_tau = (tau_ge.cpu().numpy(), tau_el.cpu().numpy())

    At = tqr.colmajor(A)
    pristine = At.clone()
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            rc = tqr.tqr_factor_noalloc(At, nb, ib, elims, tau_ge, tau_el, status, stream=stream)
    assert rc == 0, tqr.tqr_strerror(rc)
    for rep in range(2):
        At.copy_(pristine)
        tau_ge.zero_()
        tau_el.zero_()
        if rep == 1:                                        # another problem in between, uncaptured
            B = tqr.colmajor(workloads.gaussian(300, 100, seed=121))
            e2 = tqr.tqr_elimination_list(-(-300 // 32), -(-100 // 32), tqr.BINARY)
            t2 = torch.zeros(10 * 4 * 32, dtype=torch.float64, device="cuda")
            assert tqr.tqr_factor_noalloc(B, 32, 8, e2, t2, t2.clone(), status) == 0
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(tqr.to_numpy(At), want)
        assert np.array_equal(tau_ge.cpu().numpy(), want_tau[0])
        assert np.array_equal(tau_el.cpu().numpy(), want_tau[1])
