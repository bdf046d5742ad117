"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Element-wise tolerance.  The library and the oracle run the same reflectors
in the same order but sum dot products in a different order, so each result
is a backward-stable QR of A with its own rounding.  Perturbation theory of
QR bounds the difference of two such R (and of the reflectors, whose entries
are at most 1 in magnitude) by about kappa(A) * m * u * ||A||; the tests take
TOL * max|R| with TOL = 8 * kappa(A) * m * u (u = 2^-53), floored at 1e-13.
Independently of the oracle, every GPU result must meet the absolute targets
||A - QR||_F / ||A||_F <= 1e-13 and ||I - Q^T Q||_F <= 1e-13.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import FLAT_TS as O_FLAT_TS
from oracle import tiled_qr as otq
from oracle import trees as otrees
import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()
    tqr.tqr_set_timeout_ms(0)


def tol_for(A):
    kappa = np.linalg.cond(A)
    return max(1e-13, 8 * kappa * A.shape[0] * U)


def gpu_factor(A, nb, ib, tree, BS=1):
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, nb, ib, tree, BS)
    tqr.tqr_sync(f)
    return f, tqr.to_numpy(At)


def gpu_q_explicit(f, m, n):
    E = np.zeros((m, n))
    E[:n, :n] = np.eye(n)
    Et = tqr.colmajor(E)
    tqr.tqr_apply_q(f, Et)
    tqr.tqr_sync(f)
    return tqr.to_numpy(Et)


def check_targets(f, A, Aout):
    m, n = A.shape
    R = np.triu(Aout[:n, :n])
    Q = gpu_q_explicit(f, m, n)
    res = np.linalg.norm(A - Q @ R) / np.linalg.norm(A)
    orth = np.linalg.norm(np.eye(n) - Q.T @ Q)
    assert res <= 1e-13, res
    assert orth <= 1e-13, orth
    return Q, R


def compare(gpu, ref, scale, tol, what):
    err = np.abs(gpu - ref).max() / scale
    assert err <= tol, "%s: %.3e > %.3e" % (what, err, tol)
    return err


def test_small_config_parity():
    """1024 x 256, nb 64, ib 16, Greedy, N(0,1): R, V, T, Q^T b against the
    oracle; residual and orthogonality targets."""
    A, b = workloads.small_config(0)
    f, Aout = gpu_factor(A, 64, 16, tqr.GREEDY)
    F = otq.factor(A, 64, 16, tqr.GREEDY)
    tol = tol_for(A)
    scale = np.abs(F.r()).max()
    compare(Aout, F.A, scale, tol, "R and V")
    info = f.info()
    assert info["p"] == 16 and info["q"] == 4 and info["n_elims"] == 54 and info["critical_path"] == 86
    # T factors formed from the stored reflectors.
    p, q, ib, nb = 16, 4, 16, 64
    Tge = torch.zeros(p * q * ib * nb, dtype=torch.float64, device="cuda")
    Tel = torch.zeros_like(Tge)
    tqr.tqr_form_t(f, Tge, Tel)
    tqr.tqr_sync(f)
    Tge = Tge.cpu().numpy().reshape(q, p, nb, ib).transpose(1, 0, 3, 2)
    Tel = Tel.cpu().numpy().reshape(q, p, nb, ib).transpose(1, 0, 3, 2)
    compare(Tge, F.Tge, 1.0, tol, "T of GEQRT")
    compare(Tel, F.Tel, 1.0, tol, "T of TTQRT")
    # Q^T b
    bt = tqr.colmajor(b)
    tqr.tqr_apply_qt(f, bt)
    tqr.tqr_sync(f)
    compare(tqr.to_numpy(bt)[:, 0], otq.apply_qt(F, b), np.linalg.norm(b), tol, "Q^T b")
    check_targets(f, A, Aout)
    f.free()


TREES = [(tqr.FLAT_TS, 1), (tqr.FLAT_TT, 1), (tqr.SAMEH_KUCK, 1), (tqr.BINARY, 1), (tqr.FIBONACCI, 1),
         (tqr.GREEDY, 1), (tqr.PLASMA, 1), (tqr.PLASMA, 3), (tqr.PLASMA, 10), (tqr.ASAP, 1),
         (tqr.GRASAP, 2), (tqr.PLASMA_TS, 1), (tqr.PLASMA_TS, 3), (tqr.PLASMA_TS, 10)]


SPLIT_CASES = [(1400, 600, 128, 32, tqr.GREEDY, 1), (1400, 600, 128, 16, tqr.FLAT_TS, 1),
               (1300, 520, 128, 32, tqr.PLASMA_TS, 3), (1200, 500, 128, 64, tqr.BINARY, 1),
               (1100, 404, 128, 16, tqr.FIBONACCI, 1), (1536, 768, 256, 32, tqr.GREEDY, 1),
               (1600, 530, 256, 32, tqr.PLASMA_TS, 2)]


@pytest.mark.parametrize("m,n,nb,ib,tree,BS", SPLIT_CASES)
def test_split_panels_against_the_oracle(m, n, nb, ib, tree, BS):
    """Tiles of nb >= 128, whose panels run as one task per block of ib
    columns plus look-ahead and trailing update tasks: R, V, Q^T b and every
    tau element-wise against the oracle, ragged last tile row and column
    included (the 404- and 530-column cases leave whole blocks of the last
    tile column empty)."""
    A = workloads.uniform(m, n, seed=m + n + ib)
    b = workloads.rhs(m, 1, seed=7)[:, 0]
    f, Aout = gpu_factor(A, nb, ib, tree, BS)
    F = otq.factor(A, nb, ib, tree, BS)
    tol = tol_for(A)
    compare(Aout, F.A, np.abs(F.r()).max(), tol, "R and V")
    bt = tqr.colmajor(b)
    tqr.tqr_apply_qt(f, bt)
    tqr.tqr_sync(f)
    compare(tqr.to_numpy(bt)[:, 0], otq.apply_qt(F, b), np.linalg.norm(b), tol, "Q^T b")
    p, q = -(-m // nb), -(-n // nb)
    Tge = torch.zeros(p * q * ib * nb, dtype=torch.float64, device="cuda")
    Tel = torch.zeros_like(Tge)
    tqr.tqr_form_t(f, Tge, Tel)
    tqr.tqr_sync(f)
    Tge = Tge.cpu().numpy().reshape(q, p, nb, ib).transpose(1, 0, 3, 2)
    Tel = Tel.cpu().numpy().reshape(q, p, nb, ib).transpose(1, 0, 3, 2)
    compare(Tge, F.Tge, 1.0, tol, "T of GEQRT (tau on its diagonal)")
    compare(Tel, F.Tel, 1.0, tol, "T of the eliminations")
    check_targets(f, A, Aout)
    f.free()


@pytest.mark.parametrize("tree,BS", TREES)
def test_every_tree_ragged(tree, BS):
    """300 x 130, nb 32, ib 8: 10 x 5 tiles with a ragged last tile row and
    column, uniform entries."""
    A = workloads.uniform(300, 130, seed=tree * 10 + BS)
    f, Aout = gpu_factor(A, 32, 8, tree, BS)
    F = otq.factor(A, 32, 8, tree, BS)
    compare(Aout, F.A, np.abs(F.r()).max(), tol_for(A), "R and V")
    check_targets(f, A, Aout)
    f.free()


@pytest.mark.parametrize("m,n,nb,ib,tree", [
    (64, 64, 64, 16, tqr.GREEDY),       # one tile
    (50, 30, 64, 16, tqr.GREEDY),       # one partial tile
    (40, 40, 16, 4, tqr.FLAT_TT),       # ragged square
    (512, 512, 64, 8, tqr.GREEDY),      # square, p = q
    (512, 512, 64, 8, tqr.FLAT_TS),
    (1000, 64, 64, 32, tqr.FIBONACCI),  # q = 1
    (1000, 64, 64, 64, tqr.BINARY),     # ib = nb
    (1536, 512, 256, 32, tqr.GREEDY),   # nb 256: four strips per tile column
    (2000, 700, 256, 32, tqr.FLAT_TS),  # nb 256, ragged
    (700, 300, 48, 16, tqr.GREEDY),     # nb not a power of two
    (2000, 700, 256, 32, tqr.PLASMA_TS),  # TS domains + TT merges, nb 256, ragged
])
def test_shapes(m, n, nb, ib, tree):
    A = workloads.gaussian(m, n, seed=m + n)
    BS = 3 if tree == tqr.PLASMA_TS else 1
    f, Aout = gpu_factor(A, nb, ib, tree, BS)
    F = otq.factor(A, nb, ib, tree, BS)
    compare(Aout, F.A, np.abs(F.r()).max(), tol_for(A), "R and V")
    check_targets(f, A, Aout)
    f.free()


def test_apply_roundtrip_and_multiple_rhs():
    A = workloads.gaussian(640, 320, seed=3)
    f, Aout = gpu_factor(A, 64, 16, tqr.GREEDY)
    F = otq.factor(A, 64, 16, tqr.GREEDY)
    B = workloads.rhs(640, 70, seed=4)                 # 70 columns: two strips, ragged
    Bt = tqr.colmajor(B)
    tqr.tqr_apply_qt(f, Bt)
    tqr.tqr_sync(f)
    QtB = tqr.to_numpy(Bt)
    compare(QtB, otq.apply_qt(F, B), np.abs(B).max(), tol_for(A), "Q^T B")
    tqr.tqr_apply_q(f, Bt)
    tqr.tqr_sync(f)
    compare(tqr.to_numpy(Bt), B, np.abs(B).max(), 1e-13, "Q Q^T B")
    f.free()


def test_caller_given_list():
    """A random valid elimination list (neither tree's) through tqr_factor_list."""
    rng = np.random.default_rng(9)
    p, q, nb, ib = 9, 4, 32, 8
    zeroed, el = set(), []
    while len(el) < sum(p - k for k in range(1, q + 1)):
        cands = []
        for k in range(1, q + 1):
            for i in range(k + 1, p + 1):
                if (i, k) in zeroed or any((i, kp) not in zeroed for kp in range(1, k)):
                    continue
                pivs = [r for r in range(k, i) if (r, k) not in zeroed
                        and all((r, kp) in zeroed for kp in range(1, k))]
                cands += [(i, r, k) for r in pivs]
        e = cands[rng.integers(len(cands))]
        el.append(e)
        zeroed.add((e[0], e[2]))
    assert otrees.validate(p, q, el) is None
    A = workloads.gaussian(p * nb - 5, q * nb - 3, seed=5)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor_list(At, nb, ib, np.array(el) - 1)
    tqr.tqr_sync(f)
    F = otq.factor(A, nb, ib, tqr.GREEDY, elims=el)
    compare(tqr.to_numpy(At), F.A, np.abs(F.r()).max(), tol_for(A), "R and V")
    bad = list(el)
    bad[0], bad[-1] = bad[-1], bad[0]
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_factor_list(tqr.colmajor(A), nb, ib, np.array(bad) - 1)
    assert e.value.code == tqr.TQR_ERR_INVALID_LIST
    f.free()


def test_ts_list_with_triangle_tile_is_rejected():
    """TS kernels need the zeroed tile square: a BinaryTree list eliminates
    rows that were pivots earlier in the column, so it is invalid with TS."""
    p, q, nb, ib = 8, 2, 32, 8
    el = np.array(otrees.binary_tree(p, q)) - 1
    A = workloads.gaussian(p * nb, q * nb, seed=12)
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_factor_list(tqr.colmajor(A), nb, ib, el, ts=True)
    assert e.value.code == tqr.TQR_ERR_INVALID_LIST
    At = tqr.colmajor(A)
    f = tqr.tqr_factor_list(At, nb, ib, el, ts=False)     # the same list with TT kernels is fine
    tqr.tqr_sync(f)
    F = otq.factor(A, nb, ib, tqr.BINARY)
    compare(tqr.to_numpy(At), F.A, np.abs(F.r()).max(), tol_for(A), "R and V")
    f.free()


def test_reuse_allocates_nothing_and_repeats():
    A = workloads.gaussian(512, 256, seed=6)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, 64, 16, tqr.GREEDY)
    tqr.tqr_sync(f)
    first = tqr.to_numpy(At)
    At2 = tqr.colmajor(A)
    g = tqr.tqr_factor(At2, 64, 16, tqr.GREEDY, reuse=f)
    assert g is f
    tqr.tqr_sync(g)
    assert np.array_equal(tqr.to_numpy(At2), first)   # the executor is deterministic per task
    f.free()


def test_host_end_to_end():
    A = np.asfortranarray(workloads.gaussian(768, 256, seed=7))
    b = np.asfortranarray(workloads.rhs(768, 1, seed=8))
    Ah, bh = A.copy(order="F"), b.copy(order="F")
    f = tqr.tqr_factor_host(Ah, 64, 16, tqr.GREEDY, B=bh)
    F = otq.factor(A, 64, 16, tqr.GREEDY)
    compare(Ah, F.A, np.abs(F.r()).max(), tol_for(A), "R and V")
    compare(bh[:, 0], otq.apply_qt(F, b[:, 0]), np.linalg.norm(b), tol_for(A), "Q^T b")
    f.free()


def test_nonfinite_input_reports_status():
    A = workloads.gaussian(256, 128, seed=1)
    A[17, 3] = np.nan
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, 64, 16, tqr.GREEDY)
    assert tqr.tqr_sync(f, raise_on_error=False) == tqr.TQR_ERR_NONFINITE
    f.free()


def test_timeout_is_reported_and_context_survives():
    """Failure detection without a GPU fault: the host drops the ready tasks,
    every device wait runs out after 500 ms, the status says so, and the next
    factorization on the same context is correct."""
    A = workloads.gaussian(256, 128, seed=2)
    tqr.tqr_set_timeout_ms(500)
    try:
        tqr.tqr_inject_fault(1)
        At = tqr.colmajor(A)
        f = tqr.tqr_factor(At, 64, 16, tqr.GREEDY)
        assert tqr.tqr_sync(f, raise_on_error=False) == tqr.TQR_ERR_TIMEOUT
        f.free()
        # The allocation-free entry point honours the same limit and injection.
        nb, ib = 64, 16
        p, q = -(-A.shape[0] // nb), -(-A.shape[1] // nb)
        tau = torch.zeros(p * q * nb, dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        tqr.tqr_inject_fault(1)
        rc = tqr.tqr_factor_noalloc(tqr.colmajor(A), nb, ib, tqr.tqr_elimination_list(p, q, tqr.GREEDY), tau,
                                    tau.clone(), status)
        assert rc == 0, tqr.tqr_strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == tqr.TQR_ERR_TIMEOUT
    finally:
        tqr.tqr_inject_fault(0)
        tqr.tqr_set_timeout_ms(0)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, 64, 16, tqr.GREEDY)
    tqr.tqr_sync(f)
    F = otq.factor(A, 64, 16, tqr.GREEDY)
    compare(tqr.to_numpy(At), F.A, np.abs(F.r()).max(), tol_for(A), "R and V after timeout")
    f.free()


# ------------------------------------------------------------ degenerate cases
def _degenerate(case):
    rng = np.random.default_rng(21)
    if case == "zero":
        return np.zeros((300, 130)), 32, 8
    if case == "zero_column":
        A = rng.standard_normal((300, 130))
        A[:, 40] = 0.0                                  # inside the second tile column
        A[:, 64] = 0.0                                  # first column of the third tile column
        return A, 32, 8
    if case == "identity":
        return np.eye(256, 128), 32, 8
    if case == "one_by_one":
        return np.array([[3.0]]), 8, 4
    if case == "column_vector":
        return rng.standard_normal((1000, 1)), 64, 16
    if case == "rank_deficient":
        return rng.standard_normal((400, 12)) @ rng.standard_normal((12, 96)), 32, 8
    raise ValueError(case)


@pytest.mark.parametrize("case", ["zero", "zero_column", "identity", "one_by_one", "column_vector",
                                  "rank_deficient"])
@pytest.mark.parametrize("tree", [tqr.GREEDY, tqr.FLAT_TS])
def test_degenerate_inputs(case, tree):
    """Zero reflectors (x = 0 gives tau = 0 and a zero tail, LAPACK's
    convention), a 1 x 1 matrix, a single column and a rank-deficient matrix:
    R and V against the oracle, and A = QR with orthogonal Q."""
    A, nb, ib = _degenerate(case)
    f, Aout = gpu_factor(A, nb, ib, tree)
    assert tqr.tqr_sync(f) == 0
    F = otq.factor(A, nb, ib, tree)
    m, n = A.shape
    if case in ("zero", "identity", "one_by_one"):
        assert np.array_equal(Aout, F.A)                 # no rounding happens at all
    else:
        scale = np.abs(F.r()).max()
        if case == "rank_deficient":
            # The first 12 columns are independent: R's leading 12 rows are determined
            # as for A[:, :12]; the trailing rows are rounding noise.
            compare(np.triu(Aout[:12, :n]), np.triu(F.A[:12, :n]), scale, tol_for(A[:, :12]), "leading R rows")
        elif case == "zero_column":
            # Zero columns give identity reflectors; the rest is as well determined as
            # the matrix without them.
            keep = [c for c in range(n) if c not in (40, 64)]
            compare(Aout, F.A, scale, tol_for(A[:, keep]), "R and V")
        else:
            compare(Aout, F.A, scale, tol_for(A), "R and V")
    if case == "zero":
        Q = gpu_q_explicit(f, m, n)
        assert np.array_equal(Q, np.eye(m, n))           # every reflector is the identity
    else:
        check_targets(f, A, Aout)
    f.free()


def test_host_async_on_two_streams_matches_sync():
    """tqr_factor_host_async: two matrices enqueued on two streams, then
    tqr_sync; results equal the synchronous call's bit for bit."""
    mats = [np.asfortranarray(workloads.gaussian(768, 256, seed=31)),
            np.asfortranarray(workloads.uniform(1000, 300, seed=32))]
    want = []
    for A in mats:
        a = A.copy(order="F")
        f = tqr.tqr_factor_host(a, 64, 16, tqr.GREEDY)
        want.append(a)
        f.free()
    pinned = [torch.from_numpy(A.T.copy()).pin_memory() for A in mats]   # row-major view of A^T = A in F order
    views = [p.numpy().T for p in pinned]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hs = [tqr.tqr_factor_host(v, 64, 16, tqr.GREEDY, stream=s, wait=False) for v, s in zip(views, streams)]
    for h in hs:
        assert tqr.tqr_sync(h) == 0
    for v, w in zip(views, want):
        assert np.array_equal(v, w)
    for h in hs:
        h.free()


def test_host_handles_of_one_shape_with_other_tiles_stay_independent():
    """tqr_factor_host given a previous handle of the same m x n but another
    tile size makes a new handle with a device copy of A of its own: the
    previous handle still applies its own Q^T afterwards, a call with the
    previous handle's parameters reuses it (bit for bit the same result), and
    both handles free cleanly."""
    A = np.asfortranarray(workloads.gaussian(768, 256, seed=41))
    b = workloads.rhs(768, 1, seed=42)
    a1 = A.copy(order="F")
    f1 = tqr.tqr_factor_host(a1, 64, 16, tqr.GREEDY)
    a2 = A.copy(order="F")
    f2 = tqr.tqr_factor_host(a2, 128, 16, tqr.GREEDY, reuse=f1)
    assert f2 is not f1 and f2.ptr != f1.ptr
    F1 = otq.factor(A, 64, 16, tqr.GREEDY)
    F2 = otq.factor(A, 128, 16, tqr.GREEDY)
    compare(a1, F1.A, np.abs(F1.r()).max(), tol_for(A), "R and V, nb 64")
    compare(a2, F2.A, np.abs(F2.r()).max(), tol_for(A), "R and V, nb 128")
    bt = tqr.colmajor(b)
    tqr.tqr_apply_qt(f1, bt)
    assert tqr.tqr_sync(f1) == 0
    compare(tqr.to_numpy(bt)[:, 0], otq.apply_qt(F1, b[:, 0]), np.linalg.norm(b), tol_for(A), "Q^T b, first handle")
    a3 = A.copy(order="F")
    f3 = tqr.tqr_factor_host(a3, 64, 16, tqr.GREEDY, reuse=f1)
    assert f3 is f1
    assert np.array_equal(a3, a1)
    f2.free()
    f1.free()


def test_release_plans_keeps_live_handles_valid():
    """tqr_release_plans drops the cached plans no handle uses; a live
    handle still applies Q^T and refactors, and a released plan is rebuilt
    with the same result bit for bit."""
    A = workloads.gaussian(640, 192, seed=43)
    b = workloads.rhs(640, 1, seed=44)
    At = tqr.colmajor(A)
    f = tqr.tqr_factor(At, 64, 16, tqr.BINARY)
    assert tqr.tqr_sync(f) == 0
    first = tqr.to_numpy(At)
    Ag = tqr.colmajor(A)
    g = tqr.tqr_factor(Ag, 64, 16, tqr.FIBONACCI)
    assert tqr.tqr_sync(g) == 0
    fib = tqr.to_numpy(Ag)
    g.free()
    assert tqr.tqr_release_plans() >= 1                  # at least the Fibonacci plan
    F = otq.factor(A, 64, 16, tqr.BINARY)
    bt = tqr.colmajor(b)
    tqr.tqr_apply_qt(f, bt)
    assert tqr.tqr_sync(f) == 0
    compare(tqr.to_numpy(bt)[:, 0], otq.apply_qt(F, b[:, 0]), np.linalg.norm(b), tol_for(A), "Q^T b after release")
    At2 = tqr.colmajor(A)
    assert tqr.tqr_factor(At2, 64, 16, tqr.BINARY, reuse=f) is f
    assert tqr.tqr_sync(f) == 0
    assert np.array_equal(tqr.to_numpy(At2), first)
    Ag2 = tqr.colmajor(A)
    g2 = tqr.tqr_factor(Ag2, 64, 16, tqr.FIBONACCI)
    assert tqr.tqr_sync(g2) == 0
    assert np.array_equal(tqr.to_numpy(Ag2), fib)
    g2.free()
    f.free()


def test_apply_binding_rejects_b_with_another_row_count():
    """B must have the factorization's m rows (a taller view with ld >= m
    would pass the library's ldb check but apply Q to the wrong rows)."""
    A = workloads.gaussian(256, 64, seed=45)
    f, _ = gpu_factor(A, 64, 16, tqr.GREEDY)
    with pytest.raises(ValueError):
        tqr.tqr_apply_qt(f, tqr.colmajor(np.zeros((255, 1))))
    with pytest.raises(ValueError):
        tqr.tqr_apply_q(f, tqr.colmajor(np.zeros((300, 2)))[:255])
    f.free()
