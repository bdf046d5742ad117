"""Batched factorization: many matrices with their own (nb, ib, tree) in one
persistent launch, each checked against the oracle; a CUDA graph capturing a
relaunch reproduces the eager result bit for bit."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tiled_qr as otq
import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
CONFIGS = [(32, 8, tqr.GREEDY, 1), (32, 16, tqr.FLAT_TS, 1), (64, 16, tqr.BINARY, 1), (64, 32, tqr.FIBONACCI, 1),
           (32, 32, tqr.PLASMA, 3), (64, 16, tqr.ASAP, 1), (16, 8, tqr.GREEDY, 1)]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()


def make_batch(count, seed):
    rng = np.random.default_rng(seed)
    mats, cfgs = [], []
    for c in range(count):
        n = int(rng.choice([32, 64, 96]))
        m = int(rng.integers(max(n, 100), 1500))
        mats.append(workloads.gaussian(m, n, seed=1000 + c))
        cfgs.append(CONFIGS[c % len(CONFIGS)])
    return mats, cfgs


def test_batched_matches_oracle():
    mats, cfgs = make_batch(28, 0)
    As = [tqr.colmajor(A) for A in mats]
    b = tqr.tqr_factor_batched(As, [c[0] for c in cfgs], [c[1] for c in cfgs], [c[2] for c in cfgs],
                               [c[3] for c in cfgs])
    tqr.tqr_batch_sync(b)
    info = b.info()
    assert info["count"] == 28 and info["n_tasks"] > 28
    for A, At, (nb, ib, tree, BS) in zip(mats, As, cfgs):
        F = otq.factor(A, nb, ib, tree, BS)
        tol = max(1e-13, 8 * np.linalg.cond(A) * A.shape[0] * U)
        err = np.abs(tqr.to_numpy(At) - F.A).max() / np.abs(F.r()).max()
        assert err <= tol, (A.shape, nb, ib, tree, err)
    b.free()


def test_batched_relaunch_and_cuda_graph():
    mats, cfgs = make_batch(12, 1)
    src = [tqr.colmajor(A) for A in mats]
    As = [torch.empty_like(s.t()).t() for s in src]
    for a, s in zip(As, src):
        a.copy_(s)
    nbs, ibs, trs, bss = ([c[i] for c in cfgs] for i in range(4))
    b = tqr.tqr_factor_batched(As, nbs, ibs, trs, bss)
    tqr.tqr_batch_sync(b)
    eager = [tqr.to_numpy(a) for a in As]
    for a, s in zip(As, src):
        a.copy_(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            b2 = tqr.tqr_factor_batched(As, nbs, ibs, trs, bss, stream=stream, reuse=b)
    assert b2 is b
    for rep in range(2):
        for a, s in zip(As, src):
            a.copy_(s)
        g.replay()
        torch.cuda.synchronize()
        assert tqr.tqr_batch_sync(b) == 0
        for a, e in zip(As, eager):
            assert np.array_equal(tqr.to_numpy(a), e)
    b.free()


# --------------------------------------------- one tile column, FlatTree-TS
from oracle import FLAT_TS as O_FLAT_TS
from oracle import kernels as oK

ONE_COLUMN = [(300, 32, 64), (1000, 64, 64), (517, 100, 128), (64, 64, 64), (70, 48, 64), (500, 1, 64),
              (1200, 128, 128), (40, 32, 256), (2000, 64, 256), (777, 33, 64), (129, 96, 128)]


def test_one_column_flat_ts_matches_oracle_with_tau():
    """FlatTree-TS with n <= nb runs whole matrices in one CTA each; R, V
    and every tau equal the oracle's (Proposition 2's chain GEQRT, TSQRT, ...)."""
    mats = [workloads.gaussian(m, n, seed=50 + c) for c, (m, n, nb) in enumerate(ONE_COLUMN)]
    nbs = [nb for (_, _, nb) in ONE_COLUMN]
    As = [tqr.colmajor(A) for A in mats]
    b = tqr.tqr_factor_batched(As, nbs, 8, tqr.FLAT_TS, 1)
    assert tqr.tqr_batch_sync(b) == 0
    info = b.info()
    assert info["n_fused"] == len(mats) and info["n_tasks"] == 0
    for c, (A, At, nb) in enumerate(zip(mats, As, nbs)):
        m, n = A.shape
        F = otq.factor(A, nb, 8, O_FLAT_TS)
        tol = max(1e-13, 8 * np.linalg.cond(A) * m * U)
        scale = np.abs(F.r()).max()
        assert np.abs(tqr.to_numpy(At) - F.A).max() / scale <= tol, (m, n, nb)
        tg, te = tqr.tqr_batch_tau(b, c, m, n, nb)
        p = -(-m // nb)
        assert np.abs(tg[:nb] - oK.tau_of(F.Tge[0, 0])).max() <= tol
        for i in range(1, p):
            assert np.abs(te[i * nb:(i + 1) * nb] - oK.tau_of(F.Tel[i, 0])).max() <= tol, (m, n, nb, i)
    b.free()


def test_one_column_mixed_with_executor_and_graph():
    """A batch mixing one-column FlatTree-TS matrices with executor trees;
    a CUDA-graph relaunch reproduces the eager result bit for bit."""
    cfgs = [(800, 64, 64, tqr.FLAT_TS), (900, 96, 32, tqr.GREEDY), (600, 32, 128, tqr.FLAT_TS),
            (1000, 128, 64, tqr.FLAT_TS), (700, 64, 32, tqr.BINARY), (300, 200, 256, tqr.FLAT_TS)]
    mats = [workloads.gaussian(m, n, seed=70 + c) for c, (m, n, nb, t) in enumerate(cfgs)]
    src = [tqr.colmajor(A) for A in mats]
    As = [torch.empty_like(s.t()).t() for s in src]
    for a, s in zip(As, src):
        a.copy_(s)
    nbs, trs = [c[2] for c in cfgs], [c[3] for c in cfgs]
    b = tqr.tqr_factor_batched(As, nbs, 8, trs, 1)
    assert tqr.tqr_batch_sync(b) == 0
    assert b.info()["n_fused"] == 2                   # 800x64/64, 600x32/128 (1000x128 has n > nb; 300x200 n > 128)
    eager = [tqr.to_numpy(a) for a in As]
    for A, e, (m, n, nb, t) in zip(mats, eager, cfgs):
        F = otq.factor(A, nb, 8, t)
        tol = max(1e-13, 8 * np.linalg.cond(A) * m * U)
        assert np.abs(e - F.A).max() / np.abs(F.r()).max() <= tol, (m, n, nb, t)
    for a, s in zip(As, src):
        a.copy_(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            b2 = tqr.tqr_factor_batched(As, nbs, 8, trs, 1, stream=stream, reuse=b)
    assert b2 is b
    for a, s in zip(As, src):
        a.copy_(s)
    g.replay()
    torch.cuda.synchronize()
    assert tqr.tqr_batch_sync(b) == 0
    for a, e in zip(As, eager):
        assert np.array_equal(tqr.to_numpy(a), e)
    b.free()


U32 = 2.0 ** -24


def test_fp32_batch_matches_oracle():
    """FP32 one-column batch: R and V against the FP64 oracle within the
    FP32 perturbation bound 8 kappa m u32, and R^T R = A^T A to m n u32."""
    shapes = ONE_COLUMN + [(3000, 128, 256), (16384, 32, 256)]
    mats = [workloads.gaussian(m, n, seed=90 + c) for c, (m, n, nb) in enumerate(shapes)]
    As = [torch.tensor(np.asfortranarray(A, dtype=np.float32).T, device="cuda").t() for A in mats]
    nbs = [nb for (_, _, nb) in shapes]
    b = tqr.tqr_factor_batched_f32(As, nbs)
    assert tqr.tqr_batch_sync(b) == 0
    info = b.info()
    assert info["f32"] == 1 and info["n_fused"] == len(mats)
    for c, (A, At, nb) in enumerate(zip(mats, As, nbs)):
        m, n = A.shape
        A32 = A.astype(np.float32).astype(np.float64)
        F = otq.factor(A32, nb, 8, O_FLAT_TS)
        got = At.t().cpu().numpy().T.astype(np.float64)
        tol = 8 * np.linalg.cond(A32) * m * U32
        assert np.abs(got - F.A).max() / np.abs(F.r()).max() <= tol, (m, n, nb)
        R = np.triu(got[:n, :n])
        assert np.linalg.norm(R.T @ R - A32.T @ A32) / np.linalg.norm(A32) ** 2 <= m * n * U32
        tg, te = tqr.tqr_batch_tau(b, c, m, n, nb, f32=True)
        assert np.abs(tg[:nb] - oK.tau_of(F.Tge[0, 0])).max() <= tol
    b.free()


def test_fp32_batch_rejects_unsupported():
    A = torch.zeros(300, 200, dtype=torch.float32, device="cuda").t().contiguous().t()
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_factor_batched_f32([A], 256)
    assert e.value.code == tqr.TQR_ERR_UNSUPPORTED
    B = torch.zeros(300, 64, dtype=torch.float32, device="cuda").t().contiguous().t()
    with pytest.raises(tqr.TqrError):
        tqr.tqr_factor_batched_f32([B], 32)               # n > nb


def test_one_column_degenerate_inputs():
    """Zero matrices and zero columns through the one-column kernel, FP64 and
    FP32: identity reflectors (tau = 0) leave them exactly as the oracle does."""
    rng = np.random.default_rng(3)
    Z = np.zeros((500, 48))
    C = rng.standard_normal((700, 64))
    C[:, 5] = 0.0
    mats = [Z, C, np.eye(128, 96)]
    nbs = [64, 128, 128]
    As = [tqr.colmajor(A) for A in mats]
    b = tqr.tqr_factor_batched(As, nbs, 8, tqr.FLAT_TS, 1)
    assert tqr.tqr_batch_sync(b) == 0 and b.info()["n_fused"] == 3
    for A, At, nb in zip(mats, As, nbs):
        F = otq.factor(A, nb, 8, O_FLAT_TS)
        got = tqr.to_numpy(At)
        if A is C:
            keep = [c for c in range(64) if c != 5]
            tol = 8 * np.linalg.cond(A[:, keep]) * A.shape[0] * U
            assert np.abs(got - F.A).max() / np.abs(F.r()).max() <= tol
        else:
            assert np.array_equal(got, F.A)
    b.free()
    Z32 = [torch.zeros(96, 400, dtype=torch.float32, device="cuda").t()]
    b = tqr.tqr_factor_batched_f32(Z32, 128)
    assert tqr.tqr_batch_sync(b) == 0
    assert torch.count_nonzero(Z32[0]).item() == 0
    tg, te = tqr.tqr_batch_tau(b, 0, 400, 96, 128, f32=True)
    assert not tg.any() and not te.any()
    b.free()


def one_column_shapes(count, seed, f32):
    """Shapes over every (column class, tile height) pair the one-column
    kernel takes, so a batch fills all of its thread-count queues."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nb = int(rng.choice([64, 128, 256]))
        n = int(rng.integers(1, min(nb, 128) + 1))
        if not f32 and n > 64 and nb == 256:
            continue                                   # FP64 class 128 needs nb = 128
        m = int(rng.integers(n, 3000))
        out.append((m, n, nb))
    return out


@pytest.mark.parametrize("f32", [False, True])
def test_persistent_queue_equals_one_matrix_batches(f32):
    """600 matrices of every class in one persistent launch (slots of 1024,
    512 and 256 threads popping from their queues) give bit for bit what
    each matrix gives alone in a batch of one: no slot, queue position or
    phase change alters a result.  A sample is also checked against the
    oracle."""
    shapes = one_column_shapes(600, 17 + f32, f32)
    dt = torch.float32 if f32 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(3)
    src = [torch.randn(n, m, generator=g, dtype=dt, device="cuda").t() for m, n, _ in shapes]
    nbs = [nb for _, _, nb in shapes]
    work = [s.t().clone().t() for s in src]                # copies (contiguous() would return s itself)
    b = tqr.tqr_factor_batched_f32(work, nbs) if f32 else tqr.tqr_factor_batched(work, nbs, 8, tqr.FLAT_TS, 1)
    assert tqr.tqr_batch_sync(b) == 0 and b.info()["n_fused"] == len(shapes)
    b.free()
    for c in range(len(shapes)):
        one = [src[c].t().clone().t()]
        b1 = (tqr.tqr_factor_batched_f32(one, nbs[c]) if f32
              else tqr.tqr_factor_batched(one, nbs[c], 8, tqr.FLAT_TS, 1))
        assert tqr.tqr_batch_sync(b1) == 0
        assert one[0].data_ptr() != work[c].data_ptr() and not torch.equal(one[0], src[c])
        assert torch.equal(one[0], work[c]), (shapes[c], c)
        b1.free()
    for c in range(0, len(shapes), 75):
        m, n, nb = shapes[c]
        A = src[c].double().cpu().numpy()
        F = otq.factor(A, nb, 8, O_FLAT_TS)
        u = U32 if f32 else U
        tol = max(1e-13, 8 * np.linalg.cond(A) * m * u)
        got = work[c].double().cpu().numpy()
        assert np.abs(got - F.A).max() / np.abs(F.r()).max() <= tol, shapes[c]
