"""The least-squares and batched rows at the benchmark's full size and launch
configuration, where the oracle cannot process everything:

* least squares, 65536 x 4096, kappa = 1e6 (the bench's value point): the
  split-TF32 solve converges to the FP64 path's backward error and its
  solution agrees with the FP64 path's within the conditioning bound;
* the 4096-matrix batch with the autotuner's classes replaced by the
  one-column FlatTree-TS configuration it picks: sampled matrices (smallest,
  a median one, one of the largest n) against the oracle element-wise, every
  matrix's column norms preserved (||R e_c|| = ||A e_c||), FP64 and FP32.
"""

import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tiled_qr as otq
from oracle import FLAT_TS as O_FLAT_TS
import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import workloads

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()


def test_full_size_lstsq_kappa_1e6():
    A, b, x_true = workloads.ls_problem_device(bench.LS_M, bench.LS_N, 1e6, seed=3)
    tree = tqr.TREES[bench.LS_TREE]
    x64 = torch.zeros(bench.LS_N, dtype=torch.float64, device="cuda")
    i64 = tqr.tqr_lstsq(A, b, x64, bench.LS_NB, bench.LS_IB, tree, bench.LS_BS, tqr.TQR_FP64, 0.0, 0)
    xs = torch.zeros_like(x64)
    iss = tqr.tqr_lstsq(A, b, xs, bench.LS_NB, bench.LS_IB, tree, bench.LS_BS, tqr.TQR_SPLIT_TF32,
                        2 * i64["backward_error"], 50)
    assert i64["status"] == 0 and iss["status"] == 0
    assert iss["converged"] == 1 and iss["backward_error"] <= 2 * i64["backward_error"]
    rel = (torch.linalg.norm(xs - x64) / torch.linalg.norm(x64)).item()
    assert rel <= 1e6 * 1e-13, rel
    del A, b, x_true
    torch.cuda.empty_cache()


def _batch_shapes():
    rng = np.random.default_rng(bench.BT_SEED)
    ms = rng.integers(512, 16385, bench.BT_COUNT)
    ns = rng.choice([32, 64, 128], bench.BT_COUNT)
    return ms, ns


@pytest.mark.parametrize("f32", [False, True])
def test_full_size_batch_one_column(f32):
    ms, ns = _batch_shapes()
    nbs = [int(256 if (f32 or n <= 64) else 128) for n in ns]
    dt = torch.float32 if f32 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(bench.BT_SEED)
    src = [torch.randn(int(n), int(m), generator=g, dtype=dt, device="cuda").t() for m, n in zip(ms, ns)]
    work = [torch.empty_like(s.t()).t() for s in src]          # separate column-major buffers
    for w, s in zip(work, src):
        w.copy_(s)
    assert work[0].data_ptr() != src[0].data_ptr()
    if f32:
        b = tqr.tqr_factor_batched_f32(work, nbs)
    else:
        b = tqr.tqr_factor_batched(work, nbs, 8, tqr.FLAT_TS, 1)
    assert tqr.tqr_batch_sync(b) == 0 and b.info()["n_fused"] == bench.BT_COUNT
    u = 2.0 ** -24 if f32 else 2.0 ** -53
    # every matrix: column norms of R equal those of A (Q orthogonal)
    for c in range(bench.BT_COUNT):
        n = int(ns[c])
        R = torch.triu(work[c][:n, :]).double()
        rn = torch.linalg.norm(R, dim=0)
        an = torch.linalg.norm(src[c].double(), dim=0)
        assert ((rn - an).abs().max() / an.max()).item() <= 64 * n * u, c
    # sampled matrices against the oracle
    order = np.argsort(ms)
    picks = [int(order[0]), int(order[len(order) // 2]), int(np.flatnonzero(ns == 128)[0])]
    for c in picks:
        A = src[c].double().cpu().numpy()
        F = otq.factor(A, nbs[c], 8, O_FLAT_TS)
        got = work[c].double().cpu().numpy()
        tol = 8 * np.linalg.cond(A) * A.shape[0] * u
        assert np.abs(got - F.A).max() / np.abs(F.r()).max() <= max(tol, 1e-13), c
    b.free()
