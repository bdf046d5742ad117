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
