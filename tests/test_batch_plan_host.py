"""The persistent one-tile-column launch's queues, planned on the host
(tqr_ts1_plan, no GPU): every matrix sits in the queue of its thread count,
largest work first, and the shared-memory quarter covers every slot."""

import numpy as np
import pytest

import paper_1104_4475_gb300 as tqr


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1104_4475_gb300 import build
    build.build()


def threads(n, h, f32):
    """The documented rule: enough threads that one holds at most 16 FP32 / 8
    FP64 rows of its column; at least 256 (FP32) / 512 (FP64), at most 1024."""
    ncol = 32 if n <= 32 else (64 if n <= 64 else 128)
    want = h * ncol // (16 if f32 else 8)
    return ncol, min(1024, max(256 if f32 else 512, want))


def smem_bytes(n, h, f32):
    """Two published vectors (16-byte padded lane chunks), the staging tile
    (h x (ncol + 1)) and packed R."""
    ncol, t = threads(n, h, f32)
    esz = 4 if f32 else 8
    G = t // ncol
    rpt = h // G
    return esz * (2 * G * (rpt + 16 // esz) + h * (ncol + 1) + ncol * (ncol + 1) // 2)


def shapes(count, seed, f32):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nb = int(rng.choice([64, 128, 256]))
        n = int(rng.integers(1, min(nb, 128) + 1))
        if not f32 and n > 64 and nb == 256:
            continue
        out.append((int(rng.integers(n, 20000)), n, nb))
    return out


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_queues_by_thread_count_largest_first(f32, seed):
    sh = shapes(500, seed + 10 * f32, f32)
    m, n, nb = (np.array(x) for x in zip(*sh))
    order, bounds, quarter = tqr.tqr_ts1_plan(m, n, nb, f32)
    assert sorted(order.tolist()) == list(range(len(sh)))
    assert bounds[0, 0] == 0 and bounds[0, 1] == bounds[1, 0] and bounds[1, 1] == bounds[2, 0]
    assert bounds[2, 1] == len(sh)
    if not f32:
        assert bounds[2, 0] == bounds[2, 1]                  # FP64 never runs on 256 threads
    need = 0
    for k in range(3):
        idx = order[bounds[k, 0]:bounds[k, 1]]
        work = [m[c] * n[c] ** 2 for c in idx]
        assert all(a >= b for a, b in zip(work, work[1:]))
        for a, b in zip(idx, idx[1:]):                       # equal work keeps the input order
            if work[list(idx).index(a)] == work[list(idx).index(b)]:
                assert a < b
        for c in idx:
            _, t = threads(n[c], nb[c], f32)
            assert t == 1024 >> k
            need = max(need, -(-smem_bytes(n[c], nb[c], f32) // (t // 256)))
    assert quarter % 16 == 0 and quarter == max(16, -(-need // 16) * 16)
    assert 4 * quarter + 256 <= 227 * 1024


def test_one_class_and_empty():
    order, bounds, quarter = tqr.tqr_ts1_plan([4096] * 3, [128] * 3, 128)
    assert order.tolist() == [0, 1, 2] and bounds.tolist() == [[0, 3], [3, 3], [3, 3]]
    assert quarter == smem_bytes(128, 128, False) // 4
    order, bounds, quarter = tqr.tqr_ts1_plan([], [], [])
    assert order.size == 0 and bounds.tolist() == [[0, 0], [0, 0], [0, 0]] and quarter == 16


def test_refuses_matrices_the_kernel_does_not_take():
    for m, n, nb, f32 in [(300, 100, 256, False), (300, 80, 64, False), (300, 129, 256, True), (300, 32, 48, True)]:
        with pytest.raises(tqr.TqrError) as e:
            tqr.tqr_ts1_plan([m], [n], [nb], f32)
        assert e.value.code == tqr.TQR_ERR_UNSUPPORTED
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_ts1_plan([10], [20], [64])
    assert e.value.code == -3
