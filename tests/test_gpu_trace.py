"""Per-task device traces: one row per device task, the executor honours
every producer edge (no update starts before the panel whose reflectors it
applies has finished), and the Chrome-trace export covers every task."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import trace as ttrace
from paper_1104_4475_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build
    build.build()


@pytest.mark.parametrize("tree,BS,prec", [(tqr.GREEDY, 1, tqr.TQR_FP64), (tqr.PLASMA_TS, 4, tqr.TQR_FP64),
                                          (tqr.FLAT_TS, 1, tqr.TQR_SPLIT_TF32)])
def test_trace_rows_and_producer_order(tree, BS, prec, tmp_path):
    A = tqr.colmajor(workloads.uniform(2048, 768, seed=4))
    f = tqr.tqr_factor_ex(A, 128, 32, tree, BS, prec)
    tqr.tqr_sync(f)
    tqr.tqr_set_trace(f, True)
    A2 = tqr.colmajor(workloads.uniform(2048, 768, seed=4))
    g = tqr.tqr_factor_ex(A2, 128, 32, tree, BS, prec, reuse=f)
    tqr.tqr_sync(g)
    tr = tqr.tqr_get_trace(g)
    info = g.info()
    assert tr.shape == (info["n_device_tasks"], 8)
    assert np.all(tr[:, 6] >= tr[:, 5]) and np.all(tr[:, 5] > 0)
    assert np.all(tr[:, 7] < torch.cuda.get_device_properties(0).multi_processor_count)
    assert set(tr[:, 0].tolist()) <= set(range(6))
    assert ttrace.producer_violations(tr) == []
    edges = tqr.tqr_get_edges(g)
    assert len(edges) == info["n_edges"]
    assert ttrace.edge_violations(tr, edges) == []           # happens-before on every edge
    s = ttrace.summary(tr)
    assert 0.0 < s["busy_fraction"] <= 1.0 and s["tasks"] == len(tr)
    doc = ttrace.to_chrome(tr, str(tmp_path / "t.json"))
    assert len(doc["traceEvents"]) == len(tr)
    g.free()


@pytest.mark.parametrize("prec", [tqr.TQR_FP64, tqr.TQR_SPLIT_TF32])
def test_poisoned_workspace_is_never_read_before_written(prec):
    """NaN in every tau / T / V entry before a rerun: the rerun's result is
    bit-identical to the clean run and finite, so no task read workspace that
    its producers had not written yet."""
    A0 = workloads.uniform(1500, 640, seed=8)               # ragged: 12 x 5 tiles of 128
    At = tqr.colmajor(A0)
    f = tqr.tqr_factor_ex(At, 128, 32, tqr.GREEDY, 1, prec)
    assert tqr.tqr_sync(f) == 0
    clean = tqr.to_numpy(At)
    for _ in range(2):
        tqr.tqr_poison_workspace(f)
        At2 = tqr.colmajor(A0)
        g = tqr.tqr_factor_ex(At2, 128, 32, tqr.GREEDY, 1, prec, reuse=f)
        assert g is f and tqr.tqr_sync(f) == 0
        out = tqr.to_numpy(At2)
        assert np.isfinite(out).all()
        assert np.array_equal(out, clean)
    f.free()


def test_trace_enabled_from_environment():
    """TQR_TRACE=1 turns tracing on for every new handle (no tqr_set_trace call)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_1104_4475_gb300 as tqr\n"
            "from paper_1104_4475_gb300 import workloads\n"
            "A = tqr.colmajor(workloads.uniform(512, 256, seed=3))\n"
            "f = tqr.tqr_factor(A, 64, 16, tqr.GREEDY); tqr.tqr_sync(f)\n"
            "tr = tqr.tqr_get_trace(f)\n"
            "assert tr.shape[0] == f.info()['n_device_tasks'] and (tr[:, 6] >= tr[:, 5]).all()\n"
            "print('traced', tr.shape[0])\n" % root)
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, TQR_TRACE="1"), capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("traced")
