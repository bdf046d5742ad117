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
    s = ttrace.summary(tr)
    assert 0.0 < s["busy_fraction"] <= 1.0 and s["tasks"] == len(tr)
    doc = ttrace.to_chrome(tr, str(tmp_path / "t.json"))
    assert len(doc["traceEvents"]) == len(tr)
    g.free()
