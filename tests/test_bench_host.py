"""Host-side parts of bench.py's CPU baseline (no GPU): the host CPU model
and the single-core oracle time that accompany the multi-core figure."""

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_host_cpu_model_is_named():
    name = bench.host_cpu_model()
    assert isinstance(name, str) and name.strip()


def test_single_core_oracle_time():
    r = bench.single_core_oracle()
    assert r is not None and r["cores"] == 1 and r["value"] > 0
    assert "q = 1" in r["sample"]


def test_traced_critical_path_with_a_fake_library():
    """The --trace-cp step of the trees workload: build a handle, enable
    tracing, factor again with it, and reduce the trace (here a library
    stand-in whose trace is a chain of three tasks of 1, 2 and 3 ms)."""
    import numpy as np
    torch = __import__("pytest").importorskip("torch")

    class Handle:
        freed = False

        def free(self):
            Handle.freed = True

    class FakeLib:
        calls = []

        def tqr_factor(self, A, nb, ib, tree, BS, reuse=None):
            self.calls.append(("factor", tree, BS, reuse is not None))
            return reuse or Handle()

        def tqr_set_trace(self, h, on):
            self.calls.append(("trace", on))

        def tqr_sync(self, h):
            return 0

        def tqr_get_trace(self, h):
            tr = np.zeros((3, 8), dtype=np.int64)
            tr[:, 5] = [0, 1_000_000, 3_000_000]
            tr[:, 6] = [1_000_000, 3_000_000, 6_000_000]
            return tr

        def tqr_get_edges(self, h):
            return np.array([[0, 1], [1, 2]])

    lib = FakeLib()
    work, src = torch.zeros(4, 2), torch.ones(4, 2)
    r = bench.traced_critical_path(lib, work, src, 5, 1, n_sm=2)
    assert [c[0] for c in lib.calls] == ["factor", "trace", "factor"] and lib.calls[2][3]
    assert r["measured_cp_ms"] == 6.0 and r["measured_cp_tasks"] == 3
    assert r["traced_makespan_ms"] == 6.0 and r["busy_fraction"] == 0.5
    assert Handle.freed and torch.equal(work, src)
