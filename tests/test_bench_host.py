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


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the CPU oracle, no GPU) prints one JSON line
    with the contract's keys; its e2e and cpu_baseline describe the same run."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"),
                        "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]
