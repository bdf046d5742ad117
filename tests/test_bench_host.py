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
