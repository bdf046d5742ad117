import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")


def pytest_collection_modifyitems(config, items):
    """Run the full-size modules (tens of GB on the device, minutes each)
    after every small-size test, keeping the order within each group."""
    def full_size(item):
        return os.path.basename(str(item.fspath)).startswith("test_gpu_fullsize")
    items[:] = [it for it in items if not full_size(it)] + [it for it in items if full_size(it)]


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_blocks(name):
    """Parse a golden table file made of '[Name]' blocks of 'i: v1 v2 ...' lines."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            if ln.startswith("["):
                cur = ln[1:-1]
                blocks[cur] = {}
                continue
            r, vals = ln.split(":")
            blocks[cur][int(r)] = [int(v) for v in vals.split()]
    return blocks


def load_rows(name):
    """Parse a golden file of whitespace-separated integer rows."""
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                out.append([int(v) for v in ln.split()])
    return out
