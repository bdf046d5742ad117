"""Runs a few factorizations of one size, for profilers and quick timing.

    python -m paper_1104_4475_gb300.profile_case --m 16384 --q 8 --reps 2

Factors an m x (nb*q) matrix of U[-0.5, 0.5] entries with the given tree,
restoring the input before each repetition, and prints the CUDA-event time and
GFLOP/s of each factorization.
"""

import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--q", type=int, default=8)
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--ib", type=int, default=32)
    ap.add_argument("--tree", default="greedy")
    ap.add_argument("--BS", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--precision", type=int, default=0, help="0 FP64, 1 split-TF32, 2 TF32 updates")
    a = ap.parse_args(argv)
    import torch
    from . import tqr, build, workloads
    build.build()
    n = a.nb * a.q
    A0 = torch.from_numpy(np.ascontiguousarray(workloads.uniform(a.m, n, 1).T)).cuda().t()
    A = torch.empty_like(A0.t()).t()
    tree = tqr.TREES[a.tree]
    f = None
    for r in range(a.warmup + a.reps):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = tqr.tqr_factor_ex(A, a.nb, a.ib, tree, a.BS, a.precision, reuse=f)
        e1.record()
        tqr.tqr_sync(f)
        t = e0.elapsed_time(e1) / 1e3
        info = f.info()
        print("%s m=%d n=%d nb=%d ib=%d tree=%s prec=%d tasks=%d cp=%d: %.3f ms, %.1f GFLOP/s"
              % ("warmup" if r < a.warmup else "rep", a.m, n, a.nb, a.ib, a.tree, a.precision, info["n_device_tasks"],
                 info["critical_path"], 1e3 * t, info["flops"] / t / 1e9), flush=True)
    f.free()
    return 0


if __name__ == "__main__":
    sys.exit(main())
