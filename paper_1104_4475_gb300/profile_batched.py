"""Times one batched factorization configuration, for profilers and quick
measurements of the one-tile-column FlatTree-TS kernel and the executor.

    python -m paper_1104_4475_gb300.profile_batched --count 152 --m 8192 --n 128 --nb 128 --dtype f32

Factors `count` matrices m x n (N(0,1)) with the given nb / tree, restoring
the inputs before each repetition, and prints the CUDA-event time, the
GFLOP/s and the GFLOP/s per matrix of each repetition.
"""

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=152)
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--ib", type=int, default=8)
    ap.add_argument("--tree", default="flat_ts")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args(argv)
    import torch
    from . import tqr, build
    build.build()
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    g = torch.Generator(device="cuda").manual_seed(5)
    src = [torch.randn(a.n, a.m, generator=g, dtype=dt, device="cuda").t() for _ in range(a.count)]
    work = [torch.empty_like(s.t()).t() for s in src]
    flops = a.count * 2.0 * a.n * a.n * (a.m - a.n / 3.0)
    b = None
    for r in range(a.warmup + a.reps):
        for w, s in zip(work, src):
            w.copy_(s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if a.dtype == "f32":
            b = tqr.tqr_factor_batched_f32(work, a.nb, reuse=b)
        else:
            b = tqr.tqr_factor_batched(work, a.nb, a.ib, tqr.TREES[a.tree], 1, reuse=b)
        e1.record()
        tqr.tqr_batch_sync(b)
        t = e0.elapsed_time(e1) / 1e3
        info = b.info()
        print("%s count=%d m=%d n=%d nb=%d %s tree=%s one_column=%d: %.3f ms, %.1f GFLOP/s, %.2f GFLOP/s per matrix"
              % ("warmup" if r < a.warmup else "rep", a.count, a.m, a.n, a.nb, a.dtype, a.tree, info["n_fused"],
                 1e3 * t, flops / t / 1e9, flops / a.count / t / 1e9), flush=True)
    b.free()
    return 0


if __name__ == "__main__":
    sys.exit(main())
