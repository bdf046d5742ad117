"""Runs a few factorizations of one size, for profilers and quick timing.

    python -m paper_1104_4475_gb300.profile_case --m 16384 --q 8 --reps 2

Factors an m x (nb*q) matrix of U[-0.5, 0.5] entries with the given tree,
restoring the input before each repetition, and prints the CUDA-event time and
GFLOP/s of each factorization.  With --trace, every factorization after the
first records per-task device times, and the last one's trace is summarised:
SM busy fraction and time per kernel kind, the measured critical path (the
longest path through the executed graph, each task weighted by its traced
duration) against the makespan, and the Section 4 model's predicted rate
gamma_seq * T / max(T/P, cp) with gamma_seq taken from the trace.
"""

import argparse
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
    ap.add_argument("--trace", action="store_true", help="trace every factorization after the first")
    a = ap.parse_args(argv)
    import torch
    from . import tqr, build, workloads
    build.build()
    n = a.nb * a.q
    A0 = torch.from_numpy(np.ascontiguousarray(workloads.uniform(a.m, n, 1).T)).cuda().t()
    A = torch.empty_like(A0.t()).t()
    tree = tqr.TREES[a.tree]
    f = None
    traced = False
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
        if a.trace and not traced:
            tqr.tqr_set_trace(f, True)                  # from the next factorization on
            traced = r + 1 < a.warmup + a.reps
    if traced:
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        for line in trace_report(tqr.tqr_get_trace(f), tqr.tqr_get_edges(f), f.info(), n_sm):
            print(line)
    f.free()
    return 0


def trace_report(tr, edges, info, n_sm):
    """Lines summarising one traced factorization (see the module docstring);
    info is the handle's tqr_get_info dict."""
    from . import trace as ttrace
    s = ttrace.summary(tr, n_sm)
    cp_ns, path = ttrace.measured_critical_path(tr, edges)
    model = ttrace.model_prediction(tr, info["nb"], info["strip"], info["n"], info["critical_path"], n_sm,
                                    info["flops"], info.get("ib"))
    return ["trace: makespan %.3f ms, SMs busy %.1f %%, busy ms per kind %s"
            % (s["makespan_ms"], 100 * s["busy_fraction"], {k: round(v, 3) for k, v in s["busy_ms_per_kind"].items()}),
            "trace: measured critical path %.3f ms over %d tasks (%.1f %% of the makespan)"
            % (cp_ns / 1e6, len(path), 100 * cp_ns / 1e6 / s["makespan_ms"]),
            "model: T = %.0f units, cp = %d units, P = %d, bound %s; gamma_seq %.2f GFLOP/s per CTA, "
            "gamma_pred %.1f GFLOP/s, predicted %.3f ms (%.1f GFLOP/s in LAPACK flops)"
            % (model["units"], info["critical_path"], n_sm, model["bound"], model["gamma_seq_gflops"],
               model["gamma_pred_gflops"], model["predicted_ms"], model["predicted_lapack_gflops"])]


if __name__ == "__main__":
    sys.exit(main())
