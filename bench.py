"""Benchmark: FP64 tiled QR GFLOP/s on GB300 (libtqr, C ABI).

Workload ("tree sweep"): m = 16384 (p = 64 tile rows), nb = 256, ib = 32,
n = 256 q for q in {1, 2, 4, 8, 16, 32, 64}, entries iid U[-0.5, 0.5]
(seed 1), the elimination tree of each q chosen by a per-tree sweep
(Greedy for small q, Fibonacci at q = 16, PlasmaTree with TS kernels inside
domains at q >= 32).  One step factors all seven matrices; flops = sum of
2 n^2 (m - n/3) (the LAPACK count).  Inputs are resident in HBM; each step
first restores the seven matrices from pristine copies (device-to-device,
8.5 GB of traffic) after writing a 256 MiB buffer to flush L2, and both are
inside the timed region.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (numpy, the machine's host cores) on a bounded sample of the same
workload.  ``--gpus N`` under torchrun runs N independent replicas (the
factorization of one matrix does not shard), reported as weak scaling.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, NB, IB = 16384, 256, 32
QS = (1, 2, 4, 8, 16, 32, 64)
# Tree (and PlasmaTree domain size) per q: the fastest of every tree in the
# per-tree sweep of this workload on GB300 (`--workload trees`; PlasmaTree and
# PlasmaTree-TS over the critical-path model's 8 best BS and {1, p}), with
# Greedy kept where it is within about 1 % of the fastest (single timings: at
# q <= 4 the differences were 0.2 ms at most); the paper's experiments
# likewise keep the best domain size.  FlatTree-TS at q = 64 is PlasmaTree-TS
# with one domain (BS = p), which timed the same.
SWEEP_TREES = {1: ("greedy", 1), 2: ("greedy", 1), 4: ("greedy", 1), 8: ("plasma_ts", 8), 16: ("plasma_ts", 8),
               32: ("plasma_ts", 18), 64: ("flat_ts", 1)}
TREE_NAME = "tuned per q: " + ", ".join("q=%d %s%s" % (q, t, "(BS=%d)" % b if t.startswith("plasma") else "")
                                        for q, (t, b) in SWEEP_TREES.items())
SEED = 1
# FP64 peak from unit counts: 152 SMs x 2 DFMA/clk/SM (4 flop) x 2.070 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# FP32 (FFMA) peak from unit counts: 152 SMs x 128 FMA/clk/SM (256 flop) x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 256 * 2.070e9 / 1e12
# Sweep points the CPU oracle is timed on: in the GPU arm's cpu_baseline (one
# pass, about 25 s on 16 Arm cores) and, per step, in the reference arm.
CPU_SAMPLE_QS = (1, 2, 4)
REF_SAMPLE_QS = (1, 2)
# DRAM bytes per algorithmic flop of the FP64 executor: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the q = 16 PlasmaTree-TS(8)
# launch of this sweep (9.244 + 8.424 GB for 5.039e11 flop; the q = 8 Greedy
# launch gave 5.362 GB for 1.3174e11, 0.0407 bytes per flop).  The traffic
# comes from re-staging reflector blocks and strips per update task, so it
# grows with the number of strip tasks, i.e. in proportion to the flops at
# fixed nb and ib; the sweep's per-step traffic is this ratio times the
# sweep's flops.
TRAFFIC_BYTES_PER_FLOP = 17.6678e9 / 5.0394e11


def flops(m, n):
    return 2.0 * n * n * (m - n / 3.0)


PEAK_KINDS = (("dfma_tflops", 0), ("dmma_tflops", 1), ("ffma_tflops", 2), ("tf32_mma_tflops", 3))


def measure_peaks(tqr, torch, seconds=0.2):
    """Peak rates of this GPU (TFLOP/s) from the library's probes
    (tqr_peak_probe): FP64 FMA, FP64 mma.sync, FP32 FMA and TF32 mma.sync,
    each one launch of about `seconds` timed with CUDA events after a
    calibration launch."""
    stream = torch.cuda.current_stream()
    out = {}
    for name, kind in PEAK_KINDS:
        iters = 2000
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = tqr.tqr_peak_probe(kind, iters, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            rate = fl / t
            iters = max(1000, int(iters * seconds / max(t, 1e-6)))
        out[name] = rate / 1e12
    out["how"] = ("tqr_peak_probe: 2 CTAs x 8 warps per SM, independent chains of one instruction "
                  "(8 FMA chains per thread; 4 mma accumulators per warp), one launch of ~%.1f s each, CUDA events"
                  % seconds)
    return out


def workload_flops(qs=QS):
    return sum(flops(M, NB * q) for q in qs)


_JSONL = None


def emit(line):
    """Prints the result line; with --jsonl also appends it to that file."""
    text = json.dumps(line)
    print(text, flush=True)
    if _JSONL:
        with open(_JSONL, "a") as fh:
            fh.write(text + "\n")


def max_over_ranks(x, dist=None, device="cuda"):
    """Largest x over all ranks (x itself without a process group): the
    job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank, world, seconds):
    """Whole-job throughput of N independent replicas: all ranks' units / job time."""
    return units_per_rank * world / seconds


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle (CPU)
def oracle_sample(qs=CPU_SAMPLE_QS):
    """Time the CPU oracle on complete factorizations of the sweep points qs."""
    from oracle import tiled_qr as otq
    from paper_1104_4475_gb300 import workloads
    fl, t = 0.0, 0.0
    for q in qs:
        A = workloads.uniform(M, NB * q, SEED)
        t0 = time.perf_counter()
        otq.factor(A, NB, IB, 5)
        t += time.perf_counter() - t0
        fl += flops(M, NB * q)
    return fl, t


def run_oracle_subprocess(steps=1, threads=None, qs=CPU_SAMPLE_QS):
    """The oracle in a fresh process (spawned, before/independent of CUDA) with
    its BLAS threads set to `threads` (default: the host's core count), timed
    on the sweep points qs.  Returns ([(flop, seconds)] per step, threads)."""
    cores = threads or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = [bench.oracle_sample(%r) for _ in range(%d)]; print(json.dumps(r))" % (ROOT, tuple(qs), steps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1]), cores


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def single_core_oracle():
    """The oracle on one core (one BLAS thread) on the q = 1 sweep point:
    {"value": GFLOP/s, "sample": ...}, or None if the run fails."""
    try:
        res, _ = run_oracle_subprocess(1, threads=1, qs=(1,))
    except (OSError, subprocess.SubprocessError, ValueError):
        return None
    return {"value": res[0][0] / res[0][1] / 1e9, "unit": "GFLOP/s", "cores": 1,
            "sample": "one complete CPU-oracle factorization of the q = 1 point (m=%d, n=%d, nb=%d, ib=%d, Greedy)"
                      % (M, NB, NB, IB)}


def sample_desc(qs=CPU_SAMPLE_QS):
    return ("complete CPU-oracle factorizations of the q in %s points of the sweep (m=%d, nb=%d, ib=%d, Greedy, "
            "the bench's tree for these q), %.3g flop = %.2f %% of the sweep's flops"
            % (list(qs), M, NB, IB, workload_flops(qs), 100.0 * workload_flops(qs) / workload_flops()))


def cpu_estimate(rate_gflops):
    """The whole sweep on the CPU oracle at the sampled rate (a stated
    estimate: the oracle's rate depends little on q, all BLAS-2 work)."""
    return {"sweep_seconds_estimate": workload_flops() / (rate_gflops * 1e9),
            "basis": "sweep flops / the sampled rate (not measured: the full sweep would take hours on the oracle)"}


def reference_main(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    res, cores = run_oracle_subprocess(args.warmup + args.steps, qs=REF_SAMPLE_QS)
    timed = res[args.warmup:]
    fl = sum(r[0] for r in timed)
    t = sum(r[1] for r in timed)
    value = fl / t / 1e9
    line = {
        "impl": "reference", "metric": "tiled-QR GFLOP/s (FP64)", "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample_desc(REF_SAMPLE_QS) + ", per step",
                         "cpu_model": host_cpu_model(), "single_core": single_core_oracle()},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)
    return 0


def config_dict():
    return {"workload": "FP64 tree sweep: m=16384 (p=64), nb=256, ib=32, n=256q for q in "
                        "{1,2,4,8,16,32,64}, U[-0.5,0.5] entries, tree autotuned per q",
            "m": M, "nb": NB, "ib": IB, "q": list(QS), "tree": TREE_NAME, "parallelism": "replicas",
            "l2": "256 MiB flush write + input restore (8.5 GB D2D) each step, inside the timed region"}


# ---------------------------------------------------------------- GPU arm
def gpu_main(args):
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import build, workloads

    rank, world, local = dist_env()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res, cores = run_oracle_subprocess(1)        # before any CUDA call
        rate = res[0][0] / res[0][1] / 1e9
        cpu = {"value": rate, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample_desc(),
               "seconds": res[0][1], "cpu_model": host_cpu_model(), "single_core": single_core_oracle()}
        cpu.update(cpu_estimate(rate))
    build.build()
    torch.cuda.set_device(local)
    peaks = measure_peaks(tqr, torch)
    fp64_peak = peaks["dfma_tflops"]
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()

    # Inputs resident in HBM: pristine copies and working buffers.
    pristine, work = {}, {}
    for q in QS:
        a = workloads.uniform(M, NB * q, SEED)
        pristine[q] = torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
        work[q] = torch.empty_like(pristine[q].t()).t()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    handles = {}
    launches = 0

    def step(kernel_times=None):
        nonlocal launches
        flush.fill_(1.0)
        for q in QS:
            work[q].copy_(pristine[q])
        for q in QS:
            if kernel_times is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            tree, bs = SWEEP_TREES[q]
            handles[q] = tqr.tqr_factor(work[q], NB, IB, tqr.TREES[tree], bs, stream=stream, reuse=handles.get(q))
            launches += 2                               # init + executor
            if kernel_times is not None:
                e1.record(stream)
                kernel_times.append((q, e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for q in QS:
        tqr.tqr_sync(handles[q])
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = 0
    kt = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(kt)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    for q in QS:
        rc = tqr.tqr_sync(handles[q], raise_on_error=False)
        if rc != 0:
            raise RuntimeError("device status %d (%s) at q=%d" % (rc, tqr.tqr_strerror(rc), q))
    timed_launches = launches
    elapsed = max_over_ranks(elapsed, dist)
    value = weak_value(workload_flops() * args.steps, world, elapsed) / 1e9

    per_q = {}
    for q, e0, e1 in kt:
        per_q.setdefault(q, []).append(e0.elapsed_time(e1) / 1e3)
    kernel_time = sum(sum(v) for v in per_q.values()) / args.steps
    achieved = workload_flops() / kernel_time / 1e12
    detail = {str(q): {"gflops": flops(M, NB * q) / statistics.median(v) / 1e9,
                       "ms": 1e3 * statistics.median(v),
                       "critical_path_units": handles[q].info()["critical_path"]} for q, v in per_q.items()}

    # End to end through the public API with host buffers (pinned).
    e2e = None
    if not args.no_e2e:
        hosts, e2e_handles = {}, {}
        for q in QS:
            h = torch.empty((NB * q, M), dtype=torch.float64).pin_memory()
            hosts[q] = h
        h2d = sum(8 * M * NB * q for q in QS)

        # Two streams: matrix q's upload and download overlap the neighbouring
        # matrices' factorizations (pinned host memory, asynchronous copies).
        e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]

        def e2e_step():
            for idx, q in enumerate(QS):
                a = hosts[q].numpy().T                      # Fortran view of pinned memory
                tree, bs = SWEEP_TREES[q]
                e2e_handles[q] = tqr.tqr_factor_host(a, NB, IB, tqr.TREES[tree], bs, stream=e2e_streams[idx % 2],
                                                     reuse=e2e_handles.get(q), wait=False)
            for q in QS:
                rc = tqr.tqr_sync(e2e_handles[q], raise_on_error=False)
                if rc != 0:
                    raise RuntimeError("device status %d (%s) at q=%d" % (rc, tqr.tqr_strerror(rc), q))

        # The host inputs are refilled from a host copy before each step (outside the timing).
        host_src = {q: pristine[q].t().cpu().numpy() for q in QS}

        def refill():
            for q in QS:
                hosts[q].numpy()[:] = host_src[q]

        refill()
        e2e_step()
        torch.cuda.synchronize()
        tsum = 0.0
        for _ in range(args.e2e_steps):
            refill()
            if dist:
                dist.barrier()
            t_s = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            tsum += time.perf_counter() - t_s
        tsum = max_over_ranks(tsum, dist)
        e2e = {"value": weak_value(workload_flops() * args.e2e_steps, world, tsum) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d, "steps": args.e2e_steps,
               "api": "tqr_factor_host_async on two streams (pinned host A in, R and V out), tqr_sync"}
        for h in e2e_handles.values():
            h.free()

    if rank == 0:
        line = {
            "metric": "tiled-QR GFLOP/s (FP64)", "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak,
                         "traffic": args.traffic if args.traffic is not None
                         else TRAFFIC_BYTES_PER_FLOP * workload_flops(),
                         "traffic_unit": "bytes per step (7 launches), estimated from the DRAM bytes per "
                                         "flop of an ncu capture of the q = 16 PlasmaTree-TS(8) launch",
                         "algorithmic_bytes": sum(16.0 * M * NB * q for q in QS),
                         "kernel": "exec_kernel<4> (persistent executor; events around each tqr_factor)",
                         "peak_source": "measured in this run: FP64 FMA probe (DFMA; the executor's "
                                        "arithmetic), of measured",
                         "peak_unit_count": FP64_PEAK_TFLOPS,
                         "frac_of_unit_count": achieved / FP64_PEAK_TFLOPS},
            "measured_peaks": peaks,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": timed_launches,
            "fp64_pct_of_peak": 100.0 * value / 1e3 / fp64_peak / world,
            "detail": detail,
        }
    for h in handles.values():
        h.free()
    handles.clear()
    del pristine, work, flush
    torch.cuda.empty_cache()
    if rank == 0:
        if world == 1 and not args.no_next_rows:
            line["next_rows"] = next_rows(args)
        emit(line)
    if dist:
        dist.destroy_process_group()
    return 0


def next_rows(args):
    """The rest of the headline metric, measured after the sweep (outside its
    timed region): the mixed-precision least-squares speedup at the FP64
    path's backward error, the batched tall-skinny rates and the learned cost
    model's pick, each from its own workload (--workload lstsq / batched /
    costmodel) run with one timed step.  A row that fails records its error."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = 1, 3
    out = {}
    try:
        ls = lstsq_line(a)
        out["lstsq"] = {"metric": ls["metric"], "value": ls["value"], "unit": "x", "config": ls["config"]["workload"],
                        "per_kappa": {k: {x: v[x] for x in ("speedup", "fp64_seconds", "mixed_seconds",
                                                             "fp64_backward_error", "mixed_backward_error",
                                                             "converged", "refine_iterations", "cgls_iterations",
                                                             "forward_error_mixed_vs_fp64")}
                                      for k, v in ls["detail"].items()}}
    except Exception as e:                       # noqa: BLE001 - reported, not hidden
        out["lstsq"] = {"error": repr(e)}
    try:
        bt = batched_line(a)
        d = bt["detail"]
        out["batched"] = {"metric": bt["metric"], "value": bt["value"], "unit": "GFLOP/s",
                          "fp64_kernel_gflops": d["tuned"]["kernel_gflops"], "fp64_frac": bt["roofline"]["frac"],
                          "fp32_gflops": d["fp32_tuned"]["gflops"], "fp32_kernel_gflops": d["fp32_tuned"]["kernel_gflops"],
                          "fp32_frac": bt["roofline"]["fp32_frac"],
                          "fixed_config_gflops": d["fixed_nb64_ib16_greedy"]["gflops"],
                          "speedup_tuned_vs_fixed": d["speedup_tuned_vs_fixed"],
                          "peaks_of_measured": {"fp64": bt["roofline"]["peak"], "fp32": bt["roofline"]["fp32_peak"]}}
    except Exception as e:                       # noqa: BLE001
        out["batched"] = {"error": repr(e)}
    try:
        cm = costmodel_line(a)
        out["costmodel"] = {"metric": cm["metric"], "value": cm["value"], "unit": "x", "data": cm["data"],
                            "fp64": cm["detail"]["fp64"], "split_tf32": cm["detail"]["split_tf32"]}
    except Exception as e:                       # noqa: BLE001
        out["costmodel"] = {"error": repr(e)}
    return out


# ----------------------------------------------------- mixed-precision LS
LS_M, LS_N, LS_NB, LS_IB = 65536, 4096, 256, 32
# Tree for both arithmetic paths: PlasmaTree with TS kernels inside domains of
# 32 tile rows, the fastest of Greedy, PlasmaTree-TS(32) and PlasmaTree-TS(64)
# on GB300 for both paths (whole solves: FP64 2.07 / 2.15 / 2.12 s,
# split-TF32 0.405 / 0.439 / 0.436 s at kappa = 1e2).
LS_TREE, LS_BS = "plasma_ts", 32
LS_KAPPAS = (1e2, 1e6, 1e10)


def lstsq_main(args):
    emit(lstsq_line(args))
    return 0


def lstsq_line(args):
    """Mixed-precision least squares (split-TF32 updates, FP64 panels, FP64
    refinement) against the FP64 path on A = U diag(sigma) V^T, 65536 x 4096,
    kappa in {1e2, 1e6, 1e10}, b = A x_true + 1e-10 N(0,1).  Times are wall
    clock around tqr_lstsq (A, b, x resident on the device), best of
    ``--steps`` after one warm-up call."""
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import build, workloads
    build.build()
    torch.cuda.set_device(0)
    detail = {}
    for kappa in LS_KAPPAS:
        A, b, x_true = workloads.ls_problem_device(LS_M, LS_N, kappa, seed=3)
        torch.cuda.synchronize()

        def run(prec, tol, maxit):
            best, info, x = None, None, None
            for rep in range(1 + max(1, args.steps)):
                x = torch.zeros(LS_N, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = tqr.tqr_lstsq(A, b, x, LS_NB, LS_IB, tqr.TREES[args.ls_tree], args.ls_bs, prec, tol, maxit)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if rep > 0:
                    best = dt if best is None else min(best, dt)
            return best, info, x

        t64, i64, x64 = run(tqr.TQR_FP64, 0.0, 0)
        eta64 = i64["backward_error"]
        tmx, imx, xmx = run(tqr.TQR_SPLIT_TF32, eta64, 200)
        nx = float(torch.linalg.norm(x_true))
        rec = {
            "fp64_seconds": t64, "mixed_seconds": tmx,
            "speedup": (t64 / tmx) if imx["converged"] else None,
            "fp64_backward_error": eta64, "mixed_backward_error": imx["backward_error"],
            "converged": bool(imx["converged"]),
            "refine_iterations": imx["refine_iterations"], "cgls_iterations": imx["cgls_iterations"],
            "fp64_factor_seconds": i64["factor_seconds"], "mixed_factor_seconds": imx["factor_seconds"],
            "forward_error_fp64_vs_true": float(torch.linalg.norm(x64 - x_true)) / nx,
            "forward_error_mixed_vs_true": float(torch.linalg.norm(xmx - x_true)) / nx,
            "forward_error_mixed_vs_fp64": float(torch.linalg.norm(xmx - x64)) / float(torch.linalg.norm(x64)),
        }
        detail["%g" % kappa] = rec
        del A, b, x_true
        torch.cuda.empty_cache()
    head = detail["%g" % 1e6]
    line = {"metric": "mixed-prec LS speedup at FP64 backward error", "value": head["speedup"], "unit": "x",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+tf32x3", "data": "synthetic",
            "config": {"workload": "least squares A = U diag(sigma) V^T, m=65536, n=4096, sigma log-spaced "
                                   "1..1/kappa, b = A x + 1e-10 N(0,1); value at kappa=1e6",
                       "nb": LS_NB, "ib": LS_IB, "tree": "%s(BS=%d)" % (args.ls_tree, args.ls_bs),
                       "kappas": list(LS_KAPPAS)},
            "detail": detail}
    return line


# --------------------------------------------------- batched tall-skinny QR
BT_COUNT, BT_SEED = 4096, 3


def batched_main(args):
    emit(batched_line(args))
    return 0


DATA_DIR = os.path.join(ROOT, "paper_1104_4475_gb300", "data")
TUNE_DB = os.path.join(DATA_DIR, "autotune_batched_gb300.json")
TUNE_DB32 = os.path.join(DATA_DIR, "autotune_batched_f32_gb300.json")


def load_or_tune(autotune, path, sample, f32=False):
    """The tuner database at `path` if it exists, else a fresh tuning run
    (written to `path` when one is given).  Returns (db, tuning seconds or
    None when loaded)."""
    if path and os.path.exists(path):
        return autotune.load(path), None
    t = time.perf_counter()
    db = autotune.tune(sample=sample, f32=f32)
    t = time.perf_counter() - t
    if path:
        autotune.save(db, path)
    return db, t


def batched_line(args):
    """4096 independent FP64 matrices, m ~ U[512, 16384], n in {32, 64, 128},
    N(0,1) entries, factored in one persistent launch captured in a CUDA
    graph, with (nb, ib, tree) per size class from the autotuner.  A step
    restores the inputs from pristine copies and replays the graph; the same
    batch with one fixed configuration is timed the same way."""
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import autotune, build
    build.build()
    torch.cuda.set_device(0)
    peaks = measure_peaks(tqr, torch)
    rng = np.random.default_rng(BT_SEED)
    ms = rng.integers(512, 16385, BT_COUNT)
    ns = rng.choice([32, 64, 128], BT_COUNT)
    db, t_tune = load_or_tune(autotune, args.tune_db, args.tune_sample)
    g = torch.Generator(device="cuda").manual_seed(BT_SEED)
    src = [torch.randn(int(n), int(m), generator=g, dtype=torch.float64, device="cuda").t() for m, n in zip(ms, ns)]
    work = [torch.empty_like(s.t()).t() for s in src]
    flops = float(sum(2.0 * n * n * (m - n / 3.0) for m, n in zip(ms, ns)))

    def measure(cfgs, f32=False):
        nb, ib, tree, BS = (list(x) for x in zip(*cfgs))
        for w, s in zip(work, src):
            w.copy_(s)
        if f32:
            b = tqr.tqr_factor_batched_f32(work, nb)
        else:
            b = tqr.tqr_factor_batched(work, nb, ib, tree, BS)
        tqr.tqr_batch_sync(b)
        stream = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                if f32:
                    tqr.tqr_factor_batched_f32(work, nb, stream=stream, reuse=b)
                else:
                    tqr.tqr_factor_batched(work, nb, ib, tree, BS, stream=stream, reuse=b)
        for _ in range(args.warmup):
            for w, s in zip(work, src):
                w.copy_(s)
            graph.replay()
        torch.cuda.synchronize()
        step_t, kern_t = 0.0, 0.0
        for _ in range(args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            for w, s in zip(work, src):
                w.copy_(s)
            e1.record()
            graph.replay()
            e2.record()
            torch.cuda.synchronize()
            step_t += e0.elapsed_time(e2) / 1e3
            kern_t += e1.elapsed_time(e2) / 1e3
        rc = tqr.tqr_batch_sync(b)
        info = b.info()
        b.free()
        return {"gflops": flops * args.steps / step_t / 1e9, "ms_per_step": 1e3 * step_t / args.steps,
                "graph_ms": 1e3 * kern_t / args.steps, "kernel_gflops": flops * args.steps / kern_t / 1e9,
                "status": rc, "tasks": info["n_tasks"], "one_column_matrices": info["n_fused"]}

    tuned_cfgs = [autotune.lookup(db, int(m), int(n)) for m, n in zip(ms, ns)]
    tuned = measure(tuned_cfgs)
    fixed_cfgs = [(min(64, int(n)), 16, tqr.GREEDY, 1) for n in ns]
    fixed = measure(fixed_cfgs)
    # FP32: the same shapes, FlatTree-TS with one tile column, tile height tuned per class.
    db32, t32 = load_or_tune(autotune, args.tune_db32, args.tune_sample, f32=True)
    src = [s.float() for s in src]
    src = [s.t().contiguous().t() for s in src]
    work = [torch.empty_like(s.t()).t() for s in src]
    fp32 = measure([autotune.lookup(db32, int(m), int(n)) for m, n in zip(ms, ns)], f32=True)
    fp32["tuning_seconds"] = t32
    fp32["classes"] = [{k: c[k] for k in ("n", "m_lo", "m_hi", "nb", "gflops")} for c in db32["classes"]]
    line = {"metric": "batched tall-skinny QR GFLOP/s (FP64)", "value": tuned["gflops"], "unit": "GFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tuned["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4096 FP64 matrices, m ~ U[512,16384], n in {32,64,128}, N(0,1); one "
                                   "persistent launch replayed from a CUDA graph; step = input restore + replay",
                       "count": BT_COUNT, "flops_per_step": flops},
            "roofline": {"bound": "alu", "achieved": tuned["kernel_gflops"] / 1e3, "peak": peaks["dfma_tflops"],
                         "unit": "TFLOP/s", "frac": tuned["kernel_gflops"] / 1e3 / peaks["dfma_tflops"],
                         "traffic": None,
                         "kernel": "ts1_all_kernel<double>: the whole batch in one persistent launch "
                                   "(one-column FlatTree-TS; slots of 1024/512/256 threads pop matrices from "
                                   "size-sorted queues), replayed from a CUDA graph with one memset node",
                         "peak_source": "measured in this run: FP64 FMA probe, of measured",
                         "fp32_frac": fp32["kernel_gflops"] / 1e3 / peaks["ffma_tflops"],
                         "fp32_peak": peaks["ffma_tflops"], "fp32_peak_source": "measured: FP32 FMA probe"},
            "detail": {"tuned": tuned, "fixed_nb64_ib16_greedy": fixed, "fp32_tuned": fp32,
                       "speedup_tuned_vs_fixed": tuned["gflops"] / fixed["gflops"],
                       "tuning_seconds": t_tune,
                       "classes": [{k: c[k] for k in ("n", "m_lo", "m_hi", "nb", "ib", "tree", "BS", "gflops")}
                                   for c in db["classes"]]}}
    return line


# ------------------------------------------------------ per-tree comparison
def plasma_bs_candidates(tqr, p, q, tree, top=8):
    """Domain sizes timed for PlasmaTree / PlasmaTree-TS at p x q tiles: the
    `top` smallest unit-weight critical paths over BS = 1..p (ties: smaller
    BS first), together with BS = 1 and BS = p."""
    cps = sorted((tqr.tqr_critical_path(p, q, tree, bs), bs) for bs in range(1, p + 1))
    return sorted({bs for _, bs in cps[:top]} | {1, p})



def trees_main(args):
    """The tree sweep for every tree: GFLOP/s per (tree, q) and the measured
    makespan against the unit-weight critical path (Section 2.3 model),
    converted to time at one SM's FP64 rate (nb^3/3 flop per unit).
    PlasmaTree and PlasmaTree-TS take the fastest measured BS of
    plasma_bs_candidates (the critical-path model's best 8 and {1, p}).  Each
    entry is the median of ``--steps`` factorizations after one warm-up."""
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import build, workloads
    build.build()
    torch.cuda.set_device(0)
    peaks = measure_peaks(tqr, torch)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    unit_s = NB ** 3 / 3.0 / (peaks["dfma_tflops"] * 1e12 / n_sm)
    trees = [("FlatTree-TS", tqr.FLAT_TS), ("FlatTree-TT", tqr.FLAT_TT), ("BinaryTree", tqr.BINARY),
             ("Fibonacci", tqr.FIBONACCI), ("Greedy", tqr.GREEDY), ("ASAP", tqr.ASAP),
             ("PlasmaTree", tqr.PLASMA), ("PlasmaTree-TS", tqr.PLASMA_TS)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    t_all = time.perf_counter()
    for q in QS:
        src = torch.from_numpy(np.ascontiguousarray(workloads.uniform(M, NB * q, SEED).T)).cuda().t()
        work = torch.empty_like(src.t()).t()
        for name, tree in trees:
            bss = plasma_bs_candidates(tqr, M // NB, q, tree) if tree in (tqr.PLASMA, tqr.PLASMA_TS) else [1]
            best, tried = None, {}
            for BS in bss:
                times, h = [], None
                for rep in range(args.steps + 1):
                    flush.fill_(1.0)
                    work.copy_(src)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    h = tqr.tqr_factor(work, NB, IB, tree, BS, reuse=h)
                    e1.record()
                    tqr.tqr_sync(h)
                    if rep > 0:
                        times.append(e0.elapsed_time(e1) / 1e3)
                cp = h.info()["critical_path"]
                h.free()
                t = statistics.median(times)
                tried[BS] = 1e3 * t
                if best is None or t < best["ms"] / 1e3:
                    best = {"BS": BS, "ms": 1e3 * t, "gflops": flops(M, NB * q) / t / 1e9,
                            "critical_path_units": cp, "cp_bound_ms": 1e3 * cp * unit_s,
                            "makespan_over_cp_bound": t / (cp * unit_s)}
            if len(bss) > 1:
                best["ms_per_BS"] = tried
            if args.trace_cp:
                best.update(traced_critical_path(tqr, work, src, tree, best["BS"], n_sm))
            out.setdefault(name, {})[str(q)] = best
        del src, work
    sweep = {name: workload_flops() / sum(v[str(q)]["ms"] / 1e3 for q in QS) / 1e9 for name, v in out.items()}
    line = {"metric": "tiled-QR GFLOP/s (FP64) per tree", "value": max(sweep.values()), "unit": "GFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 tree sweep for every tree: m=16384 (p=64), nb=256, ib=32, n=256q, "
                                   "q in {1,2,4,8,16,32,64}, U[-0.5,0.5]; PlasmaTree and PlasmaTree-TS BS "
                                   "measured over the critical-path model's 8 best BS and {1, p}",
                       "l2": "256 MiB flush write before each factorization"},
            "measured_peaks": peaks,
            "best_tree": max(sweep, key=sweep.get), "sweep_gflops": sweep, "per_tree": out,
            "unit_ms": 1e3 * unit_s, "seconds": time.perf_counter() - t_all}
    emit(line)
    return 0


def traced_critical_path(tqr, work, src, tree, BS, n_sm):
    """One traced factorization (after an untraced one that builds the
    handle): its traced makespan, SM busy fraction and measured critical path,
    the longest path through the executed graph with traced task durations."""
    from paper_1104_4475_gb300 import trace as ttrace
    work.copy_(src)
    h = tqr.tqr_factor(work, NB, IB, tree, BS)
    tqr.tqr_set_trace(h, True)
    work.copy_(src)
    h = tqr.tqr_factor(work, NB, IB, tree, BS, reuse=h)
    tqr.tqr_sync(h)
    tr, edges = tqr.tqr_get_trace(h), tqr.tqr_get_edges(h)
    h.free()
    s = ttrace.summary(tr, n_sm)
    cp_ns, path = ttrace.measured_critical_path(tr, edges)
    return {"traced_makespan_ms": s["makespan_ms"], "busy_fraction": s["busy_fraction"],
            "measured_cp_ms": cp_ns / 1e6, "measured_cp_tasks": len(path)}


# ------------------------------------------------------- learned cost model
def costmodel_main(args):
    emit(costmodel_line(args))
    return 0


def costmodel_line(args):
    """Trains the cost-model network on the GPU (the library's forward,
    backward and Adam kernels) from the stored executor timings, then scores
    its pick on the held-out shapes against the exhaustive best, the fixed
    default (Greedy, nb 256) and the smallest-critical-path rule."""
    import torch
    from paper_1104_4475_gb300 import build, costmodel
    build.build()
    torch.cuda.set_device(0)
    data_dir = os.path.join(ROOT, "paper_1104_4475_gb300", "data")
    path = args.cost_data or os.path.join(data_dir, "costmodel_timings_gb300.csv")
    heldout = os.path.join(data_dir, "costmodel_heldout_gb300.csv")
    recs = costmodel.load_records(path)
    if args.cost_data is None and os.path.exists(heldout):
        train = recs                                            # 100 training shapes; 200 held-out shapes,
        test = costmodel.disjoint(train, costmodel.load_records(heldout))   # minus any (m, n) seen in training
        recs = recs + test
    else:
        train, test = costmodel.split(recs)
    X, y = costmodel.design(train)
    steps = 3000
    costmodel.train(X[:64], y[:64], steps=10)                # warm-up (build, first launches)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    model, losses = costmodel.train(X, y, steps=steps)
    e1.record()
    torch.cuda.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    fp64 = costmodel.summarize(costmodel.evaluate(model, test, 0))
    lp = costmodel.summarize(costmodel.evaluate(model, test, 1))
    Xt, yt = costmodel.design(test)
    rmse = float(np.sqrt(np.mean((model.predict_log_seconds(Xt) - yt) ** 2)))
    line = {"metric": "cost-model pick makespan / exhaustive best (held-out shapes, FP64)",
            "value": fp64["model_over_best"], "unit": "x", "n_gpus": 1, "steps": steps, "warmup": 10,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "executor timings on GB300 (%d runs; %d training shapes, %d held-out shapes)"
                    % (len(recs), len(costmodel.by_shape(train)), len(costmodel.by_shape(test))),
            "config": {"workload": "3-layer MLP (width 64, FP32), full-batch Adam on %d training runs; m in "
                                   "[4096,65536], n in [256,m], at most 5e11 flop per run; 12 FP64 and 6 "
                                   "split-TF32 candidates per shape" % len(train)},
            "detail": {"fp64": fp64, "split_tf32": lp, "test_rmse_log_seconds": rmse,
                       "train_seconds": train_s, "train_steps_per_s": steps / train_s,
                       "final_train_loss": losses[-1][1]}}
    return line


# ------------------------------------------------------ profiling drivers
def case_main(args):
    """One factorization size, for profilers and quick timing: factors an
    m x (nb q) matrix of U[-0.5, 0.5] entries (seed 1) with the given tree,
    BS and update arithmetic, restoring the input before each repetition,
    and prints the CUDA-event time and GFLOP/s of each.  With --trace the
    repetitions after the first are traced and the last one is summarised
    (trace.report: SM busy fraction, time per kernel kind, measured critical
    path, the Section 4 model's prediction)."""
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import build, workloads, trace as ttrace
    build.build()
    n = args.nb * args.q
    A0 = torch.from_numpy(np.ascontiguousarray(workloads.uniform(args.m, n, SEED).T)).cuda().t()
    A = torch.empty_like(A0.t()).t()
    tree = tqr.TREES[args.tree]
    f, traced = None, False
    for r in range(args.warmup + args.steps):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = tqr.tqr_factor_ex(A, args.nb, args.ib, tree, args.BS, args.precision, reuse=f)
        e1.record()
        tqr.tqr_sync(f)
        t = e0.elapsed_time(e1) / 1e3
        info = f.info()
        print("%s m=%d n=%d nb=%d ib=%d tree=%s BS=%d prec=%d tasks=%d cp=%d: %.3f ms, %.1f GFLOP/s"
              % ("warmup" if r < args.warmup else "rep", args.m, n, args.nb, args.ib, args.tree, args.BS,
                 args.precision, info["n_device_tasks"], info["critical_path"], 1e3 * t, info["flops"] / t / 1e9),
              flush=True)
        if args.trace and not traced:
            tqr.tqr_set_trace(f, True)                  # from the next factorization on
            traced = r + 1 < args.warmup + args.steps
    if traced:
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        for ln in ttrace.report(tqr.tqr_get_trace(f), tqr.tqr_get_edges(f), f.info(), n_sm):
            print(ln)
    f.free()
    return 0


def batch_case_main(args):
    """One batched configuration, for profilers and quick timing: factors
    --count matrices m x n (N(0,1)) with the given nb, ib and tree (FP64) or
    the one-column FP32 kernel (--dtype f32), restoring the inputs before each
    repetition, and prints the CUDA-event time, GFLOP/s and GFLOP/s per
    matrix."""
    import torch
    import paper_1104_4475_gb300 as tqr
    from paper_1104_4475_gb300 import build
    build.build()
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    g = torch.Generator(device="cuda").manual_seed(5)
    src = [torch.randn(args.n, args.m, generator=g, dtype=dt, device="cuda").t() for _ in range(args.count)]
    work = [torch.empty_like(x.t()).t() for x in src]
    fl = args.count * 2.0 * args.n * args.n * (args.m - args.n / 3.0)
    b = None
    for r in range(args.warmup + args.steps):
        for w, x in zip(work, src):
            w.copy_(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.dtype == "f32":
            b = tqr.tqr_factor_batched_f32(work, args.nb, reuse=b)
        else:
            b = tqr.tqr_factor_batched(work, args.nb, args.ib, tqr.TREES[args.tree], args.BS, reuse=b)
        e1.record()
        tqr.tqr_batch_sync(b)
        t = e0.elapsed_time(e1) / 1e3
        print("%s count=%d m=%d n=%d nb=%d %s tree=%s one_column=%d: %.3f ms, %.1f GFLOP/s, %.2f GFLOP/s per matrix"
              % ("warmup" if r < args.warmup else "rep", args.count, args.m, args.n, args.nb, args.dtype, args.tree,
                 b.info()["n_fused"], 1e3 * t, fl / t / 1e9, fl / args.count / t / 1e9), flush=True)
    b.free()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "lstsq", "batched", "trees", "costmodel", "case", "batch-case"],
                    help="sweep: FP64 tree sweep (default); lstsq: mixed-precision least squares; "
                         "batched: 4096 tall-skinny matrices in one launch; trees: the sweep for every tree; "
                         "costmodel: train and score the learned cost model; case / batch-case: one size, "
                         "timed per repetition (for profilers; --steps repetitions after --warmup)")
    ap.add_argument("--m", type=int, default=M, help="case / batch-case: rows")
    ap.add_argument("--q", type=int, default=8, help="case: tile columns (n = nb q)")
    ap.add_argument("--n", type=int, default=128, help="batch-case: columns")
    ap.add_argument("--nb", type=int, default=NB, help="case / batch-case: tile size")
    ap.add_argument("--ib", type=int, default=IB, help="case / batch-case: inner blocking")
    ap.add_argument("--tree", default="greedy", help="case / batch-case: tree name (tqr.TREES)")
    ap.add_argument("--BS", type=int, default=1, help="case / batch-case: PlasmaTree domain size")
    ap.add_argument("--precision", type=int, default=0, help="case: 0 FP64, 1 split-TF32, 2 TF32 updates")
    ap.add_argument("--trace", action="store_true", help="case: trace and summarise the last repetition")
    ap.add_argument("--count", type=int, default=152, help="batch-case: matrices")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"], help="batch-case: FP64 or FP32")
    ap.add_argument("--cost-data", default=None, help="executor timings CSV for --workload costmodel")
    ap.add_argument("--jsonl", default=None, help="also append the result line to this JSONL file")
    ap.add_argument("--tune-db", default=TUNE_DB,
                    help="FP64 batch autotune database to load, or to write after tuning (default: the stored "
                         "GB300 database; '' to tune afresh)")
    ap.add_argument("--tune-db32", default=TUNE_DB32, help="the same for the FP32 batch")
    ap.add_argument("--ls-tree", default=LS_TREE, help="least squares: elimination tree of both paths")
    ap.add_argument("--ls-bs", type=int, default=LS_BS, help="least squares: PlasmaTree domain size")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="default workload: skip the least-squares, batched and cost-model measurements that "
                         "follow the sweep")
    ap.add_argument("--tune-sample", type=int, default=32, help="matrices per size class when tuning")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trace-cp", action="store_true",
                    help="--workload trees: trace one more factorization per (tree, q) at its best BS and report "
                         "the measured critical path (longest traced path through the executed graph)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per executor launch from an ncu capture (for the roofline line)")
    args = ap.parse_args()
    global _JSONL
    _JSONL = args.jsonl
    if args.workload == "case":
        return case_main(args)
    if args.workload == "batch-case":
        return batch_case_main(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_main(args)
    if args.workload == "lstsq":
        return lstsq_main(args)
    if args.workload == "batched":
        return batched_main(args)
    if args.workload == "trees":
        return trees_main(args)
    if args.workload == "costmodel":
        return costmodel_main(args)
    return gpu_main(args)


if __name__ == "__main__":
    sys.exit(main())
