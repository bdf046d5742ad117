"""Autotuner for batched tall-skinny factorizations.

For each size class -- a column count n and a range of row counts m -- every
candidate (nb, ib, tree, BS) is timed on a sample batch of that class (one
batched launch per candidate, CUDA events, best of ``reps`` after a warm-up)
and the fastest is kept.  Results form a versioned JSON database that can be
saved and reloaded; :func:`lookup` maps any (m, n) to its class's choice.

The search is exhaustive over the candidate set; a learned cost model can
replace it by ranking candidates without timing them (see ``costmodel``).
"""

import json

import numpy as np

from . import tqr

DB_VERSION = 2
M_BUCKETS = [(512, 1024), (1024, 2048), (2048, 4096), (4096, 8192), (8192, 16385)]
N_CLASSES = [32, 64, 128]
TREE_CANDIDATES = [(tqr.GREEDY, 1), (tqr.BINARY, 1), (tqr.FIBONACCI, 1), (tqr.FLAT_TT, 1), (tqr.FLAT_TS, 1),
                   (tqr.PLASMA, 4), (tqr.PLASMA, 16), (tqr.ASAP, 1)]


ONE_COLUMN_NB = (64, 128, 256)
SQUARE_NB = (16, 32, 64, 128)


def candidates(n, m_lo):
    """(nb, ib, tree, BS) candidates for matrices with n columns: square tiles
    nb <= n with every tree, plus FlatTree-TS with one tile column (nb >= n),
    which runs each matrix in one CTA."""
    out = []
    for nb in SQUARE_NB:
        if nb > n or nb > m_lo:
            continue
        for ib in (8, 16, 32):
            if ib > nb or nb % ib:
                continue
            for tree, BS in TREE_CANDIDATES:
                p_min = -(-m_lo // nb)
                out.append((nb, ib, tree, min(BS, p_min)))
    for nb in ONE_COLUMN_NB:
        if nb >= n and (nb, 8, tqr.FLAT_TS, 1) not in out:
            out.append((nb, 8, tqr.FLAT_TS, 1))
    return out


def candidates_f32(n):
    """Tile heights for FP32 batches (FlatTree-TS, one tile column)."""
    return [(nb, nb, tqr.FLAT_TS, 1) for nb in ONE_COLUMN_NB if nb >= n]


def sample_class(n, m_lo, m_hi, count, seed):
    rng = np.random.default_rng(seed)
    return [int(m) for m in rng.integers(m_lo, m_hi, count)]


def time_batch(ms, n, cfg, reps=2, seed=0, f32=False):
    """Seconds for one batched launch of matrices (ms[i] x n) with config cfg."""
    import torch
    nb, ib, tree, BS = cfg
    g = torch.Generator(device="cuda").manual_seed(seed)
    dt = torch.float32 if f32 else torch.float64
    src = [torch.randn(n, m, generator=g, dtype=dt, device="cuda").t() for m in ms]
    work = [torch.empty_like(s.t()).t() for s in src]
    b = None
    best = None
    for r in range(reps + 1):
        for w, s in zip(work, src):
            w.copy_(s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if f32:
            b = tqr.tqr_factor_batched_f32(work, nb, reuse=b)
        else:
            b = tqr.tqr_factor_batched(work, nb, ib, tree, BS, reuse=b)
        e1.record()
        tqr.tqr_batch_sync(b)
        t = e0.elapsed_time(e1) / 1e3
        if r > 0:
            best = t if best is None else min(best, t)
    b.free()
    return best


def tune(n_classes=N_CLASSES, m_buckets=M_BUCKETS, sample=32, reps=2, seed=7, log=None, f32=False, full=304,
         shortlist=3):
    """Exhaustive search in two stages; returns the database (a dict).

    Stage 1 times every candidate on `sample` matrices of the class.  A small
    sample favours configurations that spread one matrix over many SMs, so
    stage 2 re-times the `shortlist` best of stage 1 and every one-column
    candidate (one CTA per matrix) on `full` matrices (the sample repeated),
    enough to fill the GPU, and keeps the fastest per matrix."""
    import torch
    classes = []
    for n in n_classes:
        for (lo, hi) in m_buckets:
            ms = sample_class(n, lo, hi, sample, seed + n + lo)
            results = []
            for cfg in (candidates_f32(n) if f32 else candidates(n, lo)):
                try:
                    t = time_batch(ms, n, cfg, reps=reps, seed=seed, f32=f32)
                except tqr.TqrError:
                    continue
                results.append((t, cfg))
            results.sort()
            if full and full > sample:
                big = [ms[i % len(ms)] for i in range(full)]
                short = [cfg for _, cfg in results[:shortlist]]
                short += [cfg for _, cfg in results if cfg[2] == tqr.FLAT_TS and cfg[0] >= n and cfg not in short]
                results = []
                for cfg in short:
                    try:
                        t = time_batch(big, n, cfg, reps=1, seed=seed, f32=f32) * len(ms) / len(big)
                    except tqr.TqrError:
                        continue
                    results.append((t, cfg))
                results.sort()
            t, (nb, ib, tree, BS) = results[0]
            flops = sum(2.0 * n * n * (m - n / 3.0) for m in ms)
            rec = {"n": n, "m_lo": lo, "m_hi": hi, "nb": nb, "ib": ib, "tree": tree, "BS": BS, "seconds": t,
                   "gflops": flops / t / 1e9, "candidates": len(results),
                   "worst_seconds": results[-1][0]}
            classes.append(rec)
            if log:
                log(rec)
    return {"version": DB_VERSION, "gpu": torch.cuda.get_device_name(0), "sample": sample, "classes": classes,
            "dtype": "f32" if f32 else "f64"}


def save(db, path):
    with open(path, "w") as fh:
        json.dump(db, fh, indent=1)


def load(path):
    with open(path) as fh:
        db = json.load(fh)
    if db.get("version") != DB_VERSION:
        raise ValueError("autotune database version %r, expected %d" % (db.get("version"), DB_VERSION))
    return db


def lookup(db, m, n):
    """The tuned (nb, ib, tree, BS) for an m x n matrix: its class, or the
    nearest class in n and m.  A square-tile choice whose nb exceeds n takes
    the largest candidate tile size that fits n (one-column FlatTree-TS when
    none does), so the result is always a valid configuration for (m, n)."""
    best, key = None, None
    for c in db["classes"]:
        dn = abs(np.log2(n) - np.log2(c["n"]))
        dm = 0.0 if c["m_lo"] <= m < c["m_hi"] else min(abs(np.log2(m / c["m_lo"])), abs(np.log2(m / c["m_hi"])))
        d = (dn, dm)
        if best is None or d < key:
            best, key = c, d
    fits = [c for c in SQUARE_NB if c <= min(best["nb"], n)]
    if best["tree"] == tqr.FLAT_TS and best["nb"] >= best["n"]:     # one tile column
        return min(max(best["nb"], -(-n // 4) * 4), 256), 8, tqr.FLAT_TS, 1
    if not fits:                                                     # n below every square tile
        return max(ONE_COLUMN_NB[0], -(-n // 4) * 4), 8, tqr.FLAT_TS, 1
    nb = fits[-1]
    ib = min(best["ib"], nb)
    BS = best["BS"]
    if best["tree"] == tqr.PLASMA:
        BS = max(1, min(BS, -(-m // nb)))
    return nb, ib, best["tree"], BS
