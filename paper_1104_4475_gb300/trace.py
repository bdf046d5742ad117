"""Per-task device traces of the executor (tqr_set_trace / tqr_get_trace):
Chrome-trace export and summaries.

A trace row is (kind, i, piv, k, w, start ns, end ns, SM), 0-based tile
indices, one row per device task.  For an update strip w = j * 65536 + strip;
for a panel run as one task w = -1; for a task of block b of a panel split
into blocks, w = b << 32 | c_lo << 16 | c_hi: it factors the block's own
columns (c_lo = b * ib) or applies the block to columns [c_lo, c_hi).
"""

import json

import numpy as np

KIND_NAMES = ("GEQRT", "UNMQR", "TTQRT", "TTMQR", "TSQRT", "TSMQR")


PANEL_KINDS = (0, 2, 4)


def panel_part(w):
    """(block, c_lo, c_hi) of a panel task's trace word, or None for a panel
    run as one task."""
    if w < 0:
        return None
    return w >> 32, (w >> 16) & 0xffff, w & 0xffff


def task_label(kind, i, piv, k, w):
    if kind in PANEL_KINDS:
        part = panel_part(w)
        extra = "" if part is None else " b%d [%d,%d)" % part
        return "%s(%d,%d,%d)%s" % (KIND_NAMES[kind], i, piv, k, extra)
    return "%s(%d,%d,%d,%d/%d)" % (KIND_NAMES[kind], i, piv, k, w >> 16, w & 0xffff)


def to_chrome(trace, path=None):
    """Chrome trace-event JSON (one track per SM); written to path if given."""
    t0 = int(trace[:, 5].min()) if len(trace) else 0
    ev = []
    for kind, i, piv, k, js, s, e, sm in trace.tolist():
        name = task_label(kind, i, piv, k, js)
        ev.append({"name": name, "cat": KIND_NAMES[kind], "ph": "X", "pid": 0, "tid": int(sm),
                   "ts": (s - t0) / 1e3, "dur": max(0, e - s) / 1e3})
    doc = {"traceEvents": ev, "displayTimeUnit": "ns"}
    if path:
        with open(path, "w") as fh:
            json.dump(doc, fh)
    return doc


def summary(trace, n_sm=None):
    """Makespan, busy fraction of the SMs that ran tasks, and time per kernel kind."""
    if len(trace) == 0:
        return {"tasks": 0}
    start, end = trace[:, 5], trace[:, 6]
    makespan = int(end.max() - start.min())
    busy = (end - start).astype(np.float64)
    sms = n_sm or len(np.unique(trace[:, 7]))
    per_kind = {KIND_NAMES[k]: float(busy[trace[:, 0] == k].sum()) / 1e6 for k in range(6) if (trace[:, 0] == k).any()}
    return {"tasks": int(len(trace)), "makespan_ms": makespan / 1e6, "sms": int(sms),
            "busy_fraction": float(busy.sum() / (makespan * sms)) if makespan > 0 else 0.0,
            "busy_ms_per_kind": per_kind}


def producer_violations(trace):
    """Update tasks that started before the panel task whose reflectors they
    apply had finished (UNMQR after GEQRT(i,k), TTMQR after TTQRT(i,piv,k),
    TSMQR after TSQRT(i,piv,k)); an empty list means the executor honoured
    every producer edge."""
    end = {}
    for kind, i, piv, k, js, s, e, sm in trace.tolist():
        if kind in PANEL_KINDS:                 # a split panel ends with its last task
            key = (kind, i, piv if kind else -1, k)
            end[key] = max(end.get(key, e), e)
    bad = []
    for kind, i, piv, k, js, s, e, sm in trace.tolist():
        if kind in (1, 3, 5):
            key = (kind - 1, i, piv if kind != 1 else -1, k)
            if key not in end or s < end[key]:
                bad.append((kind, i, piv, k, js))
    return bad


def edge_violations(trace, edges):
    """Dependency edges (u, v) of the graph whose task v started before task u
    ended -- the happens-before check of a traced run (empty when the
    executor honoured every edge)."""
    if len(edges) == 0:
        return []
    u, v = edges[:, 0], edges[:, 1]
    bad = trace[v, 5] < trace[u, 6]
    return [tuple(e) for e in edges[bad].tolist()]


# Weights of the six kernels in units of nb^3/3 flops (Table 1), indexed by kind.
KERNEL_WEIGHT = (4, 6, 2, 6, 6, 12)


def measured_critical_path(trace, edges):
    """Longest path through the executed task graph with every task weighted
    by its traced duration (end - start): the measured counterpart of the
    unit-weight critical path of the Section 2.3 model.  Every edge (u, v)
    of the executor's graphs runs from a task to a later one (task ids follow
    program order), so one pass in id order finds it.  Returns
    (length_ns, path), path being the task ids along it, first to last."""
    n = len(trace)
    if n == 0:
        return 0, []
    dur = (trace[:, 6] - trace[:, 5]).astype(np.int64)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if len(edges) and not np.all(edges[:, 0] < edges[:, 1]):
        raise ValueError("an edge does not run from an earlier task to a later one")
    order = np.argsort(edges[:, 1], kind="stable")
    src, dst = edges[order, 0], edges[order, 1]
    ptr = np.searchsorted(dst, np.arange(n + 1))
    best = np.zeros(n, dtype=np.int64)
    back = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        lo, hi = ptr[v], ptr[v + 1]
        if hi > lo:
            preds = src[lo:hi]
            a = int(np.argmax(best[preds]))
            back[v] = preds[a]
            best[v] = best[preds[a]] + dur[v]
        else:
            best[v] = dur[v]
    v = int(np.argmax(best))
    length = int(best[v])
    path = []
    while v >= 0:
        path.append(v)
        v = int(back[v])
    return length, path[::-1]


def panel_part_flops(kind, nb, ib, b, c_lo, c_hi, ncol):
    """Flops of one task of a split panel (block b, columns [c_lo, c_hi)):
    applying reflector j to one column costs 4 (t_j + 1) flops with t_j the
    length of its tail (nb - j - 1 for GEQRT, j + 1 for TTQRT, nb for TSQRT);
    forming it, about 3 t_j.  The factor task forms the block's reflectors and
    applies each to the block's later columns; an update task applies the
    block to its columns."""
    def tail(j):
        return nb - j - 1 if kind == 0 else (j + 1 if kind == 2 else nb)
    j0 = b * ib
    if c_lo == j0:                               # the factor task
        if j0 >= ncol:
            return 0.0
        return float(sum(3 * tail(j) + 4 * (tail(j) + 1) * (j0 + ib - 1 - j) for j in range(j0, j0 + ib)))
    return float(sum(4 * (tail(j) + 1) * (c_hi - c_lo) for j in range(j0, j0 + ib)))


def task_units(trace, nb, strip, n, ib=None):
    """Work of every traced task in units of nb^3/3 flops: the kernel's
    weight (Table 1) for a panel run as one task; for a task of a split panel
    (needs ib) the weight times its share of the panel's flops
    (panel_part_flops over the panel's tasks); for an update task the weight
    times the fraction of the tile's nb columns its strip covers (strips of
    `strip` columns; the last tile column holds n - (q-1) nb columns).  Over a
    whole factorization with n a multiple of nb they sum to the total weight
    of the list (6pq^2 - 2q^3 for TT kernels, Section 2.2)."""
    q = -(-n // nb)
    last_cols = n - (q - 1) * nb
    units = np.empty(len(trace), dtype=np.float64)
    parts = {}                                   # panel -> [(task, flops)]
    for t, (kind, i, piv, k, js, s, e, sm) in enumerate(trace.tolist()):
        w = KERNEL_WEIGHT[kind]
        if kind in PANEL_KINDS:
            part = panel_part(js)
            if part is None:
                units[t] = float(w)
            else:
                if ib is None:
                    raise ValueError("a split panel's work needs ib")
                ncol = last_cols if k == q - 1 else nb
                parts.setdefault((kind, i, piv, k), []).append(
                    (t, panel_part_flops(kind, nb, ib, part[0], part[1], part[2], ncol)))
        else:
            j, st = js >> 16, js & 0xffff
            cols = last_cols if j == q - 1 else nb
            units[t] = w * min(strip, cols - st * strip) / nb
    for (kind, i, piv, k), lst in parts.items():
        tot = sum(f for _, f in lst)
        for t, f in lst:
            units[t] = KERNEL_WEIGHT[kind] * (f / tot if tot > 0 else 1.0 / len(lst))
    return units


def model_prediction(trace, nb, strip, n, critical_path, n_cta, flops, ib=None):
    """The paper's performance model (Section 4) fed with measured rates:
    gamma_seq, one CTA's rate, is the traced work over the traced busy time;
    with T units of work, P CTAs and a unit-weight critical path cp, the model
    predicts a makespan of max(T/P, cp) units at gamma_seq, i.e. a rate of
    gamma_seq * T / max(T/P, cp) (flops counted per unit as nb^3/3).  Also
    returns the makespan and rate that `flops` (the LAPACK count) gives."""
    units = task_units(trace, nb, strip, n, ib)
    busy_s = float((trace[:, 6] - trace[:, 5]).sum()) / 1e9
    unit_flops = nb ** 3 / 3.0
    T = float(units.sum())
    gamma_seq = T * unit_flops / busy_s if busy_s > 0 else 0.0
    bound_units = max(T / n_cta, float(critical_path))
    t_pred = bound_units * unit_flops / gamma_seq if gamma_seq > 0 else 0.0
    return {"units": T, "gamma_seq_gflops": gamma_seq / 1e9, "bound": "cp" if critical_path > T / n_cta else "work",
            "bound_units": bound_units, "gamma_pred_gflops": gamma_seq * T / bound_units / 1e9 if bound_units else 0.0,
            "predicted_ms": 1e3 * t_pred, "predicted_lapack_gflops": flops / t_pred / 1e9 if t_pred > 0 else 0.0}


def report(tr, edges, info, n_sm):
    """Lines summarising one traced factorization: SM busy fraction and time
    per kernel kind, the measured critical path against the makespan, and the
    Section 4 model's predicted rate with gamma_seq taken from the trace;
    info is the handle's tqr_get_info dict."""
    s = summary(tr, n_sm)
    cp_ns, path = measured_critical_path(tr, edges)
    model = model_prediction(tr, info["nb"], info["strip"], info["n"], info["critical_path"], n_sm,
                             info["flops"], info.get("ib"))
    return ["trace: makespan %.3f ms, SMs busy %.1f %%, busy ms per kind %s"
            % (s["makespan_ms"], 100 * s["busy_fraction"], {k: round(v, 3) for k, v in s["busy_ms_per_kind"].items()}),
            "trace: measured critical path %.3f ms over %d tasks (%.1f %% of the makespan)"
            % (cp_ns / 1e6, len(path), 100 * cp_ns / 1e6 / s["makespan_ms"]),
            "model: T = %.0f units, cp = %d units, P = %d, bound %s; gamma_seq %.2f GFLOP/s per CTA, "
            "gamma_pred %.1f GFLOP/s, predicted %.3f ms (%.1f GFLOP/s in LAPACK flops)"
            % (model["units"], info["critical_path"], n_sm, model["bound"], model["gamma_seq_gflops"],
               model["gamma_pred_gflops"], model["predicted_ms"], model["predicted_lapack_gflops"])]
