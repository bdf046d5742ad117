"""Per-task device traces of the executor (tqr_set_trace / tqr_get_trace):
Chrome-trace export and summaries.

A trace row is (kind, i, piv, k, j * 65536 + strip, start ns, end ns, SM),
0-based tile indices, one row per device task.
"""

import json

import numpy as np

KIND_NAMES = ("GEQRT", "UNMQR", "TTQRT", "TTMQR", "TSQRT", "TSMQR")


def to_chrome(trace, path=None):
    """Chrome trace-event JSON (one track per SM); written to path if given."""
    t0 = int(trace[:, 5].min()) if len(trace) else 0
    ev = []
    for kind, i, piv, k, js, s, e, sm in trace.tolist():
        j, strip = (js >> 16, js & 0xffff) if js >= 0 else (-1, 0)
        name = "%s(%d,%d,%d%s)" % (KIND_NAMES[kind], i, piv, k, "" if j < 0 else ",%d/%d" % (j, strip))
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
        if kind in (0, 2, 4):
            end[(kind, i, piv if kind else -1, k)] = e
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
