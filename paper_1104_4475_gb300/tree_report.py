"""The Section 4 comparisons for a measured tree sweep.

    python bench.py --workload trees --steps 1 --warmup 3 > trees.jsonl
    python -m paper_1104_4475_gb300.tree_report trees.jsonl

Reads the JSON line of `bench.py --workload trees` (per tree and q: time,
GFLOP/s, unit-weight critical path) and prints, per (tree, q):

* the predicted rate of the paper's model, gamma_pred = gamma_seq * T /
  max(T/P, cp), with T = 6pq^2 - 2q^3 units of nb^3/3 flops (every list's
  total weight, Section 2.2), P CTAs (one per SM) and gamma_seq one SM's FP64
  peak; and the measured rate as a fraction of it.  The model runs every tile
  kernel on one processor.  The executor splits each update into nb/W column
  strips on different SMs, which shortens the critical path below cp units, so
  the measured rate can exceed gamma_pred where the critical path binds;
* the overhead with respect to Greedy (Greedy = 1) in critical-path length and
  in time, as the paper's overhead figures show them;
* with `bench.py --workload trees --trace-cp`, the measured critical path (the
  longest path through the executed graph, traced task durations) against the
  traced makespan.

For m and n multiples of nb, T * nb^3/3 equals the LAPACK count 2n^2(m - n/3),
so gamma_pred and the measured GFLOP/s count the same flops.
"""

import argparse
import json
import sys


def sweep_report(line, m, nb, n_sm, peak_gflops):
    """{tree: {q: row}} from the trees bench line; row holds gflops, ms, cp,
    T, bound ("cp" or "work"), gamma_pred, frac_of_pred, cp_over_greedy and
    time_over_greedy (None where Greedy has no entry for that q)."""
    p = m // nb
    gamma_seq = peak_gflops / n_sm
    per = line["per_tree"]
    greedy = per.get("Greedy", {})
    out = {}
    for tree, by_q in per.items():
        rows = {}
        for qs, r in by_q.items():
            q = int(qs)
            T = 6 * p * q * q - 2 * q ** 3
            cp = r["critical_path_units"]
            bound = max(T / n_sm, cp)
            pred = gamma_seq * T / bound
            g = greedy.get(qs)
            rows[q] = {"BS": r.get("BS"), "gflops": r["gflops"], "ms": r["ms"], "cp": cp, "T": T,
                       "bound": "cp" if cp > T / n_sm else "work", "gamma_pred": pred,
                       "frac_of_pred": r["gflops"] / pred,
                       "cp_over_greedy": cp / g["critical_path_units"] if g else None,
                       "time_over_greedy": r["ms"] / g["ms"] if g else None,
                       "measured_cp_ms": r.get("measured_cp_ms"), "traced_makespan_ms": r.get("traced_makespan_ms")}
        out[tree] = dict(sorted(rows.items()))
    return out


def markdown(rep, n_sm=152):
    """Markdown tables: measured / predicted rate, overhead vs Greedy, and (when
    traced) measured critical path vs traced makespan."""
    qs = sorted({q for rows in rep.values() for q in rows})
    head = "| tree | " + " | ".join("q=%d" % q for q in qs) + " |"
    sep = "|---" * (len(qs) + 1) + "|"
    a = ["Measured GFLOP/s / model gamma_pred GFLOP/s (fraction):", "", head, sep]
    for tree, rows in rep.items():
        a.append("| %s | " % tree + " | ".join(
            "%.0f / %.0f (%.2f)" % (rows[q]["gflops"], rows[q]["gamma_pred"], rows[q]["frac_of_pred"])
            if q in rows else "" for q in qs) + " |")
    b = ["", "Overhead with respect to Greedy (Greedy = 1): critical path / time:", "", head, sep]
    for tree, rows in rep.items():
        b.append("| %s | " % tree + " | ".join(
            "%.2f / %.2f" % (rows[q]["cp_over_greedy"], rows[q]["time_over_greedy"])
            if q in rows and rows[q]["cp_over_greedy"] is not None else "" for q in qs) + " |")
    d = ["", "Unit-weight critical path (units of nb^3/3; PlasmaTree BS after the slash) and the work "
         "bound T/P:", "", head, sep]
    for tree, rows in rep.items():
        d.append("| %s | " % tree + " | ".join(
            ("%d/%d" % (rows[q]["cp"], rows[q]["BS"]) if rows[q].get("BS", 1) not in (None, 1) or "Plasma" in tree
             else "%d" % rows[q]["cp"]) + (" (cp)" if rows[q]["bound"] == "cp" else "")
            if q in rows else "" for q in qs) + " |")
    any_rows = next(iter(rep.values()))
    d.append("| T/P | " + " | ".join("%.0f" % (any_rows[q]["T"] / n_sm) if q in any_rows else "" for q in qs) + " |")
    c = []
    if any(r["measured_cp_ms"] is not None for rows in rep.values() for r in rows.values()):
        c = ["", "Measured critical path / traced makespan, ms (bench --trace-cp):", "", head, sep]
        for tree, rows in rep.items():
            c.append("| %s | " % tree + " | ".join(
                "%.1f / %.1f" % (rows[q]["measured_cp_ms"], rows[q]["traced_makespan_ms"])
                if q in rows and rows[q]["measured_cp_ms"] is not None else "" for q in qs) + " |")
    return "\n".join(a + d + b + c)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("path", help="output of bench.py --workload trees (its last JSON line is read)")
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--sms", type=int, default=152)
    ap.add_argument("--peak", type=float, default=None,
                    help="FP64 GFLOP/s of the whole GPU (default: the DFMA peak the bench line measured)")
    a = ap.parse_args(argv)
    with open(a.path) as fh:
        lines = [ln for ln in fh.read().splitlines() if ln.strip().startswith("{")]
    line = json.loads(lines[-1])
    peak = a.peak
    if peak is None:
        peak = 1e3 * line["measured_peaks"]["dfma_tflops"] if "measured_peaks" in line else 152 * 4 * 2.07
    print(markdown(sweep_report(line, a.m, a.nb, a.sms, peak), a.sms))
    return 0


if __name__ == "__main__":
    sys.exit(main())
