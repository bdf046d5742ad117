"""Host-side trace analysis (no GPU): the measured critical path against an
independent longest-path computation, the per-task work accounting against
the total weight of an elimination list (Section 2.2), and the Section 4
performance model on traces whose rates are known by construction."""

import numpy as np
import pytest

import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import trace as ttrace

nx = pytest.importorskip("networkx")


def _random_dag_trace(n, p_edge, seed):
    rng = np.random.default_rng(seed)
    start = rng.integers(1, 1000, n)
    dur = rng.integers(0, 500, n)
    tr = np.zeros((n, 8), dtype=np.int64)
    tr[:, 5] = start
    tr[:, 6] = start + dur
    edges = [(u, v) for v in range(n) for u in range(v) if rng.random() < p_edge]
    return tr, np.array(edges, dtype=np.int64).reshape(-1, 2), dur


@pytest.mark.parametrize("n,p_edge,seed", [(1, 0.0, 0), (12, 0.3, 1), (60, 0.08, 2), (200, 0.02, 3)])
def test_measured_critical_path_matches_networkx(n, p_edge, seed):
    tr, edges, dur = _random_dag_trace(n, p_edge, seed)
    length, path = ttrace.measured_critical_path(tr, edges)
    G = nx.DiGraph()
    G.add_node("src")
    for v in range(n):
        G.add_edge("src", v, w=int(dur[v]))
    for u, v in edges.tolist():
        G.add_edge(u, v, w=int(dur[v]))
    assert length == nx.dag_longest_path_length(G, weight="w")
    assert sum(int(dur[v]) for v in path) == length             # the path carries the length
    es = set(map(tuple, edges.tolist()))
    assert all((a, b) in es for a, b in zip(path, path[1:]))     # and is a path of the graph


def test_measured_critical_path_rejects_backward_edges():
    tr, _, _ = _random_dag_trace(3, 0.0, 4)
    with pytest.raises(ValueError):
        ttrace.measured_critical_path(tr, np.array([[2, 1]]))


def _tile_trace(p, q, tree, nb, strip, n, BS=1):
    """Trace rows (zero durations) of the device tasks of a factorization:
    the tile tasks of the library's host planner with each update split into
    strips of `strip` columns, as the executor splits them."""
    tasks, _ = tqr.tqr_tasks(p, q, tree, BS)
    last_cols = n - (q - 1) * nb
    rows = []
    for kind, i, piv, k, j in tasks.tolist():
        if kind in (1, 3, 5):
            cols = last_cols if j == q - 1 else nb
            for s in range(-(-cols // strip)):
                rows.append((kind, i, piv, k, j * 65536 + s, 0, 0, 0))
        else:
            rows.append((kind, i, piv, k, -1, 0, 0, 0))
    return np.array(rows, dtype=np.int64)


@pytest.mark.parametrize("p,q,tree", [(6, 3, tqr.GREEDY), (8, 8, tqr.FLAT_TT), (7, 4, tqr.FLAT_TS),
                                      (9, 5, tqr.PLASMA_TS)])
@pytest.mark.parametrize("strip", [64, 16])
def test_task_units_sum_to_the_lists_total_weight(p, q, tree, strip):
    """Any elimination list of a p x q tile matrix does 6pq^2 - 2q^3 units
    of work with TT kernels (Section 2.2); TS kernels do the same work per
    zeroed tile (GEQRT + UNMQRs + TTQRT + TTMQRs = 6 + 12 per column to the
    right = TSQRT + TSMQRs), so every tree and kernel family sums to it, for
    any strip width."""
    nb = 64
    tr = _tile_trace(p, q, tree, nb, strip, q * nb, BS=3)
    units = ttrace.task_units(tr, nb, strip, q * nb)
    assert units.sum() == pytest.approx(6 * p * q * q - 2 * q ** 3)


def test_task_units_of_a_ragged_last_column():
    """n = 2 nb + 20 with strips of 16 columns: the last tile column's
    updates cover 16 and 4 of its 20 columns."""
    nb, strip, n = 64, 16, 148
    tr = np.array([(1, 0, -1, 0, 2 * 65536 + 0, 0, 0, 0),     # UNMQR into the last tile column, strip 0
                   (1, 0, -1, 0, 2 * 65536 + 1, 0, 0, 0),     # its strip 1: 4 columns
                   (5, 1, 0, 0, 1 * 65536 + 3, 0, 0, 0),      # TSMQR into a full column
                   (2, 1, 0, 0, -1, 0, 0, 0)], dtype=np.int64)
    got = ttrace.task_units(tr, nb, strip, n)
    assert got.tolist() == pytest.approx([6 * 16 / 64, 6 * 4 / 64, 12 * 16 / 64, 2.0])


def test_model_prediction_on_a_trace_of_known_rate():
    """Every task lasts c ns per unit, so one CTA runs nb^3/3 flops per c ns;
    the model then predicts max(T/P, cp) * c ns."""
    p, q, nb, strip, c = 8, 4, 64, 16, 1000
    n = q * nb
    tr = _tile_trace(p, q, tqr.GREEDY, nb, strip, n)
    units = ttrace.task_units(tr, nb, strip, n)
    tr[:, 5] = np.arange(len(tr)) * 10 ** 6
    tr[:, 6] = tr[:, 5] + np.round(units * c).astype(np.int64)
    T = 6 * p * q * q - 2 * q ** 3
    cp = tqr.tqr_critical_path(p, q, tqr.GREEDY)
    flops = 2.0 * n * n * (p * nb - n / 3.0)
    unit_flops = nb ** 3 / 3.0
    for P, bound in ((2, "work"), (10 ** 4, "cp")):
        r = ttrace.model_prediction(tr, nb, strip, n, cp, P, flops)
        assert r["units"] == pytest.approx(T)
        assert r["gamma_seq_gflops"] == pytest.approx(unit_flops / c, rel=1e-6)
        assert r["bound"] == bound
        b = max(T / P, cp)
        assert r["predicted_ms"] == pytest.approx(b * c / 1e6, rel=1e-6)
        assert r["gamma_pred_gflops"] == pytest.approx(unit_flops / c * T / b, rel=1e-6)
        assert r["predicted_lapack_gflops"] == pytest.approx(flops / (b * c), rel=1e-6)


def test_trace_report_on_a_synthetic_trace():
    """The report that bench.py --workload case --trace prints, on a trace
    built from the host task list with a chain of edges (every task after
    the previous)."""
    p, q, nb, strip, c = 6, 3, 64, 32, 500
    n = q * nb
    tr = _tile_trace(p, q, tqr.GREEDY, nb, strip, n)
    units = ttrace.task_units(tr, nb, strip, n)
    dur = np.round(units * c).astype(np.int64)
    tr[:, 5] = np.concatenate([[1000], 1000 + np.cumsum(dur)[:-1]])
    tr[:, 6] = tr[:, 5] + dur
    edges = np.stack([np.arange(len(tr) - 1), np.arange(1, len(tr))], axis=1)
    info = {"nb": nb, "n": n, "strip": strip, "critical_path": tqr.tqr_critical_path(p, q, tqr.GREEDY),
            "flops": 2.0 * n * n * (p * nb - n / 3.0)}
    lines = ttrace.report(tr, edges, info, 4)
    assert len(lines) == 3
    assert "(100.0 % of the makespan)" in lines[1]               # a chain: the path is everything
    assert "T = %d units" % (6 * p * q * q - 2 * q ** 3) in lines[2]


def test_tree_report_on_a_synthetic_sweep_line():
    """gamma_pred = gamma_seq T / max(T/P, cp) with T = 6pq^2 - 2q^3, and the
    overheads against Greedy, on a bench line with made-up times."""
    from paper_1104_4475_gb300 import tree_report
    line = {"per_tree": {
        "Greedy": {"1": {"BS": 1, "ms": 10.0, "gflops": 50.0, "critical_path_units": 16},
                   "8": {"BS": 1, "ms": 100.0, "gflops": 800.0, "critical_path_units": 198}},
        "BinaryTree": {"1": {"BS": 1, "ms": 20.0, "gflops": 25.0, "critical_path_units": 16},
                       "8": {"BS": 1, "ms": 150.0, "gflops": 533.0, "critical_path_units": 338}}}}
    rep = tree_report.sweep_report(line, m=64 * 256, nb=256, n_sm=152, peak_gflops=152 * 8.0)
    g1 = rep["Greedy"][1]
    assert g1["T"] == 6 * 64 - 2 and g1["bound"] == "cp"           # 382 units, cp 16 > 382 / 152
    assert g1["gamma_pred"] == pytest.approx(8.0 * 382 / 16)
    assert g1["frac_of_pred"] == pytest.approx(50.0 / (8.0 * 382 / 16))
    b8 = rep["BinaryTree"][8]
    T8 = 6 * 64 * 64 - 2 * 512
    assert b8["T"] == T8 and b8["bound"] == "cp"
    assert b8["gamma_pred"] == pytest.approx(8.0 * T8 / 338)
    assert b8["cp_over_greedy"] == pytest.approx(338 / 198) and b8["time_over_greedy"] == pytest.approx(1.5)
    wide = tree_report.sweep_report(line, m=64 * 256, nb=256, n_sm=2, peak_gflops=2 * 8.0)
    assert wide["Greedy"][8]["bound"] == "work"                    # T / 2 > 198
    assert wide["Greedy"][8]["gamma_pred"] == pytest.approx(8.0 * 2)
    md = tree_report.markdown(rep)
    assert "| Greedy |" in md and "1.00 / 1.00" in md and "Measured critical path" not in md
    line["per_tree"]["Greedy"]["8"].update(measured_cp_ms=61.5, traced_makespan_ms=99.0)
    md = tree_report.markdown(tree_report.sweep_report(line, m=64 * 256, nb=256, n_sm=152, peak_gflops=1216.0))
    assert "Measured critical path" in md and "61.5 / 99.0" in md
