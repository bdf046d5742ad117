"""Learned cost model: predicts the makespan of a factorization from
(m, n, nb, ib, tree, BS, precision) so that a configuration can be chosen
without timing every candidate.

* Network: the library's 3-layer perceptron (in -> 64 -> 64 -> 1, ReLU, FP32),
  trained on the GPU by the CUDA kernels behind tqr_mlp_loss_grad /
  tqr_mlp_adam_step on log(seconds).
* Features: log sizes, tile counts, ib/nb, one-hot tree, BS relative to p,
  one-hot precision, plus the LAPACK flop count and the unit-weight critical
  path from the host simulator (tqr_critical_path), both in log scale.
* Data: wall times of the executor itself (CUDA events around tqr_factor_ex),
  collected by :func:`collect`.

* Candidates: 22 FP64 configurations (nb 128/256, ib 16/32, the Greedy,
  Fibonacci, binary, flat TS/TT, PlasmaTree and PlasmaTree-TS trees with BS
  2..32) and 8 split-TF32 ones; shapes up to 65536 x 8192 and 2e11 flops.

Command line (the stored GB300 sets: 100 training shapes of seed 11, 200
held-out shapes of seed 23 outside them):
  python -m paper_1104_4475_gb300.costmodel collect --shapes 100 --seed 11 --out timings.csv
  python -m paper_1104_4475_gb300.costmodel collect --shapes 200 --seed 23 --exclude-seed 11 --out heldout.csv
  python -m paper_1104_4475_gb300.costmodel evaluate --data timings.csv --heldout heldout.csv
"""

import argparse
import csv
import json
import math
import sys
import time

import numpy as np

from . import tqr

TREE_IDS = list(range(10))                   # every generator of the library, PlasmaTree-TS included
BS_TREES = (tqr.PLASMA, tqr.GRASAP, tqr.PLASMA_TS)
# (nb, ib, tree, BS) of the FP64 candidates; BS is clipped to p.  ib takes both
# values the low-precision path allows, BS spans a domain of 2 to 32 tiles.
FP64_CONFIGS = ([(nb, ib, tree, 1) for nb in (128, 256) for ib in (16, 32)
                 for tree in (tqr.GREEDY, tqr.FLAT_TS, tqr.FIBONACCI)]
                + [(nb, 32, tree, 1) for nb in (128, 256) for tree in (tqr.BINARY, tqr.FLAT_TT)]
                + [(256, 32, tqr.PLASMA, BS) for BS in (2, 8, 32)]
                + [(256, 32, tqr.PLASMA_TS, BS) for BS in (8, 32)] + [(128, 32, tqr.PLASMA_TS, 32)])
LP_CONFIGS = ([(256, ib, tree, 1) for ib in (16, 32) for tree in (tqr.GREEDY, tqr.FLAT_TS)]
              + [(256, 32, tree, 1) for tree in (tqr.FIBONACCI, tqr.BINARY)]
              + [(256, 32, tqr.PLASMA_TS, 32), (128, 32, tqr.GREEDY, 1)])
DEFAULT = (256, 32, tqr.GREEDY, 1, 0)        # the configuration used without a model
FEATURES = 23
VERSION = 2


def features(m, n, nb, ib, tree, BS, prec):
    if tree not in TREE_IDS:
        raise ValueError("tree %d is outside the cost model's one-hot trees %s" % (tree, TREE_IDS))
    if prec not in (0, 1, 2):
        raise ValueError("precision %d is not 0, 1 or 2" % prec)
    p, q = -(-m // nb), -(-n // nb)
    cp = tqr.tqr_critical_path(p, q, tree, BS)
    flops = 2.0 * n * n * (m - n / 3.0)
    f = [math.log2(m) / 16, math.log2(n) / 16, math.log2(nb) / 8, ib / nb, math.log2(p) / 9, math.log2(q) / 9]
    f += [1.0 if tree == t else 0.0 for t in TREE_IDS]
    f += [BS / p if tree in BS_TREES else 0.0]
    f += [1.0 if prec == k else 0.0 for k in range(3)]
    f += [math.log2(flops) / 48, math.log2(cp * nb ** 3 / 3.0) / 48, math.log2(cp) / 12]
    assert len(f) == FEATURES
    return np.array(f, dtype=np.float32)


def configs_for(m, with_lp=True):
    """Every candidate (nb, ib, tree, BS, precision) for m rows: 22 FP64 and
    8 split-TF32 configurations."""
    out = []
    for prec, grid in ((0, FP64_CONFIGS), (1, LP_CONFIGS if with_lp else [])):
        for nb, ib, tree, BS in grid:
            out.append((nb, ib, tree, min(BS, -(-m // nb)), prec))
    return out


def random_shapes(count, seed, m_range=(4096, 65536), n_range=(256, 8192), max_flops=2e11, exclude=()):
    """Log-uniform shapes with n <= m, at most max_flops LAPACK flops, none of
    them in exclude (the training shapes, when drawing held-out ones)."""
    rng = np.random.default_rng(seed)
    out = []
    exclude = set(exclude)
    while len(out) < count:
        m = int(2 ** rng.uniform(math.log2(m_range[0]), math.log2(m_range[1])))
        n = int(2 ** rng.uniform(math.log2(n_range[0]), math.log2(min(n_range[1], m))))
        m, n = m // 64 * 64, max(256, n // 64 * 64)
        if n <= m and 2.0 * n * n * (m - n / 3.0) <= max_flops and (m, n) not in exclude:
            out.append((m, n))
    return out


def collect(shapes, with_lp=True, log=None, seed=1, out=None, max_seconds=None):
    """Time every candidate configuration on each shape with CUDA events
    around tqr_factor_ex (the second of two runs, so the cached plan is
    reused as in steady use); returns a list of records.  With max_seconds,
    stops after the first shape that ends past that much wall time."""
    import torch
    from . import build
    build.build()
    recs = []
    t0 = time.time()
    g = torch.Generator(device="cuda").manual_seed(seed)
    for si, (m, n) in enumerate(shapes):
        src = (torch.rand(n, m, generator=g, dtype=torch.float64, device="cuda") - 0.5).t()
        work = torch.empty_like(src.t()).t()
        for cfg in configs_for(m, with_lp):
            nb, ib, tree, BS, prec = cfg
            for rep in range(2):
                work.copy_(src)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                f = tqr.tqr_factor_ex(work, nb, ib, tree, BS, prec)
                e1.record()
                tqr.tqr_sync(f)
                secs = e0.elapsed_time(e1) / 1e3
                f.free()
            recs.append({"shape": si, "m": m, "n": n, "nb": nb, "ib": ib, "tree": tree, "BS": BS, "prec": prec,
                         "seconds": secs})
        if log:
            log("shape %d/%d (%d x %d) done" % (si + 1, len(shapes), m, n))
        if out:
            save_records(recs, out)                    # after every shape: a cut-off run keeps its data
        del src, work
        if max_seconds is not None and time.time() - t0 > max_seconds:
            break
    return recs


def save_records(recs, path):
    with open(path, "w", newline="") as fh:
        w = csv.DictWriter(fh, fieldnames=["shape", "m", "n", "nb", "ib", "tree", "BS", "prec", "seconds"])
        w.writeheader()
        for r in recs:
            w.writerow(r)


def load_records(path):
    out = []
    with open(path) as fh:
        for r in csv.DictReader(fh):
            out.append({k: (float(v) if k == "seconds" else int(v)) for k, v in r.items()})
    return out


def design(recs):
    X = np.stack([features(r["m"], r["n"], r["nb"], r["ib"], r["tree"], r["BS"], r["prec"]) for r in recs])
    y = np.log(np.array([r["seconds"] for r in recs], dtype=np.float64)).astype(np.float32)
    return X, y


def init_params(d, seed=0):
    """He-style initialization, flat in the library's parameter order."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, d)) * np.sqrt(2.0 / d)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    W3 = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [0.0]]).astype(np.float32)


class Model:
    """Feature standardization + network parameters (a CUDA float32 tensor)."""

    def __init__(self, params, mu, sd, ymu):
        self.params, self.mu, self.sd, self.ymu = params, mu, sd, ymu

    def predict_log_seconds(self, X):
        import torch
        Xs = torch.from_numpy(((X - self.mu) / self.sd).astype(np.float32)).cuda()
        y = tqr.tqr_mlp_forward(self.params, Xs)
        return y.cpu().numpy().astype(np.float64) + self.ymu

    def to_json(self):
        return {"version": VERSION, "features": FEATURES, "params": self.params.cpu().numpy().tolist(),
                "mu": self.mu.tolist(), "sd": self.sd.tolist(), "ymu": self.ymu}

    @staticmethod
    def from_json(d):
        if d.get("version") != VERSION or d.get("features") != FEATURES:
            raise ValueError("model file version %r with %r features; this code reads version %d with %d"
                             % (d.get("version"), d.get("features"), VERSION, FEATURES))
        import torch
        return Model(torch.tensor(d["params"], dtype=torch.float32, device="cuda"), np.array(d["mu"], np.float32),
                     np.array(d["sd"], np.float32), float(d["ymu"]))


def train(X, y, steps=3000, lr=3e-3, seed=0, log_every=0, log=None):
    """Full-batch Adam on the GPU with the library's kernels; returns (Model, losses)."""
    import torch
    mu = X.mean(axis=0)
    sd = X.std(axis=0) + 1e-3
    ymu = float(y.mean())
    Xs = torch.from_numpy(((X - mu) / sd).astype(np.float32)).cuda()
    ts = torch.from_numpy((y - ymu).astype(np.float32)).cuda()
    params = torch.from_numpy(init_params(X.shape[1], seed)).cuda()
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(Xs.shape[0] * (4 * 64 + 2), dtype=torch.float32, device="cuda")
    losses = []
    for step in range(1, steps + 1):
        tqr.tqr_mlp_loss_grad(params, Xs, ts, grad, loss, work)
        tqr.tqr_mlp_adam_step(params, grad, m, v, lr, step)
        if step % 100 == 0 or step == 1:
            losses.append((step, float(loss.item())))
            if log and log_every and step % log_every == 0:
                log("step %d loss %.4f" % (step, losses[-1][1]))
    return Model(params, mu, sd, ymu), losses


def pick(model, m, n, precisions=(0,)):
    """The candidate (nb, ib, tree, BS, precision) with the smallest predicted
    makespan for an m x n factorization (no timing); exhaustive timing
    (:func:`collect`) stays the fallback and decides whether this choice was right."""
    cands = [c for c in configs_for(m, with_lp=True) if c[4] in precisions]
    X = np.stack([features(m, n, *c) for c in cands])
    return cands[int(np.argmin(model.predict_log_seconds(X)))]


def by_shape(recs):
    out = {}
    for r in recs:
        out.setdefault(r["shape"], []).append(r)
    return out


def evaluate(model, recs, prec=0):
    """For each shape: measured time of the model's pick among the timed
    candidates of that precision, of the exhaustive best, of the fixed default
    and of the smallest-critical-path pick."""
    rows = []
    for sid, rs in by_shape(recs).items():
        rs = [r for r in rs if r["prec"] == prec]
        if not rs:
            continue
        X, _ = design(rs)
        pred = model.predict_log_seconds(X)
        t = np.array([r["seconds"] for r in rs])
        best = t.min()
        pick = t[int(np.argmin(pred))]
        dflt = [r["seconds"] for r in rs if (r["nb"], r["ib"], r["tree"]) == DEFAULT[:3]]
        cps = [tqr.tqr_critical_path(-(-r["m"] // r["nb"]), -(-r["n"] // r["nb"]), r["tree"], r["BS"])
               * r["nb"] ** 3 for r in rs]
        rows.append({"shape": sid, "m": rs[0]["m"], "n": rs[0]["n"], "best": best, "model": pick / best,
                     "default": (dflt[0] / best) if dflt else float("nan"),
                     "min_cp": t[int(np.argmin(cps))] / best, "exact": bool(pick == best)})
    return rows


def disjoint(train, test):
    """The test records whose (m, n) does not occur in the training records."""
    seen = {(r["m"], r["n"]) for r in train}
    return [r for r in test if (r["m"], r["n"]) not in seen]


def split(recs, holdout_frac=0.25, seed=0):
    shapes = sorted(by_shape(recs))
    rng = np.random.default_rng(seed)
    rng.shuffle(shapes)
    k = max(1, int(round(len(shapes) * holdout_frac)))
    test = set(shapes[:k])
    return [r for r in recs if r["shape"] not in test], [r for r in recs if r["shape"] in test]


def summarize(rows):
    a = lambda key: float(np.mean([r[key] for r in rows]))
    return {"shapes": len(rows), "model_over_best": a("model"), "default_over_best": a("default"),
            "min_cp_over_best": a("min_cp"), "model_exact_fraction": float(np.mean([r["exact"] for r in rows])),
            "model_worst": float(max(r["model"] for r in rows))}


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--shapes", type=int, default=120)
    c.add_argument("--seed", type=int, default=11)
    c.add_argument("--out", required=True)
    c.add_argument("--exclude-seed", type=int, default=None,
                   help="draw shapes outside those of this seed (and --exclude-count): held-out shapes")
    c.add_argument("--exclude-count", type=int, default=100)
    c.add_argument("--max-seconds", type=float, default=None)
    e = sub.add_parser("evaluate")
    e.add_argument("--data", required=True)
    e.add_argument("--heldout", default=None, help="separate held-out timings (train on all of --data)")
    e.add_argument("--steps", type=int, default=3000)
    e.add_argument("--model-out", default=None)
    a = ap.parse_args(argv)
    if a.cmd == "collect":
        t0 = time.time()
        skip = random_shapes(a.exclude_count, a.exclude_seed) if a.exclude_seed is not None else ()
        recs = collect(random_shapes(a.shapes, a.seed, exclude=skip),
                       log=lambda s: print(s, file=sys.stderr, flush=True), out=a.out, max_seconds=a.max_seconds)
        print(json.dumps({"records": len(recs), "seconds": time.time() - t0}))
    else:
        recs = load_records(a.data)
        tr, te = (recs, disjoint(recs, load_records(a.heldout))) if a.heldout else split(recs)
        X, y = design(tr)
        model, losses = train(X, y, steps=a.steps)
        Xt, yt = design(te)
        rmse = float(np.sqrt(np.mean((model.predict_log_seconds(Xt) - yt) ** 2)))
        out = {"train_records": len(tr), "test_records": len(te), "final_train_loss": losses[-1][1],
               "test_rmse_log_seconds": rmse, "fp64": summarize(evaluate(model, te, 0))}
        if any(r["prec"] == 1 for r in te):
            out["split_tf32"] = summarize(evaluate(model, te, 1))
        if a.model_out:
            with open(a.model_out, "w") as fh:
                json.dump(model.to_json(), fh)
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
