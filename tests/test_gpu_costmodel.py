"""Cost-model network on the GPU: forward pass, loss gradient and Adam step
of the library's kernels against the FP64 reference, and a training run."""

import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4475_gb300 import build, tqr as t
    build.build()
    return t


def case(B, d, seed):
    rng = np.random.default_rng(seed)
    theta = mlp.init(d, seed) + 0.02 * rng.standard_normal(mlp.param_count(d))
    X = rng.standard_normal((B, d))
    t = rng.standard_normal(B)
    return theta, X, t


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("B,d", [(1, 1), (97, 22), (1000, 22), (300, 32)])
def test_forward_matches_reference(tqr, B, d):
    theta, X, _ = case(B, d, B + d)
    th32 = np.float32(theta).astype(np.float64)
    X32 = np.float32(X).astype(np.float64)
    y = tqr.tqr_mlp_forward(dev(theta), dev(X)).cpu().numpy()
    ref = mlp.forward(th32, X32)
    scale = np.abs(ref).max() + 1.0
    assert np.abs(y - ref).max() <= 2e-5 * scale


@pytest.mark.parametrize("B,d", [(1, 3), (257, 22), (2000, 22)])
def test_loss_grad_matches_reference(tqr, B, d):
    theta, X, t = case(B, d, 7 * B + d)
    th32, X32, t32 = (np.float32(a).astype(np.float64) for a in (theta, X, t))
    lref, gref = mlp.loss_and_grad(th32, X32, t32)
    P = mlp.param_count(d)
    assert tqr.tqr_mlp_param_count(d) == P
    grad = torch.full((P,), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    tqr.tqr_mlp_loss_grad(dev(theta), dev(X), dev(t), grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(lref, rel=1e-5)
    assert np.all(np.isfinite(g))
    assert np.abs(g - gref).max() <= 1e-4 * (np.abs(gref).max() + 1e-30)


def test_loss_grad_deterministic(tqr):
    theta, X, t = case(500, 22, 3)
    P = mlp.param_count(22)
    outs = []
    for _ in range(2):
        grad = torch.zeros(P, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        tqr.tqr_mlp_loss_grad(dev(theta), dev(X), dev(t), grad, loss)
        outs.append((grad.cpu().numpy(), loss.item()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_adam_matches_reference(tqr):
    rng = np.random.default_rng(9)
    n = 5000
    theta, g = rng.standard_normal(n), rng.standard_normal(n)
    m, v = 0.1 * rng.standard_normal(n), np.abs(rng.standard_normal(n))
    tw, gw, mw, vw = dev(theta), dev(g), dev(m), dev(v)
    tqr.tqr_mlp_adam_step(tw, gw, mw, vw, 3e-3, 4)
    f = lambda a: np.float32(a).astype(np.float64)
    tr, mr, vr = mlp.adam_step(f(theta), f(g), f(m), f(v), 4, lr=3e-3)
    assert np.allclose(mw.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)
    assert np.allclose(vw.cpu().numpy(), vr, rtol=1e-5, atol=1e-7)
    assert np.abs(tw.cpu().numpy() - tr).max() <= 1e-6 * (np.abs(tr).max() + 1)


def test_invalid_arguments(tqr):
    with pytest.raises(tqr.TqrError):
        tqr.tqr_mlp_param_count(0)
    with pytest.raises(tqr.TqrError):
        tqr.tqr_mlp_param_count(33)
    theta = torch.zeros(mlp.param_count(40), dtype=torch.float32, device="cuda")
    with pytest.raises(tqr.TqrError):
        tqr.tqr_mlp_forward(theta, torch.zeros(4, 40, dtype=torch.float32, device="cuda"))


def test_training_fits_smooth_function(tqr):
    # A smooth target of 4 inputs: full-batch Adam through the library's
    # kernels must drive the loss well below its starting value, and the
    # trained network must agree with the FP64 reference forward pass.
    from paper_1104_4475_gb300 import costmodel
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (800, 4)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 3] ** 2).astype(np.float32)
    model, losses = costmodel.train(X, y, steps=1500, lr=3e-3)
    assert losses[-1][1] < 0.02 * losses[0][1]
    assert losses[-1][1] < 5e-3
    Xs = ((X - model.mu) / model.sd).astype(np.float32)
    ref = mlp.forward(model.params.cpu().numpy().astype(np.float64), Xs.astype(np.float64)) + model.ymu
    assert np.abs(model.predict_log_seconds(X) - ref).max() < 1e-4


def test_trained_model_gains_over_fixed_configuration(tqr):
    """Trained on executor timings of 100 shapes (GB300, 30 configurations
    each: nb, ib, tree, BS and precision all vary), the network's pick on 200
    other shapes (timed the same way) is within 2 % of the exhaustive best on
    average, and better than both the fixed default (Greedy, nb 256) and the
    smallest-critical-path rule, in FP64 and split-TF32."""
    import os
    from paper_1104_4475_gb300 import costmodel
    data = os.path.join(os.path.dirname(costmodel.__file__), "data")
    train = costmodel.load_records(os.path.join(data, "costmodel_timings_gb300.csv"))
    test = costmodel.disjoint(train, costmodel.load_records(os.path.join(data, "costmodel_heldout_gb300.csv")))
    assert len(costmodel.by_shape(test)) == 200
    X, y = costmodel.design(train)
    model, losses = costmodel.train(X, y, steps=3000)
    assert losses[-1][1] < 0.01 * losses[0][1]
    s = costmodel.summarize(costmodel.evaluate(model, test, 0))
    assert s["model_over_best"] <= 1.02
    assert s["model_over_best"] < s["default_over_best"]
    assert s["model_over_best"] <= s["min_cp_over_best"]
    assert s["model_worst"] <= 1.12
    lp = costmodel.summarize(costmodel.evaluate(model, test, 1))
    assert lp["shapes"] == 200 and lp["model_over_best"] <= 1.02
    assert lp["model_over_best"] < lp["default_over_best"] and lp["model_over_best"] <= lp["min_cp_over_best"]
    m, n = test[0]["m"], test[0]["n"]
    c = costmodel.pick(model, m, n)
    assert c in costmodel.configs_for(m) and c[4] == 0
    # the trained model saves and reloads (versioned JSON) with identical predictions
    import json
    again = costmodel.Model.from_json(json.loads(json.dumps(model.to_json())))
    Xt, _ = costmodel.design(test[:50])
    assert np.array_equal(again.predict_log_seconds(Xt), model.predict_log_seconds(Xt))
