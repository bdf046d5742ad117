"""Host logic of the learned cost model: features, candidates, shapes, data
split and the stored timing set (no GPU)."""

import os

import numpy as np
import pytest

from paper_1104_4475_gb300 import costmodel, tqr

DATA = os.path.join(os.path.dirname(costmodel.__file__), "data", "costmodel_timings_gb300.csv")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1104_4475_gb300 import build
    build.build()


def test_features_shape_and_encoding():
    f = costmodel.features(16384, 2048, 256, 32, tqr.PLASMA, 8, 1)
    assert f.shape == (costmodel.FEATURES,) and f.dtype == np.float32
    assert costmodel.FEATURES <= 32                   # the network's input limit
    trees = f[6:16]
    assert trees.sum() == 1 and trees[tqr.PLASMA] == 1
    assert f[16] == pytest.approx(8 / 64)             # BS / p
    assert list(f[17:20]) == [0, 1, 0]                # precision one-hot
    # the critical-path feature comes from the library's simulator
    cp = tqr.tqr_critical_path(64, 8, tqr.PLASMA, 8)
    assert f[22] == pytest.approx(np.log2(cp) / 12)
    # PlasmaTree-TS has its own tree slot and its BS feature
    g = costmodel.features(16384, 2048, 256, 32, tqr.PLASMA_TS, 32, 0)
    assert g[6 + tqr.PLASMA_TS] == 1 and g[16] == pytest.approx(32 / 64)
    assert costmodel.features(16384, 2048, 256, 32, tqr.GREEDY, 1, 0)[16] == 0


def test_candidates_span_ib_bs_and_trees():
    c = costmodel.configs_for(20000)
    assert len(c) == 30 and len(set(c)) == 30
    assert costmodel.DEFAULT in c
    fp64 = [x for x in c if x[4] == 0]
    lp = [x for x in c if x[4] == 1]
    assert len(fp64) == 22 and len(lp) == 8
    for prec in (0, 1):
        assert {x[1] for x in c if x[4] == prec} == {16, 32}          # ib
        assert {x[2] for x in c if x[4] == prec} >= {tqr.GREEDY, tqr.FLAT_TS, tqr.FIBONACCI, tqr.BINARY,
                                                     tqr.PLASMA_TS}
    assert {x[3] for x in fp64 if x[2] == tqr.PLASMA} == {2, 8, 32}
    assert {x[3] for x in fp64 if x[2] == tqr.PLASMA_TS} == {8, 32}
    assert all(x[3] == 1 for x in c if x[2] not in costmodel.BS_TREES)
    assert all(x[0] >= 64 and x[1] in (16, 32) for x in lp)           # the low-precision path's layouts
    # BS never exceeds p
    small = costmodel.configs_for(4096)
    assert all(x[3] <= -(-4096 // x[0]) for x in small)
    shapes = costmodel.random_shapes(50, 3)
    assert shapes == costmodel.random_shapes(50, 3)
    for m, n in shapes:
        assert 4096 <= m <= 65536 and 256 <= n <= m and m % 64 == 0 and n % 64 == 0
        assert 2.0 * n * n * (m - n / 3.0) <= 2e11
    held = costmodel.random_shapes(200, 23, exclude=costmodel.random_shapes(100, 11))
    assert len(held) == 200 and not set(held) & set(costmodel.random_shapes(100, 11))


def test_stored_timings_and_split():
    recs = costmodel.load_records(DATA)
    shapes = costmodel.by_shape(recs)
    assert len(recs) == 3000 and len(shapes) == 100
    assert [(rs[0]["m"], rs[0]["n"]) for _, rs in sorted(shapes.items())] == costmodel.random_shapes(100, 11)
    for sid, rs in shapes.items():
        assert sorted((r["nb"], r["ib"], r["tree"], r["BS"], r["prec"]) for r in rs) == \
            sorted(costmodel.configs_for(rs[0]["m"]))
        assert all(r["seconds"] > 0 for r in rs)
    tr, te = costmodel.split(recs)
    assert len(tr) + len(te) == len(recs)
    assert not {r["shape"] for r in tr} & {r["shape"] for r in te}
    assert costmodel.split(recs)[1] == te               # deterministic


def test_stored_heldout_timings():
    recs = costmodel.load_records(DATA.replace("costmodel_timings_gb300", "costmodel_heldout_gb300"))
    shapes = costmodel.by_shape(recs)
    assert len(recs) == 6000 and len(shapes) == 200
    train = {(r["m"], r["n"]) for r in costmodel.load_records(DATA)}
    held = {(r["m"], r["n"]) for r in recs}
    assert not held & train                              # drawn outside the training shapes
    assert len(costmodel.by_shape(costmodel.disjoint(costmodel.load_records(DATA), recs))) == 200
    for rs in shapes.values():
        assert len(rs) == 30 and all(r["seconds"] > 0 for r in rs)


def test_records_roundtrip(tmp_path):
    recs = [{"shape": 0, "m": 4096, "n": 256, "nb": 128, "ib": 32, "tree": 5, "BS": 1, "prec": 0,
             "seconds": 0.0125}]
    p = tmp_path / "t.csv"
    costmodel.save_records(recs, str(p))
    assert costmodel.load_records(str(p)) == recs


def test_features_refuse_trees_and_precisions_outside_the_model():
    """A tree id beyond the library's generators has no one-hot slot; asking
    for it is an error, not an all-zero tree encoding."""
    from paper_1104_4475_gb300 import costmodel, tqr
    with pytest.raises(ValueError):
        costmodel.features(16384, 2048, 256, 32, 10, 16, 0)
    with pytest.raises(ValueError):
        costmodel.features(16384, 2048, 256, 32, tqr.GREEDY, 1, 3)
    assert costmodel.features(16384, 2048, 256, 32, tqr.GREEDY, 1, 0).shape == (costmodel.FEATURES,)


def test_model_file_of_another_feature_set_is_refused():
    from paper_1104_4475_gb300 import costmodel
    with pytest.raises(ValueError):
        costmodel.Model.from_json({"version": costmodel.VERSION, "features": costmodel.FEATURES + 1,
                                   "params": [], "mu": [], "sd": [], "ymu": 0.0})
    with pytest.raises(ValueError):
        costmodel.Model.from_json({"version": 1, "features": costmodel.FEATURES, "params": [],
                                   "mu": [], "sd": [], "ymu": 0.0})
