"""Host logic of the batched autotuner: candidate sets, database round trip
and lookup (no GPU)."""

import pytest

from paper_1104_4475_gb300 import autotune, tqr


def test_candidates_cover_square_tiles_and_one_column():
    c = autotune.candidates(64, 512)
    assert all(nb <= 64 or (tree == tqr.FLAT_TS and nb >= 64) for (nb, ib, tree, BS) in c)
    one = [x for x in c if x[2] == tqr.FLAT_TS and x[0] >= 64]
    assert sorted({x[0] for x in one}) == [64, 128, 256]
    assert len(set(c)) == len(c)
    for nb, ib, tree, BS in c:
        assert nb % ib == 0 and BS >= 1
        if tree == tqr.PLASMA:
            assert BS <= -(-512 // nb)
    assert [x[0] for x in autotune.candidates_f32(128)] == [128, 256]
    assert [x[0] for x in autotune.candidates_f32(32)] == [64, 128, 256]


def test_database_roundtrip_and_lookup(tmp_path):
    db = {"version": autotune.DB_VERSION, "gpu": "x", "sample": 4, "dtype": "f64", "classes": [
        {"n": 32, "m_lo": 512, "m_hi": 1024, "nb": 256, "ib": 8, "tree": tqr.FLAT_TS, "BS": 1},
        {"n": 64, "m_lo": 512, "m_hi": 1024, "nb": 32, "ib": 8, "tree": tqr.PLASMA, "BS": 16},
        {"n": 128, "m_lo": 1024, "m_hi": 2048, "nb": 64, "ib": 16, "tree": tqr.GREEDY, "BS": 1}]}
    p = tmp_path / "db.json"
    autotune.save(db, str(p))
    assert autotune.load(str(p)) == db
    assert autotune.lookup(db, 700, 32) == (256, 8, tqr.FLAT_TS, 1)
    assert autotune.lookup(db, 600, 64) == (32, 8, tqr.PLASMA, 16)      # 16 <= p = 19
    assert autotune.lookup(db, 100, 64)[3] == 4                          # BS capped at p = ceil(100/32)
    assert autotune.lookup(db, 1500, 128) == (64, 16, tqr.GREEDY, 1)
    bad = dict(db, version=0)
    autotune.save(bad, str(p))
    with pytest.raises(ValueError):
        autotune.load(str(p))
