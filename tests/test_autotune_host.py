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


def _valid(cfg, m, n):
    nb, ib, tree, BS = cfg
    p = -(-m // nb)
    return (8 <= nb <= 256 and nb % 4 == 0 and 1 <= ib <= 64 and nb % ib == 0
            and (tree != tqr.PLASMA or 1 <= BS <= p))


def test_lookup_always_returns_a_valid_configuration():
    """Shapes outside the tuned classes (n below the class's tile size, very
    small n, n above 256) still get a configuration the library accepts."""
    db = {"version": autotune.DB_VERSION, "classes": [
        {"n": 32, "m_lo": 512, "m_hi": 1024, "nb": 32, "ib": 8, "tree": tqr.GREEDY, "BS": 1},
        {"n": 128, "m_lo": 512, "m_hi": 1024, "nb": 256, "ib": 8, "tree": tqr.FLAT_TS, "BS": 1},
        {"n": 64, "m_lo": 512, "m_hi": 1024, "nb": 64, "ib": 32, "tree": tqr.PLASMA, "BS": 16}]}
    assert autotune.lookup(db, 700, 30) == (16, 8, tqr.GREEDY, 1)      # nb 32 > n: largest tile <= 30
    assert autotune.lookup(db, 700, 10) == (64, 8, tqr.FLAT_TS, 1)     # no square tile fits: one column
    assert autotune.lookup(db, 700, 300) == (256, 8, tqr.FLAT_TS, 1)
    for m in (40, 513, 5000, 20000):
        for n in (1, 7, 16, 30, 33, 50, 64, 100, 128, 200, 300):
            if n <= m:
                assert _valid(autotune.lookup(db, m, n), m, n), (m, n)
