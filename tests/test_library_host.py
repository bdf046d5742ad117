"""libtqr on the CPU: the library loads, exports every entry point of
include/tqr.h, and its host-only integer outputs (elimination lists,
validity verdicts, task lists, unit-weight schedules, critical paths,
zero-out tables) equal the oracle's bit for bit."""

import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import dag as odag
from oracle import trees as otrees
import paper_1104_4475_gb300 as tqr
from paper_1104_4475_gb300 import build as tbuild

KIND_MAP = {odag.GEQRT: tqr.GEQRT, odag.UNMQR: tqr.UNMQR, odag.TTQRT: tqr.TTQRT,
            odag.TTMQR: tqr.TTMQR, odag.TSQRT: tqr.TSQRT, odag.TSMQR: tqr.TSMQR}
TREES = [tqr.FLAT_TS, tqr.FLAT_TT, tqr.SAMEH_KUCK, tqr.BINARY, tqr.FIBONACCI, tqr.GREEDY]


@pytest.fixture(scope="module", autouse=True)
def built():
    tbuild.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "tqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tqr_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = header_functions()
    assert len(names) >= 14
    L = tqr.lib()
    for name in names:
        assert hasattr(L, name), name
    out = os.popen("nm -D --defined-only %s" % tbuild.LIB).read()
    for name in names:
        assert re.search(r"\bT %s$" % name, out, flags=re.M), name


def header_signatures():
    """{name: number of parameters} of every function declared in tqr.h."""
    src = open(os.path.join(ROOT, "include", "tqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(tqr_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_declares_every_function_with_its_parameter_count():
    """Each C entry point has ctypes argument types in the binding, as many
    as the header declares parameters (a missing or extra argument would be
    passed silently through ctypes)."""
    sigs = header_signatures()
    assert set(sigs) == set(header_functions())
    L = tqr.lib()
    for name, count in sigs.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == count, (name, len(fn.argtypes), count)


def test_library_is_built_for_sm103a():
    out = os.popen("cuobjdump --list-elf %s 2>/dev/null" % tbuild.LIB).read()
    if out:
        assert "sm_103a" in out


def lists_equal(p, q, tree, BS=1):
    got = tqr.tqr_elimination_list(p, q, tree, BS)
    want = np.array(otrees.elimination_list(p, q, tree, BS), dtype=np.int32).reshape(-1, 3) - 1
    return got.shape == want.shape and np.array_equal(got, want)


@pytest.mark.parametrize("tree", TREES)
def test_elimination_lists_match_oracle(tree):
    for p in range(1, 34):
        for q in range(1, p + 1):
            assert lists_equal(p, q, tree), (p, q)


@pytest.mark.parametrize("tree", [tqr.ASAP, tqr.GRASAP])
def test_dynamic_lists_match_oracle(tree):
    for p in range(1, 19):
        for q in range(1, p + 1):
            for k in (range(0, q + 1) if tree == tqr.GRASAP else [1]):
                got = tqr.tqr_elimination_list(p, q, tree, k)
                want = np.array(otrees.elimination_list(p, q, tree, k), dtype=np.int32).reshape(-1, 3) - 1
                assert np.array_equal(got, want), (p, q, k)


def test_asap_biggermat_library():
    """The library's ASAP on the whole biggermat table (p up to 128).  Reading:
    the 128 x 64 entry is printed 1748; this ASAP rule, which matches the other
    nine entries and Table table.15x2x3 (b), gives 1734."""
    from conftest import load_rows
    for p, q, g, a in load_rows("biggermat_cp.txt"):
        assert tqr.tqr_critical_path(p, q, tqr.GREEDY) == g
        if (p, q) == (128, 64):
            assert tqr.tqr_critical_path(p, q, tqr.ASAP) == 1734
        else:
            assert tqr.tqr_critical_path(p, q, tqr.ASAP) == a, (p, q)


def test_plasma_lists_match_oracle():
    for p in range(1, 26):
        for q in range(1, p + 1):
            for BS in range(1, p + 1):
                assert lists_equal(p, q, tqr.PLASMA, BS), (p, q, BS)


@pytest.mark.parametrize("p,q,tree,BS", [(16, 4, tqr.GREEDY, 1), (15, 6, tqr.FIBONACCI, 1), (40, 17, tqr.PLASMA, 7),
                                         (64, 64, tqr.GREEDY, 1), (64, 8, tqr.FLAT_TS, 1), (33, 20, tqr.BINARY, 1),
                                         (9, 9, tqr.FLAT_TT, 1), (1, 1, tqr.GREEDY, 1), (7, 1, tqr.FLAT_TS, 1),
                                         (15, 3, tqr.ASAP, 1), (21, 9, tqr.GRASAP, 3), (12, 12, tqr.GRASAP, 12),
                                         (40, 17, tqr.PLASMA_TS, 7), (16, 16, tqr.PLASMA_TS, 3),
                                         (9, 4, tqr.PLASMA_TS, 9), (13, 5, tqr.PLASMA_TS, 1)])
def test_tasks_schedule_and_cp_match_oracle(p, q, tree, BS):
    el = otrees.elimination_list(p, q, tree, BS)
    otasks = odag.expand(p, q, el, otrees.ts_flags(tree, BS, el))
    ofin, ocp = odag.simulate(otasks)
    tasks, fin = tqr.tqr_tasks(p, q, tree, BS)
    want = np.array([[KIND_MAP[k], i - 1, piv - 1 if piv else -1, kk - 1, j - 1 if j else -1]
                     for (k, i, piv, kk, j) in otasks], dtype=np.int32).reshape(-1, 5)
    assert np.array_equal(tasks, want)
    assert np.array_equal(fin, np.array(ofin, dtype=np.int64))
    cp, zt = tqr.tqr_critical_path(p, q, tree, BS, zero_time=True)
    assert cp == ocp
    ozt = odag.zero_times(otasks, ofin)
    for i in range(p):
        for k in range(q):
            assert zt[i, k] == ozt.get((i + 1, k + 1), -1)


def test_critical_paths_sweep_match_oracle():
    for p in (2, 5, 16, 40):
        for q in range(1, p + 1, 3):
            for tree in TREES:
                el = otrees.elimination_list(p, q, tree)
                assert tqr.tqr_critical_path(p, q, tree) == odag.critical_path(p, q, el, tree == tqr.FLAT_TS)


def test_plasma_ts_critical_paths_match_oracle():
    for p in range(1, 22):
        for q in range(1, p + 1, 2):
            for BS in range(1, p + 1, 3):
                el = otrees.elimination_list(p, q, tqr.PLASMA_TS, BS)
                want = odag.critical_path(p, q, el, otrees.ts_flags(tqr.PLASMA_TS, BS, el))
                assert tqr.tqr_critical_path(p, q, tqr.PLASMA_TS, BS) == want, (p, q, BS)
                assert lists_equal(p, q, tqr.PLASMA_TS, BS)


BENCH_QS = (1, 2, 4, 8, 16, 32, 64)


@pytest.mark.parametrize("q", BENCH_QS)
def test_bench_sweep_plans_match_oracle_at_p64(q):
    """At the benchmark's p = 64: the list, task list, ASAP finish times,
    zero times and critical path of the tree the bench runs at this q, bit
    for bit against the oracle; and for PlasmaTree and PlasmaTree-TS the
    lists and critical paths at every domain size the per-tree sweep times
    (the critical-path model's 8 best BS and {1, p})."""
    import bench
    p = 64
    name, bs = bench.SWEEP_TREES[q]
    tree = tqr.TREES[name]
    el = otrees.elimination_list(p, q, tree, bs)
    otasks = odag.expand(p, q, el, otrees.ts_flags(tree, bs, el))
    ofin, ocp = odag.simulate(otasks)
    tasks, fin = tqr.tqr_tasks(p, q, tree, bs)
    want = np.array([[KIND_MAP[k], i - 1, piv - 1 if piv else -1, kk - 1, j - 1 if j else -1]
                     for (k, i, piv, kk, j) in otasks], dtype=np.int32).reshape(-1, 5)
    assert np.array_equal(tasks, want)
    assert np.array_equal(fin, np.array(ofin, dtype=np.int64))
    cp, zt = tqr.tqr_critical_path(p, q, tree, bs, zero_time=True)
    assert cp == ocp
    ozt = odag.zero_times(otasks, ofin)
    assert all(zt[i, k] == ozt.get((i + 1, k + 1), -1) for i in range(p) for k in range(q))
    for t in (tqr.PLASMA, tqr.PLASMA_TS):
        for BS in bench.plasma_bs_candidates(tqr, p, q, t):
            el = otrees.elimination_list(p, q, t, BS)
            assert lists_equal(p, q, t, BS), (q, t, BS)
            assert tqr.tqr_critical_path(p, q, t, BS) == odag.critical_path(p, q, el, otrees.ts_flags(t, BS, el))


def test_validator_agrees_with_oracle():
    rng = np.random.default_rng(0)
    p, q = 7, 3
    good = otrees.greedy(p, q)
    assert tqr.tqr_validate_list(p, q, np.array(good) - 1) == 0
    agree = 0
    for trial in range(400):
        el = [list(e) for e in good]
        kind = trial % 4
        if kind == 0:                                     # swap two entries
            a, b = rng.integers(0, len(el), 2)
            el[a], el[b] = el[b], el[a]
        elif kind == 1:                                   # change a pivot
            a = rng.integers(0, len(el))
            el[a][1] = int(rng.integers(el[a][2], p + 1))
        elif kind == 2:                                   # drop an entry
            del el[rng.integers(0, len(el))]
        else:                                             # duplicate an entry
            el.append(list(el[rng.integers(0, len(el))]))
        ok_oracle = otrees.validate(p, q, [tuple(e) for e in el]) is None
        rc = tqr.tqr_validate_list(p, q, np.array(el, dtype=np.int32) - 1)
        assert (rc == 0) == ok_oracle, el
        agree += 1
    assert agree == 400


def test_argument_errors():
    L = tqr.lib()
    assert L.tqr_critical_path(0, 1, 5, 1, None, None) == -1
    cp = np.zeros(1, dtype=np.int64)
    assert tqr.lib().tqr_critical_path(4, 5, 5, 1, cp.ctypes.data_as(tqr.tqr.ctypes.POINTER(tqr.tqr.ctypes.c_int64)),
                                       None) == -2
    assert tqr.lib().tqr_elimination_list(8, 2, 6, 0, None, 0, None) == -4
    with pytest.raises(tqr.TqrError):
        tqr.tqr_critical_path(4, 2, 99)
    assert tqr.tqr_strerror(tqr.TQR_ERR_TIMEOUT) == "device wait timed out"


def test_factor_argument_errors_before_any_device_work():
    """Argument checks of the factorization entry points run on the host
    before any CUDA call, so they are testable without a GPU."""
    L = tqr.lib()
    ct = tqr.tqr.ctypes
    fake = ct.c_void_p(0x1000)                            # never dereferenced: rejected earlier
    out = ct.c_void_p(None)
    # tqr_factor(A, m, n, nb, ib, tree, BS, stream, out)
    assert L.tqr_factor(None, 64, 32, 32, 8, tqr.GREEDY, 1, None, ct.byref(out)) == -1
    assert L.tqr_factor(fake, 0, 32, 32, 8, tqr.GREEDY, 1, None, ct.byref(out)) == -2
    assert L.tqr_factor(fake, 64, 65, 32, 8, tqr.GREEDY, 1, None, ct.byref(out)) == -3     # n > m
    assert L.tqr_factor(fake, 64, 32, 30, 5, tqr.GREEDY, 1, None, ct.byref(out)) == -4     # nb % 4
    assert L.tqr_factor(fake, 64, 32, 4, 4, tqr.GREEDY, 1, None, ct.byref(out)) == -4      # nb < 8
    assert L.tqr_factor(fake, 64, 32, 32, 12, tqr.GREEDY, 1, None, ct.byref(out)) == -5    # ib does not divide nb
    assert L.tqr_factor(fake, 64, 32, 32, 8, 42, 1, None, ct.byref(out)) == -6             # unknown tree
    assert L.tqr_factor(fake, 64, 32, 32, 8, tqr.PLASMA, 0, None, ct.byref(out)) == -7     # BS < 1
    assert L.tqr_factor(fake, 64, 32, 32, 8, tqr.PLASMA_TS, 3, None, ct.byref(out)) == -7  # BS > p = 2
    assert L.tqr_factor(fake, 64, 32, 32, 8, tqr.GRASAP, 2, None, ct.byref(out)) == -7     # k > q = 1
    assert L.tqr_factor(fake, 64, 32, 32, 8, tqr.GREEDY, 1, None, None) == -9
    # tqr_factor_ex(..., precision, stream, out)
    assert L.tqr_factor_ex(fake, 64, 32, 32, 8, tqr.GREEDY, 1, 7, None, ct.byref(out)) == -8
    # maximum sizes: more than 65535 tile rows, and a task graph beyond int32 task ids
    assert L.tqr_factor(fake, 65536 * 16 + 16, 32, 16, 8, tqr.GREEDY, 1, None, ct.byref(out)) == -2
    assert L.tqr_factor(fake, 65536, 65536, 16, 8, tqr.GREEDY, 1, None, ct.byref(out)) == tqr.TQR_ERR_CAPACITY
    cp = ct.c_int64(0)
    assert L.tqr_critical_path(4096, 4096, tqr.GREEDY, 1, ct.byref(cp), None) == tqr.TQR_ERR_CAPACITY
    assert out.value is None


def test_factor_host_argument_errors_before_any_device_work():
    """tqr_factor_host / _async check A, m, n, nb and ib (the positions
    tqr_factor uses) before they allocate or copy anything."""
    L = tqr.lib()
    ct = tqr.tqr.ctypes
    fake = ct.c_void_p(0x1000)
    out = ct.c_void_p(None)
    for fn in (L.tqr_factor_host, L.tqr_factor_host_async):
        # (A_host, m, n, nb, ib, tree, BS, B_host, nrhs, stream, out)
        assert fn(None, 64, 32, 32, 8, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -1
        assert fn(fake, 0, 32, 32, 8, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -2
        assert fn(fake, -5, 32, 32, 8, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -2
        assert fn(fake, 64, 65, 32, 8, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -3
        assert fn(fake, 64, 32, 30, 5, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -4
        assert fn(fake, 64, 32, 32, 12, tqr.GREEDY, 1, None, 0, None, ct.byref(out)) == -5
        assert fn(fake, 64, 32, 32, 8, tqr.GREEDY, 1, None, 0, None, None) == -11
        assert fn(fake, 64, 32, 32, 8, tqr.GREEDY, 1, fake, -1, None, ct.byref(out)) == -9
    assert out.value is None


def test_release_plans_without_cached_plans():
    """With no plan built in this process (no GPU here), releasing drops
    nothing and touches no device."""
    assert tqr.tqr_release_plans() == 0


def test_lstsq_argument_errors_before_any_device_work():
    """tqr_lstsq reports each invalid argument by its own position, before it
    allocates anything (nb, ib, tree and BS under tqr_factor's rules)."""
    L = tqr.lib()
    ct = tqr.tqr.ctypes
    fake = ct.c_void_p(0x1000)

    def call(A=fake, m=64, n=32, b=fake, x=fake, nb=32, ib=8, tree=tqr.GREEDY, BS=1, prec=1, tol=1e-14, maxit=5):
        return L.tqr_lstsq(A, m, n, b, x, nb, ib, tree, BS, prec, tol, maxit, None, None)

    assert call(A=None) == -1
    assert call(m=0) == -2
    assert call(n=65) == -3
    assert call(b=None) == -4
    assert call(x=None) == -5
    assert call(nb=30, ib=5) == -6
    assert call(ib=12) == -7
    assert call(tree=42) == -8
    assert call(tree=tqr.PLASMA, BS=0) == -9
    assert call(tree=tqr.GRASAP, BS=2) == -9                    # k > q = 1
    assert call(prec=3) == -10
    assert call(tol=-1.0) == -11
    assert call(tol=float("nan")) == -11
    assert call(tol=float("inf")) == -11
    assert call(maxit=-1) == -12
    assert call(m=65536, n=65536, nb=16, ib=8) == tqr.TQR_ERR_CAPACITY


def test_mlp_bindings_check_tensors_before_the_call():
    """The cost-model bindings reject anything but contiguous float32 CUDA
    tensors of the right size before calling the library (here: CPU tensors,
    a float64 tensor, a feature count the network does not take)."""
    torch = pytest.importorskip("torch")
    P = tqr.tqr_mlp_param_count(4)
    params, X = torch.zeros(P), torch.zeros(3, 4)
    with pytest.raises(TypeError):
        tqr.tqr_mlp_forward(params, X)
    with pytest.raises(TypeError):
        tqr.tqr_mlp_loss_grad(params, X, torch.zeros(3), torch.zeros(P), torch.zeros(1))
    with pytest.raises(TypeError):
        tqr.tqr_mlp_adam_step(params.double(), params, params, params, 1e-3, 1)
    with pytest.raises(tqr.TqrError):
        tqr.tqr_mlp_forward(params, torch.zeros(3, 40))              # more than TQR_MLP_MAX_IN features


def test_vector_bindings_check_tensors_before_the_call():
    """The device-array check that tqr_lstsq (b, x), tqr_form_t (T arrays) and
    tqr_factor_noalloc (tau, status) apply before calling the library: on a
    machine without a GPU it rejects every tensor, naming the argument."""
    torch = pytest.importorskip("torch")
    for t, dt in ((torch.zeros(64, dtype=torch.float64), "float64"), (torch.zeros(1, dtype=torch.int32), "int32")):
        with pytest.raises(TypeError, match="status must be a contiguous %s CUDA tensor" % dt):
            tqr.tqr._dev(t, "status", dt)


def test_build_rebuilds_a_library_for_another_cpu(tmp_path, monkeypatch):
    """A libtqr.so for another CPU (the tree copied between an x86 and an Arm
    machine) counts as missing, whatever its time stamp."""
    import platform
    from paper_1104_4475_gb300 import build as b
    codes = b._ELF_MACHINE
    here = codes.get(platform.machine())
    if here is None:
        pytest.skip("unknown host CPU")
    other = next(c for c in codes.values() if c != here)
    for code, ok in ((here, True), (other, False)):
        lib = tmp_path / ("lib%d.so" % code)
        lib.write_bytes(b"\x7fELF" + bytes(14) + code.to_bytes(2, "little") + bytes(40))
        monkeypatch.setattr(b, "LIB", str(lib))
        assert b._lib_matches_host() is ok
    monkeypatch.setattr(b, "LIB", str(tmp_path / "missing.so"))
    assert b._lib_matches_host() is False and b.needs_build()


def test_binding_constants_equal_the_header():
    """Tree ids, kernel kinds, precisions and status codes of the Python
    binding are the values tqr.h defines (and the oracle's tree ids too)."""
    import oracle
    src = open(os.path.join(ROOT, "include", "tqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define (TQR_[A-Z_]+) \(?(-?\d+)\)?\s*$", src, flags=re.M)}
    consts.update({k: int(v) for k, v in re.findall(r"\b(TQR_[A-Z0-9_]+) = (\d+)", src)})
    trees = {"TQR_FLAT_TS": "FLAT_TS", "TQR_FLAT_TT": "FLAT_TT", "TQR_SAMEH_KUCK": "SAMEH_KUCK",
             "TQR_BINARY": "BINARY", "TQR_FIBONACCI": "FIBONACCI", "TQR_GREEDY": "GREEDY", "TQR_PLASMA": "PLASMA",
             "TQR_ASAP": "ASAP", "TQR_GRASAP": "GRASAP", "TQR_PLASMA_TS": "PLASMA_TS"}
    for c, py in trees.items():
        assert getattr(tqr, py) == consts[c], c
        if hasattr(oracle, py):
            assert getattr(oracle, py) == consts[c], c
    for kind in ("GEQRT", "UNMQR", "TTQRT", "TTMQR", "TSQRT", "TSMQR"):
        assert getattr(tqr.tqr, kind) == consts["TQR_" + kind], kind
    for name in ("TQR_FP64", "TQR_SPLIT_TF32", "TQR_TF32"):
        assert getattr(tqr, name) == consts[name], name
    errs = [k for k in consts if k.startswith("TQR_ERR_")]
    assert len(errs) == 9
    for name in errs:
        assert getattr(tqr, name) == consts[name], name


def test_binding_structs_match_the_header():
    """tqr_info, tqr_batch_info and tqr_lstsq_info: the ctypes structures
    have the header's fields, in its order, with its types."""
    import ctypes
    src = open(os.path.join(ROOT, "include", "tqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    ctype = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    structs = re.findall(r"typedef struct \{(.*?)\}\s*(tqr_[a-z_]+);", src, flags=re.S)
    assert {name for _, name in structs} == {"tqr_info", "tqr_batch_info", "tqr_lstsq_info"}
    for body, name in structs:
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, names = decl.split(None, 1)
            fields += [(nm.strip(), ctype[typ]) for nm in names.split(",")]
        py = getattr(tqr.tqr, name)._fields_
        assert [(f, t) for f, t in py] == fields, name


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without libtqr.so every entry point raises: there is no fallback."""
    from paper_1104_4475_gb300 import build as b
    monkeypatch.setattr(b, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(tqr.tqr, "_lib", None)
    with pytest.raises(ImportError):
        tqr.tqr_elimination_list(4, 2, tqr.GREEDY)
    with pytest.raises(ImportError):
        tqr.tqr_critical_path(4, 2, tqr.GREEDY)
