"""The device task graph (tqr_device_graph, built on the host) is race-free.

The executor runs a task as soon as its in-edges are satisfied, so the graph
alone decides the order of conflicting memory accesses.  From the kernel
semantics of every device task (what it writes and which reflectors it reads)
these tests check, with the transitive closure of the graph:

* every two tasks that write overlapping rows of the same column of a tile
  are ordered, the earlier one in program order (the sequential algorithm)
  first -- rows by the kernels' definitions: block b of GEQRT writes rows
  b ib.. of its tile, of TTQRT rows ..(b+1) ib of the zeroed tile, of TSQRT
  all its rows, and of both eliminations rows b ib..(b+1) ib of the pivot;
* every task that applies reflectors runs after the task that formed them;
* a panel split into blocks is exactly that: one factor task per block of ib
  columns and update tasks that cover the columns right of the block once.

They also pin the look-ahead the finer graph exists for: the elimination of a
tile's first column block does not wait for the rest of that tile's GEQRT.
"""

import numpy as np
import pytest

import paper_1104_4475_gb300 as tqr

GE_CLASS, EL_CLASS = 0, 1
PANELS = (tqr.GEQRT, tqr.TTQRT, tqr.TSQRT)


def closure(n, edges):
    """reach[v]: bitset (Python int) of the tasks with a path to v."""
    preds = [[] for _ in range(n)]
    for u, v in edges.tolist():
        assert u < v, "edge %d -> %d runs backwards" % (u, v)
        preds[v].append(u)
    reach = [0] * n
    for v in range(n):
        r = 0
        for u in preds[v]:
            r |= reach[u] | (1 << u)
        reach[v] = r
    return reach


def accesses(tasks, m, n, nb, ib, strip):
    """Per task: the writes ((tile row, tile column, column), row_lo, row_hi)
    it makes, the reflector blocks (class, i, k, b) it reads and those it
    forms."""
    q = -(-n // nb)

    def ncol(j):
        return n - (q - 1) * nb if j == q - 1 else nb

    nblk = nb // ib
    out = []
    for kind, i, piv, k, j, st in tasks.tolist():
        if kind in PANELS:
            cls = GE_CLASS if kind == tqr.GEQRT else EL_CLASS
            if j < 0:                                   # the whole panel: every row
                cols, vr, vw = range(ncol(k)), [], [(cls, i, k, b) for b in range(nblk)]
                rows = [(i, 0, nb)] + ([] if kind == tqr.GEQRT else [(piv, 0, nb)])
            else:
                j0 = j * ib
                bot = {tqr.GEQRT: (j0, nb), tqr.TTQRT: (0, j0 + ib), tqr.TSQRT: (0, nb)}[kind]
                rows = [(i,) + bot] + ([] if kind == tqr.GEQRT else [(piv, j0, j0 + ib)])
                if st < 0:                              # factor block j
                    cols = range(j0, min(j0 + ib, ncol(k)))
                    vr, vw = [], [(cls, i, k, j)]
                else:                                   # apply block j to [c_lo, c_hi)
                    cols = range(st & 0xffff, st >> 16)
                    vr, vw = [(cls, i, k, j)], []
            tc = k
        else:
            cls = GE_CLASS if kind == tqr.UNMQR else EL_CLASS
            cols = range(st * strip, min((st + 1) * strip, ncol(j)))
            vr, vw = [(cls, i, k, b) for b in range(nblk)], []
            rows = [(i, 0, nb)] + ([] if kind == tqr.UNMQR else [(piv, 0, nb)])
            tc = j
        out.append(([((r, tc, c), lo, hi) for r, lo, hi in rows for c in cols], vr, vw))
    return out


CASES = [
    # m, n, nb, ib, tree, BS, strip
    (1024, 512, 128, 16, tqr.GREEDY, 1, 64),
    (1400, 600, 128, 32, tqr.FLAT_TS, 1, 64),       # ragged rows and columns, TS kernels
    (1024, 384, 128, 32, tqr.PLASMA_TS, 2, 64),     # TS inside domains, TT merges
    (1200, 500, 128, 16, tqr.BINARY, 1, 32),
    (512, 512, 128, 8, tqr.FIBONACCI, 1, 16),       # square
    (1040, 404, 128, 16, tqr.GREEDY, 1, 64),        # last tile column: 20 columns, 6 empty blocks
    (1200, 600, 128, 64, tqr.GREEDY, 1, 64),        # two blocks per tile
    (768, 256, 128, 4, tqr.FLAT_TT, 1, 64),         # ib < 8: panels stay whole
    (600, 250, 48, 16, tqr.BINARY, 1, 32),          # nb < 128: panels stay whole
    (1536, 512, 256, 32, tqr.GREEDY, 1, 64),        # the benchmark's tile shape
]


@pytest.mark.parametrize("m,n,nb,ib,tree,BS,strip", CASES)
def test_device_graph_orders_every_conflict(m, n, nb, ib, tree, BS, strip):
    tasks, edges = tqr.tqr_device_graph(m, n, nb, ib, tree, BS, strip)
    N = len(tasks)
    reach = closure(N, edges)
    acc = accesses(tasks, m, n, nb, ib, strip)
    writers, former = {}, {}
    for t, (cells, vr, vw) in enumerate(acc):
        for cell, lo, hi in cells:
            for a, alo, ahi in writers.get(cell, ()):
                if alo < hi and lo < ahi:
                    assert (reach[t] >> a) & 1, "writers %d and %d of rows of %s are not ordered" % (a, t, cell)
            writers.setdefault(cell, []).append((t, lo, hi))
        for blk in vw:
            assert blk not in former, "reflector block %s formed twice" % (blk,)
            former[blk] = t
        for blk in vr:
            f = former.get(blk)
            assert f is not None, "task %d applies reflector block %s before any task forms it" % (t, blk)
            assert (reach[t] >> f) & 1, "task %d applies %s without waiting for task %d" % (t, blk, f)


@pytest.mark.parametrize("m,n,nb,ib,tree,BS,strip", [c for c in CASES if c[4] != tqr.PLASMA_TS])
def test_noalloc_graph_orders_every_conflict(m, n, nb, ib, tree, BS, strip):
    """tqr_factor_noalloc's own graph builder (whole panels), under the same
    checks, and with the same tile-level task list as the library's."""
    p, q = -(-m // nb), -(-n // nb)
    elims = tqr.tqr_elimination_list(p, q, tree, BS)
    tasks, edges = tqr.tqr_noalloc_graph(m, n, nb, ib, elims, tree == tqr.FLAT_TS, strip)
    assert (tasks[[k in PANELS for k in tasks[:, 0]], 4] == -1).all()
    reach = closure(len(tasks), edges)
    writers, former = {}, {}
    for t, (cells, vr, vw) in enumerate(accesses(tasks, m, n, nb, ib, strip)):
        for cell, lo, hi in cells:
            for a, alo, ahi in writers.get(cell, ()):
                if alo < hi and lo < ahi:
                    assert (reach[t] >> a) & 1, "writers %d and %d of rows of %s are not ordered" % (a, t, cell)
            writers.setdefault(cell, []).append((t, lo, hi))
        for blk in vw:
            former[blk] = t
        for blk in vr:
            assert (reach[t] >> former[blk]) & 1
    tile = []
    for kind, i, piv, k, j, st in tasks.tolist():
        key = (kind, i, piv, k, -1 if kind in PANELS else j)
        if not tile or tile[-1] != key:
            tile.append(key)
    want, _ = tqr.tqr_tasks(p, q, tree, BS)
    assert tile == [tuple(x) for x in want.tolist()]


@pytest.mark.parametrize("m,n,nb,ib,tree,BS,strip", CASES)
def test_split_panels_cover_their_tiles_once(m, n, nb, ib, tree, BS, strip):
    tasks, _ = tqr.tqr_device_graph(m, n, nb, ib, tree, BS, strip)
    p, q = -(-m // nb), -(-n // nb)
    split = nb >= 128 and ib >= 8 and nb // ib >= 2
    # Collapsing the device tasks gives the tile-level task list, in order.
    tile = []
    for kind, i, piv, k, j, st in tasks.tolist():
        key = (kind, i, piv, k, -1 if kind in PANELS else j)
        if not tile or tile[-1] != key:
            tile.append(key)
    want, _ = tqr.tqr_tasks(p, q, tree, BS)
    assert tile == [tuple(x) for x in want.tolist()]
    panels = {}
    for kind, i, piv, k, j, st in tasks.tolist():
        if kind in PANELS:
            panels.setdefault((kind, i, piv, k), []).append((j, st))
    for (kind, i, piv, k), parts in panels.items():
        ncol = n - (q - 1) * nb if k == q - 1 else nb
        if not split:
            assert parts == [(-1, 0)]
            continue
        assert [j for j, st in parts if st < 0] == list(range(nb // ib))
        for b in range(nb // ib):
            ranges = [(st & 0xffff, st >> 16) for j, st in parts if j == b and st >= 0]
            covered = [c for lo, hi in ranges for c in range(lo, hi)]
            assert covered == list(range((b + 1) * ib, ncol)) if (b + 1) * ib < ncol else covered == []
            if ranges:                                   # the look-ahead part comes first
                assert ranges[0][0] == (b + 1) * ib and ranges[0][1] - ranges[0][0] <= max(ib, 32)


def test_elimination_starts_before_the_geqrt_finishes():
    """Greedy on a 4 x 1 tile matrix: TTQRT's first block waits for the
    first blocks of both GEQRTs, not for their last blocks, and so does the
    update of the last column unit by TTQRT's first block (row block 0 of
    that unit is final once GEQRT's first block has been applied to it)."""
    nb, ib = 128, 32
    tasks, edges = tqr.tqr_device_graph(4 * nb, nb, nb, ib, tqr.GREEDY, 1, 64)
    reach = closure(len(tasks), edges)
    idx = {tuple(r): t for t, r in enumerate(tasks.tolist())}
    first_tt = [t for t, r in enumerate(tasks.tolist()) if r[0] == tqr.TTQRT][0]
    _, i, piv, k, _, _ = tasks[first_tt].tolist()
    tt_f0 = idx[(tqr.TTQRT, i, piv, k, 0, -1)]
    tt_u0 = [t for t, r in enumerate(tasks.tolist())
             if r[:5] == [tqr.TTQRT, i, piv, k, 0] and r[5] >= 0 and (r[5] >> 16) == nb][0]
    for row in (i, piv):
        first = idx[(tqr.GEQRT, row, -1, k, 0, -1)]
        last = idx[(tqr.GEQRT, row, -1, k, nb // ib - 1, -1)]
        for t in (tt_f0, tt_u0):
            assert (reach[t] >> first) & 1
            assert not (reach[t] >> last) & 1


def test_device_graph_rejects_bad_arguments():
    for args, code in [((0, 1, 64, 16, tqr.GREEDY, 1, 64), -2), ((64, 128, 64, 16, tqr.GREEDY, 1, 64), -3),
                       ((64, 64, 64, 7, tqr.GREEDY, 1, 64), -5), ((64, 64, 64, 16, 99, 1, 64), -6),
                       ((640, 64, 64, 16, tqr.PLASMA, 11, 64), -7), ((64, 64, 64, 16, tqr.GREEDY, 1, 48), -8)]:
        with pytest.raises(tqr.TqrError) as e:
            tqr.tqr_device_graph(*args)
        assert e.value.code == code
