"""Kernel tasks of an elimination list, their dependencies, and the
unit-weight as-soon-as-possible simulator.

Part of the test oracle (see ``oracle/__init__.py``).  1-based indices.

A task is a tuple ``(kind, i, piv, k, j)``:

* ``GEQRT (x, 0, k, 0)``      factor tile (x,k) into a triangle;
* ``UNMQR (x, 0, k, j)``      apply its reflectors to tile (x,j), j > k;
* ``TTQRT/TSQRT (i, piv, k, 0)`` zero tile (i,k) against the triangle (piv,k);
* ``TTMQR/TSMQR (i, piv, k, j)`` apply that transformation to rows piv, i of
  tile column j.

Expansion follows Algorithm 2 (TS) and Algorithm 3 (TT) of Section 2.1, with
the rule that a tile already in triangle form is not factored again (and its
updates are not repeated).  Readings:

* In TT every tile (x,k), x >= k, is factored by exactly one GEQRT; it is
  emitted at the first elimination of column k that involves row x.  The
  diagonal tile of the last column of a square matrix takes part in no
  elimination; its GEQRT (and nothing else) is appended at the end.
* In TS only pivot tiles are factored by GEQRT; the zeroed tile is square.
* Dependencies (Section 2.3, and the V-NODEP / T-INPUT flags of Section 4):
  a task depends on the task that produced the reflectors it applies (V and
  T are read-only after that), and on the previous writer of every tile it
  writes, in list order.  Readers of V never delay a later writer of the
  other half of the same tile, so there are no write-after-read edges.
"""

GEQRT, UNMQR, TTQRT, TTMQR, TSQRT, TSMQR = range(6)
KIND_NAMES = ["GEQRT", "UNMQR", "TTQRT", "TTMQR", "TSQRT", "TSMQR"]

# Table 1: cost of each kernel in units of nb^3/3 floating-point operations.
WEIGHT = {GEQRT: 4, UNMQR: 6, TSQRT: 6, TSMQR: 12, TTQRT: 2, TTMQR: 6}


def expand(p, q, elims, ts=False):
    """Kernel tasks of an elimination list, in program (list) order.  ``ts``
    is one kernel family for the whole list (True = TS) or one flag per
    elimination."""
    flags = [bool(ts)] * len(elims) if isinstance(ts, (bool, int)) else list(ts)
    if len(flags) != len(elims):
        raise ValueError("one TS flag per elimination")
    tasks = []
    triangle = set()

    def factor(x, k):
        if (x, k) in triangle:
            return
        triangle.add((x, k))
        tasks.append((GEQRT, x, 0, k, 0))
        for j in range(k + 1, q + 1):
            tasks.append((UNMQR, x, 0, k, j))

    for (i, piv, k), use_ts in zip(elims, flags):
        if use_ts:
            if (i, k) in triangle:
                raise ValueError("TS elimination of a tile already in triangle form")
            factor(piv, k)
            tasks.append((TSQRT, i, piv, k, 0))
            for j in range(k + 1, q + 1):
                tasks.append((TSMQR, i, piv, k, j))
        else:
            factor(piv, k)
            factor(i, k)
            tasks.append((TTQRT, i, piv, k, 0))
            for j in range(k + 1, q + 1):
                tasks.append((TTMQR, i, piv, k, j))
    for k in range(1, min(p, q) + 1):
        factor(k, k)
    return tasks


def dependencies(tasks):
    """Predecessor index lists, one per task (producer and last-writer edges)."""
    last_writer = {}
    producer = {}          # (x,k) -> GEQRT task;  ('e', i, k) -> TTQRT/TSQRT task
    preds = []
    for t, (kind, i, piv, k, j) in enumerate(tasks):
        d = set()
        if kind == GEQRT:
            writes = [(i, k)]
            producer[(i, k)] = t
        elif kind == UNMQR:
            d.add(producer[(i, k)])
            writes = [(i, j)]
        elif kind in (TTQRT, TSQRT):
            writes = [(piv, k), (i, k)]
            producer[("e", i, k)] = t
        else:  # TTMQR, TSMQR
            d.add(producer[("e", i, k)])
            writes = [(piv, j), (i, j)]
        for w in writes:
            if w in last_writer:
                d.add(last_writer[w])
        for w in writes:
            last_writer[w] = t
        preds.append(sorted(d))
    return preds


def simulate(tasks, preds=None):
    """Unit-weight ASAP schedule with unbounded processors.

    Returns ``(finish, cp)``: the finish time of every task in units of
    nb^3/3 flops, and the critical path (finish time of the last task).
    """
    if preds is None:
        preds = dependencies(tasks)
    finish = []
    for t, task in enumerate(tasks):
        start = max((finish[d] for d in preds[t]), default=0)
        finish.append(start + WEIGHT[task[0]])
    return finish, max(finish, default=0)


def zero_times(tasks, finish):
    """{(i,k): time at which tile (i,k) is zeroed} (finish of its TTQRT/TSQRT)."""
    out = {}
    for t, (kind, i, piv, k, j) in enumerate(tasks):
        if kind in (TTQRT, TSQRT):
            out[(i, k)] = finish[t]
    return out


def critical_path(p, q, elims, ts=False):
    tasks = expand(p, q, elims, ts)
    _, cp = simulate(tasks)
    return cp


def total_weight(tasks):
    return sum(WEIGHT[t[0]] for t in tasks)


class Incremental:
    """The expansion, dependencies and ASAP times of a list built one
    elimination at a time (used by the dynamic ASAP / GRASAP trees, whose
    next elimination depends on the times of the previous ones)."""

    def __init__(self, p, q, ts=False):
        self.p, self.q, self.ts = p, q, ts
        self.tasks, self.finish = [], []
        self.triangle = set()
        self.last_writer, self.producer = {}, {}

    def _add(self, task):
        kind, i, piv, k, j = task
        d = []
        if kind == GEQRT:
            writes = [(i, k)]
        elif kind == UNMQR:
            d.append(self.producer[(i, k)])
            writes = [(i, j)]
        elif kind in (TTQRT, TSQRT):
            writes = [(piv, k), (i, k)]
        else:
            d.append(self.producer[("e", i, k)])
            writes = [(piv, j), (i, j)]
        d += [self.last_writer[w] for w in writes if w in self.last_writer]
        t = len(self.tasks)
        for w in writes:
            self.last_writer[w] = t
        if kind == GEQRT:
            self.producer[(i, k)] = t
        elif kind in (TTQRT, TSQRT):
            self.producer[("e", i, k)] = t
        self.tasks.append(task)
        self.finish.append(max((self.finish[x] for x in d), default=0) + WEIGHT[kind])
        return t

    def _factor(self, x, k):
        if (x, k) in self.triangle:
            return
        self.triangle.add((x, k))
        self._add((GEQRT, x, 0, k, 0))
        for j in range(k + 1, self.q + 1):
            self._add((UNMQR, x, 0, k, j))

    def add_elim(self, i, piv, k):
        """Append elim(i, piv, k) (Algorithm 3, or 2 when ts); returns the
        finish time of its TTQRT/TSQRT."""
        self._factor(piv, k)
        if not self.ts:
            self._factor(i, k)
        t = self._add(((TSQRT if self.ts else TTQRT), i, piv, k, 0))
        for j in range(k + 1, self.q + 1):
            self._add(((TSMQR if self.ts else TTMQR), i, piv, k, j))
        return self.finish[t]

    def triangle_time(self, x, k):
        """When GEQRT(x,k) would finish if emitted now: last writer of tile
        (x,k) plus the GEQRT weight (tile (x,k) must have all its writers)."""
        if (x, k) in self.triangle:
            return self.finish[self.producer[(x, k)]]
        lw = self.last_writer.get((x, k))
        return (self.finish[lw] if lw is not None else 0) + WEIGHT[GEQRT]

    def close(self):
        """Factor the diagonal tiles that took part in no elimination."""
        for k in range(1, min(self.p, self.q) + 1):
            self._factor(k, k)
        return max(self.finish, default=0)
