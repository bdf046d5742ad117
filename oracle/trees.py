"""Elimination lists of the tiled QR trees, their validity rules, and the
coarse-grain time-step model.

Part of the test oracle (see ``oracle/__init__.py``).  Everything here is
1-based: an elimination ``(i, piv, k)`` is the paper's ``elim(i, piv(i,k), k)``
-- it zeroes tile ``(i, k)`` using row ``piv`` (Section 2, Algorithm 1).

Readings of points the paper leaves open are stated beside each generator.
"""

from . import FLAT_TS, FLAT_TT, SAMEH_KUCK, BINARY, FIBONACCI, GREEDY, PLASMA, ASAP, GRASAP, PLASMA_TS


# --------------------------------------------------------------------------
# Sameh-Kuck / FlatTree (Section 3.1, "Sameh-Kuck algorithm"; Section 3.2
# notes that tiled Sameh-Kuck is PLASMA's FlatTree).
# --------------------------------------------------------------------------
def sameh_kuck(p, q):
    """Column k uses the panel row k to zero rows k+1..p, top to bottom."""
    out = []
    for k in range(1, min(p, q) + 1):
        for i in range(k + 1, p + 1):
            out.append((i, k, k))
    return out


# --------------------------------------------------------------------------
# Fibonacci scheme of order 1 (Section 3.1, "Fibonacci algorithm").
# --------------------------------------------------------------------------
def fibonacci_x(p):
    """Least integer x with x(x+1)/2 >= p-1 (number of coarse steps of column 1)."""
    x = 0
    while x * (x + 1) // 2 < p - 1:
        x += 1
    return x


def fibonacci_coarse(p, i, k):
    """coarse(i,k) of the Fibonacci scheme for i > k.

    Column 1: coarse(i,1) = x - y + 1 with y the least integer such that
    i <= y(y+1)/2 + 1.  Column k is column k-1 shifted down one row plus two
    time-units: coarse(i,k) = coarse(i-1,k-1) + 2, i.e.
    coarse(i,k) = coarse(i-k+1, 1) + 2(k-1).  x always uses the full p.
    """
    x = fibonacci_x(p)
    r = i - k + 1
    y = 0
    while not (r <= y * (y + 1) // 2 + 1):
        y += 1
    return x - y + 1 + 2 * (k - 1)


def fibonacci(p, q):
    """Fibonacci elimination list.

    In every column the rows sharing one coarse time-step form a contiguous
    block of z rows; each is paired with the row z above it (piv = i - z),
    z being that column's block size (the bottom block of a later column may
    be shorter than in column 1).  Order: column, then time-step ascending,
    then row ascending.
    """
    out = []
    for k in range(1, min(p, q) + 1):
        groups = {}
        for i in range(k + 1, p + 1):
            groups.setdefault(fibonacci_coarse(p, i, k), []).append(i)
        for step in sorted(groups):
            rows = sorted(groups[step])
            z = len(rows)
            for i in rows:
                out.append((i, i - z, k))
    return out


# --------------------------------------------------------------------------
# Greedy for tiles (Section 3.2, Algorithm 4, TT kernels).
# --------------------------------------------------------------------------
def greedy(p, q):
    """Greedy tiled elimination list (Algorithm 4).

    nT(j) counts triangularized tiles and nZ(j) zeroed tiles of column j,
    both counted from the bottom row p upwards.  One outer step sweeps the
    columns j = q..1.  Column 1 triangularizes all p rows at once; column
    j > 1 triangularizes every tile whose left neighbour is zero, reading
    nZ(j-1) as it stood at the end of the previous step (the sweep is
    right-to-left).  Then half of the triangularized-but-not-zeroed tiles are
    zeroed, bottom first, tile p-kk paired with p-kk-(nZnew-nZ(j)).
    The loop stops when every column j <= min(p,q) holds p-j zeros.
    Order of the list: step, then column descending, then kk ascending.
    """
    qq = min(p, q)
    nZ = [0] * (q + 1)
    nT = [0] * (q + 1)
    out = []

    def finished():
        return all(nZ[j] == p - j for j in range(1, qq + 1))

    while not finished():
        for j in range(q, 0, -1):
            if j == 1:
                nT_new = p
            else:
                nT_new = nZ[j - 1]
            nZ_new = nZ[j] + (nT[j] - nZ[j]) // 2
            for kk in range(nZ[j], nZ_new):
                out.append((p - kk, p - kk - nZ_new + nZ[j], j))
            nT[j] = nT_new
            nZ[j] = nZ_new
    return out


# --------------------------------------------------------------------------
# BinaryTree (Section 3.2, Proposition 1).
# --------------------------------------------------------------------------
def binary_tree(p, q):
    """Binary reduction per column.

    With offsets d = i - k from the panel row, level s = 1, 2, 4, ... zeroes
    every row k+d with d = s (mod 2s) using row k+d-s.  Order: column, level,
    row.
    """
    out = []
    for k in range(1, min(p, q) + 1):
        n = p - k + 1
        s = 1
        while s < n:
            for d in range(s, n, 2 * s):
                out.append((k + d, k + d - s, k))
            s *= 2
    return out


# --------------------------------------------------------------------------
# PlasmaTree(BS) (Section 3.2, domains of BS rows).
# --------------------------------------------------------------------------
def plasma_tree(p, q, BS):
    """Flat trees inside domains of BS consecutive rows, binary merge on top.

    Domains of column k start at the panel row k: {k..k+BS-1}, {k+BS..}, ...;
    the bottom domain is truncated as k grows.  Inside a domain the first row
    zeroes the others; the domain heads are then merged by the BinaryTree
    pairing over the list of heads.  Order: domains top-down, then merge
    levels.
    """
    if BS < 1:
        raise ValueError("BS must be >= 1")
    out = []
    for k in range(1, min(p, q) + 1):
        heads = list(range(k, p + 1, BS))
        for h in heads:
            for i in range(h + 1, min(h + BS - 1, p) + 1):
                out.append((i, h, k))
        s = 1
        while s < len(heads):
            for d in range(s, len(heads), 2 * s):
                out.append((heads[d], heads[d - s], k))
            s *= 2
    return out


def elimination_list(p, q, tree, BS=1):
    """The elimination list of a tree (1-based triplets).  BS is PlasmaTree's
    domain size, or the k of GRASAP(k)."""
    if not (p >= q >= 1):
        raise ValueError("need p >= q >= 1")
    if tree in (FLAT_TS, FLAT_TT, SAMEH_KUCK):
        return sameh_kuck(p, q)
    if tree == BINARY:
        return binary_tree(p, q)
    if tree == FIBONACCI:
        return fibonacci(p, q)
    if tree == GREEDY:
        return greedy(p, q)
    if tree in (PLASMA, PLASMA_TS):
        return plasma_tree(p, q, BS)
    if tree == ASAP:
        return asap(p, q)
    if tree == GRASAP:
        return grasap(p, q, BS)
    raise ValueError("unknown tree %r" % (tree,))


def ts_flags(tree, BS, elims):
    """Kernel family of each elimination: True = TS (TSQRT/TSMQR), False = TT.

    FlatTree-TS uses TS kernels throughout (Proposition 2).  PlasmaTree-TS is
    PlasmaTree with TS kernels inside each domain -- the domain's first row
    zeroes the others with the triangle-on-top-of-square kernels, as the
    library the paper compares against does -- and TT kernels for the binary
    merge of the domain heads.  Domains of column k start at row k, so rows i
    and piv share a domain exactly when (i - k) // BS == (piv - k) // BS.
    Every other tree uses TT kernels.
    """
    if tree == FLAT_TS:
        return [True] * len(elims)
    if tree == PLASMA_TS:
        return [(i - k) // BS == (piv - k) // BS for (i, piv, k) in elims]
    return [False] * len(elims)


# --------------------------------------------------------------------------
# Validity of an elimination list (Section 2.2).
# --------------------------------------------------------------------------
def validate(p, q, elims):
    """Return None if ``elims`` is a valid elimination list, else a reason.

    Rules: exactly one entry per tile (i,k) with i > k, k <= min(p,q);
    both rows ready (every elimination of rows i and piv in columns k' < k
    comes earlier); piv still a potential annihilator (the elimination of
    tile (piv,k), if any, comes later).
    """
    qq = min(p, q)
    pos = {}
    for t, e in enumerate(elims):
        if len(e) != 3:
            return "entry %d is not a triplet" % t
        i, piv, k = e
        if not (1 <= k <= qq):
            return "entry %d: column %d out of range" % (t, k)
        if not (k < i <= p):
            return "entry %d: row %d does not lie below the diagonal" % (t, i)
        if not (k <= piv <= p) or piv == i:
            return "entry %d: pivot %d invalid" % (t, piv)
        if (i, k) in pos:
            return "entry %d: tile (%d,%d) zeroed twice" % (t, i, k)
        pos[(i, k)] = t
    for k in range(1, qq + 1):
        for i in range(k + 1, p + 1):
            if (i, k) not in pos:
                return "tile (%d,%d) never zeroed" % (i, k)
    for t, (i, piv, k) in enumerate(elims):
        for kp in range(1, k):
            for r in (i, piv):
                if pos[(r, kp)] > t:
                    return "entry %d: row %d not ready (tile (%d,%d) zeroed later)" % (t, r, r, kp)
        if piv > k and pos[(piv, k)] < t:
            return "entry %d: pivot row %d already zeroed in column %d" % (t, piv, k)
    return None


# --------------------------------------------------------------------------
# Coarse-grain model (Section 3.1): one time-unit per row-pair transformation.
# --------------------------------------------------------------------------
def coarse_asap(p, q, elims):
    """Time-step of each elimination when every transformation costs one unit
    and a row takes part in one transformation at a time, in list order."""
    busy = [0] * (p + 1)
    steps = {}
    for (i, piv, k) in elims:
        t = max(busy[i], busy[piv]) + 1
        busy[i] = busy[piv] = t
        steps[(i, k)] = t
    return steps


def coarse_greedy(p, q):
    """Coarse-grain Greedy: at every step each column zeroes as many tiles as
    possible, bottom rows first, pairing the z bottom active rows with the z
    rows just above them.  A row zeroed in column k-1 at step s becomes
    active in column k at step s+1.  Returns {(i,k): step}."""
    qq = min(p, q)
    ready_at = {}  # (row, k) -> first step at which row is active in column k
    for r in range(1, p + 1):
        ready_at[(r, 1)] = 1
    zeroed = {}
    step = 0
    while len(zeroed) < sum(p - k for k in range(1, qq + 1)):
        step += 1
        new = []
        for k in range(1, qq + 1):
            active = [r for r in range(k, p + 1)
                      if ready_at.get((r, k), None) is not None
                      and ready_at[(r, k)] <= step and (r, k) not in zeroed]
            active.sort()
            z = len(active) // 2
            for t in range(z):
                row = active[len(active) - z + t]
                new.append((row, k))
        for (row, k) in new:
            zeroed[(row, k)] = step
            if k + 1 <= qq:
                ready_at[(row, k + 1)] = step + 1
    return zeroed


def coarse_fibonacci(p, q):
    """Coarse-grain Fibonacci time-steps from the closed form."""
    return {(i, k): fibonacci_coarse(p, i, k)
            for k in range(1, min(p, q) + 1) for i in range(k + 1, p + 1)}


# --------------------------------------------------------------------------
# ASAP and GRASAP(k) (Section 3.2): dynamic trees on the tiled time model.
# --------------------------------------------------------------------------
def asap(p, q, greedy_columns=0):
    """ASAP: in every column, as soon as at least two rows are ready (their
    tile of the column is a triangle and no elimination is using it), pair
    them.  With 2s ready rows r_1 < ... < r_2s the first is paired with row
    s+1, the second with s+2, ...: r_{s+j} is zeroed by r_j.  With an odd
    number of ready rows the one closest to the diagonal waits.
    GRASAP(k): ``greedy_columns = q - k`` first columns follow Greedy
    (Algorithm 4), the last k columns follow ASAP.  Returns the list (in
    order of decision time, then column, then row)."""
    from . import dag
    qq = min(p, q)
    inc = dag.Incremental(p, q)
    out = []
    zeroed = set()
    busy_until = {}
    if greedy_columns > 0:
        for e in greedy(p, q):
            if e[2] <= greedy_columns:
                out.append(e)
                inc.add_elim(*e)
                zeroed.add((e[0], e[2]))
    total = sum(p - k for k in range(1, qq + 1))
    t = 0
    while len(zeroed) < total:
        progressed = False
        for k in range(greedy_columns + 1, qq + 1):
            ready = []
            for r in range(k, p + 1):
                if (r, k) in zeroed:
                    continue
                if k > 1 and any((r, kp) not in zeroed for kp in range(1, k)):
                    continue
                if busy_until.get(r, 0) > t:
                    continue
                if inc.triangle_time(r, k) <= t:
                    ready.append(r)
            if len(ready) < 2:
                continue
            s = len(ready) // 2
            rows = ready[len(ready) - 2 * s:]
            for jj in range(s):
                piv, i = rows[jj], rows[s + jj]
                out.append((i, piv, k))
                end = inc.add_elim(i, piv, k)
                zeroed.add((i, k))
                busy_until[i] = busy_until[piv] = end
                progressed = True
        t += 1
        if t > 100000 * (p + q) and not progressed:
            raise RuntimeError("ASAP made no progress")
    return out


def grasap(p, q, k):
    """GRASAP(k): Greedy on columns 1..q-k, ASAP on the last k columns."""
    return asap(p, q, greedy_columns=max(0, min(p, q) - k))
