// Host planner of libtqr: elimination lists of the seven trees, the validity
// rules of an elimination list, the TS/TT expansion into kernel tasks, the
// unit-weight critical-path simulator, and the device task graphs.
//
// Paper: "Tiled QR factorization algorithms" (Bouwmeester, Jacquelin, Langou,
// Robert, 2011).  All indices here are 0-based.
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <algorithm>
#include <cstring>

namespace tqr {

// ---------------------------------------------------------------------------
// Elimination lists (Section 3).
// ---------------------------------------------------------------------------

// Sameh-Kuck / FlatTree: column k zeroes rows k+1..p-1 with the panel row k.
static void flat_list(int p, int q, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    for (int k = 0; k < qq; ++k)
        for (int i = k + 1; i < p; ++i) out.push_back({i, k, k});
}

// BinaryTree (Proposition 1): level s = 1,2,4,... zeroes the rows whose
// offset d from the panel row is an odd multiple of s, with the row s above.
static void binary_list(int p, int q, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    for (int k = 0; k < qq; ++k) {
        const int rows = p - k;
        for (int s = 1; s < rows; s *= 2)
            for (int d = s; d < rows; d += 2 * s) out.push_back({k + d, k + d - s, k});
    }
}

// Fibonacci scheme of order 1 (Section 3.1).  In column 1 the rows at offset
// r = i - k + 1 (1-based) from the panel row fall into groups y = 1, 2, ...
// holding the offsets y(y-1)/2+2 .. y(y+1)/2+1; group y is zeroed at coarse
// step x - y + 1, larger groups first.  Column k repeats the pattern shifted
// down by k-1 rows, the bottom group being cut at row p.  Each row of a
// group of z rows is paired with the row z above it.
static void fibonacci_list(int p, int q, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    for (int k = 0; k < qq; ++k) {
        const int rmax = p - k;                    // largest offset r in this column
        if (rmax < 2) continue;
        int ymax = 1;
        while (ymax * (ymax + 1) / 2 + 1 < rmax) ++ymax;
        for (int y = ymax; y >= 1; --y) {
            const int lo = y * (y - 1) / 2 + 2;
            const int hi = std::min(y * (y + 1) / 2 + 1, rmax);
            const int z = hi - lo + 1;
            for (int r = lo; r <= hi; ++r) {
                const int i = k + r - 1;           // 0-based row of offset r
                out.push_back({i, i - z, k});
            }
        }
    }
}

// Greedy for tiles (Algorithm 4).  nT[j] / nZ[j] count the tiles of column j
// that are triangularized / zeroed, from the bottom row upwards.  Each outer
// step sweeps j from right to left, so column j reads nZ[j-1] as it stood at
// the end of the previous step.  The loop ends when every column
// j < min(p,q) holds p-1-j zeros.
static void greedy_list(int p, int q, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    std::vector<int> nZ(q, 0), nT(q, 0);
    auto finished = [&]() {
        for (int j = 0; j < qq; ++j)
            if (nZ[j] != p - 1 - j) return false;
        return true;
    };
    while (!finished()) {
        for (int j = q - 1; j >= 0; --j) {
            const int tri = (j == 0) ? p : nZ[j - 1];
            const int zn = nZ[j] + (nT[j] - nZ[j]) / 2;
            const int shift = zn - nZ[j];
            for (int kk = nZ[j]; kk < zn; ++kk) {
                const int row = p - 1 - kk;
                out.push_back({row, row - shift, j});
            }
            nT[j] = tri;
            nZ[j] = zn;
        }
    }
}

// PlasmaTree(BS) (Section 3.2): flat trees inside domains of BS rows that
// start at the panel row (the bottom domain shrinks as k grows), then a binary
// merge of the domain heads.
static void plasma_list(int p, int q, int BS, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    std::vector<int> heads;
    for (int k = 0; k < qq; ++k) {
        heads.clear();
        for (int h = k; h < p; h += BS) heads.push_back(h);
        for (int h : heads)
            for (int i = h + 1; i < std::min(h + BS, p); ++i) out.push_back({i, h, k});
        const int nh = static_cast<int>(heads.size());
        for (int s = 1; s < nh; s *= 2)
            for (int d = s; d < nh; d += 2 * s) out.push_back({heads[d], heads[d - s], k});
    }
}

// ---------------------------------------------------------------------------
// ASAP and GRASAP(k) (Section 3.2).  These trees are dynamic: the next
// eliminations depend on when rows become ready in the tiled time model, so
// the list is built together with an incremental unit-weight simulation of
// its kernel tasks (Algorithm 3 expansion, producer + last-writer edges).
// ---------------------------------------------------------------------------
namespace {

class IncSim {
public:
    IncSim(int p, int q)
        : p_(p), q_(q), last_(static_cast<size_t>(p) * q, -1), prod_ge_(static_cast<size_t>(p) * q, -1),
          prod_el_(static_cast<size_t>(p) * q, -1), tri_(static_cast<size_t>(p) * q, 0) {}

    // Appends elim(i, piv, k) with TT kernels; returns its TTQRT's finish.
    int64_t add_elim(int i, int piv, int k) {
        factor(piv, k);
        factor(i, k);
        const int64_t t = add(TTQRT, i, piv, k, -1);
        for (int j = k + 1; j < q_; ++j) add(TTMQR, i, piv, k, j);
        return t;
    }

    // Finish of GEQRT(x,k) if it were emitted now.
    int64_t triangle_time(int x, int k) const {
        const size_t a = idx(x, k);
        if (tri_[a]) return fin_[prod_ge_[a]];
        return (last_[a] >= 0 ? fin_[last_[a]] : 0) + kernel_weight(GEQRT);
    }

private:
    int p_, q_;
    std::vector<int64_t> fin_;
    std::vector<int64_t> last_, prod_ge_, prod_el_;
    std::vector<char> tri_;

    size_t idx(int r, int c) const { return static_cast<size_t>(c) * p_ + r; }

    void factor(int x, int k) {
        if (tri_[idx(x, k)]) return;
        tri_[idx(x, k)] = 1;
        add(GEQRT, x, -1, k, -1);
        for (int j = k + 1; j < q_; ++j) add(UNMQR, x, -1, k, j);
    }

    int64_t add(int kind, int i, int piv, int k, int j) {
        int64_t start = 0;
        size_t w[2];
        int nw = 0;
        if (kind == GEQRT) {
            w[nw++] = idx(i, k);
        } else if (kind == UNMQR) {
            start = fin_[prod_ge_[idx(i, k)]];
            w[nw++] = idx(i, j);
        } else if (kind == TTQRT) {
            w[nw++] = idx(piv, k);
            w[nw++] = idx(i, k);
        } else {
            start = fin_[prod_el_[idx(i, k)]];
            w[nw++] = idx(piv, j);
            w[nw++] = idx(i, j);
        }
        for (int a = 0; a < nw; ++a)
            if (last_[w[a]] >= 0) start = std::max(start, fin_[last_[w[a]]]);
        const int64_t t = static_cast<int64_t>(fin_.size());
        fin_.push_back(start + kernel_weight(kind));
        for (int a = 0; a < nw; ++a) last_[w[a]] = t;
        if (kind == GEQRT) prod_ge_[idx(i, k)] = t;
        if (kind == TTQRT) prod_el_[idx(i, k)] = t;
        return fin_.back();
    }
};

}  // namespace

// ASAP: in every column, as soon as two or more rows are ready (tile of the
// column triangularized, row not zeroed in it, not inside an elimination),
// the 2s bottom ready rows are paired first-with-(s+1)-th, second-with-
// (s+2)-th, ...; with an odd count the row nearest the diagonal waits.
// GRASAP(kk): columns 0..q-kk-1 keep the Greedy list, the last kk columns run
// ASAP.  List order: the Greedy part, then decision time, column, pair.
static void asap_list(int p, int q, int greedy_cols, std::vector<Elim>& out) {
    const int qq = std::min(p, q);
    IncSim sim(p, q);
    std::vector<int> zc(p, 0);               // leading columns zeroed in each row
    std::vector<int64_t> busy(p, 0);
    int64_t remaining = 0;
    for (int k = 0; k < qq; ++k) remaining += p - 1 - k;
    if (greedy_cols > 0) {
        std::vector<Elim> g;
        greedy_list(p, q, g);
        for (const Elim& e : g)
            if (e.k < greedy_cols) {
                out.push_back(e);
                sim.add_elim(e.i, e.piv, e.k);
                zc[e.i] = e.k + 1;
                --remaining;
            }
    }
    std::vector<std::vector<int>> ready(qq);
    for (int64_t t = 0; remaining > 0; ++t) {
        for (int k = 0; k < qq; ++k) ready[k].clear();
        for (int r = 0; r < p; ++r) {
            const int k = zc[r];                 // column in which row r is active
            if (k >= qq || k < greedy_cols || r < k) continue;
            if (busy[r] > t || sim.triangle_time(r, k) > t) continue;
            ready[k].push_back(r);
        }
        for (int k = greedy_cols; k < qq; ++k) {
            const std::vector<int>& rd = ready[k];
            const int s = static_cast<int>(rd.size()) / 2;
            if (s < 1) continue;
            const int base = static_cast<int>(rd.size()) - 2 * s;
            for (int a = 0; a < s; ++a) {
                const int piv = rd[base + a], i = rd[base + s + a];
                out.push_back({i, piv, k});
                const int64_t end = sim.add_elim(i, piv, k);
                zc[i] = k + 1;
                busy[i] = busy[piv] = end;
                --remaining;
            }
        }
    }
}

int make_elims(int p, int q, int tree, int BS, std::vector<Elim>& out) {
    out.clear();
    switch (tree) {
        case TQR_FLAT_TS:
        case TQR_FLAT_TT:
        case TQR_SAMEH_KUCK: flat_list(p, q, out); return TQR_OK;
        case TQR_BINARY: binary_list(p, q, out); return TQR_OK;
        case TQR_FIBONACCI: fibonacci_list(p, q, out); return TQR_OK;
        case TQR_GREEDY: greedy_list(p, q, out); return TQR_OK;
        case TQR_PLASMA:
        case TQR_PLASMA_TS:
            if (BS < 1 || BS > p) return -4;
            plasma_list(p, q, BS, out);
            return TQR_OK;
        case TQR_ASAP: asap_list(p, q, 0, out); return TQR_OK;
        case TQR_GRASAP:
            if (BS < 0 || BS > std::min(p, q)) return -4;
            asap_list(p, q, std::min(p, q) - BS, out);
            return TQR_OK;
        default: return -3;
    }
}

// ---------------------------------------------------------------------------
// Validity rules (Section 2.2).
// ---------------------------------------------------------------------------
int validate_elims(int p, int q, const Elim* e, int64_t count) {
    const int qq = std::min(p, q);
    if (p < 1 || q < 1 || p < q) return TQR_ERR_INVALID_LIST;
    std::vector<int64_t> pos(static_cast<size_t>(p) * qq, -1);
    auto at = [&](int i, int k) -> int64_t& { return pos[static_cast<size_t>(k) * p + i]; };
    for (int64_t t = 0; t < count; ++t) {
        const Elim& x = e[t];
        if (x.k < 0 || x.k >= qq) return TQR_ERR_INVALID_LIST;
        if (x.i <= x.k || x.i >= p) return TQR_ERR_INVALID_LIST;
        if (x.piv < x.k || x.piv >= p || x.piv == x.i) return TQR_ERR_INVALID_LIST;
        if (at(x.i, x.k) >= 0) return TQR_ERR_INVALID_LIST;   // zeroed twice
        at(x.i, x.k) = t;
    }
    for (int k = 0; k < qq; ++k)
        for (int i = k + 1; i < p; ++i)
            if (at(i, k) < 0) return TQR_ERR_INVALID_LIST;    // never zeroed
    for (int64_t t = 0; t < count; ++t) {
        const Elim& x = e[t];
        for (int kp = 0; kp < x.k; ++kp)                         // both rows ready
            if (at(x.i, kp) > t || at(x.piv, kp) > t) return TQR_ERR_INVALID_LIST;
        if (x.piv > x.k && at(x.piv, x.k) < t) return TQR_ERR_INVALID_LIST;  // annihilator
    }
    return TQR_OK;
}

// ---------------------------------------------------------------------------
// TS / TT expansion (Algorithms 2 and 3).  A tile already in triangle form
// is not factored again.  In TT every tile (x,k), x >= k, is factored once,
// at the first elimination of column k that involves row x; the diagonal
// tile of the last column of a square matrix, which takes part in no
// elimination, is factored at the end.
// ---------------------------------------------------------------------------
// Kernel family per elimination (1 = TS, 0 = TT).  FlatTree-TS is TS
// throughout; PlasmaTree-TS uses TS when row i lies in its pivot's domain
// (domains of column k start at row k, BS rows each) and TT for the merges of
// domain heads; every other tree is TT.
std::vector<char> ts_flags(int tree, int BS, const std::vector<Elim>& elims) {
    std::vector<char> f(elims.size(), tree == TQR_FLAT_TS ? 1 : 0);
    if (tree == TQR_PLASMA_TS)
        for (size_t t = 0; t < elims.size(); ++t)
            f[t] = (elims[t].i - elims[t].k) / BS == (elims[t].piv - elims[t].k) / BS;
    return f;
}

bool expand_tasks(int p, int q, const std::vector<Elim>& elims, bool ts, std::vector<TileTask>& out) {
    return expand_tasks(p, q, elims, std::vector<char>(elims.size(), ts ? 1 : 0), out);
}

// Returns false when a TS elimination meets a tile already in triangle form
// (a row that was a pivot earlier in the same column): the TS kernels need a
// square tile there, so such a list is invalid for them.
bool expand_tasks(int p, int q, const std::vector<Elim>& elims, const std::vector<char>& ts_of,
                  std::vector<TileTask>& out) {
    out.clear();
    std::vector<char> tri(static_cast<size_t>(p) * q, 0);
    auto factor = [&](int x, int k) {
        char& f = tri[static_cast<size_t>(k) * p + x];
        if (f) return;
        f = 1;
        out.push_back({GEQRT, x, -1, k, -1});
        for (int j = k + 1; j < q; ++j) out.push_back({UNMQR, x, -1, k, j});
    };
    for (size_t t = 0; t < elims.size(); ++t) {
        const Elim& e = elims[t];
        const bool ts = ts_of[t] != 0;
        if (ts && tri[static_cast<size_t>(e.k) * p + e.i]) return false;
        factor(e.piv, e.k);
        if (!ts) factor(e.i, e.k);
        out.push_back({ts ? TSQRT : TTQRT, e.i, e.piv, e.k, -1});
        for (int j = e.k + 1; j < q; ++j) out.push_back({ts ? TSMQR : TTMQR, e.i, e.piv, e.k, j});
    }
    for (int k = 0; k < std::min(p, q); ++k) factor(k, k);
    return true;
}

// Dependencies of tile tasks: the producer of the reflectors a task applies,
// and the previous writer (in program order) of every tile it writes.
// Readers of V never delay a writer of the other half of the tile (V: NODEP,
// T: INPUT, Section 4), hence no write-after-read edges.
template <class Fn>
static void for_each_dep(int p, int q, const std::vector<TileTask>& tasks, Fn&& fn) {
    const size_t nt = static_cast<size_t>(p) * q;
    std::vector<int64_t> last(nt, -1), prod_ge(nt, -1), prod_el(nt, -1);
    auto idx = [&](int r, int c) { return static_cast<size_t>(c) * p + r; };
    int64_t d[4];
    for (int64_t t = 0; t < static_cast<int64_t>(tasks.size()); ++t) {
        const TileTask& x = tasks[t];
        int nd = 0;
        size_t w[2];
        int nw = 0;
        switch (x.kind) {
            case GEQRT: w[nw++] = idx(x.i, x.k); prod_ge[idx(x.i, x.k)] = t; break;
            case UNMQR: d[nd++] = prod_ge[idx(x.i, x.k)]; w[nw++] = idx(x.i, x.j); break;
            case TTQRT:
            case TSQRT:
                w[nw++] = idx(x.piv, x.k); w[nw++] = idx(x.i, x.k);
                prod_el[idx(x.i, x.k)] = t;
                break;
            default:  // TTMQR, TSMQR
                d[nd++] = prod_el[idx(x.i, x.k)];
                w[nw++] = idx(x.piv, x.j); w[nw++] = idx(x.i, x.j);
                break;
        }
        for (int a = 0; a < nw; ++a) d[nd++] = last[w[a]];
        for (int a = 0; a < nw; ++a) last[w[a]] = t;
        fn(t, d, nd);
    }
}

int64_t simulate(int p, int q, const std::vector<TileTask>& tasks, std::vector<int64_t>* finish) {
    std::vector<int64_t> fin(tasks.size(), 0);
    int64_t cp = 0;
    for_each_dep(p, q, tasks, [&](int64_t t, const int64_t* d, int nd) {
        int64_t s = 0;
        for (int a = 0; a < nd; ++a)
            if (d[a] >= 0) s = std::max(s, fin[d[a]]);
        fin[t] = s + kernel_weight(tasks[t].kind);
        cp = std::max(cp, fin[t]);
    });
    if (finish) finish->swap(fin);
    return cp;
}

// ---------------------------------------------------------------------------
// Device task graphs.
// ---------------------------------------------------------------------------
static void finish_graph(const std::vector<std::pair<int32_t, int32_t>>& edges, Graph& g) {
    const size_t nt = g.tasks.size();
    g.indeg.assign(nt, 0);
    g.succ_ptr.assign(nt + 1, 0);
    for (auto& e : edges) { g.succ_ptr[e.first + 1]++; g.indeg[e.second]++; }
    for (size_t t = 0; t < nt; ++t) g.succ_ptr[t + 1] += g.succ_ptr[t];
    g.succ.assign(edges.size(), 0);
    std::vector<int32_t> fill(g.succ_ptr.begin(), g.succ_ptr.end() - 1);
    for (auto& e : edges) g.succ[fill[e.first]++] = e.second;
    g.ready.clear();
    for (size_t t = 0; t < nt; ++t)
        if (g.indeg[t] == 0) g.ready.push_back(static_cast<int32_t>(t));
}

// Tiles of fewer than 128 columns stay whole: their blocks are too small for
// a task each to pay for its scheduling.
bool split_panels(int nb, int ib) { return nb >= 128 && ib >= 8 && nb / ib >= 2; }

// Updates are split into strips of W columns.  Panels are one task each, or,
// when split_panels(nb, ib), one task per block b of ib columns that factors
// it, then tasks that apply it to the columns right of it: first the next
// look-ahead columns (max(ib, 32) of them, which the next block's factor
// waits for), then the rest in strips of W.
//
// Writers of a tile are chained per cell of (row block, column unit) --
// blocks of ib rows (all nb rows when panels stay whole) and units of
// gcd(ib, W) columns -- in list order: a task depends on the last writer of
// every cell it writes, and a task applying reflectors on the task that
// formed them (for an update of another tile column: the factor task of the
// panel's last block, which follows every other task of the panel).  Rows a
// task writes: block b of GEQRT rows [b ib, nb) of its tile; of TTQRT rows
// [0, (b+1) ib) of the zeroed tile and [b ib, (b+1) ib) of the pivot tile;
// of TSQRT all rows of the zeroed tile and [b ib, (b+1) ib) of the pivot;
// whole panels and update strips all rows.  So block b of an elimination
// waits only for the blocks <= b of the tasks before it on those rows, and
// the elimination tree proceeds as a wavefront over column blocks.  Panel
// factor tasks, look-ahead updates and the updates of the next tile column
// (k + 1) carry kHighPriority.  Readers
// of a panel's reflectors do not wait for later writers of the other
// triangle of the same tile (the reflectors' NODEP of Section 4).
void build_factor_graph(int p, int q, int nb, int ib, int W, int n_cols_last,
                        const std::vector<TileTask>& tt, Graph& g) {
    const bool split = split_panels(nb, ib);
    int cu = W;                                       // column unit of the writer chains
    if (split) {
        int a = ib, b = W;
        while (b) { const int r = a % b; a = b; b = r; }
        cu = a;
    }
    const int rbs = split ? ib : nb;                  // rows per row block
    const int umax = (nb + cu - 1) / cu, rmax = (nb + rbs - 1) / rbs;
    const int cells = umax * rmax;
    auto cols_of = [&](int j) { return (j == q - 1) ? n_cols_last : nb; };
    const size_t ntile = static_cast<size_t>(p) * q;
    std::vector<int32_t> last(ntile * cells, -1), prod(ntile * 2, -1);
    auto L = [&](int r, int c, int rb, int u) -> int32_t& {
        return last[(static_cast<size_t>(c) * p + r) * cells + static_cast<size_t>(rb) * umax + u];
    };
    g.tasks.clear();
    std::vector<std::pair<int32_t, int32_t>> edges;
    edges.reserve(tt.size() * 4);
    std::vector<int32_t> deps;
    deps.reserve(2 * cells + 4);
    auto add_edges = [&](int32_t t) {
        std::sort(deps.begin(), deps.end());
        for (size_t a = 0; a < deps.size(); ++a)
            if (deps[a] >= 0 && (a == 0 || deps[a] != deps[a - 1])) edges.push_back({deps[a], t});
        deps.clear();
    };
    // Task t writes rows [r0, r1) of columns [c0, c1) of tile (tr, tc).
    auto writes = [&](int32_t t, int tr, int tc, int r0, int r1, int c0, int c1) {
        const int u0 = c0 / cu, u1 = (c1 + cu - 1) / cu;
        const int b0 = r0 / rbs, b1 = (r1 + rbs - 1) / rbs;
        for (int rb = b0; rb < b1; ++rb)
            for (int u = u0; u < u1; ++u) {
                deps.push_back(L(tr, tc, rb, u));
                L(tr, tc, rb, u) = t;
            }
    };
    auto push = [&](int32_t kind, int i, int piv, int k, int j, int strip) {
        const int32_t t = static_cast<int32_t>(g.tasks.size());
        g.tasks.push_back({kind, i, piv, k, j, strip});
        return t;
    };
    // Rows block b of a panel of `kind` writes in the zeroed / factored tile
    // (bottom) and in the pivot tile (top).
    auto panel_rows = [&](int kind, int b, int* blo, int* bhi, int* tlo, int* thi) {
        const int j0 = b * ib;
        *blo = (kind == GEQRT) ? j0 : 0;
        *bhi = (kind == TTQRT) ? std::min(nb, j0 + ib) : nb;
        *tlo = j0;
        *thi = std::min(nb, j0 + ib);
    };
    const int la = ((ib > 32 ? ib : 32) + ib - 1) / ib * ib;   // look-ahead columns
    for (const TileTask& x : tt) {
        if (x.kind == GEQRT || x.kind == TTQRT || x.kind == TSQRT) {
            const bool pair = x.kind != GEQRT;
            const int ncol = cols_of(x.k);
            int32_t sink;
            if (!split) {
                sink = push(x.kind | kHighPriority, x.i, x.piv, x.k, -1, 0);
                writes(sink, x.i, x.k, 0, nb, 0, ncol);
                if (pair) writes(sink, x.piv, x.k, 0, nb, 0, ncol);
                add_edges(sink);
            } else {
                int32_t prev = -1;
                for (int b = 0; b < nb / ib; ++b) {
                    const int j0 = b * ib;
                    int blo, bhi, tlo, thi;
                    panel_rows(x.kind, b, &blo, &bhi, &tlo, &thi);
                    const int32_t f = push(x.kind | kHighPriority, x.i, x.piv, x.k, b, -1);
                    deps.push_back(prev);
                    if (j0 < ncol) {
                        const int c1 = std::min(j0 + ib, ncol);
                        writes(f, x.i, x.k, blo, bhi, j0, c1);
                        if (pair) writes(f, x.piv, x.k, tlo, thi, j0, c1);
                    }
                    add_edges(f);
                    prev = f;
                    for (int c0 = j0 + ib; c0 < ncol;) {
                        const int c1 = std::min(ncol, c0 == j0 + ib ? c0 + la : c0 + W);
                        const int32_t hp = (c0 == j0 + ib) ? kHighPriority : 0;   // the look-ahead part
                        const int32_t u = push(x.kind | hp, x.i, x.piv, x.k, b, c0 | (c1 << 16));
                        deps.push_back(f);
                        writes(u, x.i, x.k, blo, bhi, c0, c1);
                        if (pair) writes(u, x.piv, x.k, tlo, thi, c0, c1);
                        add_edges(u);
                        c0 = c1;
                    }
                }
                sink = prev;
            }
            prod[(static_cast<size_t>(x.k) * p + x.i) * 2 + (x.kind == GEQRT ? 0 : 1)] = sink;
        } else {
            const int32_t pr = prod[(static_cast<size_t>(x.k) * p + x.i) * 2 + (x.kind == UNMQR ? 0 : 1)];
            const int ncol = cols_of(x.j);
            const int32_t hp = (x.j == x.k + 1) ? kHighPriority : 0;      // feeds the next panel column
            for (int s = 0; s * W < ncol; ++s) {
                const int32_t t = push(x.kind | hp, x.i, x.piv, x.k, x.j, s);
                const int c0 = s * W, c1 = std::min(ncol, (s + 1) * W);
                deps.push_back(pr);
                writes(t, x.i, x.j, 0, nb, c0, c1);
                if (x.kind != UNMQR) writes(t, x.piv, x.j, 0, nb, c0, c1);
                add_edges(t);
            }
        }
    }
    finish_graph(edges, g);
}

void build_apply_graph(int p, const std::vector<TileTask>& tt, int nstrips, bool trans, Graph& g) {
    std::vector<const TileTask*> panels;
    for (const TileTask& x : tt)
        if (x.kind == GEQRT || x.kind == TTQRT || x.kind == TSQRT) panels.push_back(&x);
    if (!trans) std::reverse(panels.begin(), panels.end());
    std::vector<int32_t> last(static_cast<size_t>(p) * nstrips, -1);
    g.tasks.clear();
    std::vector<std::pair<int32_t, int32_t>> edges;
    for (const TileTask* x : panels) {
        const int kind = (x->kind == GEQRT) ? UNMQR : (x->kind == TTQRT ? TTMQR : TSMQR);
        for (int s = 0; s < nstrips; ++s) {
            const int32_t t = static_cast<int32_t>(g.tasks.size());
            g.tasks.push_back({kind, x->i, x->piv, x->k, -1, s});
            int32_t& a = last[static_cast<size_t>(x->i) * nstrips + s];
            if (a >= 0) edges.push_back({a, t});
            a = t;
            if (kind != UNMQR) {
                int32_t& b = last[static_cast<size_t>(x->piv) * nstrips + s];
                if (b >= 0) edges.push_back({b, t});
                b = t;
            }
        }
    }
    finish_graph(edges, g);
}

}  // namespace tqr
