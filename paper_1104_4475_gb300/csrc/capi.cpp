// C ABI of libtqr (declared in include/tqr.h): argument checking, the cache of
// task-graph plans, factorization handles, and the host-only integer entry
// points.  No C++ exception crosses this boundary.
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

namespace tqr {

// A task graph uploaded to the device.
struct DevGraphOwner {
    DevGraph d;
    ~DevGraphOwner() {
        cudaFree(d.tasks);
        cudaFree(d.succ_ptr);
        cudaFree(d.succ);
        cudaFree(d.indeg);
        cudaFree(d.ready);
    }
};

template <class T>
static cudaError_t upload(T** dst, const std::vector<T>& src) {
    *dst = nullptr;
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

static cudaError_t upload_graph(const Graph& g, DevGraphOwner& o) {
    cudaError_t e;
    if ((e = upload(&o.d.tasks, g.tasks)) != cudaSuccess) return e;
    if ((e = upload(&o.d.succ_ptr, g.succ_ptr)) != cudaSuccess) return e;
    if ((e = upload(&o.d.succ, g.succ)) != cudaSuccess) return e;
    if ((e = upload(&o.d.indeg, g.indeg)) != cudaSuccess) return e;
    // The initially ready tasks, high-priority ones first (program order kept).
    std::vector<int32_t> ready;
    ready.reserve(g.ready.size());
    for (int32_t t : g.ready)
        if (g.tasks[t].kind & kHighPriority) ready.push_back(t);
    o.d.nready_hi = static_cast<int32_t>(ready.size());
    for (int32_t t : g.ready)
        if (!(g.tasks[t].kind & kHighPriority)) ready.push_back(t);
    o.d.n_hi = 0;
    for (const DevTask& x : g.tasks)
        if (x.kind & kHighPriority) ++o.d.n_hi;
    if ((e = upload(&o.d.ready, ready)) != cudaSuccess) return e;
    o.d.ntasks = static_cast<int32_t>(g.tasks.size());
    o.d.nready = static_cast<int32_t>(g.ready.size());
    o.d.nedges = static_cast<int64_t>(g.succ.size());
    return cudaSuccess;
}

struct PlanKey {
    int64_t m, n;
    int nb, ib, tree, BS, ts, device;
    std::vector<Elim> list;   // only for caller-given lists (tree = -1)
    bool operator<(const PlanKey& o) const {
        auto a = std::tie(m, n, nb, ib, tree, BS, ts, device);
        auto b = std::tie(o.m, o.n, o.nb, o.ib, o.tree, o.BS, o.ts, o.device);
        if (a != b) return a < b;
        if (list.size() != o.list.size()) return list.size() < o.list.size();
        return std::memcmp(list.data(), o.list.data(), list.size() * sizeof(Elim)) < 0;
    }
};

// Everything derived from (m, n, nb, ib, elimination list, kernel family).
struct Plan {
    PlanKey key;
    int p = 0, q = 0, G = 0, W = 0, smem = 0;
    int ts = 0;                // 0 TT, 1 TS, 2 TS inside PlasmaTree domains
    std::vector<Elim> elims;
    std::vector<TileTask> tt;
    int64_t cp = 0;
    Graph g;
    DevGraphOwner dg;
    int32_t* d_panels = nullptr;   // (kind, i, k) of every panel task
    int npanels = 0;
    std::mutex mu;
    std::map<std::pair<int, int>, std::unique_ptr<DevGraphOwner>> apply;   // (nstrips, trans)
    ~Plan() { cudaFree(d_panels); }
};

static std::mutex g_plans_mu;
static std::map<PlanKey, std::shared_ptr<Plan>>& plans() {
    static auto* m = new std::map<PlanKey, std::shared_ptr<Plan>>();   // lives until exit
    return *m;
}

// Trees whose BS argument matters (PlasmaTree domain size, GRASAP's k).
static bool uses_bs(int tree) { return tree == TQR_PLASMA || tree == TQR_PLASMA_TS || tree == TQR_GRASAP; }

// Kernel family recorded in the plan key: 0 TT, 1 TS, 2 TS inside domains.
static int kernel_mode(int tree) { return tree == TQR_FLAT_TS ? 1 : tree == TQR_PLASMA_TS ? 2 : 0; }

// The plan key of a factorization with a generated tree on device `dev`
// (Sameh-Kuck lowers to the same TT list as FlatTree).
static PlanKey tree_key(int64_t m, int64_t n, int nb, int ib, int tree, int BS, int dev) {
    return PlanKey{m, n, nb, ib, tree == TQR_SAMEH_KUCK ? TQR_FLAT_TT : tree, uses_bs(tree) ? BS : 0,
                   kernel_mode(tree), dev, {}};
}

static bool same_key(const PlanKey& a, const PlanKey& b) { return !(a < b) && !(b < a); }

static double lapack_flops(int64_t m, int64_t n) {
    const double M = static_cast<double>(m), N = static_cast<double>(n);
    return 2.0 * N * N * (M - N / 3.0);
}

// Upper bound of the device tasks of a factorization graph: at most q tile
// tasks per elimination and tile (p q of them), each update split into at
// most nb / 8 + 1 strips, plus, for split panels, at most nb / 8 blocks per
// panel (two panels per tile) with at most nb / 8 + 2 tasks each.  Task ids
// are int32 on the device.
static bool plan_fits(int64_t p, int64_t q, int nb) {
    const double pq = static_cast<double>(p) * q;
    const double bound = pq * (q + 1) * (nb / 8 + 1) + 2.0 * pq * (nb / 8) * (nb / 8 + 2);
    return bound < 2.0e9;
}

static int make_plan(const PlanKey& key, std::shared_ptr<Plan>& out) {
    auto P = std::make_shared<Plan>();
    P->key = key;
    P->p = static_cast<int>((key.m + key.nb - 1) / key.nb);
    P->q = static_cast<int>((key.n + key.nb - 1) / key.nb);
    if (!plan_fits(P->p, P->q, key.nb)) return TQR_ERR_CAPACITY;
    P->ts = key.ts;
    if (key.tree >= 0) {
        int rc = make_elims(P->p, P->q, key.tree, key.BS, P->elims);
        if (rc != TQR_OK) return rc;
    } else {
        P->elims = key.list;
    }
    if (validate_elims(P->p, P->q, P->elims.data(), static_cast<int64_t>(P->elims.size())) != TQR_OK)
        return TQR_ERR_INVALID_LIST;
    const std::vector<char> ts_of = key.tree >= 0 ? ts_flags(key.tree, key.BS, P->elims)
                                                  : std::vector<char>(P->elims.size(), key.ts ? 1 : 0);
    if (!expand_tasks(P->p, P->q, P->elims, ts_of, P->tt)) return TQR_ERR_INVALID_LIST;
    P->cp = simulate(P->p, P->q, P->tt, nullptr);
    if (!choose_layout(key.nb, key.ib, &P->G, &P->smem)) return TQR_ERR_UNSUPPORTED;
    P->W = strip_width(P->G);
    const int last_cols = static_cast<int>(key.n - static_cast<int64_t>(P->q - 1) * key.nb);
    build_factor_graph(P->p, P->q, key.nb, key.ib, P->W, last_cols, P->tt, P->g);
    if (upload_graph(P->g, P->dg) != cudaSuccess) return TQR_ERR_CUDA;
    std::vector<int32_t> panels;
    for (const TileTask& x : P->tt)
        if (x.kind == GEQRT || x.kind == TTQRT || x.kind == TSQRT) {
            panels.push_back(x.kind);
            panels.push_back(x.i);
            panels.push_back(x.k);
        }
    P->npanels = static_cast<int>(panels.size() / 3);
    if (upload(&P->d_panels, panels) != cudaSuccess) return TQR_ERR_CUDA;
    out = P;
    return TQR_OK;
}

static int get_plan(const PlanKey& key, std::shared_ptr<Plan>& out) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    auto it = plans().find(key);
    if (it != plans().end()) {
        out = it->second;
        return TQR_OK;
    }
    std::shared_ptr<Plan> P;
    int rc = make_plan(key, P);
    if (rc != TQR_OK) return rc;
    plans()[key] = P;
    out = P;
    return TQR_OK;
}

static int get_apply_graph(Plan& P, int nstrips, bool trans, const DevGraph** out) {
    std::lock_guard<std::mutex> lk(P.mu);
    auto key = std::make_pair(nstrips, trans ? 1 : 0);
    auto it = P.apply.find(key);
    if (it == P.apply.end()) {
        Graph g;
        build_apply_graph(P.p, P.tt, nstrips, trans, g);
        auto o = std::make_unique<DevGraphOwner>();
        if (upload_graph(g, *o) != cudaSuccess) return TQR_ERR_CUDA;
        it = P.apply.emplace(key, std::move(o)).first;
    }
    *out = &it->second->d;
    return TQR_OK;
}

// Process-wide test hooks; atomic because any host thread may set them while
// another launches.
static std::atomic<double> g_timeout_ms{0.0};   // set by tqr_set_timeout_ms
static std::atomic<int> g_fault{0};             // set by tqr_inject_fault

uint64_t exec_timeout_ns(double flops) {
    const double ms = g_timeout_ms.load();
    if (ms > 0) return static_cast<uint64_t>(ms * 1e6);
    if (const char* s = std::getenv("TQR_TIMEOUT_MS")) {
        const double env_ms = std::atof(s);
        if (env_ms > 0) return static_cast<uint64_t>(env_ms * 1e6);
    }
    // Longest legitimate wait is below the whole run; assume >= 50 GFLOP/s.
    return static_cast<uint64_t>((10.0 + flops / 5e10) * 1e9);
}

static void free_state(ExecState& s) {
    cudaFree(s.deps);
    cudaFree(s.queue);
    cudaFree(s.ctr);
    s = ExecState();
}

static cudaError_t alloc_state(ExecState& s, int32_t cap, int32_t* status) {
    free_state(s);
    cudaError_t e;
    const size_t n = std::max<int32_t>(1, cap);
    if ((e = cudaMalloc(&s.deps, n * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s.queue, n * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s.ctr, 4 * sizeof(uint32_t))) != cudaSuccess) return e;
    s.status = status;
    s.capacity = cap;
    return cudaSuccess;
}

// Host-side plan of one matrix of a batch: its factor graph for strips of W.
struct HostPlan {
    int p = 0, q = 0;
    int64_t cp = 0;
    Graph g;
};

static std::mutex g_hplans_mu;
static std::map<std::tuple<int64_t, int64_t, int, int, int, int, int>, std::shared_ptr<HostPlan>>& hplans() {
    static auto* m = new std::map<std::tuple<int64_t, int64_t, int, int, int, int, int>, std::shared_ptr<HostPlan>>();
    return *m;
}

static int host_plan(int64_t m, int64_t n, int nb, int ib, int tree, int BS, int W, std::shared_ptr<HostPlan>& out) {
    const auto key = std::make_tuple(m, n, nb, ib, tree, BS, W);
    {
        std::lock_guard<std::mutex> lk(g_hplans_mu);
        auto it = hplans().find(key);
        if (it != hplans().end()) {
            out = it->second;
            return TQR_OK;
        }
    }
    auto H = std::make_shared<HostPlan>();
    H->p = static_cast<int>((m + nb - 1) / nb);
    H->q = static_cast<int>((n + nb - 1) / nb);
    std::vector<Elim> el;
    int rc = make_elims(H->p, H->q, tree, BS, el);
    if (rc != TQR_OK) return rc;
    std::vector<TileTask> tt;
    if (!expand_tasks(H->p, H->q, el, ts_flags(tree, BS, el), tt)) return TQR_ERR_INVALID_LIST;
    H->cp = simulate(H->p, H->q, tt, nullptr);
    build_factor_graph(H->p, H->q, nb, ib, W, static_cast<int>(n - static_cast<int64_t>(H->q - 1) * nb), tt, H->g);
    std::lock_guard<std::mutex> lk(g_hplans_mu);
    hplans()[key] = H;
    out = H;
    return TQR_OK;
}

}  // namespace tqr

using namespace tqr;

struct tqr_batch {
    int count = 0;
    bool f32 = false;          // FP32 matrices (tqr_factor_batched_f32)
    std::vector<double*> A;    // identity of the matrices (FP32 pointers stored as is)
    std::vector<int64_t> m, n;
    std::vector<int32_t> nb, ib, tree, BS;
    DevGraphOwner dg;
    MatDesc* d_mats = nullptr;
    double* tau_ge = nullptr;
    double* tau_el = nullptr;
    int32_t* status = nullptr;
    ExecState st;
    int G = 4, smem = 0;
    int64_t max_cp = 0;
    double flops = 0.0;
    cudaStream_t stream = nullptr;
    // Matrices on the one-tile-column FlatTree-TS kernel: descriptors by
    // thread count (1024, 512, 256), largest first within each, and the
    // queues of the one persistent launch that runs them all.
    Ts1Desc* ts1 = nullptr;
    Ts1Phases ts1_ph{};
    int n_fused = 0;
    bool has_exec = false;
    ~tqr_batch() {
        cudaFree(ts1);
        cudaFree(d_mats);
        cudaFree(tau_ge);
        cudaFree(tau_el);
        cudaFree(status);
        cudaFree(st.deps);
        cudaFree(st.queue);
        cudaFree(st.ctr);
    }
    bool same(int c, double* const* a, const int64_t* mm, const int64_t* nn, const int32_t* b, const int32_t* ii,
              const int32_t* tr, const int32_t* bs) const {
        if (c != count) return false;
        for (int x = 0; x < c; ++x)
            if (A[x] != a[x] || m[x] != mm[x] || n[x] != nn[x] || nb[x] != b[x] || ib[x] != ii[x] ||
                tree[x] != tr[x] || BS[x] != bs[x])
                return false;
        return true;
    }
};

struct tqr_factors {
    std::shared_ptr<Plan> plan;
    double* A = nullptr;
    cudaStream_t stream = nullptr;
    double* tau_ge = nullptr;
    double* tau_el = nullptr;
    int32_t* status = nullptr;
    ExecState fst, ast;
    float* T_ge = nullptr;       // compact-WY T blocks, FP32 (low-precision factorizations)
    float* T_el = nullptr;
    float* V_ge = nullptr;       // reflectors in FP32 with unit/zero structure (same)
    float* V_el = nullptr;
    int prec = 0;
    uint64_t* trace = nullptr;   // per-task (start, duration | sm << 56) when tracing
    int trace_on = 0;
    double* own_A = nullptr;     // device copies used by tqr_factor_host
    double* own_B = nullptr;
    size_t own_B_elems = 0;
    ~tqr_factors() {
        free_state(fst);
        free_state(ast);
        cudaFree(tau_ge);
        cudaFree(tau_el);
        cudaFree(T_ge);
        cudaFree(T_el);
        cudaFree(V_ge);
        cudaFree(V_el);
        cudaFree(trace);
        cudaFree(status);
        cudaFree(own_A);
        cudaFree(own_B);
    }
};

// A launch's graph, with the initially ready tasks dropped when a fault
// injection is pending (the counters and edges are untouched).
namespace tqr {
DevGraph graph_for_launch(const DevGraph& g) {
    DevGraph x = g;
    if (g_fault.exchange(0) == 1) x.nready = x.nready_hi = 0;   // one launch consumes the injection
    return x;
}
}  // namespace tqr
using tqr::graph_for_launch;

static ExecParams base_params(const tqr_factors* f) {
    const Plan& P = *f->plan;
    ExecParams x{};
    x.A = f->A;
    x.lda = P.key.m;
    x.m = P.key.m;
    x.n = P.key.n;
    x.nb = P.key.nb;
    x.ib = P.key.ib;
    x.p = P.p;
    x.q = P.q;
    x.tau_ge = f->tau_ge;
    x.tau_el = f->tau_el;
    x.trans = 1;
    x.prec = f->prec;
    x.T_ge = f->T_ge;
    x.T_el = f->T_el;
    x.V_ge = f->V_ge;
    x.V_el = f->V_el;
    x.trace = nullptr;
    x.mats = nullptr;
    x.timeout_ns = exec_timeout_ns(lapack_flops(P.key.m, P.key.n));
    return x;
}

// TQR_TRACE set (and not "0") in the environment: every new handle records
// per-task traces, as if tqr_set_trace(f, 1) had been called.
static bool trace_from_env() {
    static const bool on = [] {
        const char* e = std::getenv("TQR_TRACE");
        return e && e[0] && !(e[0] == '0' && e[1] == 0);
    }();
    return on;
}

static int new_handle(const std::shared_ptr<Plan>& plan, tqr_factors** out) {
    tqr_factors* f = new (std::nothrow) tqr_factors();
    if (!f) return TQR_ERR_NOMEM;
    f->plan = plan;
    f->trace_on = trace_from_env() ? 1 : 0;
    const size_t ntau = static_cast<size_t>(plan->p) * plan->q * plan->key.nb;
    if (cudaMalloc(&f->tau_ge, ntau * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f->tau_el, ntau * sizeof(double)) != cudaSuccess ||
        cudaMemset(f->tau_ge, 0, ntau * sizeof(double)) != cudaSuccess ||     // slots no reflector uses stay 0
        cudaMemset(f->tau_el, 0, ntau * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f->status, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(f->status, 0, sizeof(int32_t)) != cudaSuccess ||
        alloc_state(f->fst, plan->dg.d.ntasks, f->status) != cudaSuccess) {
        delete f;
        return TQR_ERR_NOMEM;
    }
    *out = f;
    return TQR_OK;
}

static int run_factor(const PlanKey& key, double* A, void* stream, tqr_factors** out, int prec = 0) {
    std::shared_ptr<Plan> plan;
    int rc = get_plan(key, plan);
    if (rc != TQR_OK) return rc;
    int smem = plan->smem;
    if (prec != 0) {
        if (!lp_supported(key.nb, key.ib, plan->G)) return TQR_ERR_UNSUPPORTED;
        smem = std::max(smem, lp_smem_bytes(key.nb, key.ib, plan->G));
        int dev = 0, maxsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (smem > maxsm - 1024) return TQR_ERR_UNSUPPORTED;
    }
    tqr_factors* f = *out;
    if (f && f->plan && same_key(f->plan->key, key)) {
        f->plan = plan;                       // same graph (the cached copy may have been released)
    } else {
        f = nullptr;
        rc = new_handle(plan, &f);
        if (rc != TQR_OK) return rc;
    }
    if (prec != 0 && !f->T_ge) {
        const size_t nt = static_cast<size_t>(plan->p) * plan->q * key.ib * key.nb;
        const size_t nv = static_cast<size_t>(plan->p) * plan->q * key.nb * key.nb;
        if (cudaMalloc(&f->T_ge, nt * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&f->T_el, nt * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&f->V_ge, nv * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&f->V_el, nv * sizeof(float)) != cudaSuccess) {
            if (f != *out) delete f;
            return TQR_ERR_NOMEM;
        }
    }
    f->A = A;
    f->prec = prec;
    f->stream = static_cast<cudaStream_t>(stream);
    if (f->trace_on && !f->trace) {
        if (cudaMalloc(&f->trace, 2 * sizeof(uint64_t) * std::max<int32_t>(1, plan->dg.d.ntasks)) != cudaSuccess) {
            f->trace = nullptr;
            if (f != *out) delete f;
            return TQR_ERR_NOMEM;
        }
    }
    ExecParams P = base_params(f);
    P.trace = f->trace_on ? f->trace : nullptr;
    cudaError_t e = launch_factor_exec(P, graph_for_launch(plan->dg.d), f->fst, plan->G, smem, true, f->stream);
    *out = f;
    return e == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

static int check_common(double* A, int64_t m, int64_t n, int nb, int ib) {
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1 || n > m) return -3;
    if (nb < 8 || nb > 256 || nb % 4 != 0) return -4;
    if (ib < 1 || ib > 64 || nb % ib != 0) return -5;
    const int64_t p = (m + nb - 1) / nb, q = (n + nb - 1) / nb;
    if (p > 65535 || q > 65535) return -2;
    if (!plan_fits(p, q, nb)) return TQR_ERR_CAPACITY;
    return TQR_OK;
}

namespace tqr {

int check_factor_args(int64_t m, int64_t n, int nb, int ib, int tree, int BS) {
    static double probe;                               // a non-null stand-in for A
    const int rc = check_common(&probe, m, n, nb, ib);
    if (rc != TQR_OK) return rc;
    if (tree < TQR_FLAT_TS || tree > TQR_PLASMA_TS) return -6;
    const int64_t p = (m + nb - 1) / nb, q = (n + nb - 1) / nb;
    if ((tree == TQR_PLASMA || tree == TQR_PLASMA_TS) && (BS < 1 || BS > p)) return -7;
    if (tree == TQR_GRASAP && (BS < 0 || BS > q)) return -7;
    return TQR_OK;
}

}  // namespace tqr

extern "C" {

int tqr_factor(double* A, int64_t m, int64_t n, int nb, int ib, int tree, int BS, void* stream,
               tqr_factors** out) {
    try {
        if (!A) return -1;
        const int rc = check_factor_args(m, n, nb, ib, tree, BS);
        if (rc != TQR_OK) return rc;
        if (!out) return -9;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
        return run_factor(tree_key(m, n, nb, ib, tree, BS, dev), A, stream, out);
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_factor_ex(double* A, int64_t m, int64_t n, int nb, int ib, int tree, int BS, int precision, void* stream,
                  tqr_factors** out) {
    try {
        if (!A) return -1;
        const int rc = check_factor_args(m, n, nb, ib, tree, BS);
        if (rc != TQR_OK) return rc;
        if (precision < TQR_FP64 || precision > TQR_TF32) return -8;
        if (!out) return -10;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
        return run_factor(tree_key(m, n, nb, ib, tree, BS, dev), A, stream, out, precision);
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_factor_list(double* A, int64_t m, int64_t n, int nb, int ib, const int32_t* list, int64_t count,
                    int ts, void* stream, tqr_factors** out) {
    try {
        int rc = check_common(A, m, n, nb, ib);
        if (rc != TQR_OK) return rc;
        if (!list && count > 0) return -6;
        if (count < 0) return -7;
        if (ts != 0 && ts != 1) return -8;
        if (!out) return -10;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
        PlanKey key{m, n, nb, ib, -1, 0, ts, dev, {}};
        key.list.resize(static_cast<size_t>(count));
        for (int64_t t = 0; t < count; ++t) key.list[t] = {list[3 * t], list[3 * t + 1], list[3 * t + 2]};
        const int p = static_cast<int>((m + nb - 1) / nb), q = static_cast<int>((n + nb - 1) / nb);
        if (validate_elims(p, q, key.list.data(), count) != TQR_OK) return TQR_ERR_INVALID_LIST;
        return run_factor(key, A, stream, out);
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

static int apply_common(tqr_factors* f, double* B, int64_t ldb, int64_t nrhs, void* stream, bool trans) {
    try {
        if (!f || !f->plan) return -1;
        if (!B) return -2;
        const Plan& P = *f->plan;
        if (ldb < P.key.m) return -3;
        if (nrhs < 0) return -4;
        if (nrhs == 0) return TQR_OK;
        const int64_t ns = (nrhs + P.W - 1) / P.W;
        if (ns * static_cast<int64_t>(P.npanels) > 0x7fffffff) return -4;
        const DevGraph* g = nullptr;
        int rc = get_apply_graph(*f->plan, static_cast<int>(ns), trans, &g);
        if (rc != TQR_OK) return rc;
        if (g->ntasks > f->ast.capacity) {
            if (alloc_state(f->ast, g->ntasks, f->status) != cudaSuccess) return TQR_ERR_NOMEM;
        }
        f->stream = static_cast<cudaStream_t>(stream);
        ExecParams x = base_params(f);
        x.B = B;
        x.ldb = ldb;
        x.nrhs = nrhs;
        x.trans = trans ? 1 : 0;
        x.timeout_ns = exec_timeout_ns(4.0 * static_cast<double>(P.key.m) * P.key.n * nrhs);
        cudaError_t e = launch_factor_exec(x, graph_for_launch(*g), f->ast, P.G, P.smem, false, f->stream);
        return e == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_apply_qt(tqr_factors* f, double* B, int64_t ldb, int64_t nrhs, void* stream) {
    return apply_common(f, B, ldb, nrhs, stream, true);
}

int tqr_apply_q(tqr_factors* f, double* B, int64_t ldb, int64_t nrhs, void* stream) {
    return apply_common(f, B, ldb, nrhs, stream, false);
}

int tqr_form_t(tqr_factors* f, double* T_geqrt, double* T_elim, void* stream) {
    try {
        if (!f || !f->plan) return -1;
        const Plan& P = *f->plan;
        const size_t elems = static_cast<size_t>(P.p) * P.q * P.key.ib * P.key.nb;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (T_geqrt && cudaMemsetAsync(T_geqrt, 0, elems * sizeof(double), s) != cudaSuccess) return TQR_ERR_CUDA;
        if (T_elim && cudaMemsetAsync(T_elim, 0, elems * sizeof(double), s) != cudaSuccess) return TQR_ERR_CUDA;
        if (!T_geqrt && !T_elim) return TQR_OK;
        ExecParams x = base_params(f);
        f->stream = s;
        return launch_form_t(x, P.d_panels, P.npanels, T_geqrt, T_elim, s) == cudaSuccess ? TQR_OK
                                                                                           : TQR_ERR_CUDA;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_set_trace(tqr_factors* f, int enable) {
    if (!f) return -1;
    f->trace_on = enable ? 1 : 0;
    return TQR_OK;
}

int tqr_get_edges(const tqr_factors* f, int32_t* src, int32_t* dst, int64_t cap, int64_t* count) {
    try {
        if (!f || !f->plan) return -1;
        if (!count) return -5;
        const Graph& g = f->plan->g;
        const int64_t ne = static_cast<int64_t>(g.succ.size());
        *count = ne;
        if (cap < ne) return TQR_ERR_CAPACITY;
        if ((!src || !dst) && ne > 0) return -2;
        int64_t e = 0;
        for (size_t u = 0; u + 1 < g.succ_ptr.size(); ++u)
            for (int32_t k = g.succ_ptr[u]; k < g.succ_ptr[u + 1]; ++k, ++e) {
                src[e] = static_cast<int32_t>(u);
                dst[e] = g.succ[k];
            }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_poison_workspace(tqr_factors* f) {
    if (!f || !f->plan) return -1;
    const Plan& P = *f->plan;
    const size_t ntau = static_cast<size_t>(P.p) * P.q * P.key.nb;
    const size_t nt = static_cast<size_t>(P.p) * P.q * P.key.ib * P.key.nb;
    const size_t nv = static_cast<size_t>(P.p) * P.q * P.key.nb * P.key.nb;
    // All-ones bytes are a NaN in both FP64 and FP32.
    if (cudaMemsetAsync(f->tau_ge, 0xff, ntau * sizeof(double), f->stream) != cudaSuccess ||
        cudaMemsetAsync(f->tau_el, 0xff, ntau * sizeof(double), f->stream) != cudaSuccess)
        return TQR_ERR_CUDA;
    if (f->T_ge && (cudaMemsetAsync(f->T_ge, 0xff, nt * sizeof(float), f->stream) != cudaSuccess ||
                    cudaMemsetAsync(f->T_el, 0xff, nt * sizeof(float), f->stream) != cudaSuccess ||
                    cudaMemsetAsync(f->V_ge, 0xff, nv * sizeof(float), f->stream) != cudaSuccess ||
                    cudaMemsetAsync(f->V_el, 0xff, nv * sizeof(float), f->stream) != cudaSuccess))
        return TQR_ERR_CUDA;
    return TQR_OK;
}

int tqr_get_trace(tqr_factors* f, int64_t* out, int64_t cap, int64_t* count) {
    try {
        if (!f || !f->plan) return -1;
        if (!count) return -4;
        const Plan& P = *f->plan;
        const int64_t nt = P.dg.d.ntasks;
        *count = nt;
        if (!f->trace) return TQR_ERR_UNSUPPORTED;     // tracing was not enabled
        if (cap < nt) return TQR_ERR_CAPACITY;
        if (!out) return -2;
        if (cudaStreamSynchronize(f->stream) != cudaSuccess) return TQR_ERR_CUDA;
        std::vector<uint64_t> raw(2 * static_cast<size_t>(nt));
        if (cudaMemcpy(raw.data(), f->trace, raw.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TQR_ERR_CUDA;
        for (int64_t t = 0; t < nt; ++t) {
            const DevTask& x = P.g.tasks[t];
            int64_t* o = out + 8 * t;
            o[0] = x.kind & kKindMask;
            o[1] = x.i;
            o[2] = x.piv;
            o[3] = x.k;
            const int kind = x.kind & kKindMask;
            if (kind == GEQRT || kind == TTQRT || kind == TSQRT) {
                // Whole panel: -1.  Block b of a split panel: b << 32 | c_lo << 16 | c_hi,
                // [c_lo, c_hi) the columns it factors (the block's) or updates.
                if (x.j < 0) {
                    o[4] = -1;
                } else {
                    const int64_t j0 = static_cast<int64_t>(x.j) * P.key.ib;
                    const int64_t lo = x.strip < 0 ? j0 : (x.strip & 0xffff);
                    const int64_t hi = x.strip < 0 ? j0 + P.key.ib : (x.strip >> 16);
                    o[4] = (static_cast<int64_t>(x.j) << 32) | (lo << 16) | hi;
                }
            } else {
                o[4] = static_cast<int64_t>(x.j) * 65536 + x.strip;
            }
            o[5] = static_cast<int64_t>(raw[2 * t]);
            o[6] = static_cast<int64_t>(raw[2 * t] + (raw[2 * t + 1] & 0x00ffffffffffffffull));
            o[7] = static_cast<int64_t>(raw[2 * t + 1] >> 56);
        }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_sync(tqr_factors* f) {
    if (!f) return -1;
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) return TQR_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpy(&st, f->status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return TQR_ERR_CUDA;
    return st;
}

int tqr_get_info(const tqr_factors* f, tqr_info* info) {
    if (!f || !f->plan) return -1;
    if (!info) return -2;
    const Plan& P = *f->plan;
    info->m = P.key.m;
    info->n = P.key.n;
    info->nb = P.key.nb;
    info->ib = P.key.ib;
    info->p = P.p;
    info->q = P.q;
    info->tree = P.key.tree;
    info->BS = P.key.BS;
    info->ts = P.ts;
    info->strip = P.W;
    info->n_elims = static_cast<int64_t>(P.elims.size());
    info->n_tile_tasks = static_cast<int64_t>(P.tt.size());
    info->n_device_tasks = P.dg.d.ntasks;
    info->n_edges = P.dg.d.nedges;
    info->critical_path = P.cp;
    info->flops = lapack_flops(P.key.m, P.key.n);
    return TQR_OK;
}

void tqr_free(tqr_factors* f) {
    if (!f) return;
    cudaStreamSynchronize(f->stream);
    delete f;
}

static int factor_host_impl(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS,
                            double* B_host, int64_t nrhs, void* stream, tqr_factors** out, bool wait);

int tqr_factor_host(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS, double* B_host,
                    int64_t nrhs, void* stream, tqr_factors** out) {
    return factor_host_impl(A_host, m, n, nb, ib, tree, BS, B_host, nrhs, stream, out, true);
}

int tqr_factor_host_async(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS, double* B_host,
                          int64_t nrhs, void* stream, tqr_factors** out) {
    return factor_host_impl(A_host, m, n, nb, ib, tree, BS, B_host, nrhs, stream, out, false);
}

static int factor_host_impl(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS,
                            double* B_host, int64_t nrhs, void* stream, tqr_factors** out, bool wait) {
    try {
        int rc = check_common(A_host, m, n, nb, ib);     // same argument positions as tqr_factor
        if (rc != TQR_OK) return rc;
        if (!out) return -11;
        if (B_host && nrhs < 0) return -9;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        tqr_factors* prev = *out;
        // Reuse the previous handle's device copy of A only if tqr_factor will reuse
        // the handle itself (same plan key); a new handle gets a buffer of its own, so
        // that the previous handle's data is left untouched.
        const bool same = prev && prev->plan && prev->own_A &&
                          same_key(prev->plan->key, tree_key(m, n, nb, ib, tree, BS, dev));
        double* dA = same ? prev->own_A : nullptr;
        if (!same) {
            if (cudaMalloc(&dA, static_cast<size_t>(m) * n * sizeof(double)) != cudaSuccess) return TQR_ERR_NOMEM;
        }
        if (cudaMemcpyAsync(dA, A_host, static_cast<size_t>(m) * n * sizeof(double), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return TQR_ERR_CUDA;
        tqr_factors* f = same ? prev : nullptr;
        rc = tqr_factor(dA, m, n, nb, ib, tree, BS, stream, &f);
        if (rc != TQR_OK) {
            if (!same) cudaFree(dA);
            return rc;
        }
        if (!same) f->own_A = dA;     // the new handle adopts the buffer
        *out = f;                     // from here on the caller owns f, also on error
        if (B_host && nrhs > 0) {
            const size_t be = static_cast<size_t>(m) * nrhs;
            if (f->own_B_elems < be) {
                cudaFree(f->own_B);
                f->own_B = nullptr;
                f->own_B_elems = 0;
                if (cudaMalloc(&f->own_B, be * sizeof(double)) != cudaSuccess) return TQR_ERR_NOMEM;
                f->own_B_elems = be;
            }
            if (cudaMemcpyAsync(f->own_B, B_host, be * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return TQR_ERR_CUDA;
            rc = tqr_apply_qt(f, f->own_B, m, nrhs, stream);
            if (rc != TQR_OK) return rc;
            if (cudaMemcpyAsync(B_host, f->own_B, be * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return TQR_ERR_CUDA;
        }
        if (cudaMemcpyAsync(A_host, dA, static_cast<size_t>(m) * n * sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            return TQR_ERR_CUDA;
        return wait ? tqr_sync(f) : TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

// ------------------------------------------------------------- host only
int tqr_elimination_list(int p, int q, int tree, int BS, int32_t* out, int64_t cap, int64_t* count) {
    try {
        if (p < 1 || p > 65535) return -1;
        if (q < 1 || q > p) return -2;
        if (tree < TQR_FLAT_TS || tree > TQR_PLASMA_TS) return -3;
        if ((tree == TQR_PLASMA || tree == TQR_PLASMA_TS) && (BS < 1 || BS > p)) return -4;
        if (tree == TQR_GRASAP && (BS < 0 || BS > q)) return -4;
        if (!count) return -7;
        std::vector<Elim> el;
        int rc = make_elims(p, q, tree, BS, el);
        if (rc != TQR_OK) return rc;
        *count = static_cast<int64_t>(el.size());
        if (static_cast<int64_t>(el.size()) > cap) return TQR_ERR_CAPACITY;
        if (!out && !el.empty()) return -5;
        for (size_t t = 0; t < el.size(); ++t) {
            out[3 * t] = el[t].i;
            out[3 * t + 1] = el[t].piv;
            out[3 * t + 2] = el[t].k;
        }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_validate_list(int p, int q, const int32_t* list, int64_t count) {
    try {
        if (p < 1) return -1;
        if (q < 1 || q > p) return -2;
        if (!list && count > 0) return -3;
        if (count < 0) return -4;
        std::vector<Elim> el(static_cast<size_t>(count));
        for (int64_t t = 0; t < count; ++t) el[t] = {list[3 * t], list[3 * t + 1], list[3 * t + 2]};
        return validate_elims(p, q, el.data(), count);
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_critical_path(int p, int q, int tree, int BS, int64_t* cp, int32_t* zero_time) {
    try {
        if (p < 1 || p > 65535) return -1;
        if (q < 1 || q > p) return -2;
        if (tree < TQR_FLAT_TS || tree > TQR_PLASMA_TS) return -3;
        if ((tree == TQR_PLASMA || tree == TQR_PLASMA_TS) && (BS < 1 || BS > p)) return -4;
        if (tree == TQR_GRASAP && (BS < 0 || BS > q)) return -4;
        if (!cp) return -5;
        if (!plan_fits(p, q, 0)) return TQR_ERR_CAPACITY;   // tile tasks alone would not fit
        std::vector<Elim> el;
        int rc = make_elims(p, q, tree, BS, el);
        if (rc != TQR_OK) return rc;
        std::vector<TileTask> tt;
        if (!expand_tasks(p, q, el, ts_flags(tree, BS, el), tt)) return TQR_ERR_INTERNAL;
        std::vector<int64_t> fin;
        *cp = simulate(p, q, tt, &fin);
        if (zero_time) {
            for (int64_t t = 0; t < static_cast<int64_t>(p) * q; ++t) zero_time[t] = -1;
            for (size_t t = 0; t < tt.size(); ++t)
                if (tt[t].kind == TTQRT || tt[t].kind == TSQRT)
                    zero_time[static_cast<int64_t>(tt[t].i) * q + tt[t].k] = static_cast<int32_t>(fin[t]);
        }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_tasks(int p, int q, int tree, int BS, int32_t* out, int64_t* finish, int64_t cap, int64_t* count) {
    try {
        if (p < 1 || p > 65535) return -1;
        if (q < 1 || q > p) return -2;
        if (tree < TQR_FLAT_TS || tree > TQR_PLASMA_TS) return -3;
        if ((tree == TQR_PLASMA || tree == TQR_PLASMA_TS) && (BS < 1 || BS > p)) return -4;
        if (tree == TQR_GRASAP && (BS < 0 || BS > q)) return -4;
        if (!count) return -8;
        if (!plan_fits(p, q, 0)) return TQR_ERR_CAPACITY;   // tile tasks alone would not fit
        std::vector<Elim> el;
        int rc = make_elims(p, q, tree, BS, el);
        if (rc != TQR_OK) return rc;
        std::vector<TileTask> tt;
        if (!expand_tasks(p, q, el, ts_flags(tree, BS, el), tt)) return TQR_ERR_INTERNAL;
        *count = static_cast<int64_t>(tt.size());
        if (static_cast<int64_t>(tt.size()) > cap) return TQR_ERR_CAPACITY;
        if (!out && !tt.empty()) return -5;
        std::vector<int64_t> fin;
        simulate(p, q, tt, &fin);
        for (size_t t = 0; t < tt.size(); ++t) {
            out[5 * t] = tt[t].kind;
            out[5 * t + 1] = tt[t].i;
            out[5 * t + 2] = tt[t].piv;
            out[5 * t + 3] = tt[t].k;
            out[5 * t + 4] = tt[t].j;
            if (finish) finish[t] = fin[t];
        }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_device_graph(int64_t m, int64_t n, int nb, int ib, int tree, int BS, int strip, int32_t* tasks,
                     int64_t task_cap, int64_t* ntasks, int32_t* src, int32_t* dst, int64_t edge_cap,
                     int64_t* nedges) {
    try {
        static double probe;
        const int rc = check_common(&probe, m, n, nb, ib);
        if (rc != TQR_OK) return rc == -1 ? TQR_ERR_INTERNAL : rc;   // -2 m, -3 n, -4 nb, -5 ib
        if (tree < TQR_FLAT_TS || tree > TQR_PLASMA_TS) return -6;
        const int p = static_cast<int>((m + nb - 1) / nb), q = static_cast<int>((n + nb - 1) / nb);
        if ((tree == TQR_PLASMA || tree == TQR_PLASMA_TS) && (BS < 1 || BS > p)) return -7;
        if (tree == TQR_GRASAP && (BS < 0 || BS > q)) return -7;
        if (strip != 16 && strip != 32 && strip != 64) return -8;
        if (!ntasks || !nedges) return !ntasks ? -11 : -15;
        if (!plan_fits(p, q, nb)) return TQR_ERR_CAPACITY;
        const int t = tree == TQR_SAMEH_KUCK ? TQR_FLAT_TT : tree;
        std::vector<Elim> el;
        int r2 = make_elims(p, q, t, BS, el);
        if (r2 != TQR_OK) return r2;
        std::vector<TileTask> tt;
        if (!expand_tasks(p, q, el, ts_flags(t, BS, el), tt)) return TQR_ERR_INTERNAL;
        Graph g;
        build_factor_graph(p, q, nb, ib, strip, static_cast<int>(n - static_cast<int64_t>(q - 1) * nb), tt, g);
        *ntasks = static_cast<int64_t>(g.tasks.size());
        *nedges = static_cast<int64_t>(g.succ.size());
        if (*ntasks > task_cap || *nedges > edge_cap) return TQR_ERR_CAPACITY;
        if ((!tasks && *ntasks) || ((!src || !dst) && *nedges)) return TQR_ERR_CAPACITY;
        for (size_t x = 0; x < g.tasks.size(); ++x) {
            const DevTask& d = g.tasks[x];
            int32_t* o = tasks + 6 * x;
            o[0] = d.kind & kKindMask;
            o[1] = d.i;
            o[2] = d.piv;
            o[3] = d.k;
            o[4] = d.j;
            o[5] = d.strip;
        }
        int64_t e = 0;
        for (size_t u = 0; u + 1 < g.succ_ptr.size(); ++u)
            for (int32_t k = g.succ_ptr[u]; k < g.succ_ptr[u + 1]; ++k, ++e) {
                src[e] = static_cast<int32_t>(u);
                dst[e] = g.succ[k];
            }
        return TQR_OK;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_release_plans(void) {
    try {
        release_lstsq_cache();                          // its handle holds a plan
        int dropped = 0;
        {
            std::lock_guard<std::mutex> lk(g_plans_mu);
            auto& mp = plans();
            for (auto it = mp.begin(); it != mp.end();) {
                if (it->second.use_count() == 1) {      // held by the cache alone
                    it = mp.erase(it);
                    ++dropped;
                } else {
                    ++it;
                }
            }
        }
        std::lock_guard<std::mutex> lk(g_hplans_mu);
        hplans().clear();                               // batches copy what they use
        return dropped;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_set_timeout_ms(double ms) {
    g_timeout_ms.store(ms > 0 ? ms : 0.0);
    return TQR_OK;
}

int tqr_inject_fault(int kind) {
    if (kind != 0 && kind != 1) return -1;
    g_fault.store(kind);
    return TQR_OK;
}

static int launch_batch(tqr_batch* b) {
    // status word and the persistent launch's three queue counters
    if (cudaMemsetAsync(b->status, 0, 4 * sizeof(int32_t), b->stream) != cudaSuccess) return TQR_ERR_CUDA;
    if (b->n_fused > 0 && launch_ts1_all(b->ts1, b->ts1_ph, b->f32, b->tau_ge, b->tau_el, b->status, b->status + 1,
                                         b->stream) != cudaSuccess)
        return TQR_ERR_CUDA;
    if (!b->has_exec) return TQR_OK;
    ExecParams P{};
    P.tau_ge = b->tau_ge;
    P.tau_el = b->tau_el;
    P.trans = 1;
    P.mats = b->d_mats;
    P.timeout_ns = exec_timeout_ns(b->flops);
    P.nb = b->nb.empty() ? 0 : b->nb[0];
    P.ib = b->ib.empty() ? 0 : b->ib[0];
    const cudaError_t e = launch_factor_exec(P, b->dg.d, b->st, b->G, b->smem, false, b->stream);
    return e == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

// Plans the one-tile-column matrices of a batch into the persistent launch's
// queues (plan_ts1) and uploads the descriptors.
static int build_ts1(tqr_batch* b, const std::vector<Ts1Desc>& fused) {
    std::vector<Ts1Desc> q;
    plan_ts1(fused, b->f32 ? 4 : 8, &q, &b->ts1_ph, &b->max_cp);
    b->n_fused = static_cast<int>(q.size());
    if (!q.empty() && upload(&b->ts1, q) != cudaSuccess) return TQR_ERR_NOMEM;
    return TQR_OK;
}

int tqr_ts1_plan(int count, const int64_t* m, const int64_t* n, const int32_t* nb, int f32, int32_t* order,
                 int32_t* bounds, int32_t* quarter_bytes) {
    try {
        if (count < 0 || count > (1 << 23)) return -1;
        if (count > 0 && (!m || !n || !nb)) return -2;
        if (!order || !bounds || !quarter_bytes) return -5;
        const int esz = f32 ? 4 : 8;
        std::vector<Ts1Desc> fused(count);
        for (int c = 0; c < count; ++c) {
            if (m[c] < 1) return -2;
            if (n[c] < 1 || n[c] > m[c]) return -3;
            if (!ts1_supported(m[c], n[c], nb[c], esz)) return TQR_ERR_UNSUPPORTED;
            // the matrix's index in place of its pointer: this plan is never launched
            fused[c] = Ts1Desc{reinterpret_cast<void*>(static_cast<intptr_t>(c) + 1), m[c], static_cast<int32_t>(n[c]),
                               nb[c], 0};
        }
        std::vector<Ts1Desc> q;
        Ts1Phases ph{};
        int64_t cp = 0;
        plan_ts1(fused, esz, &q, &ph, &cp);
        for (int i = 0; i < count; ++i) order[i] = static_cast<int32_t>(reinterpret_cast<intptr_t>(q[i].A) - 1);
        for (int k = 0; k < 3; ++k) {
            bounds[2 * k] = ph.begin[k];
            bounds[2 * k + 1] = ph.end[k];
        }
        *quarter_bytes = ph.quarter_bytes;
        return TQR_OK;
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_factor_batched(int count, double* const* A, const int64_t* m, const int64_t* n, const int32_t* nb,
                       const int32_t* ib, const int32_t* tree, const int32_t* BS, void* stream,
                       tqr_batch** out) {
    try {
        if (count < 1 || count > (1 << 23)) return -1;
        if (!A) return -2;
        if (!m) return -3;
        if (!n) return -4;
        if (!nb) return -5;
        if (!ib) return -6;
        if (!tree) return -7;
        if (!BS) return -8;
        if (!out) return -10;
        int nbmax = 0, ibmax = 0;
        for (int c = 0; c < count; ++c) {
            const int rc = check_common(A[c], m[c], n[c], nb[c], ib[c]);
            if (rc != TQR_OK) {
                if (rc < -99) return rc;                  // named code (capacity)
                return rc == -1 ? -2 : (rc == -2 ? -3 : (rc == -3 ? -4 : (rc == -4 ? -5 : -6)));
            }
            if (tree[c] < TQR_FLAT_TS || tree[c] > TQR_PLASMA_TS) return -7;
            const int p = static_cast<int>((m[c] + nb[c] - 1) / nb[c]);
            const int q = static_cast<int>((n[c] + nb[c] - 1) / nb[c]);
            if ((tree[c] == TQR_PLASMA || tree[c] == TQR_PLASMA_TS) && (BS[c] < 1 || BS[c] > p)) return -8;
            if (tree[c] == TQR_GRASAP && (BS[c] < 0 || BS[c] > q)) return -8;
            nbmax = std::max(nbmax, nb[c]);
            ibmax = std::max(ibmax, ib[c]);
        }
        tqr_batch* b = *out;
        if (b && b->same(count, A, m, n, nb, ib, tree, BS)) {
            b->stream = static_cast<cudaStream_t>(stream);
            return launch_batch(b);
        }
        auto nbh = std::make_unique<tqr_batch>();
        b = nbh.get();
        b->count = count;
        b->A.assign(A, A + count);
        b->m.assign(m, m + count);
        b->n.assign(n, n + count);
        b->nb.assign(nb, nb + count);
        b->ib.assign(ib, ib + count);
        b->tree.assign(tree, tree + count);
        b->BS.assign(BS, BS + count);
        if (!choose_layout(nbmax, ibmax, &b->G, &b->smem)) return TQR_ERR_UNSUPPORTED;
        const int W = strip_width(b->G);
        Graph all;
        std::vector<MatDesc> mats(count);
        std::vector<Ts1Desc> fused;
        int64_t tau_off = 0;
        for (int c = 0; c < count; ++c) {
            if (tree[c] == TQR_FLAT_TS && ts1_supported(m[c], n[c], nb[c], sizeof(double))) {
                const int64_t p = (m[c] + nb[c] - 1) / nb[c];
                fused.push_back(Ts1Desc{A[c], m[c], static_cast<int32_t>(n[c]), nb[c], tau_off});
                mats[c] = MatDesc{A[c], m[c], m[c], n[c], nb[c], ib[c], static_cast<int>(p), 1, tau_off};
                b->flops += lapack_flops(m[c], n[c]);
                tau_off += p * nb[c];
                continue;
            }
            b->has_exec = true;
            const int t = tree[c] == TQR_SAMEH_KUCK ? TQR_FLAT_TT : tree[c];
            const int bs = uses_bs(t) ? BS[c] : 0;
            std::shared_ptr<HostPlan> H;
            const int rc = host_plan(m[c], n[c], nb[c], ib[c], t, bs, W, H);
            if (rc != TQR_OK) return rc;
            b->smem = std::max(b->smem, fp64_smem_bytes(nb[c], ib[c], b->G));
            b->max_cp = std::max(b->max_cp, H->cp);
            b->flops += lapack_flops(m[c], n[c]);
            const int32_t off = static_cast<int32_t>(all.tasks.size());
            if (static_cast<int64_t>(off) + static_cast<int64_t>(H->g.tasks.size()) > 0x7fffffff) return TQR_ERR_UNSUPPORTED;
            for (const DevTask& x : H->g.tasks) {
                DevTask y = x;
                y.kind = x.kind | (c << 8);
                all.tasks.push_back(y);
            }
            const int32_t eoff = static_cast<int32_t>(all.succ.size());
            if (all.succ_ptr.empty()) all.succ_ptr.push_back(0);
            for (size_t t2 = 1; t2 < H->g.succ_ptr.size(); ++t2) all.succ_ptr.push_back(H->g.succ_ptr[t2] + eoff);
            for (int32_t sx : H->g.succ) all.succ.push_back(sx + off);
            all.indeg.insert(all.indeg.end(), H->g.indeg.begin(), H->g.indeg.end());
            for (int32_t r : H->g.ready) all.ready.push_back(r + off);
            mats[c] = MatDesc{A[c], m[c], m[c], n[c], nb[c], ib[c], H->p, H->q, tau_off};
            tau_off += static_cast<int64_t>(H->p) * H->q * nb[c];
        }
        if (b->has_exec && upload_graph(all, b->dg) != cudaSuccess) return TQR_ERR_NOMEM;
        if (upload(&b->d_mats, mats) != cudaSuccess) return TQR_ERR_NOMEM;
        if (cudaMalloc(&b->tau_ge, std::max<int64_t>(1, tau_off) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&b->tau_el, std::max<int64_t>(1, tau_off) * sizeof(double)) != cudaSuccess ||
            cudaMemset(b->tau_ge, 0, std::max<int64_t>(1, tau_off) * sizeof(double)) != cudaSuccess ||
            cudaMemset(b->tau_el, 0, std::max<int64_t>(1, tau_off) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&b->status, 4 * sizeof(int32_t)) != cudaSuccess ||
            (b->has_exec && alloc_state(b->st, b->dg.d.ntasks, b->status) != cudaSuccess))
            return TQR_ERR_NOMEM;
        if (build_ts1(b, fused) != TQR_OK) return TQR_ERR_NOMEM;
        b->stream = static_cast<cudaStream_t>(stream);
        const int rc = launch_batch(b);
        if (rc != TQR_OK) return rc;
        *out = nbh.release();
        return TQR_OK;
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_factor_batched_f32(int count, float* const* A, const int64_t* m, const int64_t* n, const int32_t* nb,
                           void* stream, tqr_batch** out) {
    try {
        if (count < 1 || count > (1 << 23)) return -1;
        if (!A) return -2;
        if (!m) return -3;
        if (!n) return -4;
        if (!nb) return -5;
        if (!out) return -7;
        for (int c = 0; c < count; ++c) {
            if (!A[c]) return -2;
            if (m[c] < 1) return -3;
            if (n[c] < 1 || n[c] > m[c]) return -4;
            if (nb[c] < 8 || nb[c] > 256 || nb[c] % 4 != 0 || (m[c] + nb[c] - 1) / nb[c] > 65535) return -5;
            if (!ts1_supported(m[c], n[c], nb[c], sizeof(float))) return TQR_ERR_UNSUPPORTED;
        }
        const std::vector<int32_t> ones(count, 1), flat(count, TQR_FLAT_TS);
        std::vector<double*> ids(count);
        for (int c = 0; c < count; ++c) ids[c] = reinterpret_cast<double*>(A[c]);
        tqr_batch* b = *out;
        if (b && b->f32 && b->same(count, ids.data(), m, n, nb, nb, flat.data(), ones.data())) {
            b->stream = static_cast<cudaStream_t>(stream);
            return launch_batch(b);
        }
        auto nbh = std::make_unique<tqr_batch>();
        b = nbh.get();
        b->count = count;
        b->f32 = true;
        b->A = ids;
        b->m.assign(m, m + count);
        b->n.assign(n, n + count);
        b->nb.assign(nb, nb + count);
        b->ib.assign(nb, nb + count);
        b->tree = flat;
        b->BS = ones;
        std::vector<Ts1Desc> fused(count);
        int64_t tau_off = 0;
        for (int c = 0; c < count; ++c) {
            fused[c] = Ts1Desc{A[c], m[c], static_cast<int32_t>(n[c]), nb[c], tau_off};
            tau_off += (m[c] + nb[c] - 1) / nb[c] * nb[c];
            b->flops += lapack_flops(m[c], n[c]);
        }
        if (cudaMalloc(&b->tau_ge, std::max<int64_t>(1, tau_off) * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&b->tau_el, std::max<int64_t>(1, tau_off) * sizeof(float)) != cudaSuccess ||
            cudaMemset(b->tau_ge, 0, std::max<int64_t>(1, tau_off) * sizeof(float)) != cudaSuccess ||
            cudaMemset(b->tau_el, 0, std::max<int64_t>(1, tau_off) * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&b->status, 4 * sizeof(int32_t)) != cudaSuccess)
            return TQR_ERR_NOMEM;
        if (build_ts1(b, fused) != TQR_OK) return TQR_ERR_NOMEM;
        b->stream = static_cast<cudaStream_t>(stream);
        const int rc = launch_batch(b);
        if (rc != TQR_OK) return rc;
        *out = nbh.release();
        return TQR_OK;
    } catch (const std::bad_alloc&) {
        return TQR_ERR_NOMEM;
    } catch (...) {
        return TQR_ERR_INTERNAL;
    }
}

int tqr_batch_tau(const tqr_batch* b, int c, void* tau_ge, void* tau_el) {
    if (!b) return -1;
    if (c < 0 || c >= b->count) return -2;
    if (!tau_ge) return -3;
    if (!tau_el) return -4;
    const size_t esz = b->f32 ? sizeof(float) : sizeof(double);
    int64_t off = 0;
    for (int x = 0; x < c; ++x)
        off += (b->m[x] + b->nb[x] - 1) / b->nb[x] * ((b->n[x] + b->nb[x] - 1) / b->nb[x]) * b->nb[x];
    const int64_t len = (b->m[c] + b->nb[c] - 1) / b->nb[c] * ((b->n[c] + b->nb[c] - 1) / b->nb[c]) * b->nb[c];
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TQR_ERR_CUDA;
    const char* ge = reinterpret_cast<const char*>(b->tau_ge) + off * esz;
    const char* el = reinterpret_cast<const char*>(b->tau_el) + off * esz;
    if (cudaMemcpy(tau_ge, ge, len * esz, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(tau_el, el, len * esz, cudaMemcpyDefault) != cudaSuccess)
        return TQR_ERR_CUDA;
    return TQR_OK;
}

int tqr_batch_sync(tqr_batch* b) {
    if (!b) return -1;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TQR_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpy(&st, b->status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return TQR_ERR_CUDA;
    return st;
}

int tqr_batch_get_info(const tqr_batch* b, tqr_batch_info* info) {
    if (!b) return -1;
    if (!info) return -2;
    info->count = b->count;
    info->strip = strip_width(b->G);
    info->n_tasks = b->dg.d.ntasks;
    info->n_edges = b->dg.d.nedges;
    info->max_critical_path = b->max_cp;
    info->flops = b->flops;
    info->n_fused = b->n_fused;
    info->f32 = b->f32 ? 1 : 0;
    return TQR_OK;
}

void tqr_batch_free(tqr_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    delete b;
}

const char* tqr_strerror(int status) {
    switch (status) {
        case TQR_OK: return "success";
        case TQR_ERR_INVALID_LIST: return "invalid elimination list";
        case TQR_ERR_TIMEOUT: return "device wait timed out";
        case TQR_ERR_NONFINITE: return "non-finite value in a Householder norm";
        case TQR_ERR_CUDA: return "CUDA runtime error";
        case TQR_ERR_NOMEM: return "out of memory";
        case TQR_ERR_CAPACITY: return "output array too small";
        case TQR_ERR_INTERNAL: return "internal error";
        case TQR_ERR_UNSUPPORTED: return "unsupported parameters";
        case TQR_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of tqr_factor_noalloc";
        default:
            if (status < 0 && status > -100) return "invalid argument";
            return "unknown status";
    }
}

}  // extern "C"
