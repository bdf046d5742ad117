// Internal declarations shared by the host planner, the device executor and
// the C ABI of libtqr.  Not installed; the public interface is include/tqr.h.
#pragma once

#include <cstdint>
#include <vector>
#include <memory>
#include <cuda_runtime.h>

namespace tqr {

// Kernel kinds (same numbering as tqr_kernel in tqr.h).
enum Kind : int32_t { GEQRT = 0, UNMQR = 1, TTQRT = 2, TTMQR = 3, TSQRT = 4, TSMQR = 5 };

// Table 1 of the paper: cost of each kernel in units of nb^3/3 flops.
inline int kernel_weight(int kind) {
    static const int w[6] = {4, 6, 2, 6, 6, 12};
    return w[kind];
}

struct Elim { int32_t i, piv, k; };                 // 0-based elim(i, piv, k)
struct TileTask { int32_t kind, i, piv, k, j; };     // 0-based; piv/j = -1 when unused

// One device task.  Update kernels are split into column strips: `strip`
// selects columns [strip*W, strip*W + W) of tile column j (or of B).
// Bit kHighPriority of `kind` sends the task, once ready, to the executor's
// high-priority queue, which idle CTAs serve first.
constexpr int32_t kHighPriority = 0x80;
constexpr int32_t kKindMask = 0x7f;
struct DevTask {
    int32_t kind;    // Kind in bits 0-6, kHighPriority in bit 7; matrix of a batched factorization in bits 8-31
    int32_t i;       // row of the tile factored / zeroed / updated
    int32_t piv;     // pivot row (TT/TS kernels), else -1
    int32_t k;       // panel column
    int32_t j;       // update column (updates); panels: -1, or the block of a split panel
    int32_t strip;   // column strip (updates); split panel: -1 = factor the block,
                     // else c_lo | c_hi << 16 = apply it to columns [c_lo, c_hi)
};

// One matrix of a batched factorization (device array indexed by DevTask::kind >> 8).
struct MatDesc {
    double* A;
    int64_t lda, m, n;
    int32_t nb, ib, p, q;
    int64_t tau_off;   // offset of this matrix's tau in tau_ge / tau_el
};

// ---- argument checks shared by the entry points (capi.cpp) ----
// tqr_factor's m, n, nb, ib, tree and BS: TQR_OK, TQR_ERR_CAPACITY, or -k for
// tqr_factor's invalid argument k (2 m, 3 n, 4 nb, 5 ib, 6 tree, 7 BS).
int check_factor_args(int64_t m, int64_t n, int nb, int ib, int tree, int BS);

// ---- host planner (planner.cpp) ----
int make_elims(int p, int q, int tree, int BS, std::vector<Elim>& out);
int validate_elims(int p, int q, const Elim* e, int64_t count);
bool expand_tasks(int p, int q, const std::vector<Elim>& elims, bool ts, std::vector<TileTask>& out);
bool expand_tasks(int p, int q, const std::vector<Elim>& elims, const std::vector<char>& ts_of,
                  std::vector<TileTask>& out);
std::vector<char> ts_flags(int tree, int BS, const std::vector<Elim>& elims);
// Unit-weight ASAP finish time of every tile task and the critical path.
int64_t simulate(int p, int q, const std::vector<TileTask>& tasks, std::vector<int64_t>* finish);

// Device task graph: tasks, successor lists (CSR) and in-degrees.
struct Graph {
    std::vector<DevTask> tasks;
    std::vector<int32_t> succ_ptr;   // size ntasks+1
    std::vector<int32_t> succ;
    std::vector<int32_t> indeg;
    std::vector<int32_t> ready;      // tasks with in-degree 0, program order
};

// Graph of the factorization: updates split into strips of W columns, and
// panels, when split_panels(nb, ib), into one factor task per block of ib
// columns plus tasks applying each block to column ranges right of it
// (DevTask: j = block, strip = -1 to factor, else c_lo | c_hi << 16).
// n_cols_last: number of valid columns of the last tile column.
bool split_panels(int nb, int ib);
void build_factor_graph(int p, int q, int nb, int ib, int W, int n_cols_last,
                        const std::vector<TileTask>& tt, Graph& g);
// Graph replaying the panel tasks' transformations on a right-hand side of
// nstrips strips (trans = Q^T order, else reverse order for Q).
void build_apply_graph(int p, const std::vector<TileTask>& tt, int nstrips, bool trans, Graph& g);

}  // namespace tqr

// ---------------------------------------------------------------------------
// Device side (device.cu).
// ---------------------------------------------------------------------------
namespace tqr {

constexpr int kThreads = 256;   // threads per executor CTA

// A task graph resident in device memory (immutable after upload).
struct DevGraph {
    DevTask* tasks = nullptr;
    int32_t* succ_ptr = nullptr;
    int32_t* succ = nullptr;
    int32_t* indeg = nullptr;
    int32_t* ready = nullptr;        // initially ready tasks: the high-priority ones first
    int32_t ntasks = 0, nready = 0;
    int32_t n_hi = 0, nready_hi = 0; // tasks with kHighPriority; how many of them start ready
    int64_t nedges = 0;
};

// Mutable per-run state of the executor: dependency counters, ready queues,
// their heads/tails and the status word.  queue[0, n_hi) is the high-priority
// queue, queue[n_hi, ntasks) the other one.
struct ExecState {
    int32_t* deps = nullptr;
    int32_t* queue = nullptr;
    uint32_t* ctr = nullptr;     // [0] head, [1] tail of the high queue; [2], [3] of the other
    int32_t* status = nullptr;
    int32_t capacity = 0;        // tasks the arrays can hold
};

// Everything one executor launch needs (passed by value as a kernel argument).
struct ExecParams {
    double* A; int64_t lda; int64_t m, n;       // matrix being factored (R and V)
    int nb, ib, p, q;
    double* tau_ge;                              // tau of GEQRT(i,k): [(k*p+i)*nb + r]
    double* tau_el;                              // tau of TTQRT/TSQRT zeroing (i,k)
    double* B; int64_t ldb, nrhs;                // right-hand side (apply graphs), else null
    int trans;                                   // 1: apply Q^T, 0: apply Q
    int prec;                                    // 0: FP64 updates, 1: split-TF32 (3 pass), 2: TF32
    float* T_ge;                                 // compact-WY T blocks (prec != 0), FP32: ib x nb per tile
    float* T_el;
    float* V_ge;                                 // reflectors as FP32 with unit/zero structure written
    float* V_el;                                 //   out (prec != 0): nb x nb per tile, column-major
    const DevTask* tasks; const int32_t* succ_ptr; const int32_t* succ;
    int32_t* deps; int32_t* queue; uint32_t* ctr; int32_t* status;
    int32_t ntasks;
    int32_t n_hi;                                // size of the high-priority queue (queue[0, n_hi))
    uint64_t timeout_ns;                         // limit for any single wait
    uint64_t* trace;                             // optional: 2 per task (start, duration | sm << 56)
    const MatDesc* mats;                         // batched factorization: per-matrix fields, else null
};

// Row groups per strip column (G) and dynamic shared memory for (nb, ib);
// returns false if no layout fits.
bool choose_layout(int nb, int ib, int* G, int* smem_bytes);
// Shared memory the low-precision update kernels need for (nb, ib, G), and
// whether the low-precision path supports (nb, ib) at all.
int lp_smem_bytes(int nb, int ib, int G);
bool lp_supported(int nb, int ib, int G);
int strip_width(int G);
int fp64_smem_bytes(int nb, int ib, int G);
int device_sm_count();
// exec_kernel<G, PREC> launcher; one definition per (G, PREC) in its own object.
template <int G, int PREC>
cudaError_t launch_exec(const ExecParams& P, int smem, int grid, cudaStream_t s);
cudaError_t launch_factor_exec(ExecParams P, const DevGraph& g, const ExecState& st, int G,
                               int smem, bool reset_status, cudaStream_t s);
// Limit for any single device wait of a launch doing `flops` flops: the value
// of tqr_set_timeout_ms if set, else TQR_TIMEOUT_MS from the environment, else
// 10 s + flops / 5e10 s (capi.cpp).
uint64_t exec_timeout_ns(double flops);
// The graph a launch should use: `g` itself, or `g` with no initially ready
// task when tqr_inject_fault(1) is pending (one launch consumes it), so that
// every wait of that launch runs out (capi.cpp).
DevGraph graph_for_launch(const DevGraph& g);
// Frees the workspace and factor handle tqr_lstsq keeps for its next call
// (lstsq.cu).
void release_lstsq_cache();
// Batched FlatTree-TS for one tile column (q = 1): one CTA per matrix, the tile
// in registers, R in shared memory.  A matrix of n <= 128 columns with n <= nb
// and nb in {64, 128, 256} (nb >= its column class 32 / 64 / 128; FP64 with
// class 128 needs nb = 128) runs there when its shared memory fits.
struct Ts1Desc {
    void* A;            // column-major, leading dimension m (double or float)
    int64_t m;
    int32_t n, h;       // columns, tile height nb
    int64_t tau_off;    // offset of the matrix's tau block (p * nb entries)
};
int ts1_ncol_class(int64_t n);
int ts1_smem_bytes(int ncol_class, int h, int elem_size);
bool ts1_supported(int64_t m, int64_t n, int nb, int elem_size);
// Threads a matrix of the class runs with: 256, 512 or 1024.
int ts1_threads(int ncol_class, int h, int elem_size);
// The persistent launch's queues: descriptors [begin[k], end[k]) run on slots
// of 1024 >> k threads (begin[0] = 0, end[k] = begin[k + 1], end[2] = count);
// a slot of 1024 >> k threads has (4 >> k) * quarter_bytes of shared memory.
struct Ts1Phases {
    int32_t begin[3], end[3];
    int32_t quarter_bytes;
};
// The launch's queues (host only): the matrices sorted by thread count (1024
// first), largest work m n^2 first within each, the phase bounds and the
// shared-memory quarter (a multiple of 16 bytes that covers every slot's
// need); *max_cp is raised to the longest chain (Proposition 2, q = 1).
void plan_ts1(const std::vector<Ts1Desc>& fused, int elem_size, std::vector<Ts1Desc>* queue, Ts1Phases* ph,
              int64_t* max_cp);
// One launch for every one-tile-column matrix of a batch; ctr: three counters
// that must be zero when the kernel starts.
cudaError_t launch_ts1_all(const Ts1Desc* d, const Ts1Phases& ph, bool f32, void* tau_ge, void* tau_el,
                           int32_t* status, int32_t* ctr, cudaStream_t s);
// T factors of the listed panel tasks (kind, i, k triplets on the device).
cudaError_t launch_form_t(const ExecParams& P, const int32_t* panels, int npanels,
                          double* T_ge, double* T_el, cudaStream_t s);

}  // namespace tqr
