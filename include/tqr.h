/*
 * tqr.h -- C ABI of libtqr, tiled Householder QR factorization on one GPU.
 *
 * Method: Bouwmeester, Jacquelin, Langou, Robert, "Tiled QR factorization
 * algorithms" (2011).  An m x n matrix (m >= n) is split into p x q tiles of
 * nb x nb.  An elimination tree produces an elimination list (Section 2,
 * Algorithm 1; validity rules of Section 2.2); each elimination expands into
 * TS or TT kernel tasks (Algorithms 2 and 3); the tasks run as soon as their
 * dependencies are met (Section 2.3).  The six kernels (Table 1) are GEQRT,
 * UNMQR, TSQRT, TSMQR, TTQRT and TTMQR, with inner blocking ib.
 *
 * Conventions for every entry point:
 *  - Return value: 0 (TQR_OK) on success.  A negative value -k in -1..-99
 *    means that argument k (1-based) is invalid.  Named codes below.
 *  - No C++ exception crosses this boundary.
 *  - Matrices are column-major FP64 (FP32 for tqr_factor_batched_f32 and the
 *    cost-model network).  "device" pointers are CUDA global memory of the
 *    current device; "host" pointers are ordinary host memory.
 *  - Device work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) and returns before it completes.  Errors detected on the
 *    device (timeout, non-finite values) surface at tqr_sync().
 *  - Tile indices in integer outputs are 0-based: the paper's elim(i, piv, k)
 *    with 1-based rows and columns appears as (i-1, piv-1, k-1).
 *  - Ownership: the caller owns every matrix it passes.  The library owns
 *    what a tqr_factors handle holds (reflector scalars, task graph,
 *    counters) until tqr_free().
 */
#ifndef TQR_H
#define TQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Elimination trees (Section 3).  TQR_FLAT_TS runs FlatTree with TS kernels
 * (Proposition 2) and TQR_PLASMA_TS runs PlasmaTree with TS kernels inside
 * each domain and TT kernels for the merge of the domain heads (the kernel
 * mix of the TS-based library the experiments compare against); every other
 * tree runs TT kernels.  ASAP and GRASAP(k)
 * (Section 3.2) are dynamic: their lists come from simulating the tiled time
 * model (Table 1 weights) while the list is built.  For TQR_GRASAP the BS
 * argument carries k, 0 <= k <= min(p,q) (0 = Greedy, min(p,q) = ASAP). */
typedef enum {
    TQR_FLAT_TS = 0,     /* Sameh-Kuck list, TS kernels                    */
    TQR_FLAT_TT = 1,     /* Sameh-Kuck list, TT kernels (FlatTree)         */
    TQR_SAMEH_KUCK = 2,  /* same list and kernels as TQR_FLAT_TT           */
    TQR_BINARY = 3,      /* binary reduction per column (Proposition 1)    */
    TQR_FIBONACCI = 4,   /* Fibonacci scheme of order 1 (Section 3.1)      */
    TQR_GREEDY = 5,      /* Greedy for tiles (Algorithm 4)                 */
    TQR_PLASMA = 6,      /* PlasmaTree with domain size BS (Section 3.2)   */
    TQR_ASAP = 7,        /* ASAP: pair ready rows as soon as two are ready  */
    TQR_GRASAP = 8,      /* GRASAP(k), k = BS: Greedy, then ASAP on the last k columns */
    TQR_PLASMA_TS = 9    /* PlasmaTree(BS) list, TS inside domains, TT merges */
} tqr_tree;

/* Kernel kinds, as reported by tqr_tasks(). */
typedef enum {
    TQR_GEQRT = 0, TQR_UNMQR = 1, TQR_TTQRT = 2, TQR_TTMQR = 3, TQR_TSQRT = 4, TQR_TSMQR = 5
} tqr_kernel;

#define TQR_OK 0
#define TQR_ERR_INVALID_LIST (-100) /* elimination list breaks a Section 2.2 rule */
#define TQR_ERR_TIMEOUT (-101)      /* a device wait ran past its time limit      */
#define TQR_ERR_NONFINITE (-102)    /* a Householder norm was Inf or NaN          */
#define TQR_ERR_CUDA (-103)         /* a CUDA runtime call failed                 */
#define TQR_ERR_NOMEM (-104)        /* device or host allocation failed           */
#define TQR_ERR_CAPACITY (-105)     /* caller's output array too small            */
#define TQR_ERR_INTERNAL (-106)     /* inconsistent internal state                */
#define TQR_ERR_UNSUPPORTED (-107)  /* parameters outside what the kernels handle */
#define TQR_ERR_TOO_LARGE (-108)    /* problem exceeds tqr_factor_noalloc's fixed scratch */

typedef struct tqr_factors tqr_factors;

/* Arithmetic of the update kernels (UNMQR/TSMQR/TTMQR).  Panels (reflector
 * generation, T factors) and everything a least-squares solve does with A and
 * its residual stay FP64 in every mode. */
typedef enum {
    TQR_FP64 = 0,        /* FP64 everywhere                                   */
    TQR_SPLIT_TF32 = 1,  /* updates on tensor cores, operands split hi+lo TF32, 3 products, FP32 accumulation */
    TQR_TF32 = 2         /* updates on tensor cores, one TF32 product, FP32 accumulation */
} tqr_precision;

/* Result of tqr_lstsq. */
typedef struct {
    int32_t refine_iterations;  /* FP64 refinement steps taken                       */
    int32_t cgls_iterations;    /* R-preconditioned CGLS steps taken                  */
    int32_t converged;          /* 1 if the backward error reached tol (FP64 with tol = 0: 1) */
    int32_t status;             /* device status of the factorization                */
    double backward_error;      /* ||A^T r||_2 / (||A||_F ||r||_2), r = b - A x      */
    double residual_norm;       /* ||r||_2                                           */
    double factor_seconds;      /* factorization + Q^T b, wall time                  */
    double solve_seconds;       /* solution, preconditioner and refinement, wall time */
} tqr_lstsq_info;

/* Summary of a factorization handle. */
typedef struct {
    int64_t m, n;          /* matrix size                                  */
    int32_t nb, ib;        /* tile size and inner blocking                 */
    int32_t p, q;          /* tile rows ceil(m/nb), tile columns ceil(n/nb) */
    int32_t tree, BS;      /* tree (-1 for a caller-given list), domain size */
    int32_t ts;            /* 0 TT kernels, 1 TS kernels, 2 TS inside PlasmaTree domains + TT merges */
    int32_t strip;         /* columns per update task on the device        */
    int64_t n_elims;       /* length of the elimination list               */
    int64_t n_tile_tasks;  /* kernel tasks (Algorithms 2/3)                */
    int64_t n_device_tasks;/* tasks after splitting updates into strips and
                              panels into blocks (nb >= 128, nb / ib >= 2, ib >= 8)     */
    int64_t n_edges;       /* dependency edges of the device task graph    */
    int64_t critical_path; /* unit-weight critical path, units of nb^3/3    */
    double flops;          /* 2 n^2 (m - n/3), the LAPACK count (Section 2.2) */
} tqr_info;

/* ---------------------------------------------------------------------------
 * Factorization (Sections 2.1-2.3).
 *
 * tqr_factor: A = Q R in place.  A is a device pointer to an m x n matrix,
 * column-major, leading dimension m (lda = m), m >= n >= 1.  On return (once
 * the stream reaches it) A holds R in its upper triangle and the Householder
 * reflectors V below it and in the zeroed tiles, exactly as LAPACK/PLASMA's
 * GEQRT, TTQRT and TSQRT leave them; the reflectors' tau values stay inside
 * the handle.  m and n need not be multiples of nb: the last tile row/column
 * is ragged and behaves as if zero-padded (R and V are unchanged by the
 * padding).
 *   nb:   tile size, 8 <= nb <= 256, nb % 4 == 0.
 *   ib:   inner blocking, ib divides nb, ib <= 64.
 *   tree: a tqr_tree value.  BS: PlasmaTree / PlasmaTree-TS domain size,
 *         1 <= BS <= p, or the k of GRASAP(k), 0 <= k <= q (ignored by
 *         other trees).
 *   out:  receives the handle.  If *out already holds a handle made for the
 *         same (m, n, nb, ib, tree, BS), its device buffers are reused and
 *         nothing is allocated; otherwise a new handle is created (the old
 *         one is left untouched).  Set *out = NULL before the first call.
 * Errors: -1..-9 argument errors, TQR_ERR_NOMEM, TQR_ERR_CUDA, and
 * TQR_ERR_CAPACITY when the task graph could exceed 2e9 device tasks
 * (p q (q+1) (nb/8+1) >= 2e9, e.g. 65536 x 65536 with nb = 16), checked
 * before anything is built.
 * ------------------------------------------------------------------------- */
int tqr_factor(double* A, int64_t m, int64_t n, int nb, int ib, int tree, int BS,
               void* stream, tqr_factors** out);

/* tqr_factor with a choice of update arithmetic (tqr_precision).  With
 * TQR_SPLIT_TF32 / TQR_TF32 the panel kernels also form the compact-WY T of
 * each block of ib reflectors in FP64, and the update kernels apply
 * C <- C - V (T^T (V^T C)) with both products on the tensor cores; A (R and V)
 * stays FP64.  Low precision needs nb % 16 == 0, nb >= 64 and ib in {16, 32}
 * (else TQR_ERR_UNSUPPORTED).  Argument errors: as tqr_factor, -8 for an
 * unknown precision, -10 for out. */
int tqr_factor_ex(double* A, int64_t m, int64_t n, int nb, int ib, int tree, int BS, int precision,
                  void* stream, tqr_factors** out);

/* Same with a caller-given elimination list: `list` (host) holds `count`
 * 0-based triplets (i, piv, k) in order; ts = 1 selects TS kernels, 0 TT.
 * The list is checked against the rules of Section 2.2 first
 * (TQR_ERR_INVALID_LIST); with ts = 1 a list that zeroes a tile already in
 * triangle form (a row that was a pivot earlier in the same column) is
 * invalid too, since TSQRT needs a square tile there.  *out is reused only if
 * it was made from the same list. */
int tqr_factor_list(double* A, int64_t m, int64_t n, int nb, int ib, const int32_t* list,
                    int64_t count, int ts, void* stream, tqr_factors** out);

/* B <- Q^T B (tqr_apply_qt) or B <- Q B (tqr_apply_q) with the Q of a
 * factorization.  B: device, m x nrhs, column-major, leading dimension
 * ldb >= m.  The transformations are replayed in elimination-list order (or
 * reverse order for Q), on the stream given.  The factorization must have been
 * enqueued earlier on the same stream (or be complete). */
int tqr_apply_qt(tqr_factors* f, double* B, int64_t ldb, int64_t nrhs, void* stream);
int tqr_apply_q(tqr_factors* f, double* B, int64_t ldb, int64_t nrhs, void* stream);

/* Compact-WY T factors (Section 1; LAPACK/PLASMA storage) of every GEQRT
 * and of every TTQRT/TSQRT, formed from the stored reflectors.  Each output
 * is a device array of p*q tiles of ib x nb doubles; the T of tile (i,k)
 * (0-based) starts at offset ((size_t)k*p + i)*ib*nb and is column-major
 * ib x nb: columns b*ib..b*ib+ib-1 hold the upper-triangular ib x ib factor
 * of reflectors b*ib..b*ib+ib-1.  T_geqrt receives the T of GEQRT(i,k);
 * T_elim the T of the TTQRT/TSQRT that zeroed tile (i,k).  Tiles without
 * such a kernel are set to zero.  Either pointer may be NULL. */
int tqr_form_t(tqr_factors* f, double* T_geqrt, double* T_elim, void* stream);

/* Per-task trace of the last factorization on a handle (profiling; the
 * paper's simulator has no device counterpart).  tqr_set_trace(f, 1) makes
 * later factorizations with f record, for every device task, its start and
 * end on the GPU's %globaltimer (ns) and the SM that ran it (allocates
 * 16 bytes per task once); with TQR_TRACE set (not "0") in the environment
 * every new handle starts with tracing on.  tqr_get_trace waits for the handle's work and
 * writes 8 int64 per task to out (host): kind, i, piv, k, w, start ns, end ns,
 * SM id -- in device task order; w = j * 65536 + strip for an update strip
 * (columns strip*W.. of tile column j, W = tqr_info.strip), -1 for a panel run
 * as one task, and b << 32 | c_lo << 16 | c_hi for a task of block b of a panel
 * split into blocks of ib columns: it factors the block when c_lo = b * ib,
 * else applies the block's reflectors to columns [c_lo, c_hi) of the tile
 * (pair).  cap in tasks, *count = number of tasks (TQR_ERR_CAPACITY if cap is
 * too small, TQR_ERR_UNSUPPORTED if tracing was not enabled). */
int tqr_set_trace(tqr_factors* f, int enable);
int tqr_get_trace(tqr_factors* f, int64_t* out, int64_t cap, int64_t* count);

/* Dependency edges (u -> v: v may start only after u has finished) of the
 * handle's factorization graph, in the device task numbering of
 * tqr_get_trace; host only.  With a trace, every edge must satisfy
 * end(u) <= start(v) (a happens-before check of the executor).  Every edge
 * runs from a task to a later one (u < v: tasks are numbered in program
 * order), so the task order is a topological order.  cap in edges,
 * *count = number of edges (TQR_ERR_CAPACITY if cap is too small). */
int tqr_get_edges(const tqr_factors* f, int32_t* src, int32_t* dst, int64_t cap, int64_t* count);

/* Test instrument: fills the handle's workspace -- tau arrays, and the FP32
 * T and V arrays of a low-precision handle -- with NaN on the handle's stream.
 * A following factorization with the handle reads those entries only after
 * the tasks that write them have run, so its results stay finite and equal
 * to an unpoisoned run's; a read before the write shows up as NaN. */
int tqr_poison_workspace(tqr_factors* f);

/* Waits for the handle's last enqueued work and returns its device status:
 * TQR_OK, TQR_ERR_TIMEOUT, TQR_ERR_NONFINITE or TQR_ERR_CUDA. */
int tqr_sync(tqr_factors* f);

/* Fills *info.  Host only. */
int tqr_get_info(const tqr_factors* f, tqr_info* info);

/* Releases the handle's device and host memory (synchronizes first). */
void tqr_free(tqr_factors* f);

/* The library caches one plan (elimination list, task graph on the device,
 * apply graphs) per distinct (m, n, nb, ib, tree, BS) or caller-given list it
 * has factored, so that later calls with the same arguments build nothing.
 * tqr_release_plans frees the workspace tqr_lstsq keeps, drops every cached
 * plan that no live handle uses, frees its device memory, and clears the
 * host-side plans of batched calls; it
 * returns the number of device plans dropped (>= 0) or TQR_ERR_INTERNAL.
 * Live handles keep their own plan and stay valid; a later call with released
 * arguments rebuilds the plan.  Host entry point: it frees device memory, so
 * it synchronizes with the device and must not be called during stream
 * capture. */
int tqr_release_plans(void);

/* End-to-end convenience for host data: copies A_host (m x n, column-major,
 * leading dimension m) to the device, factors it, and copies A (R and V)
 * back to A_host; if B_host is not NULL it also copies B_host (m x nrhs,
 * leading dimension m) in, applies Q^T and copies it back.  Device buffers
 * are owned by the handle and reused across calls with the same shape (set
 * *out = NULL before the first call).  Synchronizes before returning. */
int tqr_factor_host(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS,
                    double* B_host, int64_t nrhs, void* stream, tqr_factors** out);

/* tqr_factor_host without the final wait: every copy and kernel is enqueued on
 * `stream` and the call returns; tqr_sync(*out) waits and reports the status.
 * A_host (and B_host) must stay allocated and unmodified until then; with
 * pinned host memory the copies run asynchronously, so matrices handled on
 * different streams overlap their transfers with each other's factorization. */
int tqr_factor_host_async(double* A_host, int64_t m, int64_t n, int nb, int ib, int tree, int BS,
                          double* B_host, int64_t nrhs, void* stream, tqr_factors** out);

/* Least squares min ||A x - b||_2 (Section 1 names least squares as the main
 * use of the factorization).  A: device, m x n (m >= n), column-major, lda = m,
 * left unchanged (the library factors a copy); b: device, m; x: device, n,
 * output.  The copy of A is factored with `precision`; c = Q^T b is formed with
 * the reflectors in FP64; x solves R x = c[0:n] by blocked back substitution
 * in FP64.  For a low-precision factorization x is then refined in FP64 --
 * residual r = b - A x, correction R^-1 R^-T A^T r with an explicit FP64
 * inverse of the computed R as the preconditioner -- until the backward error
 * ||A^T r|| / (||A||_F ||r||) <= tol; if a step fails to halve it, CGLS on the
 * correction problem, right-preconditioned by R^-1, continues, for at most
 * maxit steps in all.  In FP64 tol is only compared with the final backward
 * error (converged = 1 when tol = 0).  info (host, may be NULL) receives iteration counts,
 * final backward error and phase times.  Synchronizes `stream` before
 * returning.  R^-1 and R^-T are applied by blocked substitution, never formed.
 * Device workspace (a copy of A, m*n doubles, plus vectors) and the factor
 * handle (with FP32 copies of the reflectors in low precision) stay allocated
 * after the call and serve the next call with the same arguments from any
 * host thread (a call made while another thread's call uses them allocates
 * its own, freed on return); tqr_release_plans() frees them.  Argument errors, checked before any device work: -k for argument k
 * (1 A, 2 m, 3 n, 4 b, 5 x, 6 nb, 7 ib, 8 tree, 9 BS, 10 precision, 11 tol
 * negative, NaN or infinite, 12 maxit), with nb, ib, tree and BS under
 * tqr_factor's rules; TQR_ERR_CAPACITY as tqr_factor. */
int tqr_lstsq(const double* A, int64_t m, int64_t n, const double* b, double* x, int nb, int ib,
              int tree, int BS, int precision, double tol, int maxit, void* stream,
              tqr_lstsq_info* info);

/* ---------------------------------------------------------------------------
 * Batched factorization: `count` independent matrices in one persistent
 * launch.  The task graphs of all matrices are concatenated; any CTA may run
 * any matrix's ready task, so small matrices fill the GPU together.
 *   A:  host array of `count` device pointers, matrix c is m[c] x n[c],
 *       column-major with leading dimension m[c], overwritten by R and V.
 *   nb, ib, tree, BS: host arrays of per-matrix parameters (as tqr_factor),
 *       so every size class can use its own tuned configuration.
 *   out: receives the batch handle.  If *out was made by a call with the same
 *       count and identical A, m, n, nb, ib, tree and BS arrays, it is launched
 *       again without any allocation or host-to-device copy (such a call can be
 *       captured into a CUDA graph); otherwise a new handle is built (allocates
 *       and copies; the old one is left untouched).
 * Argument errors: -1 count, -2 A, -3 m, -4 n, -5 nb, -6 ib, -7 tree, -8 BS,
 * -10 out, each for the first offending matrix. */
typedef struct tqr_batch tqr_batch;

typedef struct {
    int32_t count;          /* matrices                                    */
    int32_t strip;          /* columns per update task                      */
    int64_t n_tasks;        /* device tasks of the combined graph           */
    int64_t n_edges;        /* dependency edges                             */
    int64_t max_critical_path; /* largest unit-weight critical path         */
    double flops;           /* sum of 2 n^2 (m - n/3)                       */
    int32_t n_fused;        /* matrices run by the one-tile-column FlatTree-TS kernel */
    int32_t f32;            /* 1 for a tqr_factor_batched_f32 batch         */
} tqr_batch_info;

int tqr_factor_batched(int count, double* const* A, const int64_t* m, const int64_t* n, const int32_t* nb,
                       const int32_t* ib, const int32_t* tree, const int32_t* BS, void* stream,
                       tqr_batch** out);
/* One tile column, FlatTree with TS kernels (q = 1).  A matrix with
 * tree = TQR_FLAT_TS, n <= nb and n <= 128 is factored by a kernel that runs
 * the whole chain GEQRT(1,1), TSQRT(2,1,1), ..., TSQRT(p,1,1) of one matrix in
 * one CTA with the tile in registers and R resident in shared memory
 * (Proposition 2's flat tree; the batch supplies the parallelism), provided nb
 * is 64, 128 or 256 and at least n rounded up to 32 / 64 / 128; with FP64,
 * n in 65..128 needs nb = 128.  The results equal
 * tqr_factor's for the same (nb, TQR_FLAT_TS) up to rounding.  All such
 * matrices of a batch run in ONE persistent launch: one CTA of 1024 threads
 * per SM whose slots of 1024, 512 or 256 threads (the thread count of the
 * matrix's class) pop matrices, largest first, from one queue per thread
 * count.  The batch's other matrices go to the task-graph executor in a
 * second launch after it; both on `stream`, after one memset of the batch's
 * status and queue counters.
 *
 * tqr_factor_batched_f32: the same for FP32 matrices (all arithmetic FP32);
 * every matrix must satisfy the one-tile-column conditions above (FP32 also
 * allows nb = 256 with n in 65..128), otherwise
 * TQR_ERR_UNSUPPORTED.  Argument errors: -1 count, -2 A, -3 m, -4 n, -5 nb,
 * -7 out.  Reuse and graph capture as for tqr_factor_batched.
 *
 * tqr_batch_tau: copies matrix c's tau values (p*q*nb entries each, of the
 * batch's type, tile (i,k) reflector j at (k*p + i)*nb + j) into tau_ge
 * (GEQRT) and tau_el (TSQRT/TTQRT), host or device buffers; waits for the
 * batch's stream first. */
int tqr_factor_batched_f32(int count, float* const* A, const int64_t* m, const int64_t* n, const int32_t* nb,
                           void* stream, tqr_batch** out);
/* Host only (no GPU, nothing allocated on a device): the queues of the batch's
 * persistent one-tile-column launch for `count` matrices m[c] x n[c] with tile
 * height nb[c] (FP32 when f32 is nonzero), each satisfying the one-tile-column
 * conditions above.  order[i] receives the index of the i-th queued matrix
 * (count entries); bounds[2k], bounds[2k+1] the begin and end of the queue of
 * 1024 >> k threads (6 entries); *quarter_bytes the shared-memory quarter (a
 * slot of t threads owns t/256 quarters).  Returns 0; -1 count, -2 m (or a
 * null size array), -3 n, -5 a null output; TQR_ERR_UNSUPPORTED for a matrix
 * the one-tile-column kernel does not take. */
int tqr_ts1_plan(int count, const int64_t* m, const int64_t* n, const int32_t* nb, int f32, int32_t* order,
                 int32_t* bounds, int32_t* quarter_bytes);
int tqr_batch_tau(const tqr_batch* b, int c, void* tau_ge, void* tau_el);

/* Waits for the batch's last launch; returns its device status. */
int tqr_batch_sync(tqr_batch* b);
int tqr_batch_get_info(const tqr_batch* b, tqr_batch_info* info);
void tqr_batch_free(tqr_batch* b);

/* ---------------------------------------------------------------------------
 * Cost-model network (the paper has no learned component; the autotuner uses
 * it to rank configurations without timing them).  A 3-layer perceptron
 * in -> 64 -> 64 -> 1 with ReLU, FP32.  Parameters are one device array of
 * tqr_mlp_param_count(in) floats: W1 (64 x in, row-major), b1 (64), W2 (64 x
 * 64, row-major), b2 (64), W3 (64), b3 (1).  X is B x in row-major (device).
 *   tqr_mlp_forward:   y[s] = network(X[s]) for s < B.
 *   tqr_mlp_loss_grad: loss (device scalar) = (1/B) sum_s (y[s] - t[s])^2 and
 *                      its gradient w.r.t. the parameters into grad; work is a
 *                      device scratch of B * (4*64 + 2) floats.  The gradient
 *                      of every parameter is summed over samples in a fixed
 *                      order (deterministic).
 *   tqr_mlp_adam_step: one Adam update (bias-corrected, step >= 1) of count
 *                      parameters with moment arrays m, v (device, zeroed
 *                      before step 1). */
#define TQR_MLP_MAX_IN 32
int tqr_mlp_param_count(int in_dim);
int tqr_mlp_forward(const float* params, int in_dim, const float* X, int B, float* y, void* stream);
int tqr_mlp_loss_grad(const float* params, int in_dim, const float* X, const float* t, int B, float* work,
                      float* grad, float* loss, void* stream);
int tqr_mlp_adam_step(float* params, const float* grad, float* m, float* v, int count, float lr, float beta1,
                      float beta2, float eps, int step, void* stream);

/* ---------------------------------------------------------------------------
 * Host-only integer entry points (no GPU needed).
 * ------------------------------------------------------------------------- */

/* Elimination list of `tree` for p x q tiles (p >= q >= 1), as 0-based
 * triplets (i, piv, k) written to out[3*e .. 3*e+2] for e < *count.
 * cap: capacity of `out` in triplets; TQR_ERR_CAPACITY if too small (then
 * *count holds the needed size). */
int tqr_elimination_list(int p, int q, int tree, int BS, int32_t* out, int64_t cap,
                         int64_t* count);

/* TQR_OK if the list is a valid elimination list for p x q tiles (Section
 * 2.2: one entry per subdiagonal tile of the first min(p,q) columns, both
 * rows ready, pivot still a potential annihilator), else
 * TQR_ERR_INVALID_LIST. */
int tqr_validate_list(int p, int q, const int32_t* list, int64_t count);

/* Critical path of `tree` in units of nb^3/3 flops (Table 1 weights,
 * unbounded processors, every kernel starts as soon as its dependencies
 * are met).  zero_time, if not NULL, receives p*q values: zero_time[i*q+k]
 * = time at which tile (i,k) is zeroed, or -1 for tiles that are not. */
int tqr_critical_path(int p, int q, int tree, int BS, int64_t* cp, int32_t* zero_time);

/* Kernel tasks of `tree` in program order (Algorithms 2 and 3), as 5 ints
 * per task: kind (tqr_kernel), i, piv, k, j (0-based; piv = -1 for GEQRT and
 * UNMQR, j = -1 for the three panel kernels).  finish, if not NULL, receives
 * each task's unit-weight ASAP finish time.  cap in tasks. */
int tqr_tasks(int p, int q, int tree, int BS, int32_t* out, int64_t* finish, int64_t cap,
              int64_t* count);

/* The device task graph that tqr_factor executes for this problem, built on
 * the host (no GPU needed) for update strips of `strip` columns (16, 32 or 64;
 * tqr_info.strip reports the width a GPU uses: 64 for nb >= 64 with the
 * default shared-memory budget).  tasks (host) receives 6 ints per device
 * task, in device order: kind, i, piv, k, j, strip.  For an update (UNMQR,
 * TTMQR, TSMQR) j is the updated tile column and strip its column strip.  For
 * a panel (GEQRT, TTQRT, TSQRT) run as one task j = -1; a panel split into
 * blocks of ib columns (nb / ib >= 2 and ib >= 8) has for each block b one
 * task j = b, strip = -1 that factors the block, then tasks j = b,
 * strip = c_lo | c_hi << 16 that apply its reflectors to columns [c_lo, c_hi)
 * of the same tile (pair).  src/dst (host) receive the dependency edges
 * (src -> dst, src < dst).  Caps in tasks and edges; *ntasks and *nedges are
 * always set (TQR_ERR_CAPACITY if a cap is too small).  Argument errors: -2 m,
 * -3 n, -4 nb, -5 ib, -6 tree, -7 BS, -8 strip, -11 ntasks, -15 nedges NULL.
 * The dependency rule (Section 2.3 execution model, refined to column units):
 * a task depends on the previous writer, in program order, of every unit of
 * gcd(ib, strip) columns it writes in each tile, and a task applying
 * reflectors on the task that formed them. */
int tqr_device_graph(int64_t m, int64_t n, int nb, int ib, int tree, int BS, int strip, int32_t* tasks,
                     int64_t task_cap, int64_t* ntasks, int32_t* src, int32_t* dst, int64_t edge_cap,
                     int64_t* nedges);

/* Peak-rate probes: the roofline denominators of the library's kernels,
 * measured on the GPU that runs them (measurement support; the paper has no
 * counterpart).  Enqueues on `stream` one launch that keeps every SM busy
 * with independent chains of one kind of instruction for `iters` iterations
 * and sets *flops (host) to the flops that launch performs; time the launch
 * with events to get the rate.  kind: TQR_PEAK_DFMA (FP64 fma, the FP64
 * kernels' arithmetic), TQR_PEAK_DMMA (FP64 mma.sync m8n8k4), TQR_PEAK_FFMA
 * (FP32 fma), TQR_PEAK_TF32 (TF32 mma.sync m16n8k8 with FP32 accumulation).
 * The first call on a device allocates one word of device memory that the
 * library keeps until exit.  Errors: -1 kind, -2 iters < 1, -4 flops NULL,
 * TQR_ERR_CUDA, TQR_ERR_NOMEM. */
enum { TQR_PEAK_DFMA = 0, TQR_PEAK_DMMA = 1, TQR_PEAK_FFMA = 2, TQR_PEAK_TF32 = 3 };
int tqr_peak_probe(int kind, int64_t iters, void* stream, double* flops);

/* Test support for failure detection (the paper has no counterpart).
 * tqr_set_timeout_ms: limit, in milliseconds, for any single device wait of
 * later launches (ms <= 0 restores the default, which scales with the
 * problem's flop count; the TQR_TIMEOUT_MS environment variable also sets it).
 * tqr_inject_fault(1): the next factorization or apply launch drops its
 * initially ready tasks on the host, so no task ever becomes ready, every
 * wait runs out, and tqr_sync() reports TQR_ERR_TIMEOUT; the device context
 * stays usable.  tqr_inject_fault(0) cancels a pending injection. */
int tqr_set_timeout_ms(double ms);
int tqr_inject_fault(int kind);

/* ---------------------------------------------------------------------------
 * Factorization without allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate memory when they factor --
 * code running while a CUDA stream is being captured into a graph (where
 * cudaMalloc is not allowed), services confined to a device-memory budget
 * fixed at start-up, real-time loops that forbid allocation after
 * initialization.  It computes exactly what tqr_factor computes (same task
 * graph, same kernels) but calls no cudaMalloc, cudaFree or other allocating
 * routine, on the device or the host.
 *
 * Its working state (task graph, dependency counters, ready queue) lives in
 * one fixed array of TQR_NOALLOC_SCRATCH_BYTES (4 MiB) inside the library;
 * every GPU that loads the library holds that array until the process exits.
 * Limits: p*q <= TQR_NOALLOC_MAX_TILES tiles and at most
 * TQR_NOALLOC_MAX_TASKS device tasks (updates count once per strip of
 * columns; e.g. 16384 x 4096 at nb 256 fits, 16384 x 8192 does not);
 * larger problems return TQR_ERR_TOO_LARGE and nothing is launched.
 *
 *   A:     device, m x n, column-major, lda = m; overwritten by R and V.
 *   nb, ib: as for tqr_factor.
 *   list:  host, `count` 0-based triplets (i, piv, k), e.g. from
 *          tqr_elimination_list(); checked by the same validity rules as
 *          tqr_factor_list (TQR_ERR_INVALID_LIST).  ts = 1: TS kernels, 0: TT kernels;
 *          with ts = 1, zeroing a tile already in triangle form is also
 *          TQR_ERR_INVALID_LIST.
 *   tau_geqrt, tau_elim: device outputs, p*q*nb doubles each; the tau of
 *          reflector r of GEQRT(i,k) (resp. of the TTQRT/TSQRT zeroing tile
 *          (i,k)) is stored at [((size_t)k*p + i)*nb + r].
 *   status: device output, one int32: set to 0 when the work starts and to
 *          TQR_ERR_TIMEOUT or TQR_ERR_NONFINITE if the device detects one.
 *   stream: the work is enqueued on it.  Outside stream capture the task
 *          graph is uploaded with cudaMemcpyAsync from the library's pageable
 *          host arrays, and CUDA finishes the work already queued on `stream`
 *          before such a copy starts: the call blocks until then.  That wait is
 *          what lets the next call reuse the host arrays safely.  Under stream
 *          capture nothing waits (see below).  The factorization itself is not
 *          waited for in either case.
 *   Device waits are bounded like tqr_factor's (tqr_set_timeout_ms,
 *          TQR_TIMEOUT_MS), and tqr_inject_fault applies to this call too.
 *
 * The first call on each device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  On a stream that is being captured into
 * a CUDA graph, the task graph is written to the device by small kernels that
 * carry it in their parameters (a copy from the library's pageable host
 * arrays could not be captured), so the captured work replays this call's
 * problem whatever later calls do on the host; outside capture it is copied
 * with cudaMemcpyAsync.  Every call reuses the same array and
 * overwrites what the previous call left in it (each launch re-initializes
 * its counters and queue); calls whose device work overlaps -- on two
 * streams without ordering between them, say -- race on the array and give
 * wrong results.  Host threads are serialized while a call prepares its work.
 * ------------------------------------------------------------------------- */
/* Test support: the task graph tqr_factor_noalloc builds for these
 * arguments (its own fixed-capacity builder, panels as whole tasks), built on
 * the host for update strips of `strip` columns (16, 32 or 64), in the format
 * of tqr_device_graph.  No GPU is needed and nothing is allocated.  Argument
 * errors: -1 m, -2 n, -3 nb, -4 ib, -5 list, -6 count, -7 ts, -8 strip,
 * -11 ntasks, -15 nedges NULL; TQR_ERR_INVALID_LIST, TQR_ERR_TOO_LARGE and
 * TQR_ERR_CAPACITY as for the factorization. */
int tqr_noalloc_graph(int64_t m, int64_t n, int nb, int ib, const int32_t* list, int64_t count, int ts,
                      int strip, int32_t* tasks, int64_t task_cap, int64_t* ntasks, int32_t* src,
                      int32_t* dst, int64_t edge_cap, int64_t* nedges);

#define TQR_NOALLOC_SCRATCH_BYTES (4 << 20)
#define TQR_NOALLOC_MAX_TASKS 65536
#define TQR_NOALLOC_MAX_TILES 4096
int tqr_factor_noalloc(double* A, int64_t m, int64_t n, int nb, int ib, const int32_t* list,
                       int64_t count, int ts, double* tau_geqrt, double* tau_elim, int32_t* status,
                       void* stream);

/* Message for a status code. */
const char* tqr_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* TQR_H */
