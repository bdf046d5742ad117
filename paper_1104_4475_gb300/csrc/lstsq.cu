// Least squares min ||A x - b|| on top of the tiled QR (the paper's motivating
// use, Section 1), with an optional low-precision factorization refined in
// FP64:
//   1. factor a copy of A (FP64, or FP64 panels + split-TF32 / TF32 updates);
//   2. c = Q^T b with the stored reflectors applied in FP64;
//   3. x = R^-1 c[0:n] by blocked back substitution on the computed R (FP64,
//      backward stable);
//   4. low precision: the computed R preconditions a corrected
//      semi-normal-equation refinement in FP64,
//        r = b - A x,  s = A^T r,  x += R^-1 R^-T s,
//      until the backward error ||A^T r|| / (||A||_F ||r||) reaches tol; if it
//      stops decreasing, R-preconditioned CGLS (min ||A R^-1 z - b||, x =
//      R^-1 z) continues from the current x.  R^-1 and R^-T are applied by
//      blocked back and forward substitution (never formed).
// Every residual, product with A and the solution are FP64.  The workspace
// and the factor handle of the last call stay allocated for the next call of
// the same shape (release_lstsq_cache frees them).
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <cmath>
#include <vector>

namespace {

constexpr int kT = 256;

// y = b - A x  (A: m x n column-major, lda).  One thread per row; x staged
// in shared memory in chunks.
__global__ void resid_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                             const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ y) {
    __shared__ double xs[1024];
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += 1024) {
        const int64_t cn = std::min<int64_t>(1024, n - c0);
        __syncthreads();
        for (int64_t t = threadIdx.x; t < cn; t += blockDim.x) xs[t] = x[c0 + t];
        __syncthreads();
        if (r < m) {
            const double* a = A + r + c0 * lda;
            int64_t c = 0;
            for (; c + 1 < cn; c += 2) {
                acc0 = fma(a[c * lda], xs[c], acc0);
                acc1 = fma(a[(c + 1) * lda], xs[c + 1], acc1);
            }
            if (c < cn) acc0 = fma(a[c * lda], xs[c], acc0);
        }
    }
    if (r < m) y[r] = b[r] - (acc0 + acc1);
}

__device__ __forceinline__ double warp_reduce(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// s = A^T r: one warp per column.
__global__ void atr_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                           const double* __restrict__ r, double* __restrict__ s) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const double* a = A + c * lda;
    double acc = 0.0;
    for (int64_t i = lane; i < m; i += 32) acc = fma(a[i], r[i], acc);
    acc = warp_reduce(acc);
    if (lane == 0) s[c] = acc;
}

// One step of the blocked back substitution that solves R x = y for upper-
// triangular R = triu(R[0:n, 0:n]) (lda), block rows of kBk from the bottom:
// step kb solves the diagonal block R[r0:r1, r0:r1] x[r0:r1] = y[r0:r1] and
// subtracts R[0:r0, r0:r1] x[r0:r1] from y[0:r0].  Every CTA solves the small
// triangle itself (one warp, column-oriented, in shared memory) and then
// updates its own rows of y; CTA 0 writes x[r0:r1].  Rows r0.. of y are only
// read during the step, rows < r0 only written by the CTA that owns them.
constexpr int kBk = 64;
__global__ void trsv_step_kernel(const double* __restrict__ R, int64_t lda, int64_t n, int64_t r0,
                                 double* __restrict__ y, double* __restrict__ x) {
    __shared__ double Rd[kBk][kBk + 1];
    __shared__ double xs[kBk];
    const int64_t r1 = std::min<int64_t>(n, r0 + kBk);
    const int nbk = static_cast<int>(r1 - r0);
    for (int t = threadIdx.x; t < kBk * kBk; t += blockDim.x) {
        const int r = t % kBk, c = t / kBk;
        Rd[r][c] = (r < nbk && c < nbk && r <= c) ? R[(r0 + r) + (r0 + c) * lda] : 0.0;
    }
    for (int t = threadIdx.x; t < kBk; t += blockDim.x) xs[t] = t < nbk ? y[r0 + t] : 0.0;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = nbk - 1; j >= 0; --j) {
            const double xj = xs[j] / Rd[j][j];
            __syncwarp();
            if (lane == 0) xs[j] = xj;
            for (int i = lane; i < j; i += 32) xs[i] = fma(-Rd[i][j], xj, xs[i]);
            __syncwarp();
        }
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < nbk; t += blockDim.x) x[r0 + t] = xs[t];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < r0;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nbk; ++c) acc = fma(R[i + (r0 + c) * lda], xs[c], acc);
        y[i] -= acc;
    }
}

// One step of the blocked forward substitution that solves R^T x = y (R^T
// lower triangular), block rows of kBk from the top: step r0 solves
// R[r0:r1, r0:r1]^T x[r0:r1] = y[r0:r1] (every CTA, one warp, in shared
// memory) and subtracts R[r0:r1, i]^T x[r0:r1] from y[i] for i >= r1, one
// warp per row i reading column i of R over the block (coalesced); CTA 0
// writes x[r0:r1].
__global__ void trsv_t_step_kernel(const double* __restrict__ R, int64_t lda, int64_t n, int64_t r0,
                                   double* __restrict__ y, double* __restrict__ x) {
    __shared__ double Rd[kBk][kBk + 1];
    __shared__ double xs[kBk];
    const int64_t r1 = std::min<int64_t>(n, r0 + kBk);
    const int nbk = static_cast<int>(r1 - r0);
    for (int t = threadIdx.x; t < kBk * kBk; t += blockDim.x) {
        const int r = t % kBk, c = t / kBk;
        Rd[r][c] = (r < nbk && c < nbk && r <= c) ? R[(r0 + r) + (r0 + c) * lda] : 0.0;
    }
    for (int t = threadIdx.x; t < kBk; t += blockDim.x) xs[t] = t < nbk ? y[r0 + t] : 0.0;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = 0; j < nbk; ++j) {
            const double xj = xs[j] / Rd[j][j];
            __syncwarp();
            if (lane == 0) xs[j] = xj;
            for (int i = j + 1 + lane; i < nbk; i += 32) xs[i] = fma(-Rd[j][i], xj, xs[i]);
            __syncwarp();
        }
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < nbk; t += blockDim.x) x[r0 + t] = xs[t];
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    for (int64_t i = r1 + static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32; i < n;
         i += warps) {
        const double* col = R + r0 + i * lda;
        double acc = 0.0;
        for (int c = lane; c < nbk; c += 32) acc = fma(col[c], xs[c], acc);
        acc = warp_reduce(acc);
        if (lane == 0) y[i] -= acc;
    }
}

// out[0] += sum x[i]*y[i] (block partials via atomics on a zeroed slot).
__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* out) {
    __shared__ double part[kT / 32];
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        acc = fma(x[i], y[i], acc);
    acc = warp_reduce(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.0;
        v = warp_reduce(v);
        if (threadIdx.x == 0) atomicAdd(out, v);
    }
}

// y = a*x + y
__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

// p = s + beta p
__global__ void xpby_kernel(const double* __restrict__ s, double beta, double* __restrict__ p, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = fma(beta, p[i], s[i]);
}

struct Ws {
    double *Af = nullptr, *c = nullptr, *r = nullptr, *q = nullptr;
    double *s = nullptr, *u = nullptr, *d = nullptr, *t = nullptr, *pv = nullptr, *y = nullptr, *sc = nullptr;
    ~Ws() {
        for (double* p : {Af, c, r, q, s, u, d, t, pv, y, sc}) cudaFree(p);
    }
    bool alloc(int64_t m, int64_t n) {
        const size_t mn = static_cast<size_t>(m) * n;
        return cudaMalloc(&Af, mn * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c, m * sizeof(double)) == cudaSuccess && cudaMalloc(&r, m * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&q, m * sizeof(double)) == cudaSuccess && cudaMalloc(&s, n * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&u, n * sizeof(double)) == cudaSuccess && cudaMalloc(&d, n * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&t, n * sizeof(double)) == cudaSuccess && cudaMalloc(&pv, n * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&y, n * sizeof(double)) == cudaSuccess && cudaMalloc(&sc, sizeof(double)) == cudaSuccess;
    }
};

// The last call's workspace and factor handle, kept for the next call with
// the same arguments on the same device.
struct LsCache {
    std::mutex mu;
    int dev = -1;
    int64_t m = 0, n = 0;
    int nb = 0, ib = 0, tree = 0, BS = 0, prec = 0;
    Ws* w = nullptr;
    tqr_factors* f = nullptr;
    void drop() {
        if (f) tqr_free(f);
        delete w;
        f = nullptr;
        w = nullptr;
        dev = -1;
    }
};
LsCache g_ls;

struct Solver {
    const double* A;
    int64_t m, n;
    const double* b;
    double* x;
    cudaStream_t st;
    Ws* w = nullptr;
    int blocks = 1024;

    int grid_rows() const { return static_cast<int>((m + kT - 1) / kT); }
    int grid_cols(int64_t cols) const { return static_cast<int>((cols + kT / 32 - 1) / (kT / 32)); }

    double dot(const double* a, const double* b2, int64_t len) {
        cudaMemsetAsync(w->sc, 0, sizeof(double), st);
        dot_kernel<<<std::min<int64_t>(blocks, (len + kT - 1) / kT), kT, 0, st>>>(a, b2, len, w->sc);
        double h = 0.0;
        cudaMemcpyAsync(&h, w->sc, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return h;
    }
    void resid() { resid_kernel<<<grid_rows(), kT, 0, st>>>(A, m, m, n, x, b, w->r); }   // r = b - A x
    void atr(const double* r, double* s) { atr_kernel<<<grid_cols(n), kT, 0, st>>>(A, m, m, n, r, s); }
    // xo = R^-1 y for R = triu(Af[0:n, 0:n]); y (n entries) is overwritten.
    void back_substitute(double* y, double* xo) {
        for (int64_t r0 = ((n - 1) / kBk) * kBk; r0 >= 0; r0 -= kBk) {
            const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, (r0 + kT - 1) / kT)));
            trsv_step_kernel<<<g, kT, 0, st>>>(w->Af, m, n, r0, y, xo);
        }
    }
    // xo = R^-T y; y (n entries) is overwritten.
    void forward_substitute(double* y, double* xo) {
        for (int64_t r0 = 0; r0 < n; r0 += kBk) {
            const int64_t rest = n - std::min<int64_t>(n, r0 + kBk);
            const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, (rest + 7) / 8)));
            trsv_t_step_kernel<<<g, kT, 0, st>>>(w->Af, m, n, r0, y, xo);
        }
    }
    // out = R^-1 v (trans = 0) or R^-T v (trans = 1); v is left unchanged.
    void rsolve(const double* v, double* out, int trans) {
        cudaMemcpyAsync(w->y, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (trans) forward_substitute(w->y, out);
        else back_substitute(w->y, out);
    }
    int nblk(int64_t len) const { return static_cast<int>(std::min<int64_t>(blocks, (len + kT - 1) / kT)); }
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

namespace tqr {
void release_lstsq_cache() {
    std::lock_guard<std::mutex> lk(g_ls.mu);
    g_ls.drop();
}
}  // namespace tqr

extern "C" int tqr_lstsq(const double* A, int64_t m, int64_t n, const double* b, double* x, int nb, int ib,
                         int tree, int BS, int precision, double tol, int maxit, void* stream,
                         tqr_lstsq_info* info) {
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1 || n > m) return -3;
    if (!b) return -4;
    if (!x) return -5;
    // m, n, nb, ib, tree, BS as tqr_factor checks them, reported at this call's positions.
    const int fa = tqr::check_factor_args(m, n, nb, ib, tree, BS);
    if (fa != TQR_OK) return (fa <= -4 && fa >= -7) ? fa - 2 : fa;   // nb..BS: -4..-7 -> -6..-9
    if (precision < TQR_FP64 || precision > TQR_TF32) return -10;
    if (!(tol >= 0.0) || std::isinf(tol)) return -11;
    if (maxit < 0) return -12;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
    tqr_lstsq_info local{};
    tqr_lstsq_info& I = info ? *info : local;
    I = tqr_lstsq_info{};
    Solver S;
    S.A = A;
    S.m = m;
    S.n = n;
    S.b = b;
    S.x = x;
    S.st = static_cast<cudaStream_t>(stream);
    auto t0 = std::chrono::steady_clock::now();
    // The cached workspace and handle when this thread gets the cache and the
    // arguments match; a cache held by another thread leaves this call with
    // its own workspace, freed at the end.
    std::unique_lock<std::mutex> lk(g_ls.mu, std::try_to_lock);
    const bool cached = lk.owns_lock();
    std::unique_ptr<Ws> own;
    tqr_factors* f = nullptr;
    if (cached) {
        const bool same = g_ls.w && g_ls.dev == dev && g_ls.m == m && g_ls.n == n && g_ls.nb == nb &&
                          g_ls.ib == ib && g_ls.tree == tree && g_ls.BS == BS && g_ls.prec == precision;
        if (!same) {
            g_ls.drop();
            g_ls.w = new Ws();
            if (!g_ls.w->alloc(m, n)) {
                g_ls.drop();
                return TQR_ERR_NOMEM;
            }
            g_ls.dev = dev;
            g_ls.m = m;
            g_ls.n = n;
            g_ls.nb = nb;
            g_ls.ib = ib;
            g_ls.tree = tree;
            g_ls.BS = BS;
            g_ls.prec = precision;
        }
        S.w = g_ls.w;
        f = g_ls.f;
    } else {
        own.reset(new Ws());
        if (!own->alloc(m, n)) return TQR_ERR_NOMEM;
        S.w = own.get();
    }
    Ws& W = *S.w;
    const size_t mn = static_cast<size_t>(m) * n;
    cudaMemcpyAsync(W.Af, A, mn * sizeof(double), cudaMemcpyDeviceToDevice, S.st);
    int rc = tqr_factor_ex(W.Af, m, n, nb, ib, tree, BS, precision, stream, &f);
    if (cached) g_ls.f = f;
    if (rc != TQR_OK) {
        if (cached) g_ls.drop();
        else tqr_free(f);
        return rc;
    }
    auto done = [&](int code) {
        if (!cached) tqr_free(f);
        return code;
    };
    cudaMemcpyAsync(W.c, b, m * sizeof(double), cudaMemcpyDeviceToDevice, S.st);
    rc = tqr_apply_qt(f, W.c, m, 1, stream);
    if (rc == TQR_OK) rc = tqr_sync(f);
    if (rc != TQR_OK) return done(rc);
    I.factor_seconds = seconds_since(t0);
    auto t1 = std::chrono::steady_clock::now();
    S.back_substitute(W.c, x);                             // x = R^-1 c[0:n] (c[0:n] overwritten)
    const double normA = std::sqrt(S.dot(A, A, static_cast<int64_t>(mn)));
    auto backward = [&](double* rnorm) {                   // r, s = A^T r, eta
        S.resid();
        S.atr(W.r, W.s);
        const double rr = S.dot(W.r, W.r, m);
        const double ss = S.dot(W.s, W.s, n);
        *rnorm = std::sqrt(rr);
        return (rr > 0.0) ? std::sqrt(ss) / (normA * std::sqrt(rr)) : 0.0;
    };
    double rnorm = 0.0;
    double eta = backward(&rnorm);
    I.refine_iterations = 0;
    I.cgls_iterations = 0;
    if (precision != TQR_FP64) {
        double prev = eta;
        while (eta > tol && I.refine_iterations < maxit) {
            S.rsolve(W.s, W.u, 1);                         // u = R^-T s
            S.rsolve(W.u, W.d, 0);                         // d = R^-1 u
            axpy_kernel<<<S.nblk(n), kT, 0, S.st>>>(1.0, W.d, x, n);
            ++I.refine_iterations;
            eta = backward(&rnorm);
            if (eta > 0.5 * prev) break;                   // not contracting: hand over to CGLS
            prev = eta;
        }
        if (eta > tol && I.refine_iterations < maxit) {
            // CGLS on the correction problem min ||r - (A R^-1) z||, x += R^-1 z.
            // c (Q^T b) is no longer needed: it becomes the zero vector so
            // that resid(t, c) = -A t.
            cudaMemsetAsync(W.c, 0, m * sizeof(double), S.st);
            S.rsolve(W.s, W.u, 1);                         // u = R^-T A^T r
            cudaMemcpyAsync(W.pv, W.u, n * sizeof(double), cudaMemcpyDeviceToDevice, S.st);
            double gamma = S.dot(W.u, W.u, n);
            while (eta > tol && I.refine_iterations + I.cgls_iterations < maxit && gamma > 0.0) {
                S.rsolve(W.pv, W.t, 0);                    // t = R^-1 p
                resid_kernel<<<S.grid_rows(), kT, 0, S.st>>>(A, m, m, n, W.t, W.c, W.q);  // q = -A t
                const double qq = S.dot(W.q, W.q, m);
                if (qq <= 0.0) break;
                const double alpha = gamma / qq;
                axpy_kernel<<<S.nblk(n), kT, 0, S.st>>>(alpha, W.t, x, n);      // x += alpha t
                ++I.cgls_iterations;
                if (I.cgls_iterations % 4 == 0) {
                    eta = backward(&rnorm);                 // true FP64 residual replaces r
                } else {
                    axpy_kernel<<<S.nblk(m), kT, 0, S.st>>>(alpha, W.q, W.r, m);  // r -= alpha A t
                    S.atr(W.r, W.s);
                    const double rr = S.dot(W.r, W.r, m), ss = S.dot(W.s, W.s, n);
                    rnorm = std::sqrt(rr);
                    eta = rr > 0.0 ? std::sqrt(ss) / (normA * std::sqrt(rr)) : 0.0;
                }
                S.rsolve(W.s, W.u, 1);                     // u = R^-T A^T r
                const double gnew = S.dot(W.u, W.u, n);
                xpby_kernel<<<S.nblk(n), kT, 0, S.st>>>(W.u, gnew / gamma, W.pv, n);
                gamma = gnew;
            }
            eta = backward(&rnorm);
        }
    }
    cudaError_t e = cudaStreamSynchronize(S.st);
    I.solve_seconds = seconds_since(t1);
    I.backward_error = eta;
    I.residual_norm = rnorm;
    I.converged = ((precision == TQR_FP64 && tol == 0.0) || eta <= tol) ? 1 : 0;
    I.status = tqr_sync(f);
    if (e != cudaSuccess) return done(TQR_ERR_CUDA);
    return done(I.status);
}
