// Batched FlatTree with TS kernels for one tile column (q = 1, n <= nb).
//
// For a tall-skinny matrix whose n columns fit in one tile column, FlatTree-TS
// (Sameh-Kuck list with the triangle-on-top-of-square kernels, Section 2.1 and
// Proposition 2) is the chain GEQRT(1,1), TSQRT(2,1,1), ..., TSQRT(p,1,1):
// every task depends on the previous one through the triangle R of tile row 1,
// and there are no update tasks.  When thousands of such matrices are
// factored together the parallelism comes from the batch, so one CTA runs the
// whole chain of one matrix and keeps R resident in shared memory; the tiles
// below it stream through shared memory once (read, reflect, write back V).
// The results are those of tqr_factor(A, m, n, nb, ib, TQR_FLAT_TS, ...):
// R in the upper triangle of rows 0..n-1, GEQRT's V below the diagonal of tile
// row 1, TSQRT's V in the whole of every other tile row, tau per reflector in
// the handle's layout (tile i, reflector j at i*nb + j; padded columns j >= n
// get tau = 0).
//
// Reflectors are formed and applied one at a time (LAPACK dlarfg convention,
// as in the executor's panel kernels).  Within a CTA, reflector j's update of
// the A = n-j-1 trailing columns is spread over A groups of Gj lanes (Gj a
// power of two <= 32, A*Gj <= 256): a group owns one column, its lanes take
// rows g, g+Gj, ...; the dot products reduce by shuffles inside the group.
// The group that updates column j+1 also accumulates the squares of its new
// entries, forms reflector j+1 and scales its vector into the second of two
// vector buffers, so each reflector costs one block barrier.
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace tqr {

namespace {

constexpr int kTs1Threads = 256;

__device__ __forceinline__ void ts1_status(int32_t* status, int code) { atomicCAS(status, 0, code); }

template <typename Real>
__device__ __forceinline__ Real group_sum(Real x, int G, unsigned gmask) {
    for (int off = G >> 1; off > 0; off >>= 1) x += __shfl_xor_sync(gmask, x, off);
    return x;
}

// Reflector mapping (alpha, x) to (beta, 0): beta = -sign(alpha) ||(alpha, x)||
// with sign(0) = +1, tau = (beta - alpha) / beta, v = x / (alpha - beta);
// x = 0 gives tau = 0 and a zero vector.  sig = ||x||^2.  Writes beta over
// alpha and returns the scale 1 / (alpha - beta).
template <typename Real>
__device__ Real make_reflector(Real* ap, Real sig, Real* tau_out, int32_t* status) {
    const Real alpha = *ap;
    Real tau = Real(0), scale = Real(0);
    if (sig != Real(0) || !isfinite(sig)) {
        const Real nrm = sqrt(fma(alpha, alpha, sig));
        if (!isfinite(nrm)) ts1_status(status, TQR_ERR_NONFINITE);
        const Real beta = alpha >= Real(0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = Real(1) / (alpha - beta);
        *ap = beta;
    }
    *tau_out = tau;
    return scale;
}

__device__ __forceinline__ int packed(int j, int c) { return c * (c + 1) / 2 + j; }

template <typename Real, int NCOL>
__global__ void __launch_bounds__(kTs1Threads) ts1_kernel(const Ts1Desc* __restrict__ descs, Real* tau_ge,
                                                           Real* tau_el, int32_t* status) {
    extern __shared__ __align__(16) unsigned char ts1_raw[];
    constexpr int ld = NCOL + 1;
    __shared__ Real s_tau[2];
    const Ts1Desc d = descs[blockIdx.x];
    const int n = d.n, h = d.h;
    const int64_t m = d.m;
    Real* A = static_cast<Real*>(d.A);
    Real* T = reinterpret_cast<Real*>(ts1_raw);   // tile: h x ld, row-major
    Real* R = T + h * ld;                         // packed upper triangle, NCOL (NCOL+1)/2
    Real* Vb = R + NCOL * (NCOL + 1) / 2;         // two reflector vectors of h entries
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int p = static_cast<int>((m + h - 1) / h);

    for (int tile = 0; tile < p; ++tile) {
        const bool ge = tile == 0;
        const int64_t row0 = static_cast<int64_t>(tile) * h;
        const int rows = static_cast<int>(m - row0 < h ? m - row0 : h);
        Real* tau_out = (ge ? tau_ge : tau_el) + d.tau_off + static_cast<int64_t>(tile) * h;
        __syncthreads();
        for (int e = t; e < rows * n; e += kTs1Threads) {
            const int r = e % rows, c = e / rows;
            T[r * ld + c] = A[row0 + r + static_cast<int64_t>(c) * m];
        }
        for (int j = n + t; j < h; j += kTs1Threads) tau_out[j] = Real(0);   // padded columns
        __syncthreads();

        // Reflector 0 by warp 0.
        if (t < 32) {
            const int lo = ge ? 1 : 0;
            Real s = Real(0);
            for (int r = lo + lane; r < rows; r += 32) s = fma(T[r * ld], T[r * ld], s);
            s = group_sum(s, 32, 0xffffffffu);
            Real scale = Real(0);
            if (lane == 0) {
                scale = make_reflector(ge ? &T[0] : &R[0], s, &s_tau[0], status);
                tau_out[0] = s_tau[0];
            }
            scale = __shfl_sync(0xffffffffu, scale, 0);
            for (int r = lo + lane; r < rows; r += 32) {
                const Real x = T[r * ld] * scale;
                T[r * ld] = x;
                Vb[r] = x;
            }
        }
        __syncthreads();

        for (int j = 0; j < n - 1; ++j) {
            const int Acols = n - j - 1;
            int Gj = kTs1Threads / Acols;
            Gj = Gj >= 32 ? 32 : (Gj >= 16 ? 16 : (Gj >= 8 ? 8 : (Gj >= 4 ? 4 : (Gj >= 2 ? 2 : 1))));
            if (t < Acols * Gj) {
                const Real* v = Vb + (j & 1) * h;
                Real* vn = Vb + ((j + 1) & 1) * h;
                const Real tau = s_tau[j & 1];
                const int c = j + 1 + t / Gj, g = t % Gj;
                const int leader = lane & ~(Gj - 1);
                const unsigned gmask = (Gj == 32) ? 0xffffffffu : (((1u << Gj) - 1u) << leader);
                const int lo = ge ? j + 1 : 0;
                Real* rp = ge ? &T[j * ld + c] : &R[packed(j, c)];
                Real acc = Real(0);
                for (int r = lo + g; r < rows; r += Gj) acc = fma(v[r], T[r * ld + c], acc);
                if (g == 0) acc += *rp;
                acc = group_sum(acc, Gj, gmask);
                const Real wt = tau * acc;
                if (g == 0) *rp -= wt;
                const bool next = c == j + 1;
                const int nlo = ge ? j + 2 : 0;
                Real s = Real(0);
                for (int r = lo + g; r < rows; r += Gj) {
                    const Real x = fma(-v[r], wt, T[r * ld + c]);
                    T[r * ld + c] = x;
                    if (next && r >= nlo) s = fma(x, x, s);
                }
                if (next) {                 // the whole group owns column j+1
                    s = group_sum(s, Gj, gmask);
                    Real scale = Real(0);
                    if (g == 0) {
                        Real* ap = ge ? &T[(j + 1) * ld + (j + 1)] : &R[packed(j + 1, j + 1)];
                        scale = make_reflector(ap, s, &s_tau[(j + 1) & 1], status);
                        tau_out[j + 1] = s_tau[(j + 1) & 1];
                    }
                    scale = __shfl_sync(gmask, scale, leader);
                    for (int r = lo + g; r < rows; r += Gj) {
                        if (r < nlo) continue;
                        const Real x = T[r * ld + c] * scale;
                        T[r * ld + c] = x;
                        vn[r] = x;
                    }
                }
            }
            __syncthreads();
        }

        if (ge) {                                  // R = upper triangle of the factored first tile
            for (int e = t; e < n * (n + 1) / 2; e += kTs1Threads) {
                int c = 0;
                while ((c + 1) * (c + 2) / 2 <= e) ++c;
                const int j = e - c * (c + 1) / 2;
                R[e] = T[j * ld + c];
            }
        }
        for (int e = t; e < rows * n; e += kTs1Threads) {
            const int r = e % rows, c = e / rows;
            A[row0 + r + static_cast<int64_t>(c) * m] = T[r * ld + c];
        }
    }
    __syncthreads();
    if (p > 1) {                                   // final R over the first tile's upper triangle
        for (int e = t; e < n * (n + 1) / 2; e += kTs1Threads) {
            int c = 0;
            while ((c + 1) * (c + 2) / 2 <= e) ++c;
            const int j = e - c * (c + 1) / 2;
            A[j + static_cast<int64_t>(c) * m] = R[e];
        }
    }
}

template <typename Real, int NCOL>
cudaError_t launch_class(const Ts1Desc* d, int count, int hmax, void* tau_ge, void* tau_el, int32_t* status,
                         cudaStream_t s) {
    const int smem = ts1_smem_bytes(NCOL, hmax, sizeof(Real));
    cudaError_t e = cudaFuncSetAttribute(ts1_kernel<Real, NCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    ts1_kernel<Real, NCOL><<<count, kTs1Threads, smem, s>>>(d, static_cast<Real*>(tau_ge),
                                                             static_cast<Real*>(tau_el), status);
    return cudaGetLastError();
}

}  // namespace

int ts1_ncol_class(int64_t n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 0)); }

int ts1_smem_bytes(int ncol_class, int hmax, int elem_size) {
    return (hmax * (ncol_class + 1) + ncol_class * (ncol_class + 1) / 2 + 2 * hmax) * elem_size;
}

bool ts1_supported(int64_t m, int64_t n, int nb, int elem_size) {
    const int cls = ts1_ncol_class(n);
    if (cls == 0 || n > nb || m < n || nb < 8 || nb > 256) return false;
    int optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    return ts1_smem_bytes(cls, nb, elem_size) <= optin;
}

cudaError_t launch_ts1(const Ts1Desc* d, int count, int ncol_class, int hmax, bool f32, void* tau_ge, void* tau_el,
                       int32_t* status, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    switch (ncol_class) {
        case 32: return f32 ? launch_class<float, 32>(d, count, hmax, tau_ge, tau_el, status, s)
                            : launch_class<double, 32>(d, count, hmax, tau_ge, tau_el, status, s);
        case 64: return f32 ? launch_class<float, 64>(d, count, hmax, tau_ge, tau_el, status, s)
                            : launch_class<double, 64>(d, count, hmax, tau_ge, tau_el, status, s);
        case 128: return f32 ? launch_class<float, 128>(d, count, hmax, tau_ge, tau_el, status, s)
                             : launch_class<double, 128>(d, count, hmax, tau_ge, tau_el, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tqr
