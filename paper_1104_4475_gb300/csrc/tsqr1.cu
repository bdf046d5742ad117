// Batched FlatTree with TS kernels for one tile column (q = 1, n <= nb).
//
// For a tall-skinny matrix whose n columns fit in one tile column, FlatTree-TS
// (Sameh-Kuck list with the triangle-on-top-of-square kernels, Section 2.1 and
// Proposition 2) is the chain GEQRT(1,1), TSQRT(2,1,1), ..., TSQRT(p,1,1):
// every task depends on the previous one through the triangle R of tile row 1,
// and there are no update tasks.  When thousands of such matrices are
// factored together the parallelism comes from the batch, so one CTA runs the
// whole chain of one matrix and keeps R resident in shared memory; the tiles
// below it are read once, reflected in registers and written back as V.
// The results are those of tqr_factor(A, m, n, nb, ib, TQR_FLAT_TS, ...):
// R in the upper triangle of rows 0..n-1, GEQRT's V below the diagonal of tile
// row 1, TSQRT's V in the whole of every other tile row, tau per reflector in
// the handle's layout (tile i, reflector j at i*nb + j; padded columns j >= n
// get tau = 0).
//
// Reflectors are formed and applied one at a time (LAPACK dlarfg convention,
// as in the executor's panel kernels).  The tile lives in registers while it
// is factored: the CTA's NT threads form NCOL column groups of G = NT/NCOL
// adjacent lanes, lane g of column c holding rows g*RPT .. g*RPT+RPT-1 of
// column c (tile height nb = G*RPT; NT chosen so that RPT <= 16 in FP32 and
// <= 8 in FP64 where 1024 threads allow it).  Reflector j's vector u is published in
// shared memory; every column c > j computes its dot product with u from
// registers, reduces it across its G lanes by shuffles, and updates its
// registers.  For GEQRT u carries the implicit unit at row j and zeros above
// it, so the same code updates R's row j; for TSQRT R's row j lives in shared
// memory (packed) and lane 0 of each column adds and updates it.  The group of
// column j+1 forms reflector j+1 right after its own update and publishes u
// in the second of two buffers: one barrier per reflector.  Tiles move
// between global memory and registers through a shared staging tile
// (coalesced global loads and stores).
//
// The whole batch is one persistent launch (ts1_all_kernel): one CTA of 1024
// threads per SM, whose threads form slots of 1024, 512 or 256 threads (the
// thread count of a matrix's class).  Each slot pops matrices, largest first,
// from a queue per thread count and synchronises on a named barrier of its
// own, so a CTA runs up to four matrices at once and the SMs balance
// themselves without one launch per class.
#include "tqr_internal.h"
#include "reflector.cuh"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

namespace tqr {

namespace {

__device__ __forceinline__ void ts1_status(int32_t* status, int code) { atomicCAS(status, 0, code); }

template <typename Real>
__device__ __forceinline__ Real group_sum(Real x, int G, unsigned gmask) {
    for (int off = G >> 1; off > 0; off >>= 1) x += __shfl_xor_sync(gmask, x, off);
    return x;
}

__device__ __forceinline__ int packed(int j, int c) { return c * (c + 1) / 2 + j; }

__device__ __forceinline__ int ts1_ncol_class_dev(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : 128); }

// Shared-memory geometry of one (Real, NCOL, RPT) instantiation.
template <typename Real, int NCOL, int RPT, int NT>
struct Ts1Geom {
    static constexpr int G = NT / NCOL;                     // lanes per column
    static constexpr int H = G * RPT;                       // tile height nb
    static constexpr int VPAD = 16 / sizeof(Real);          // one 16-byte slot between lane chunks
    static constexpr int UCH = RPT + VPAD;                  // chunk stride of a published vector
    static constexpr int ULEN = G * UCH;                    // one published vector
    static constexpr int LD = NCOL + 1;                     // staging tile row stride
    static constexpr int ELEMS = 2 * ULEN + H * LD + NCOL * (NCOL + 1) / 2;
};

template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec2<double> { using T = double2; static constexpr int N = 2; };

// One accumulation chain: with 8 or more warps per sub-partition the other
// warps hide the chain's latency, and joining several chains would cost
// instructions (each FP64 instruction occupies the sub-partition's unit for
// as long as a dependent one waits).
template <typename Real, int RPT>
__device__ __forceinline__ Real dot_chunk(const Real* __restrict__ u, const Real (&x)[RPT]) {
    using V = typename Vec2<Real>::T;
    constexpr int N = Vec2<Real>::N;
    Real a = Real(0);
#pragma unroll
    for (int k = 0; k < RPT; k += N) {
        const V w = *reinterpret_cast<const V*>(u + k);
        if constexpr (N == 4) {
            a = fma(w.x, x[k], a);
            a = fma(w.y, x[k + 1], a);
            a = fma(w.z, x[k + 2], a);
            a = fma(w.w, x[k + 3], a);
        } else {
            a = fma(w.x, x[k], a);
            a = fma(w.y, x[k + 1], a);
        }
    }
    return a;
}

template <typename Real, int RPT>
__device__ __forceinline__ void axpy_chunk(const Real* __restrict__ u, Real wt, Real (&x)[RPT]) {
    using V = typename Vec2<Real>::T;
    constexpr int N = Vec2<Real>::N;
#pragma unroll
    for (int k = 0; k < RPT; k += N) {
        const V w = *reinterpret_cast<const V*>(u + k);
        if constexpr (N == 4) {
            x[k] = fma(-w.x, wt, x[k]);
            x[k + 1] = fma(-w.y, wt, x[k + 1]);
            x[k + 2] = fma(-w.z, wt, x[k + 2]);
            x[k + 3] = fma(-w.w, wt, x[k + 3]);
        } else {
            x[k] = fma(-w.x, wt, x[k]);
            x[k + 1] = fma(-w.y, wt, x[k + 1]);
        }
    }
}

// Forms reflector jn from column jn, held by the G lanes of its group (lane
// g has rows r0..r0+RPT-1 in x).  LAPACK convention: beta = -sign(alpha)
// ||(alpha, x)|| with sign(0) = +1, tau = (beta - alpha)/beta, v = x/(alpha -
// beta); x = 0 gives tau = 0 and v = 0.  GEQRT: alpha is row jn of the tile and
// x its rows below; the published u is (0 above jn, 1 at jn, v below).
// TSQRT: alpha is R(jn,jn) and x the whole tile column; u = v.
template <typename Real, int RPT>
__device__ __forceinline__ void ts1_form(bool ge, int jn, int r0, int g, int G, unsigned gmask, Real (&x)[RPT],
                                         Real* __restrict__ u, Real* R, Real* s_tau, Real* tau_out,
                                         int32_t* status) {
    Real a = ge ? Real(0) : R[packed(jn, jn)];   // TS: read before lane 0 overwrites it
    Real sig = Real(0);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int row = r0 + k;
        if (!ge || row > jn) sig = fma(x[k], x[k], sig);
        if (ge && row == jn) a = x[k];
    }
    sig = group_sum(sig, G, gmask);
    // GE: alpha (row jn) lives in lane jn / RPT of the group; one shuffle.
    if (ge) a = __shfl_sync(gmask, a, ((threadIdx.x & 31) & ~(G - 1)) + jn / RPT);
    Real tau = Real(0), scale = Real(0), beta = a;
    if (sig != Real(0) || !isfinite(sig)) reflector_scalars(a, sig, &beta, &tau, &scale);
    if (g == 0) {
        if (!isfinite(beta)) ts1_status(status, TQR_ERR_NONFINITE);
        *s_tau = tau;
        *tau_out = tau;
        if (!ge) R[packed(jn, jn)] = beta;
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int row = r0 + k;
        if (ge) {
            if (row > jn) {
                x[k] *= scale;
                u[k] = x[k];
            } else if (row == jn) {
                x[k] = beta;
                u[k] = Real(1);
            } else {
                u[k] = Real(0);
            }
        } else {
            x[k] *= scale;
            u[k] = x[k];
        }
    }
}

// Named barrier `id` (1..4) over the nt threads of one slot.
__device__ __forceinline__ void slot_sync(int id, int nt) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nt) : "memory");
}

// Factors one matrix with the NT threads t = 0..NT-1 of a slot; sm is the
// slot's shared memory (Ts1Geom::ELEMS elements), s_tau two scalars of it,
// bar its named barrier.
template <typename Real, int NCOL, int RPT, int NT>
__device__ __forceinline__ void ts1_body(const Ts1Desc& d, Real* sm, Real* s_tau, Real* tau_ge, Real* tau_el,
                                         int32_t* status, int t, int bar) {
    using Geo = Ts1Geom<Real, NCOL, RPT, NT>;
    constexpr int G = Geo::G, H = Geo::H, LD = Geo::LD, UCH = Geo::UCH, ULEN = Geo::ULEN;
    Real* Ub = sm;                                 // 2 published vectors (16-byte aligned chunks)
    Real* T = Ub + 2 * ULEN;                       // staging tile: H x LD, row-major
    Real* R = T + H * LD;                          // packed upper triangle of R
    const int n = d.n;
    const int64_t m = d.m;
    Real* A = static_cast<Real*>(d.A);
    const int c = t / G, g = t % G;
    const int lane = t & 31;
    const int leader = lane & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << leader);
    const int r0 = g * RPT;
    const int p = static_cast<int>((m + H - 1) / H);
    Real x[RPT];

    for (int tile = 0; tile < p; ++tile) {
        const bool ge = tile == 0;
        const int64_t row0 = static_cast<int64_t>(tile) * H;
        const int rows = static_cast<int>(m - row0 < H ? m - row0 : H);
        Real* tau_out = (ge ? tau_ge : tau_el) + d.tau_off + static_cast<int64_t>(tile) * H;
        slot_sync(bar, NT);
        for (int e = t; e < H * n; e += NT) {
            const int r = e % H, cc = e / H;
            T[r * LD + cc] = r < rows ? A[row0 + r + static_cast<int64_t>(cc) * m] : Real(0);
        }
        for (int j = n + t; j < H; j += NT) tau_out[j] = Real(0);   // padded columns
        slot_sync(bar, NT);
#pragma unroll
        for (int k = 0; k < RPT; ++k) x[k] = c < n ? T[(r0 + k) * LD + c] : Real(0);
        if (c == 0) ts1_form<Real, RPT>(ge, 0, r0, g, G, gmask, x, Ub + g * UCH, R, &s_tau[0], &tau_out[0], status);
        slot_sync(bar, NT);

        for (int j = 0; j < n - 1; ++j) {
            if (c > j && c < n) {
                const Real* u = Ub + (j & 1) * ULEN + g * UCH;
                const Real tau = s_tau[j & 1];
                Real acc = dot_chunk<Real, RPT>(u, x);
                if (!ge && g == 0) acc += R[packed(j, c)];
                acc = group_sum(acc, G, gmask);
                const Real wt = tau * acc;
                axpy_chunk<Real, RPT>(u, wt, x);
                if (!ge && g == 0) R[packed(j, c)] -= wt;
                if (c == j + 1)
                    ts1_form<Real, RPT>(ge, j + 1, r0, g, G, gmask, x, Ub + ((j + 1) & 1) * ULEN + g * UCH, R,
                                        &s_tau[(j + 1) & 1], &tau_out[j + 1], status);
            }
            slot_sync(bar, NT);
        }

        if (c < n) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) T[(r0 + k) * LD + c] = x[k];
        }
        slot_sync(bar, NT);
        if (ge) {                                  // R = upper triangle of the factored first tile
            for (int e = t; e < n * (n + 1) / 2; e += NT) {
                int cc = 0;
                while ((cc + 1) * (cc + 2) / 2 <= e) ++cc;
                const int j = e - cc * (cc + 1) / 2;
                R[e] = T[j * LD + cc];
            }
        }
        for (int e = t; e < rows * n; e += NT) {
            const int r = e % rows, cc = e / rows;
            A[row0 + r + static_cast<int64_t>(cc) * m] = T[r * LD + cc];
        }
    }
    slot_sync(bar, NT);
    if (p > 1) {                                   // final R over the first tile's upper triangle
        for (int e = t; e < n * (n + 1) / 2; e += NT) {
            int cc = 0;
            while ((cc + 1) * (cc + 2) / 2 <= e) ++cc;
            const int j = e - cc * (cc + 1) / 2;
            A[j + static_cast<int64_t>(cc) * m] = R[e];
        }
    }
}

// Threads per matrix: enough that a thread holds at most 16 FP32 / 8 FP64 rows
// of its column (RPT = nb * NCOL / NT), so that the reflector chain of one
// matrix has many warps to hide its latency; at least 256 (FP32) / 512 (FP64),
// at most 1024.  Always a power of two: 256, 512 or 1024.
constexpr int threads_for(int esz, int ncol, int h) {
    const int want = h * ncol / (esz == 4 ? 16 : 8);
    const int lo = esz == 4 ? 256 : 512;
    return want < lo ? lo : (want > 1024 ? 1024 : want);
}

int geom_elems(int ncol, int h, int esz) {
    const int G = threads_for(esz, ncol, h) / ncol, rpt = h / G, vpad = 16 / esz;
    return 2 * G * (rpt + vpad) + h * (ncol + 1) + ncol * (ncol + 1) / 2;
}

// Runs matrices of one class (threads_for == NT) with the slot's threads.
template <typename Real, int NCOL, int H, int NT>
__device__ __forceinline__ void ts1_class(const Ts1Desc& d, Real* sm, Real* s_tau, Real* tg, Real* te,
                                          int32_t* status, int t, int bar) {
    if constexpr (threads_for(sizeof(Real), NCOL, H) == NT && !(sizeof(Real) == 8 && NCOL == 128 && H == 256))
        ts1_body<Real, NCOL, H * NCOL / NT, NT>(d, sm, s_tau, tg, te, status, t, bar);
}

// One phase of the persistent kernel: slots of NT threads pop matrices of
// their phase (descriptors ph.begin..ph.end, largest first) until none is
// left.  Slot s covers threads [s NT, (s+1) NT) and shared-memory quarters
// [s NT/256, (s+1) NT/256): a slot of a later phase never shares memory or a
// barrier with a slot of an earlier phase that may still run.
template <typename Real, int NT>
__device__ __forceinline__ void ts1_phase(const Ts1Desc* __restrict__ descs, int begin, int end, int32_t* ctr,
                                          unsigned char* raw, int quarter_bytes, Real* tg, Real* te,
                                          int32_t* status, int* s_next, Real (*s_tau)[2]) {
    // s_next: this phase's own four words, so that a thread still reading the
    // previous phase's last (failed) pop never sees this phase's values.
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int q0 = slot * (NT / 256);              // first quarter of the slot
    const int bar = 1 + q0;
    Real* sm = reinterpret_cast<Real*>(raw + static_cast<size_t>(q0) * quarter_bytes);
    for (;;) {
        if (t == 0) s_next[q0] = begin + atomicAdd(ctr, 1);
        slot_sync(bar, NT);
        const int k = s_next[q0];
        if (k >= end) break;                       // uniform over the slot
        const Ts1Desc d = descs[k];
        switch (ts1_ncol_class_dev(d.n) * 1000 + d.h) {
            case 32064: ts1_class<Real, 32, 64, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 32128: ts1_class<Real, 32, 128, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 32256: ts1_class<Real, 32, 256, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 64064: ts1_class<Real, 64, 64, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 64128: ts1_class<Real, 64, 128, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 64256: ts1_class<Real, 64, 256, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 128128: ts1_class<Real, 128, 128, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            case 128256: ts1_class<Real, 128, 256, NT>(d, sm, s_tau[q0], tg, te, status, t, bar); break;
            default: break;                        // the host sorts only supported classes into a phase
        }
        slot_sync(bar, NT);                        // every thread has read s_next before it is rewritten
    }
}

// The whole one-tile-column batch in one persistent launch: one CTA of 1024
// threads per SM runs the 1024-thread matrices, then two slots of 512, then
// four slots of 256, each slot popping the next matrix from its phase's
// queue (atomic counter ctr[phase], zeroed before the launch).
template <typename Real>
__global__ void __launch_bounds__(1024, 1) ts1_all_kernel(const Ts1Desc* __restrict__ descs, Ts1Phases ph,
                                                           Real* tau_ge, Real* tau_el, int32_t* status,
                                                           int32_t* ctr) {
    extern __shared__ __align__(16) unsigned char ts1_raw[];
    __shared__ int s_next[3][4];
    __shared__ Real s_tau[4][2];
    if (ph.begin[0] < ph.end[0])
        ts1_phase<Real, 1024>(descs, ph.begin[0], ph.end[0], ctr + 0, ts1_raw, ph.quarter_bytes, tau_ge, tau_el,
                              status, s_next[0], s_tau);
    if (ph.begin[1] < ph.end[1])
        ts1_phase<Real, 512>(descs, ph.begin[1], ph.end[1], ctr + 1, ts1_raw, ph.quarter_bytes, tau_ge, tau_el,
                             status, s_next[1], s_tau);
    if (ph.begin[2] < ph.end[2])
        ts1_phase<Real, 256>(descs, ph.begin[2], ph.end[2], ctr + 2, ts1_raw, ph.quarter_bytes, tau_ge, tau_el,
                             status, s_next[2], s_tau);
}

}  // namespace

int ts1_ncol_class(int64_t n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 0)); }

int ts1_smem_bytes(int ncol_class, int h, int elem_size) { return geom_elems(ncol_class, h, elem_size) * elem_size; }

bool ts1_supported(int64_t m, int64_t n, int nb, int elem_size) {
    const int cls = ts1_ncol_class(n);
    if (cls == 0 || n > nb || m < n) return false;
    if (nb != 64 && nb != 128 && nb != 256) return false;
    if (nb < cls) return false;
    if (cls == 128 && nb == 256 && elem_size == 8) return false;    // would need 64 FP64 rows per thread
    int optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    return ts1_smem_bytes(cls, nb, elem_size) + 256 <= optin;   // + the kernel's static words and rounding
}

int ts1_threads(int ncol_class, int h, int elem_size) { return threads_for(elem_size, ncol_class, h); }

void plan_ts1(const std::vector<Ts1Desc>& fused, int elem_size, std::vector<Ts1Desc>* queue, Ts1Phases* ph,
              int64_t* max_cp) {
    auto phase = [elem_size](const Ts1Desc& d) {
        const int nt = ts1_threads(ts1_ncol_class(d.n), d.h, elem_size);
        return nt == 1024 ? 0 : (nt == 512 ? 1 : 2);
    };
    std::vector<Ts1Desc>& q = *queue;
    q = fused;
    std::stable_sort(q.begin(), q.end(), [&](const Ts1Desc& x, const Ts1Desc& y) {
        const int px = phase(x), py = phase(y);
        if (px != py) return px < py;
        return static_cast<double>(x.m) * x.n * x.n > static_cast<double>(y.m) * y.n * y.n;
    });
    Ts1Phases out{};
    int quarter = 16;
    for (int k = 0, at = 0; k < 3; ++k) {
        out.begin[k] = at;
        while (at < static_cast<int>(q.size()) && phase(q[at]) == k) {
            const Ts1Desc& d = q[at];
            const int per = (1024 >> k) / 256;                    // quarters of the slot
            const int need = (ts1_smem_bytes(ts1_ncol_class(d.n), d.h, elem_size) + per - 1) / per;
            quarter = std::max(quarter, (need + 15) / 16 * 16);
            *max_cp = std::max<int64_t>(*max_cp, 6 * ((d.m + d.h - 1) / d.h) - 2);   // Proposition 2, q = 1
            ++at;
        }
        out.end[k] = at;
    }
    out.quarter_bytes = quarter;
    *ph = out;
}

cudaError_t launch_ts1_all(const Ts1Desc* d, const Ts1Phases& ph, bool f32, void* tau_ge, void* tau_el,
                           int32_t* status, int32_t* ctr, cudaStream_t s) {
    const int count = ph.end[2];
    if (count == 0) return cudaSuccess;
    const int smem = 4 * ph.quarter_bytes;
    const int nsm = device_sm_count();
    if (nsm < 1) return cudaErrorInvalidDevice;
    const int grid = count < nsm ? count : nsm;
    if (f32) {
        auto* k = ts1_all_kernel<float>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, 1024, smem, s>>>(d, ph, static_cast<float*>(tau_ge), static_cast<float*>(tau_el), status, ctr);
    } else {
        auto* k = ts1_all_kernel<double>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, 1024, smem, s>>>(d, ph, static_cast<double*>(tau_ge), static_cast<double*>(tau_el), status, ctr);
    }
    return cudaGetLastError();
}

}  // namespace tqr
