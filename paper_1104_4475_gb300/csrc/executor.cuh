// Device code of libtqr's persistent DAG executor and the six tile
// kernels of tiled Householder QR ("Tiled QR factorization algorithms",
// Bouwmeester, Jacquelin, Langou, Robert, 2011; kernels of Section 2.1,
// execution scheme of Section 2.3).
//
// Design (sm_103a, FP64):
//  * One persistent launch runs a whole task graph.  Each CTA pops a task id
//    from a global ready queue, runs the task with all 256 threads, then
//    decrements its successors' dependency counters and pushes the ones that
//    reach zero.  Every wait is bounded by a %globaltimer limit; on expiry the
//    CTA records TQR_ERR_TIMEOUT in the status word and returns.
//  * FP64 arithmetic runs on the DFMA pipe (sm_103 has no FP64 tensor path
//    faster than DFMA), so the kernels apply Householder reflectors one at a
//    time: no T-factor products are spent on the critical path, and every
//    flop is one the LAPACK count includes.  ib only sets how many reflectors
//    are staged in shared memory at once (and the block size of T).
//  * An update kernel works on a strip of W = 256/G columns held in shared
//    memory.  Thread (c, g) owns column c and the rows r = g (mod G) of the
//    strip, so a reflector's dot product is a G-lane shuffle reduction and no
//    thread ever reads a row another thread writes.
//
// This header holds the executor's device code; exec_inst.cu instantiates
// exec_kernel<G, PREC> (one object per pair, compiled in parallel) and
// device.cu holds the host-side helpers and the small auxiliary kernels.
#pragma once

#include "tqr_internal.h"
#include "reflector.cuh"
#include "../../include/tqr.h"

#include <cuda_runtime.h>
#include <cstdint>

namespace tqr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

enum Mode { GE = 0, TT = 1, TS = 2 };

// ------------------------------------------------------------ memory order
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acq_rel(int32_t* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_status(int32_t* status, int code) {
    atomicCAS(status, 0, code);
}

// ------------------------------------------------------------ smem layout
struct Smem {
    double* Cs;    // strip: nb x W, leading dimension ldc
    double* Vs;    // reflector block: nb x ib, leading dimension ldv
    double* Ct;    // top rows: ib x max(W, ib), leading dimension ldt
    double* taus;  // ib
    int ldc, ldt, ldv;
};

__host__ __device__ inline int round16(int x) { return (x + 15) / 16 * 16; }
__host__ __device__ inline int ldc_of(int nb, int G) { return round16(nb) + (G % 16); }
// Reflector columns 8 (mod 16) doubles apart: the two columns a half-warp of
// the 8-lane helpers reads fall on disjoint shared-memory banks.
__host__ __device__ inline int ldv_of(int nb) { return round16(nb) + 8; }

__host__ __device__ inline int smem_doubles(int nb, int ib, int G) {
    const int W = kThreads / G;
    const int wt = W > ib ? W : ib;
    return ldc_of(nb, G) * W + ldv_of(nb) * ib + (ib + 1) * wt + ib;
}

template <int G>
__device__ __forceinline__ Smem layout(const ExecParams& P, double* base) {
    constexpr int W = kThreads / G;
    Smem s;
    s.ldc = ldc_of(P.nb, G);
    s.ldt = P.ib + 1;
    s.ldv = ldv_of(P.nb);
    s.Cs = base;
    s.Vs = s.Cs + s.ldc * W;
    s.Ct = s.Vs + s.ldv * P.ib;
    const int wt = W > P.ib ? W : P.ib;
    s.taus = s.Ct + s.ldt * wt;
    return s;
}

// A view of (a window of) a column-major matrix with validity bounds: rows
// >= rv and columns >= cv do not exist (they read as zero, never written).
struct View {
    double* p;
    int64_t ld;
    int rv, cv;
};

__device__ __forceinline__ View tile_view(const ExecParams& P, int i, int k) {
    View v;
    v.p = P.A + static_cast<int64_t>(k) * P.nb * P.lda + static_cast<int64_t>(i) * P.nb;
    v.ld = P.lda;
    const int64_t rr = P.m - static_cast<int64_t>(i) * P.nb;
    const int64_t cc = P.n - static_cast<int64_t>(k) * P.nb;
    v.rv = static_cast<int>(rr < P.nb ? rr : P.nb);
    v.cv = static_cast<int>(cc < P.nb ? cc : P.nb);
    return v;
}

// Row block i of the right-hand side B, columns from c0.
__device__ __forceinline__ View rhs_view(const ExecParams& P, int i, int c0) {
    View v;
    v.p = P.B + static_cast<int64_t>(c0) * P.ldb + static_cast<int64_t>(i) * P.nb;
    v.ld = P.ldb;
    const int64_t rr = P.m - static_cast<int64_t>(i) * P.nb;
    const int64_t cc = P.nrhs - c0;
    v.rv = static_cast<int>(rr < P.nb ? rr : P.nb);
    v.cv = static_cast<int>(cc < 0x40000000 ? cc : 0x40000000);
    return v;
}

// dst[(r - rbase) + c*ldd] = src(r, c0 + c) for r in [r0, r1), c in [0, nc).
// Each thread keeps eight loads in flight before storing them.
__device__ __forceinline__ void load_rect(double* dst, int ldd, int rbase, const View& v, int r0,
                                          int r1, int c0, int nc) {
    const int nr = r1 - r0;
    if (nr <= 0) return;
    const int total = nr * nc;
    for (int base = threadIdx.x; base < total; base += 8 * kThreads) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads;
            const int r = r0 + idx % nr;
            const int c = idx / nr;
            x[u] = (idx < total && r < v.rv && c0 + c < v.cv)
                       ? __ldcg(v.p + r + static_cast<int64_t>(c0 + c) * v.ld) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads;
            if (idx < total) dst[(r0 + idx % nr - rbase) + (idx / nr) * ldd] = x[u];
        }
    }
}

// src(r, c0 + c) = dst[...] for the same rectangle; upper = only r <= c0 + c.
__device__ __forceinline__ void store_rect(const double* src, int lds, int rbase, const View& v,
                                           int r0, int r1, int c0, int nc, bool upper) {
    const int nr = r1 - r0;
    if (nr <= 0) return;
    for (int idx = threadIdx.x; idx < nr * nc; idx += kThreads) {
        const int r = r0 + idx % nr;
        const int c = idx / nr;
        if (r < v.rv && c0 + c < v.cv && (!upper || r <= c0 + c))
            v.p[r + static_cast<int64_t>(c0 + c) * v.ld] = src[(r - rbase) + c * lds];
    }
}

template <int G>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ----------------------------------------------------------------------------
// Apply reflectors j0..j0+ib-1 (staged in Vs/taus) to the strip in Cs (and
// the top rows in Ct for TT/TS), forward (Q^T) or backward (Q).
//   GE: reflector j is (1 at row j, Vs[r>j]) on the strip's own rows;
//   TT: (1 at top row j, Vs[0..j] on the bottom rows);
//   TS: (1 at top row j, Vs[0..nb-1] on the bottom rows).
// Thread (c, g) owns column c and rows r = g (mod G): no shared-memory
// hazards between threads, only the G-lane reductions.
// ----------------------------------------------------------------------------
template <int G, int MODE>
__device__ __forceinline__ void apply_block(const Smem& S, int nb, int j0, int ib, int trans, int ncols) {
    const int c = threadIdx.x / G;
    const int g = threadIdx.x % G;
    if ((threadIdx.x / 32) * (32 / G) >= ncols) return;   // this warp's columns do not exist
    double* Cc = S.Cs + c * S.ldc;
    for (int s = 0; s < ib; ++s) {
        const int jj = trans ? s : ib - 1 - s;
        const int j = j0 + jj;
        const double tau = S.taus[jj];
        const double* v = S.Vs + jj * S.ldv;
        int rlo, rhi;   // own rows r in [rlo, rhi), r = g (mod G)
        double acc;
        if (MODE == GE) {
            rlo = j + 1 + ((g - j - 1) & (G - 1));
            rhi = nb;
            acc = (g == (j & (G - 1))) ? Cc[j] : 0.0;
        } else {
            rlo = g;
            rhi = (MODE == TT) ? j + 1 : nb;
            acc = (g == 0) ? S.Ct[jj + c * S.ldt] : 0.0;
        }
        // One accumulation chain: each FP64 instruction occupies its
        // sub-partition's unit for as long as its latency, and the other warp
        // on the same unit fills the gaps, so a second chain (and the add
        // that joins the two) would only cost an instruction.
        int r = rlo;
        for (; r < rhi; r += G) acc = fma(v[r], Cc[r], acc);
        acc = group_sum<G>(acc);
        const double w = tau * acc;
        if (MODE == GE) {
            if (g == (j & (G - 1))) Cc[j] -= w;
        } else {
            if (g == 0) S.Ct[jj + c * S.ldt] -= w;
        }
        for (r = rlo; r < rhi; r += G) Cc[r] = fma(-v[r], w, Cc[r]);
    }
}

// ----------------------------------------------------------------------------
// Householder panel factorization of the ib columns staged in Vs (and Ct for
// TT/TS).  Reflector j maps (alpha, x) to (beta, 0), LAPACK convention:
// beta = -sign(alpha) ||(alpha, x)||, tau = (beta - alpha)/beta,
// v = x / (alpha - beta); x = 0 gives tau = 0.
//   GE: alpha = Vs[j, jj], x = Vs[j+1.., jj]   (GEQRT)
//   TT: alpha = Ct[jj, jj], x = Vs[0..j, jj]   (TTQRT)
//   TS: alpha = Ct[jj, jj], x = Vs[0..nb-1, jj] (TSQRT)
// Warp 0 forms reflector 0.  Then, for each reflector jj, warp 0 applies it to
// column jj+1 and at once forms reflector jj+1 from that column, while warps
// 1..7 apply reflector jj to columns jj+2.. of the block: one block barrier
// per reflector, and reflector generation overlaps the other columns' updates.
// ----------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void fb_range(int j, int nb, int* rlo, int* rhi) {
    *rlo = (MODE == GE) ? j + 1 : 0;
    *rhi = (MODE == TT) ? j + 1 : nb;
}

// Warp-level: forms reflector jj of the block from column jj of Vs (and its
// alpha), writes beta over alpha, tau into S.taus[jj], and v in place.
template <int MODE>
__device__ void fb_form(const Smem& S, int nb, int j0, int jj, int lane, int32_t* status) {
    const int j = j0 + jj;
    double* v = S.Vs + jj * S.ldv;
    int rlo, rhi;
    fb_range<MODE>(j, nb, &rlo, &rhi);
    double sig = 0.0;
    for (int r = rlo + lane; r < rhi; r += 32) sig = fma(v[r], v[r], sig);
    sig = warp_sum(sig);
    double scale = 0.0;
    if (lane == 0) {
        double* ap = (MODE == GE) ? &v[j] : &S.Ct[jj + jj * S.ldt];
        const double alpha = *ap;
        double tau = 0.0;
        if (sig != 0.0 || !isfinite(sig)) {
            double beta;
            reflector_scalars(alpha, sig, &beta, &tau, &scale);
            if (!isfinite(beta)) set_status(status, TQR_ERR_NONFINITE);
            *ap = beta;
        }                                   // else x is zero: identity reflector, zero tail
        S.taus[jj] = tau;
    }
    scale = __shfl_sync(kFull, scale, 0);
    for (int r = rlo + lane; r < rhi; r += 32) v[r] *= scale;
}

// Warp-level: applies reflector jj (v in column jj, tau) to column cc of the block.
template <int MODE>
__device__ __forceinline__ void fb_apply(const Smem& S, int nb, int j0, int jj, int cc, double tau, int lane) {
    const int j = j0 + jj;
    const double* v = S.Vs + jj * S.ldv;
    double* u = S.Vs + cc * S.ldv;
    int rlo, rhi;
    fb_range<MODE>(j, nb, &rlo, &rhi);
    double acc = 0.0;
    for (int r = rlo + lane; r < rhi; r += 32) acc = fma(v[r], u[r], acc);
    if (lane == 0) acc += (MODE == GE) ? u[j] : S.Ct[jj + cc * S.ldt];
    acc = warp_sum(acc);
    const double w = tau * acc;
    if (lane == 0) {
        if (MODE == GE) u[j] -= w;
        else S.Ct[jj + cc * S.ldt] -= w;
    }
    for (int r = rlo + lane; r < rhi; r += 32) u[r] = fma(-v[r], w, u[r]);
}

// Warp-level, 8 lanes per column (4 columns per warp): applies reflector jj
// to column cc.  Lane g of a column group handles rows r = rlo + g (mod 8).
// Lanes whose column does not exist (valid false) take part in the shuffles
// and write nothing.
template <int MODE>
__device__ __forceinline__ void fb_apply8(const Smem& S, int nb, int j0, int jj, int cc, double tau, int g,
                                          bool valid) {
    const int j = j0 + jj;
    const double* v = S.Vs + jj * S.ldv;
    const int col = valid ? cc : jj;
    double* u = S.Vs + col * S.ldv;
    int rlo, rhi;
    fb_range<MODE>(j, nb, &rlo, &rhi);
    double acc = (g == 0) ? ((MODE == GE) ? u[j] : S.Ct[jj + col * S.ldt]) : 0.0;
    for (int r = rlo + g; r < rhi; r += 8) acc = fma(v[r], u[r], acc);
    acc = group_sum<8>(acc);
    const double w = tau * acc;
    if (!valid) return;
    if (g == 0) {
        if (MODE == GE) u[j] -= w;
        else S.Ct[jj + cc * S.ldt] -= w;
    }
    for (int r = rlo + g; r < rhi; r += 8) u[r] = fma(-v[r], w, u[r]);
}

// FP64 on sm_103 runs one warp instruction per 64 cycles on each of the SM's
// four sub-partitions, and a warp sharing its sub-partition with another busy
// warp waits several times longer per dependent instruction.  So warp 0, which
// carries the chain (apply reflector jj to column jj+1, form reflector jj+1),
// has its sub-partition to itself (warp 4 idles), and the six warps on the
// other sub-partitions apply reflector jj to the block's columns jj+2.., four
// columns per warp pass, 8 lanes per column.  One block barrier per reflector.
template <int MODE>
__device__ void factor_block(const Smem& S, int nb, int j0, int ib, int32_t* status) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    static_assert(kThreads == 256, "factor_block assigns eight warps");
    if (warp == 0) fb_form<MODE>(S, nb, j0, 0, lane, status);
    __syncthreads();
    const int hw = (warp < 4) ? warp - 1 : warp - 2;    // helper index 0..5 (warps 1-3, 5-7)
    for (int jj = 0; jj < ib; ++jj) {
        const double tau = S.taus[jj];
        if (warp == 0) {
            if (jj + 1 < ib) {
                fb_apply<MODE>(S, nb, j0, jj, jj + 1, tau, lane);
                __syncwarp();
                fb_form<MODE>(S, nb, j0, jj + 1, lane, status);
            }
        } else if (warp != 4) {
            for (int c0 = jj + 2 + 4 * hw; c0 < ib; c0 += 24) {
                const int cc = c0 + (lane >> 3);
                fb_apply8<MODE>(S, nb, j0, jj, cc, tau, lane & 7, cc < ib);
            }
        }
        __syncthreads();
    }
}

template <int MODE>
__device__ void form_t_block(const Smem& S, int nb, int j0, int ib, float* Tout, double* scratch);
// In low precision, panel_factor keeps the block's FP32 reflectors (unit and
// zero entries written out, leading dimension nb + 1) in the strip buffer,
// after form_t_block's Gram and T.
__device__ __forceinline__ float* lp_block_v32(double* scratch, int ib) {
    return reinterpret_cast<float*>(scratch + 2 * ib * ib);
}
template <int G, int MODE, int PREC>
__device__ void panel_lp_trailing(const ExecParams& P, int i, int k, const View& top, const View& bot, int j0,
                                  int c_lo, int c_hi, double* smem);

// ----------------------------------------------------------------------------
// Panel kernels: GEQRT(i,k) (MODE GE), TTQRT(i,piv,k) (TT), TSQRT(i,piv,k)
// (TS).  Blocks of ib columns are factored in turn; after each block its
// reflectors are applied to the rest of the tile (pair), W columns at a time.
// The executor runs a panel either as one task (panel_task) or as separate
// tasks per block -- panel_factor(b), then panel_update(b, columns) for the
// columns right of the block -- so that other CTAs apply block b while the
// next block is factored; the arithmetic on every element is the same.
// ----------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void stage_panel_block(const Smem& S, const View& top, const View& bot, int nb, int j0,
                                                  int ib) {
    if (MODE == GE) {
        load_rect(S.Vs, S.ldv, 0, bot, j0, nb, j0, ib);
    } else {
        load_rect(S.Ct, S.ldt, j0, top, j0, j0 + ib, j0, ib);
        load_rect(S.Vs, S.ldv, 0, bot, 0, (MODE == TT) ? j0 + ib : nb, j0, ib);
    }
}

// Factor block j0 of the panel: stage it, factor it, store R, V and tau (and,
// in low precision, the block's FP32 V and T).  A block right of the tile's
// last valid column only records identity reflectors (tau = 0, T = 0).
template <int G, int MODE, int PREC>
__device__ void panel_factor(const ExecParams& P, int i, int piv, int k, int j0, double* smem) {
    const Smem S = layout<G>(P, smem);
    const int nb = P.nb, ib = P.ib;
    const View bot = tile_view(P, i, k);                    // GE: the tile itself
    const View top = (MODE == GE) ? bot : tile_view(P, piv, k);
    double* tau_out = ((MODE == GE) ? P.tau_ge : P.tau_el) + (static_cast<int64_t>(k) * P.p + i) * nb;
    const int64_t tile = static_cast<int64_t>(k) * P.p + i;
    if (j0 >= bot.cv) {
        for (int t = threadIdx.x; t < ib; t += kThreads) tau_out[j0 + t] = 0.0;
        if (PREC != 0) {
            float* Tdst = ((MODE == GE) ? P.T_ge : P.T_el) + tile * ib * nb + static_cast<int64_t>(j0) * ib;
            float* Vdst = ((MODE == GE) ? P.V_ge : P.V_el) + tile * nb * nb + static_cast<int64_t>(j0) * nb;
            for (int idx = threadIdx.x; idx < ib * ib; idx += kThreads) Tdst[idx] = 0.0f;
            for (int idx = threadIdx.x; idx < nb * ib; idx += kThreads) Vdst[idx] = 0.0f;
        }
        return;
    }
    __syncthreads();
    stage_panel_block<MODE>(S, top, bot, nb, j0, ib);
    __syncthreads();
    factor_block<MODE>(S, nb, j0, ib, P.status);
    // Write the block back: R (and V) in place, tau to the handle.
    if (MODE == GE) {
        store_rect(S.Vs, S.ldv, 0, bot, j0, nb, j0, ib, false);
    } else {
        store_rect(S.Ct, S.ldt, j0, top, j0, j0 + ib, j0, ib, true);
        store_rect(S.Vs, S.ldv, 0, bot, 0, (MODE == TT) ? j0 + ib : nb, j0, ib, MODE == TT);
    }
    for (int t = threadIdx.x; t < ib; t += kThreads) tau_out[j0 + t] = S.taus[t];
    if (PREC != 0) {
        // T_b in FP64 (Cs is free here), V_b and T_b stored as FP32.
        float* Tdst = ((MODE == GE) ? P.T_ge : P.T_el) + tile * ib * nb;
        float* Vdst = ((MODE == GE) ? P.V_ge : P.V_el) + tile * nb * nb;
        float* V32 = lp_block_v32(S.Cs, ib);                   // the same FP32 block, for T's Gram
        for (int idx = threadIdx.x; idx < nb * ib; idx += kThreads) {
            const int r = idx % nb, jj = idx / nb, j = j0 + jj;
            float v;
            if (MODE == GE) v = (r < j) ? 0.0f : (r == j ? 1.0f : static_cast<float>(S.Vs[r + jj * S.ldv]));
            else if (MODE == TT) v = (r <= j) ? static_cast<float>(S.Vs[r + jj * S.ldv]) : 0.0f;
            else v = static_cast<float>(S.Vs[r + jj * S.ldv]);
            Vdst[r + static_cast<int64_t>(j) * nb] = v;
            V32[r + jj * (nb + 1)] = v;
        }
        __syncthreads();
        form_t_block<MODE>(S, nb, j0, ib, Tdst + static_cast<int64_t>(j0) * ib, S.Cs);
    }
}

template <int G, int MODE>
__device__ void panel_update_range(const ExecParams& P, const Smem& S, const View& top, const View& bot, int i,
                                   int k, int j0, int c_lo, int c_hi, bool staged);

// Apply the reflectors of block j0 (factored and stored by panel_factor) to
// columns [c_lo, c_hi) of the tile (pair).  staged: the block's V and tau are
// still in shared memory from panel_factor in this CTA; otherwise they are
// loaded from the tile and the handle.  Only columns [c_lo, c_hi) are stored.
template <int G, int MODE, int PREC>
__device__ void panel_update(const ExecParams& P, int i, int piv, int k, int j0, int c_lo, int c_hi, bool staged,
                             double* smem) {
    const int nb = P.nb;
    const View bot = tile_view(P, i, k);
    const View top = (MODE == GE) ? bot : tile_view(P, piv, k);
    if (c_hi > bot.cv) c_hi = bot.cv;
    if (c_lo >= c_hi) return;
    if (PREC != 0) {
        panel_lp_trailing<G, MODE, PREC>(P, i, k, top, bot, j0, c_lo, c_hi, smem);
        return;
    }
    const Smem S = layout<G>(P, smem);
    if (G == 4 && c_hi - c_lo <= 32) {
        // A narrow range (the look-ahead columns): 8 row groups of 32 columns,
        // so that all 8 warps work (two per FP64 unit) rather than four.
        Smem S8 = S;
        S8.ldc = ldc_of(nb, 8);
        panel_update_range<8, MODE>(P, S8, top, bot, i, k, j0, c_lo, c_hi, staged);
        return;
    }
    panel_update_range<G, MODE>(P, S, top, bot, i, k, j0, c_lo, c_hi, staged);
}

// FP64 part of panel_update in the G-row-group layout (W = 256 / G columns
// per pass), S laid out for it.
template <int G, int MODE>
__device__ void panel_update_range(const ExecParams& P, const Smem& S, const View& top, const View& bot, int i,
                                   int k, int j0, int c_lo, int c_hi, bool staged) {
    constexpr int W = kThreads / G;
    const int nb = P.nb, ib = P.ib;
    if (!staged) {
        const double* tau_in = ((MODE == GE) ? P.tau_ge : P.tau_el) + (static_cast<int64_t>(k) * P.p + i) * nb;
        __syncthreads();
        if (MODE == GE) load_rect(S.Vs, S.ldv, 0, bot, j0, nb, j0, ib);
        else load_rect(S.Vs, S.ldv, 0, bot, 0, (MODE == TT) ? j0 + ib : nb, j0, ib);
        for (int t = threadIdx.x; t < ib; t += kThreads) S.taus[t] = __ldcg(tau_in + j0 + t);
    }
    for (int c0 = c_lo; c0 < c_hi; c0 += W) {
        const int nc = (c_hi - c0 < W) ? c_hi - c0 : W;
        __syncthreads();
        if (MODE == GE) {
            load_rect(S.Cs, S.ldc, 0, bot, j0, nb, c0, nc);
        } else {
            load_rect(S.Ct, S.ldt, j0, top, j0, j0 + ib, c0, nc);
            load_rect(S.Cs, S.ldc, 0, bot, 0, (MODE == TT) ? j0 + ib : nb, c0, nc);
        }
        __syncthreads();
        apply_block<G, MODE>(S, nb, j0, ib, 1, nc);
        __syncthreads();
        if (MODE == GE) {
            store_rect(S.Cs, S.ldc, 0, bot, j0, nb, c0, nc, false);
        } else {
            store_rect(S.Ct, S.ldt, j0, top, j0, j0 + ib, c0, nc, false);
            store_rect(S.Cs, S.ldc, 0, bot, 0, (MODE == TT) ? j0 + ib : nb, c0, nc, false);
        }
    }
}

// The whole panel as one task: every block factored, then applied to the
// columns right of it.
template <int G, int MODE, int PREC>
__device__ void panel_task(const ExecParams& P, int i, int piv, int k, double* smem) {
    const int nb = P.nb, ib = P.ib;
    const int ncol = tile_view(P, i, k).cv;                 // valid columns of the tile pair
    for (int j0 = 0; j0 < nb; j0 += ib) {
        panel_factor<G, MODE, PREC>(P, i, piv, k, j0, smem);
        if (j0 < ncol) panel_update<G, MODE, PREC>(P, i, piv, k, j0, j0 + ib, ncol, true, smem);
    }
}

// A panel task of the device graph.  T.j < 0: the whole panel; otherwise one
// block b = T.j: T.strip < 0 factors it, else T.strip = c_lo | c_hi << 16
// applies it to columns [c_lo, c_hi).
template <int G, int MODE, int PREC>
__device__ __forceinline__ void panel_any(const ExecParams& P, const DevTask& T, double* smem) {
    if (T.j < 0) {
        panel_task<G, MODE, PREC>(P, T.i, T.piv, T.k, smem);
    } else if (T.strip < 0) {
        panel_factor<G, MODE, PREC>(P, T.i, T.piv, T.k, T.j * P.ib, smem);
    } else {
        panel_update<G, MODE, PREC>(P, T.i, T.piv, T.k, T.j * P.ib, T.strip & 0xffff, T.strip >> 16, false, smem);
    }
}

// load_rect by asynchronous copies (cp.async, 8 bytes each; entries outside
// the view are zero-filled without a read); the caller commits and waits.
__device__ __forceinline__ void load_rect_async(double* dst, int ldd, int rbase, const View& v, int r0, int r1,
                                                int c0, int nc) {
    const int nr = r1 - r0;
    if (nr <= 0) return;
    for (int idx = threadIdx.x; idx < nr * nc; idx += kThreads) {
        const int r = r0 + idx % nr;
        const int c = idx / nr;
        const bool in = r < v.rv && c0 + c < v.cv;
        const double* src = in ? v.p + r + static_cast<int64_t>(c0 + c) * v.ld : v.p;
        const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst + (r - rbase) + c * ldd));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(in ? 8 : 0) : "memory");
    }
}

__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ----------------------------------------------------------------------------
// Update kernels on one strip: UNMQR (GE), TTMQR (TT), TSMQR (TS).  The
// reflectors come from tile (i,k); the strip is columns [strip*W, +W) of
// tile column j (rows i and piv), or of the right-hand side B.  Reflectors
// are staged hb at a time (hb = 16 when 16 divides ib and ib >= 32, else ib):
// with two groups in the nb x ib reflector buffer, the next group (its
// reflectors, taus and, for TT/TS, the strip's top rows) arrives by
// asynchronous copies while the current one is applied.
// ----------------------------------------------------------------------------
template <int GL, int MODE>
__device__ void update_task_g(const ExecParams& P, const DevTask& T, const Smem& S, int c0);

template <int G, int MODE>
__device__ void update_task(const ExecParams& P, const DevTask& T, double* smem) {
    const Smem S = layout<G>(P, smem);
    const int c0 = T.strip * (kThreads / G);
    if (P.B && P.nrhs - c0 <= 8) {
        // A narrow right-hand side (Q^T b for a few vectors): one warp per
        // column, 32 lanes over the rows, instead of four lanes per column.
        Smem S32 = S;
        S32.ldc = ldc_of(P.nb, 32);
        update_task_g<32, MODE>(P, T, S32, c0);
        return;
    }
    update_task_g<G, MODE>(P, T, S, c0);
}

// update_task in the layout of GL row groups (W = 256 / GL columns), S laid
// out for it, strip starting at column c0.
template <int GL, int MODE>
__device__ void update_task_g(const ExecParams& P, const DevTask& T, const Smem& S, int c0) {
    constexpr int G = GL;
    constexpr int W = kThreads / G;
    const int nb = P.nb, ib = P.ib;
    const View vt = tile_view(P, T.i, T.k);
    const double* tau_in = ((MODE == GE) ? P.tau_ge : P.tau_el) + (static_cast<int64_t>(T.k) * P.p + T.i) * nb;
    View bot, top;
    if (P.B) {
        bot = rhs_view(P, T.i, 0);
        top = (MODE == GE) ? bot : rhs_view(P, T.piv, 0);
    } else {
        bot = tile_view(P, T.i, T.j);
        top = (MODE == GE) ? bot : tile_view(P, T.piv, T.j);
    }
    const bool dbl = ib >= 32 && ib % 16 == 0;
    const int hb = dbl ? 16 : ib;                            // reflectors per staged group
    const int ng = nb / hb;
    // Group gi: reflectors j0 = gi*hb.. in buffer gi & 1 (Vs columns, taus and Ct rows shifted by hb).
    auto stage = [&](int gi) {
        const int j0 = gi * hb, buf = dbl ? (gi & 1) : 0;
        double* vs = S.Vs + buf * hb * S.ldv;
        const int lo = (MODE == GE) ? j0 : 0, hi = (MODE == TT) ? j0 + hb : nb;
        load_rect_async(vs, S.ldv, 0, vt, lo, hi, j0, hb);
        for (int t = threadIdx.x; t < hb; t += kThreads) {
            const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(S.taus + buf * hb + t));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(tau_in + j0 + t) : "memory");
        }
        if (MODE != GE) load_rect_async(S.Ct + buf * hb, S.ldt, j0, top, j0, j0 + hb, c0, W);
        async_commit();
    };
    load_rect(S.Cs, S.ldc, 0, bot, 0, nb, c0, W);
    stage(P.trans ? 0 : ng - 1);
    for (int gg = 0; gg < ng; ++gg) {
        const int gi = P.trans ? gg : ng - 1 - gg;
        const int j0 = gi * hb, buf = dbl ? (gi & 1) : 0;
        __syncthreads();                                      // the other buffer is no longer read
        if (dbl && gg + 1 < ng) {
            stage(P.trans ? gi + 1 : gi - 1);
            async_wait<1>();
        } else {
            async_wait<0>();
        }
        __syncthreads();                                      // group gi has landed for every thread
        Smem Sg = S;
        Sg.Vs = S.Vs + buf * hb * S.ldv;
        Sg.taus = S.taus + buf * hb;
        Sg.Ct = S.Ct + buf * hb;
        apply_block<G, MODE>(Sg, nb, j0, hb, P.trans, bot.cv - c0);
        if (MODE != GE) {
            __syncthreads();
            store_rect(Sg.Ct, S.ldt, j0, top, j0, j0 + hb, c0, W, false);
        }
        if (!dbl && gg + 1 < ng) {
            __syncthreads();
            stage(P.trans ? gi + 1 : gi - 1);
        }
    }
    __syncthreads();
    store_rect(S.Cs, S.ldc, 0, bot, 0, nb, c0, W, false);
}

// ----------------------------------------------------------------------------
// Mixed precision (split-TF32 or TF32 updates, FP64 panels).
//
// A panel task also forms, in FP64, the compact-WY factor T_b of each block
// of ib reflectors (Schreiber-Van Loan forward accumulation) and stores it in
// the handle's T array.  An update task then applies block b as
//     C <- C - V_b (T_b^T (V_b^T C))            (GE: UNMQR)
//     [C_top; C] <- ... with V = [I; V_b]       (TT/TS: TTMQR/TSMQR)
// with both products on the tensor cores (mma.sync m16n8k8 TF32, FP32
// accumulation).  Split-TF32 writes each operand x = hi + lo (hi = tf32(x),
// lo = tf32(x - hi)) and sums hi*hi + hi*lo + lo*hi.  C stays in FP64.
// ----------------------------------------------------------------------------
// Dot product of two FP32 columns over rows [lo, hi), exact products
// (a b = p + e by one FMA) summed with TwoSum's error terms carried along:
// the result is the exact dot product to about 2^-48 relative (absent heavy
// cancellation), from FP32 instructions only.
__device__ __forceinline__ double dot_f32_compensated(const float* a, const float* b, int lo, int hi) {
    // _rn intrinsics: no contraction into FMAs, which would break the error terms.
    float s = 0.0f, err = 0.0f;
    for (int x = lo; x < hi; ++x) {
        const float p = __fmul_rn(a[x], b[x]);
        const float pe = fmaf(a[x], b[x], -p);
        const float t = __fadd_rn(s, p);
        const float bv = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        err = __fadd_rn(err, __fadd_rn(e, pe));
        s = t;
    }
    return static_cast<double>(s) + static_cast<double>(err);
}

template <int MODE>
__device__ void form_t_block(const Smem& S, int nb, int j0, int ib, float* Tout, double* scratch) {
    double* Gm = scratch;             // ib x ib Gram of the block's full reflector vectors
    double* Tb = scratch + ib * ib;   // ib x ib T
    const float* V32 = lp_block_v32(scratch, ib);
    const int ld32 = nb + 1;
    for (int idx = threadIdx.x; idx < ib * ib; idx += kThreads) {
        Gm[idx] = 0.0;
        Tb[idx] = 0.0;
    }
    __syncthreads();
    // G[r, c] (r < c) of the FP32 vectors the updates apply, one pair per thread:
    // pair p = c (c - 1) / 2 + r.  Rows: GE from c's unit entry on, TT up to
    // r's last row, TS all.  FP32 arithmetic, compensated (the FP64 unit would
    // take one 64-cycle slot per product).
    const int npairs = ib * (ib - 1) / 2;
    for (int p = threadIdx.x; p < npairs; p += kThreads) {
        int c = static_cast<int>((1.0f + sqrtf(1.0f + 8.0f * static_cast<float>(p))) * 0.5f);
        while (c * (c - 1) / 2 > p) --c;
        while ((c + 1) * c / 2 <= p) ++c;
        const int r = p - c * (c - 1) / 2;
        const int lo = (MODE == GE) ? j0 + c : 0;
        const int hi = (MODE == TT) ? j0 + r + 1 : nb;
        Gm[r + c * ib] = dot_f32_compensated(V32 + r * ld32, V32 + c * ld32, lo, hi);
    }
    __syncthreads();
    for (int c = 0; c < ib; ++c) {
        const double tc = S.taus[c];
        for (int r = threadIdx.x; r < c; r += kThreads) {
            double s = 0.0;
            for (int x = r; x < c; ++x) s = fma(Tb[r + x * ib], Gm[x + c * ib], s);
            Tb[r + c * ib] = -tc * s;
        }
        if (threadIdx.x == 0) Tb[c + c * ib] = tc;
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < ib * ib; idx += kThreads) Tout[idx] = static_cast<float>(Tb[idx]);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D += A * B with A = ahi + alo, B = bhi + blo (PREC 1: three products; 2: one).
template <int PREC>
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ahi)[4], const uint32_t (&alo)[4],
                                     uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    if (PREC == 1) {
        mma_tf32(d, alo, bh0, bh1);
        mma_tf32(d, ahi, bl0, bl1);
    }
    mma_tf32(d, ahi, bh0, bh1);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// TF32 split by truncation on the integer pipe: hi keeps the top 19 bits of x,
// lo the top 19 bits of x - hi (exact in FP32).  PREC 2: hi only.
template <int PREC>
__device__ __forceinline__ void split_t(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = (PREC == 1) ? (__float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u) : 0u;
}

// Layout of an update task in low precision: the strip of C and the strip of
// the top tile (TT/TS) in FP32, two buffers of the FP32 reflector block and of
// its T, and W / T^T W.
struct Lp2 {
    float* Cf;
    float* Ctf;
    float* Vb[2];
    float* Tb[2];
    float* Wm;
    float* W2;
    int ldc, ldv, ldw;
};

__host__ __device__ inline int lp2_ldc(int nb) { return (nb + 31) / 32 * 32 + 4; }
__host__ __device__ inline int lp2_ldv(int nb) { return (nb + 15) / 16 * 16 + 4; }
__host__ __device__ inline int lp2_bytes(int nb, int ib, int G) {
    const int W = kThreads / G;
    return 4 * (2 * lp2_ldc(nb) * W + 2 * lp2_ldv(nb) * ib + 2 * ib * ib + 2 * ib * (W + 8));
}

template <int G>
__device__ __forceinline__ Lp2 lp2_layout(int nb, int ib, double* base) {
    constexpr int W = kThreads / G;
    Lp2 L;
    L.ldc = lp2_ldc(nb);
    L.ldv = lp2_ldv(nb);
    L.ldw = W + 8;
    float* f = reinterpret_cast<float*>(base);
    L.Cf = f;
    L.Ctf = L.Cf + L.ldc * W;
    L.Vb[0] = L.Ctf + L.ldc * W;
    L.Vb[1] = L.Vb[0] + L.ldv * ib;
    L.Tb[0] = L.Vb[1] + L.ldv * ib;
    L.Tb[1] = L.Tb[0] + ib * ib;
    L.Wm = L.Tb[1] + ib * ib;
    L.W2 = L.Wm + ib * L.ldw;
    return L;
}

// Rows [r0, r1) of a strip of a column-major FP64 view <-> FP32 shared memory.
__device__ __forceinline__ void strip_to_f32(float* dst, int ldd, const View& v, int r0, int r1, int c0, int W) {
    for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
        const bool rok = r < v.rv;
#pragma unroll 8
        for (int c = 0; c < W; ++c) {
            double x = 0.0;
            if (rok && c0 + c < v.cv) x = __ldcg(v.p + r + static_cast<int64_t>(c0 + c) * v.ld);
            dst[r + c * ldd] = static_cast<float>(x);
        }
    }
}
__device__ __forceinline__ void strip_from_f32(const float* src, int lds, const View& v, int r0, int r1, int c0,
                                               int W) {
    for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
        if (r >= v.rv) continue;
#pragma unroll 8
        for (int c = 0; c < W; ++c)
            if (c0 + c < v.cv) v.p[r + static_cast<int64_t>(c0 + c) * v.ld] = static_cast<double>(src[r + c * lds]);
    }
}

// One block of ib reflectors (FP32 V_b in Vb, T_b in Tb) applied to the FP32
// strip L.Cf (rows [rlo, rhi)) and, for TT/TS, to rows j0.. of L.Ctf:
//   W = V_b^T C (+ C_top rows),  W2 = T_b^T W,  C_top rows -= W2,  C -= V_b W2.
// Both products run on the tensor cores (m16n8k8 TF32, FP32 accumulation).
template <int G, int MODE, int PREC>
__device__ void lp2_block(const Lp2& L, const float* Vb, const float* Tb, int ib, int j0, int rlo, int rhi) {
    constexpr int W = kThreads / G;
    constexpr int NNT = W / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int nmt1 = ib / 16;
        // W = V_b^T C: warp w owns m-tile w % nmt1 and n-tiles (w / nmt1) + (8 / nmt1) t
        // (at most two in the layouts the low-precision path runs: 64-column strips, ib 16
        // or 32).  Even and odd k-steps go to separate accumulators, summed at the end:
        // twice the independent MMA chains.
        {
            const int m0 = (warp % nmt1) * 16;
            constexpr int kMaxAcc = 2;
            float acc[kMaxAcc][4], acc2[kMaxAcc][4];
            const int nstep = 8 / nmt1;
#pragma unroll
            for (int a = 0; a < kMaxAcc; ++a) {
                acc[a][0] = acc[a][1] = acc[a][2] = acc[a][3] = 0.0f;
                acc2[a][0] = acc2[a][1] = acc2[a][2] = acc2[a][3] = 0.0f;
            }
            for (int k0 = rlo; k0 < rhi; k0 += 8) {
                const bool odd = ((k0 - rlo) >> 3) & 1;
                uint32_t ahi[4], alo[4];
                split_t<PREC>(Vb[(k0 + tig) + (m0 + gid) * L.ldv], ahi[0], alo[0]);
                split_t<PREC>(Vb[(k0 + tig) + (m0 + gid + 8) * L.ldv], ahi[1], alo[1]);
                split_t<PREC>(Vb[(k0 + tig + 4) + (m0 + gid) * L.ldv], ahi[2], alo[2]);
                split_t<PREC>(Vb[(k0 + tig + 4) + (m0 + gid + 8) * L.ldv], ahi[3], alo[3]);
#pragma unroll
                for (int a = 0; a < kMaxAcc; ++a) {
                    const int nt = warp / nmt1 + a * nstep;
                    if (a * nstep < NNT && nt < NNT) {
                        const int n0 = nt * 8;
                        uint32_t bh0, bl0, bh1, bl1;
                        split_t<PREC>(L.Cf[(k0 + tig) + (n0 + gid) * L.ldc], bh0, bl0);
                        split_t<PREC>(L.Cf[(k0 + tig + 4) + (n0 + gid) * L.ldc], bh1, bl1);
                        if (odd) mma3<PREC>(acc2[a], ahi, alo, bh0, bh1, bl0, bl1);
                        else mma3<PREC>(acc[a], ahi, alo, bh0, bh1, bl0, bl1);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < kMaxAcc; ++a) {
                const int nt = warp / nmt1 + a * nstep;
                if (a * nstep < NNT && nt < NNT) {
                    const int n0 = nt * 8;
                    L.Wm[(m0 + gid) * L.ldw + n0 + 2 * tig] = acc[a][0] + acc2[a][0];
                    L.Wm[(m0 + gid) * L.ldw + n0 + 2 * tig + 1] = acc[a][1] + acc2[a][1];
                    L.Wm[(m0 + gid + 8) * L.ldw + n0 + 2 * tig] = acc[a][2] + acc2[a][2];
                    L.Wm[(m0 + gid + 8) * L.ldw + n0 + 2 * tig + 1] = acc[a][3] + acc2[a][3];
                }
            }
        }
        __syncthreads();
        // W2 = T^T (W + C_top rows)
        for (int idx = threadIdx.x; idx < ib * W; idx += kThreads) {
            const int a = idx / W, n = idx % W;
            float sum = 0.0f;
            for (int x = 0; x <= a; ++x) {
                float w = L.Wm[x * L.ldw + n];
                if (MODE != GE) w += L.Ctf[(j0 + x) + n * L.ldc];
                sum = fmaf(Tb[x + a * ib], w, sum);
            }
            L.W2[a * L.ldw + n] = sum;
        }
        __syncthreads();
        if (MODE != GE)
            for (int idx = threadIdx.x; idx < ib * W; idx += kThreads) {
                const int a = idx / W, n = idx % W;
                L.Ctf[(j0 + a) + n * L.ldc] -= L.W2[a * L.ldw + n];
            }
        // C[rlo:rhi, :] -= V_b W2: warp w owns m-tiles w, w+8, ...; four n-tiles at a
        // time share each split A fragment and give four independent MMA chains.
        constexpr int kNT = 4;
        for (int mt = (rlo / 16) + warp; mt < rhi / 16; mt += 8) {
            const int r0 = mt * 16;
            for (int nt0 = 0; nt0 < NNT; nt0 += kNT) {
                float acc[kNT][4];
#pragma unroll
                for (int q = 0; q < kNT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0f;
                for (int k0 = 0; k0 < ib; k0 += 8) {
                    uint32_t ahi[4], alo[4];
                    split_t<PREC>(Vb[(r0 + gid) + (k0 + tig) * L.ldv], ahi[0], alo[0]);
                    split_t<PREC>(Vb[(r0 + gid + 8) + (k0 + tig) * L.ldv], ahi[1], alo[1]);
                    split_t<PREC>(Vb[(r0 + gid) + (k0 + tig + 4) * L.ldv], ahi[2], alo[2]);
                    split_t<PREC>(Vb[(r0 + gid + 8) + (k0 + tig + 4) * L.ldv], ahi[3], alo[3]);
#pragma unroll
                    for (int q = 0; q < kNT; ++q) {
                        if (nt0 + q < NNT) {
                            const int n0 = (nt0 + q) * 8;
                            uint32_t bh0, bl0, bh1, bl1;
                            split_t<PREC>(L.W2[(k0 + tig) * L.ldw + n0 + gid], bh0, bl0);
                            split_t<PREC>(L.W2[(k0 + tig + 4) * L.ldw + n0 + gid], bh1, bl1);
                            mma3<PREC>(acc[q], ahi, alo, bh0, bh1, bl0, bl1);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kNT; ++q) {
                    if (nt0 + q < NNT) {
                        const int n0 = (nt0 + q) * 8;
                        L.Cf[(r0 + gid) + (n0 + 2 * tig) * L.ldc] -= acc[q][0];
                        L.Cf[(r0 + gid) + (n0 + 2 * tig + 1) * L.ldc] -= acc[q][1];
                        L.Cf[(r0 + gid + 8) + (n0 + 2 * tig) * L.ldc] -= acc[q][2];
                        L.Cf[(r0 + gid + 8) + (n0 + 2 * tig + 1) * L.ldc] -= acc[q][3];
                    }
                }
            }
        }
}

// Update task in low precision: C (and C_top) converted to FP32 once, every
// block of ib reflectors applied with two tensor-core products,
//   W = V_b^T C (+ C_top rows),  W2 = T_b^T W,  C_top rows -= W2,  C -= V_b W2,
// then converted back.  Reflector blocks and T arrive in FP32 from the panel
// task (unit/zero structure written out) by double-buffered cp.async.
template <int G, int MODE, int PREC>
__device__ void update_task_lp(const ExecParams& P, const DevTask& T, double* smem) {
    constexpr int W = kThreads / G;
    const int nb = P.nb, ib = P.ib;
    const Lp2 L = lp2_layout<G>(nb, ib, smem);
    const int64_t tile = static_cast<int64_t>(T.k) * P.p + T.i;
    const float* Vt = ((MODE == GE) ? P.V_ge : P.V_el) + tile * nb * nb;
    const float* Tt = ((MODE == GE) ? P.T_ge : P.T_el) + tile * ib * nb;
    const int c0 = T.strip * W;
    const View bot = tile_view(P, T.i, T.j);
    const View top = (MODE == GE) ? bot : tile_view(P, T.piv, T.j);
    const int nblk = nb / ib;

    auto stage = [&](int b, int buf) {
        const int j0 = b * ib;
        const int rlo = (MODE == GE) ? j0 : 0;
        const int rhi = (MODE == TT) ? j0 + ib : nb;
        const int chunks = (rhi - rlo) / 4;
        for (int idx = threadIdx.x; idx < chunks * ib; idx += kThreads) {
            const int jj = idx / chunks, c = idx % chunks;
            cp_async16(L.Vb[buf] + rlo + 4 * c + jj * L.ldv, Vt + rlo + 4 * c + static_cast<int64_t>(j0 + jj) * nb);
        }
        for (int idx = threadIdx.x; idx < ib * ib / 4; idx += kThreads)
            cp_async16(L.Tb[buf] + 4 * idx, Tt + static_cast<int64_t>(j0) * ib + 4 * idx);
        cp_commit();
    };

    stage(0, 0);
    strip_to_f32(L.Cf, L.ldc, bot, 0, nb, c0, W);
    if (MODE != GE) strip_to_f32(L.Ctf, L.ldc, top, 0, nb, c0, W);
    for (int b = 0; b < nblk; ++b) {
        const int buf = b & 1;
        const int j0 = b * ib;
        const int rlo = (MODE == GE) ? j0 : 0;
        const int rhi = (MODE == TT) ? j0 + ib : nb;
        if (b + 1 < nblk) {
            stage(b + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        lp2_block<G, MODE, PREC>(L, L.Vb[buf], L.Tb[buf], ib, j0, rlo, rhi);
        __syncthreads();
    }
    strip_from_f32(L.Cf, L.ldc, bot, 0, nb, c0, W);
    if (MODE != GE) strip_from_f32(L.Ctf, L.ldc, top, 0, nb, c0, W);
}

// Trailing update of a panel block in low precision: block j0's FP32 V and T
// (written to the handle by panel_factor) come by cp.async; the columns
// [c_lo, c_hi) of the tile pair are converted to FP32 strip by strip and
// updated on the tensor cores.  The whole shared memory is free here.
template <int G, int MODE, int PREC>
__device__ void panel_lp_trailing(const ExecParams& P, int i, int k, const View& top, const View& bot, int j0,
                                  int c_lo, int c_hi, double* smem) {
    constexpr int W = kThreads / G;
    const int nb = P.nb, ib = P.ib;
    const Lp2 L = lp2_layout<G>(nb, ib, smem);
    const int64_t tile = static_cast<int64_t>(k) * P.p + i;
    const float* Vt = ((MODE == GE) ? P.V_ge : P.V_el) + tile * nb * nb;
    const float* Tt = ((MODE == GE) ? P.T_ge : P.T_el) + tile * ib * nb;
    const int rlo = (MODE == GE) ? j0 : 0;
    const int rhi = (MODE == TT) ? j0 + ib : nb;
    __syncthreads();                       // the block's V / T writes are done
    const int chunks = (rhi - rlo) / 4;
    for (int idx = threadIdx.x; idx < chunks * ib; idx += kThreads) {
        const int jj = idx / chunks, c = idx % chunks;
        cp_async16(L.Vb[0] + rlo + 4 * c + jj * L.ldv, Vt + rlo + 4 * c + static_cast<int64_t>(j0 + jj) * nb);
    }
    for (int idx = threadIdx.x; idx < ib * ib / 4; idx += kThreads)
        cp_async16(L.Tb[0] + 4 * idx, Tt + static_cast<int64_t>(j0) * ib + 4 * idx);
    cp_commit();
    cp_wait<0>();
    for (int c0 = c_lo; c0 < c_hi; c0 += W) {
        const int nc = (c_hi - c0 < W) ? c_hi - c0 : W;
        __syncthreads();
        strip_to_f32(L.Cf, L.ldc, bot, rlo, rhi, c0, nc);
        if (MODE != GE) strip_to_f32(L.Ctf, L.ldc, top, j0, j0 + ib, c0, nc);
        __syncthreads();
        lp2_block<G, MODE, PREC>(L, L.Vb[0], L.Tb[0], ib, j0, rlo, rhi);
        __syncthreads();
        strip_from_f32(L.Cf, L.ldc, bot, rlo, rhi, c0, nc);
        if (MODE != GE) strip_from_f32(L.Ctf, L.ldc, top, j0, j0 + ib, c0, nc);
    }
}

template <int G, int MODE, int PREC>
__device__ __forceinline__ void update_any(const ExecParams& P, const DevTask& T, double* smem) {
    if (PREC != 0 && !P.B) update_task_lp<G, MODE, (PREC != 0 ? PREC : 1)>(P, T, smem);
    else update_task<G, MODE>(P, T, smem);
}

template <int G, int PREC>
__device__ void run_task(const ExecParams& P, const DevTask& T, double* smem) {
    switch (T.kind & kKindMask) {
        case GEQRT: panel_any<G, GE, PREC>(P, T, smem); break;
        case TTQRT: panel_any<G, TT, PREC>(P, T, smem); break;
        case TSQRT: panel_any<G, TS, PREC>(P, T, smem); break;
        case UNMQR: update_any<G, GE, PREC>(P, T, smem); break;
        case TTMQR: update_any<G, TT, PREC>(P, T, smem); break;
        case TSMQR: update_any<G, TS, PREC>(P, T, smem); break;
        default: set_status(P.status, TQR_ERR_INTERNAL); break;
    }
}

// Warp 0: decrement the successors of task t; push those that become ready,
// each into the queue of its priority (slots reserved by one atomic per queue
// and warp, then filled with release stores).
__device__ void release_successors(const ExecParams& P, int t) {
    const int lane = threadIdx.x & 31;
    __threadfence();                      // the CTA's writes before the counters
    const int b = P.succ_ptr[t], e = P.succ_ptr[t + 1];
    const unsigned below = (1u << lane) - 1u;
    for (int base = b; base < e; base += 32) {
        const int idx = base + lane;
        int s = -1;
        bool ready = false, hi = false;
        if (idx < e) {
            s = P.succ[idx];
            ready = atom_add_acq_rel(&P.deps[s], -1) == 1;
            if (ready) hi = (P.tasks[s].kind & kHighPriority) != 0;
        }
#pragma unroll
        for (int qi = 0; qi < 2; ++qi) {
            const bool mine = ready && (hi == (qi == 0));
            const unsigned mask = __ballot_sync(kFull, mine);
            if (!mask) continue;
            const int leader = __ffs(mask) - 1;
            unsigned pos = 0;
            if (lane == leader) pos = atomicAdd(&P.ctr[qi == 0 ? 1 : 3], static_cast<unsigned>(__popc(mask)));
            pos = __shfl_sync(kFull, pos, leader);
            if (mine) {
                const unsigned slot = pos + __popc(mask & below);
                const unsigned cap = (qi == 0) ? static_cast<unsigned>(P.n_hi)
                                               : static_cast<unsigned>(P.ntasks - P.n_hi);
                if (slot < cap) st_release(&P.queue[(qi == 0 ? 0 : P.n_hi) + slot], s);
                else set_status(P.status, TQR_ERR_INTERNAL);
            }
        }
    }
}

// Thread 0 of a CTA: the next task to run, or -1 when every task has been
// taken or the run failed.  Each queue has a head (slots taken) and a tail
// (slots reserved by pushers); a CTA takes slot `head` of the high-priority
// queue when head < tail there, else of the other queue, by CAS on the head,
// then reads the task (the pusher's store may still be in flight).  Every
// wait is bounded by the run's time limit.
__device__ int next_task(const ExecParams& P) {
    const unsigned cap[2] = {static_cast<unsigned>(P.n_hi), static_cast<unsigned>(P.ntasks - P.n_hi)};
    const int base[2] = {0, P.n_hi};
    const uint64_t t0 = globaltimer();
    unsigned it = 0;
    for (;;) {
        bool all_taken = true;
        for (int qi = 0; qi < 2; ++qi) {
            const unsigned h = static_cast<unsigned>(ld_acquire(reinterpret_cast<const int32_t*>(&P.ctr[2 * qi])));
            if (h < cap[qi]) all_taken = false;
            const unsigned tl = static_cast<unsigned>(ld_acquire(reinterpret_cast<const int32_t*>(&P.ctr[2 * qi + 1])));
            if (h < tl && h < cap[qi] && atomicCAS(&P.ctr[2 * qi], h, h + 1u) == h) {
                for (;;) {
                    const int v = ld_acquire(&P.queue[base[qi] + h]);
                    if (v >= 0) return v;
                    if (ld_relaxed(P.status) != 0) return -1;
                    if ((++it & 31u) == 0 && globaltimer() - t0 > P.timeout_ns) {
                        set_status(P.status, TQR_ERR_TIMEOUT);
                        return -1;
                    }
                }
            }
        }
        if (all_taken) return -1;
        if (ld_relaxed(P.status) != 0) return -1;
        if ((++it & 31u) == 0 && globaltimer() - t0 > P.timeout_ns) {
            set_status(P.status, TQR_ERR_TIMEOUT);
            return -1;
        }
        __nanosleep(128);
    }
}

template <int G, int PREC>
__global__ void __launch_bounds__(kThreads, 1) exec_kernel(ExecParams P) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_task;
    for (;;) {
        if (threadIdx.x == 0) {
            int t = next_task(P);
            if (t >= P.ntasks) {
                set_status(P.status, TQR_ERR_INTERNAL);
                t = -1;
            }
            if (t >= 0) __threadfence();
            s_task = t;
        }
        __syncthreads();
        const int t = s_task;
        if (t < 0) return;
        const DevTask T = P.tasks[t];
        uint64_t t_begin = 0;
        if (P.trace && threadIdx.x == 0) t_begin = globaltimer();
        if (P.mats) {
            ExecParams Q = P;
            const MatDesc d = P.mats[T.kind >> 8];
            Q.A = d.A;
            Q.lda = d.lda;
            Q.m = d.m;
            Q.n = d.n;
            Q.nb = d.nb;
            Q.ib = d.ib;
            Q.p = d.p;
            Q.q = d.q;
            Q.tau_ge = P.tau_ge + d.tau_off;
            Q.tau_el = P.tau_el + d.tau_off;
            run_task<G, PREC>(Q, T, smem);
        } else {
            run_task<G, PREC>(P, T, smem);
        }
        __syncthreads();
        if (P.trace && threadIdx.x == 0) {
            uint32_t sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            P.trace[2 * t] = t_begin;
            P.trace[2 * t + 1] = ((globaltimer() - t_begin) & 0x00ffffffffffffffull) | (static_cast<uint64_t>(sm) << 56);
        }
        if (threadIdx.x < 32) release_successors(P, t);
    }
}

}  // namespace
}  // namespace tqr
