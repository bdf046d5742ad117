// Host side of libtqr's executor: layout choice, launch of the persistent
// executor (its instantiations live in exec_inst.cu), the initialization
// kernel of the dependency counters and the on-demand T-factor kernel.
#include "executor.cuh"

namespace tqr {

namespace {

// Dependency counters from the in-degrees; the initially ready tasks into
// the two queues (ready[0, nready_hi) into the high-priority queue
// queue[0, n_hi), the rest into queue[n_hi, ntasks)); every other slot -1.
__global__ void init_kernel(int32_t* deps, const int32_t* indeg, int32_t* queue, const int32_t* ready,
                            int nready, int nready_hi, int n_hi, int ntasks, uint32_t* ctr, int32_t* status,
                            int reset) {
    const int stride = gridDim.x * blockDim.x;
    const int nready_lo = nready - nready_hi;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntasks; t += stride) {
        deps[t] = indeg[t];
        int v = -1;
        if (t < n_hi) {
            if (t < nready_hi) v = ready[t];
        } else if (t - n_hi < nready_lo) {
            v = ready[nready_hi + (t - n_hi)];
        }
        queue[t] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr[0] = 0;
        ctr[1] = static_cast<uint32_t>(nready_hi);
        ctr[2] = 0;
        ctr[3] = static_cast<uint32_t>(nready_lo);
        if (reset) *status = 0;
    }
}

// ----------------------------------------------------------------------------
// T factors from stored reflectors (Schreiber-Van Loan forward accumulation):
// for each block of ib reflectors, T[:c, c] = -tau_c T[:c, :c] (V^T v_c),
// T[c, c] = tau_c, with v the full reflector vectors of the kernel.
// One CTA per panel task; panels[3*t] = kind, [3*t+1] = i, [3*t+2] = k.
// ----------------------------------------------------------------------------
__global__ void form_t_kernel(ExecParams P, const int32_t* panels, double* T_ge, double* T_el) {
    extern __shared__ __align__(16) double sm[];
    const int kind = panels[3 * blockIdx.x];
    const int i = panels[3 * blockIdx.x + 1];
    const int k = panels[3 * blockIdx.x + 2];
    const int nb = P.nb, ib = P.ib;
    double* Tout = (kind == GEQRT) ? T_ge : T_el;
    if (!Tout) return;
    Tout += (static_cast<int64_t>(k) * P.p + i) * ib * nb;
    const double* tau = ((kind == GEQRT) ? P.tau_ge : P.tau_el) + (static_cast<int64_t>(k) * P.p + i) * nb;
    const View v = tile_view(P, i, k);
    double* Vb = sm;                 // nb x ib
    double* Tb = sm + nb * ib;       // ib x ib
    double* gv = Tb + ib * ib;       // ib
    for (int j0 = 0; j0 < nb; j0 += ib) {
        __syncthreads();
        load_rect(Vb, nb, 0, v, 0, nb, j0, ib);
        for (int t = threadIdx.x; t < ib * ib; t += blockDim.x) Tb[t] = 0.0;
        __syncthreads();
        for (int c = 0; c < ib; ++c) {
            const int jc = j0 + c;
            // g[r] = v_r^T v_c for r < c (full vectors: unit entry + tail).
            for (int r = threadIdx.x; r < c; r += blockDim.x) {
                const int jr = j0 + r;
                double s = 0.0;
                if (kind == GEQRT) {
                    s = Vb[jc + r * nb];                            // tail_r . e_c
                    for (int x = jc + 1; x < nb; ++x) s = fma(Vb[x + r * nb], Vb[x + c * nb], s);
                } else {
                    const int hi = (kind == TTQRT) ? jr + 1 : nb;   // tail_r support
                    for (int x = 0; x < hi; ++x) s = fma(Vb[x + r * nb], Vb[x + c * nb], s);
                }
                gv[r] = s;
            }
            __syncthreads();
            const double tc = tau[jc];
            for (int r = threadIdx.x; r < c; r += blockDim.x) {
                double s = 0.0;
                for (int x = r; x < c; ++x) s = fma(Tb[r + x * ib], gv[x], s);
                Tb[r + c * ib] = -tc * s;
            }
            if (threadIdx.x == 0) Tb[c + c * ib] = tc;
            __syncthreads();
        }
        for (int t = threadIdx.x; t < ib * ib; t += blockDim.x) {
            const int r = t % ib, c = t / ib;
            Tout[r + static_cast<int64_t>(j0 + c) * ib] = Tb[t];
        }
    }
}

}  // namespace

// ----------------------------------------------------------------------------
// Host-side launch helpers.
// ----------------------------------------------------------------------------
int strip_width(int G) { return kThreads / G; }

int fp64_smem_bytes(int nb, int ib, int G) { return smem_doubles(nb, ib, G) * static_cast<int>(sizeof(double)); }

int lp_smem_bytes(int nb, int ib, int G) {
    const int panel = smem_doubles(nb, ib, G) * 8;
    const int upd = lp2_bytes(nb, ib, G);
    return panel > upd ? panel : upd;
}

// Low-precision updates run in the 4-row-group layout (64-column strips, nb >= 64) with
// ib 16 or 32: the configurations whose results the parity tests have checked on the
// GPU.  Other layouts compile but are refused rather than run unchecked.
bool lp_supported(int nb, int ib, int G) {
    const int W = kThreads / G;
    return G == 4 && nb % 16 == 0 && (ib == 16 || ib == 32) && W % 8 == 0 && W / 8 <= 8;
}

bool choose_layout(int nb, int ib, int* G, int* smem_bytes) {
    int dev = 0, maxsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        maxsm = 232448;
    const int budget = maxsm - 1024;   // static shared memory of the kernel
    const int cands[3] = {4, 8, 16};
    for (int g : cands) {
        const int W = kThreads / g;
        if (W > nb && g != 16) continue;
        const int bytes = smem_doubles(nb, ib, g) * static_cast<int>(sizeof(double));
        if (bytes <= budget) {
            *G = g;
            *smem_bytes = bytes;
            return true;
        }
    }
    return false;
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

template <int G>
static cudaError_t launch_g(const ExecParams& P, int smem, int grid, cudaStream_t s) {
    switch (P.B ? 0 : P.prec) {      // apply graphs always run the FP64 kernels
        case 0: return launch_exec<G, 0>(P, smem, grid, s);
        case 1: return launch_exec<G, 1>(P, smem, grid, s);
        case 2: return launch_exec<G, 2>(P, smem, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_factor_exec(ExecParams P, const DevGraph& g, const ExecState& st, int G, int smem,
                               bool reset_status, cudaStream_t s) {
    if (g.ntasks > st.capacity) return cudaErrorInvalidValue;
    P.tasks = g.tasks;
    P.succ_ptr = g.succ_ptr;
    P.succ = g.succ;
    P.deps = st.deps;
    P.queue = st.queue;
    P.ctr = st.ctr;
    P.status = st.status;
    P.ntasks = g.ntasks;
    P.n_hi = g.n_hi;
    const int nsm = device_sm_count();
    int ib = (g.ntasks + 255) / 256;
    if (ib > 4 * nsm) ib = 4 * nsm;
    if (ib < 1) ib = 1;
    init_kernel<<<ib, 256, 0, s>>>(st.deps, g.indeg, st.queue, g.ready, g.nready, g.nready_hi, g.n_hi, g.ntasks,
                                  st.ctr, st.status, reset_status ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (g.ntasks == 0) return cudaSuccess;
    int grid = nsm > 0 ? nsm : 1;                 // one 256-thread CTA per SM
    if (grid > g.ntasks) grid = g.ntasks;
    switch (G) {
        case 4: return launch_g<4>(P, smem, grid, s);
        case 8: return launch_g<8>(P, smem, grid, s);
        case 16: return launch_g<16>(P, smem, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_form_t(const ExecParams& P, const int32_t* panels, int npanels, double* T_ge,
                          double* T_el, cudaStream_t s) {
    if (npanels == 0) return cudaSuccess;
    const int smem = (P.nb * P.ib + P.ib * P.ib + P.ib) * static_cast<int>(sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(form_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    form_t_kernel<<<npanels, kThreads, smem, s>>>(P, panels, T_ge, T_el);
    return cudaGetLastError();
}

}  // namespace tqr
