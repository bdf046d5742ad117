// tqr_factor_noalloc: the factorization for callers that cannot allocate.
//
// Some callers may not allocate memory at the moment they factor: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc is not
// allowed there), services that run under a fixed device-memory budget
// reserved at start-up, or real-time loops that forbid allocation after
// initialization.  This entry point serves them: it calls no cudaMalloc,
// cudaFree or other allocating routine, on the device or on the host.
//
// All working state of the executor -- task graph, dependency counters, ready
// queue, queue head/tail -- lives in one file-scope __device__ array of fixed
// size (kScratchBytes, 4 MiB).  Every GPU that loads the library holds that
// array until the process exits.  The host-side graph is built in fixed
// static arrays and uploaded into the scratch array (by cudaMemcpyAsync, or,
// on a stream being captured into a CUDA graph, by kernels that carry the
// words in their parameters).  Problems whose task graph does not fit are
// rejected with TQR_ERR_TOO_LARGE before anything is launched.
//
// Every call shares the one array and overwrites what the previous call left
// there (the counters and queue are re-initialized by each launch); two calls
// whose device work overlaps -- e.g. on two streams without ordering between
// them -- race on the array and give wrong results.  Host threads are
// serialized by a lock while a call builds and uploads its graph.
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace tqr {
namespace {

constexpr int kMaxTasks = TQR_NOALLOC_MAX_TASKS;
constexpr int kMaxEdges = 4 * TQR_NOALLOC_MAX_TASKS;
constexpr int kMaxTiles = TQR_NOALLOC_MAX_TILES;
constexpr int kMaxStrips = 16;          // nb / W: nb <= 256, W >= 16
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of each region inside the scratch array.
constexpr size_t kOffTasks = 0;
constexpr size_t kOffSuccPtr = kOffTasks + align256(sizeof(DevTask) * kMaxTasks);
constexpr size_t kOffSucc = kOffSuccPtr + align256(sizeof(int32_t) * (kMaxTasks + 1));
constexpr size_t kOffIndeg = kOffSucc + align256(sizeof(int32_t) * kMaxEdges);
constexpr size_t kOffReady = kOffIndeg + align256(sizeof(int32_t) * kMaxTasks);
constexpr size_t kOffDeps = kOffReady + align256(sizeof(int32_t) * kMaxTasks);
constexpr size_t kOffQueue = kOffDeps + align256(sizeof(int32_t) * kMaxTasks);
constexpr size_t kOffCtr = kOffQueue + align256(sizeof(int32_t) * kMaxTasks);
constexpr size_t kScratchBytes = kOffCtr + 256;
static_assert(kScratchBytes <= TQR_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch array.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress (setup()).
static __device__ __align__(256) unsigned char g_scratch[TQR_NOALLOC_SCRATCH_BYTES];

void* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device
std::mutex g_mu;

// Host-side graph under construction (fixed capacity, no heap).
struct HostGraph {
    int64_t pos[kMaxTiles];              // list index zeroing tile (i,k), k-major
    char tri[kMaxTiles];                 // tile already factored into a triangle
    int32_t last[kMaxTiles * kMaxStrips];
    int32_t prod[kMaxTiles * 2];         // [..*2]: GEQRT, [..*2+1]: TTQRT/TSQRT
    DevTask tasks[kMaxTasks];
    int32_t epred[kMaxEdges], esucc[kMaxEdges];
    int32_t succ_ptr[kMaxTasks + 1], succ[kMaxEdges], indeg[kMaxTasks], ready[kMaxTasks];
    int32_t fill[kMaxTasks];
    int32_t ntasks, nedges, nready;
};
HostGraph g_h;

// Device address of the scratch array for the current device; looked up
// once per device, with that device current.
int setup(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TQR_ERR_UNSUPPORTED;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TQR_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TQR_OK;
}

// Section 2.2 validity rules for a 0-based list.
int validate(int p, int q, const int32_t* list, int64_t count) {
    const int qq = std::min(p, q);
    for (int t = 0; t < p * qq; ++t) g_h.pos[t] = -1;
    for (int64_t t = 0; t < count; ++t) {
        const int i = list[3 * t], piv = list[3 * t + 1], k = list[3 * t + 2];
        if (k < 0 || k >= qq || i <= k || i >= p || piv < k || piv >= p || piv == i) return TQR_ERR_INVALID_LIST;
        int64_t& s = g_h.pos[k * p + i];
        if (s >= 0) return TQR_ERR_INVALID_LIST;
        s = t;
    }
    for (int k = 0; k < qq; ++k)
        for (int i = k + 1; i < p; ++i)
            if (g_h.pos[k * p + i] < 0) return TQR_ERR_INVALID_LIST;
    for (int64_t t = 0; t < count; ++t) {
        const int i = list[3 * t], piv = list[3 * t + 1], k = list[3 * t + 2];
        for (int kp = 0; kp < k; ++kp)
            if (g_h.pos[kp * p + i] > t || g_h.pos[kp * p + piv] > t) return TQR_ERR_INVALID_LIST;
        if (piv > k && g_h.pos[k * p + piv] < t) return TQR_ERR_INVALID_LIST;
    }
    return TQR_OK;
}

// Task graph of Algorithms 2/3 with updates split into strips of W columns;
// dependencies: producer of the applied reflectors + previous writer of each
// written (tile, strip) in list order (V read-only, no write-after-read).
class Builder {
public:
    Builder(int p, int q, int nb, int W, int last_cols, bool ts)
        : p_(p), q_(q), W_(W), ts_(ts), nb_(nb), last_cols_(last_cols), smax_((nb + W - 1) / W) {}

    int build(const int32_t* list, int64_t count) {
        g_h.ntasks = g_h.nedges = 0;
        for (int t = 0; t < p_ * q_; ++t) g_h.tri[t] = 0;
        for (int t = 0; t < p_ * q_ * smax_; ++t) g_h.last[t] = -1;
        for (int t = 0; t < p_ * q_ * 2; ++t) g_h.prod[t] = -1;
        for (int64_t e = 0; e < count; ++e) {
            const int i = list[3 * e], piv = list[3 * e + 1], k = list[3 * e + 2];
            if (ts_ && g_h.tri[k * p_ + i]) return TQR_ERR_INVALID_LIST;   // TS needs a square tile
            if (!factor(piv, k) || (!ts_ && !factor(i, k))) return TQR_ERR_TOO_LARGE;
            if (!panel(ts_ ? TSQRT : TTQRT, i, piv, k)) return TQR_ERR_TOO_LARGE;
            for (int j = k + 1; j < q_; ++j)
                if (!update(ts_ ? TSMQR : TTMQR, i, piv, k, j)) return TQR_ERR_TOO_LARGE;
        }
        for (int k = 0; k < std::min(p_, q_); ++k)
            if (!factor(k, k)) return TQR_ERR_TOO_LARGE;
        finish();
        return TQR_OK;
    }

private:
    int p_, q_, W_;
    bool ts_;
    int nb_, last_cols_, smax_;
    int32_t deps_[2 * kMaxStrips + 2];

    int nstrips(int j) const { return ((j == q_ - 1 ? last_cols_ : nb_) + W_ - 1) / W_; }
    int32_t& L(int r, int c, int s) { return g_h.last[(c * p_ + r) * smax_ + s]; }

    bool new_task(DevTask x, int nd) {
        if (g_h.ntasks >= kMaxTasks) return false;
        const int32_t t = g_h.ntasks++;
        g_h.tasks[t] = x;
        std::sort(deps_, deps_ + nd);
        for (int a = 0; a < nd; ++a) {
            if (deps_[a] < 0 || (a > 0 && deps_[a] == deps_[a - 1])) continue;
            if (g_h.nedges >= kMaxEdges) return false;
            g_h.epred[g_h.nedges] = deps_[a];
            g_h.esucc[g_h.nedges] = t;
            ++g_h.nedges;
        }
        return true;
    }

    bool factor(int x, int k) {
        char& f = g_h.tri[k * p_ + x];
        if (f) return true;
        f = 1;
        if (!panel(GEQRT, x, -1, k)) return false;
        for (int j = k + 1; j < q_; ++j)
            if (!update(UNMQR, x, -1, k, j)) return false;
        return true;
    }

    bool panel(int kind, int i, int piv, int k) {
        const int32_t t = g_h.ntasks;
        int nd = 0;
        const int rows[2] = {i, piv};
        for (int a = 0; a < (kind == GEQRT ? 1 : 2); ++a)
            for (int s = 0; s < nstrips(k); ++s) {
                deps_[nd++] = L(rows[a], k, s);
                L(rows[a], k, s) = t;
            }
        g_h.prod[(k * p_ + i) * 2 + (kind == GEQRT ? 0 : 1)] = t;
        return new_task({kind, i, piv, k, -1, 0}, nd);
    }

    bool update(int kind, int i, int piv, int k, int j) {
        const int32_t pr = g_h.prod[(k * p_ + i) * 2 + (kind == UNMQR ? 0 : 1)];
        for (int s = 0; s < nstrips(j); ++s) {
            const int32_t t = g_h.ntasks;
            int nd = 0;
            deps_[nd++] = pr;
            deps_[nd++] = L(i, j, s);
            L(i, j, s) = t;
            if (kind != UNMQR) {
                deps_[nd++] = L(piv, j, s);
                L(piv, j, s) = t;
            }
            if (!new_task({kind, i, piv, k, j, s}, nd)) return false;
        }
        return true;
    }

    void finish() {
        const int nt = g_h.ntasks;
        for (int t = 0; t <= nt; ++t) g_h.succ_ptr[t] = 0;
        for (int t = 0; t < nt; ++t) g_h.indeg[t] = 0;
        for (int e = 0; e < g_h.nedges; ++e) {
            g_h.succ_ptr[g_h.epred[e] + 1]++;
            g_h.indeg[g_h.esucc[e]]++;
        }
        for (int t = 0; t < nt; ++t) g_h.succ_ptr[t + 1] += g_h.succ_ptr[t];
        for (int t = 0; t < nt; ++t) g_h.fill[t] = g_h.succ_ptr[t];
        for (int e = 0; e < g_h.nedges; ++e) g_h.succ[g_h.fill[g_h.epred[e]]++] = g_h.esucc[e];
        g_h.nready = 0;
        for (int t = 0; t < nt; ++t)
            if (g_h.indeg[t] == 0) g_h.ready[g_h.nready++] = t;
    }
};

// Upload for a stream that is being captured into a CUDA graph.  A copy from
// pageable host memory (the static graph above) cannot be captured, so the
// words travel as kernel parameters instead: each launch carries 1000 words
// (4000 bytes, inside the 4 KiB parameter limit), and a captured launch keeps
// its parameters by value, so the graph replays this call's task graph even
// after later calls have rewritten the static arrays.
constexpr int kPutWords = 1000;
struct PutChunk {
    uint32_t w[kPutWords];
};

__global__ void put_words_kernel(uint32_t* __restrict__ dst, const PutChunk c, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = c.w[t];
}

cudaError_t put_words(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    static_assert(sizeof(DevTask) % 4 == 0, "device tasks are whole words");
    const uint32_t* w = static_cast<const uint32_t*>(src);
    uint32_t* d = static_cast<uint32_t*>(dst);
    const size_t nw = bytes / 4;
    PutChunk c;
    for (size_t off = 0; off < nw; off += kPutWords) {
        const int n = static_cast<int>(std::min<size_t>(kPutWords, nw - off));
        std::memcpy(c.w, w + off, static_cast<size_t>(n) * 4);
        put_words_kernel<<<1, 256, 0, s>>>(d + off, c, n);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace tqr

using namespace tqr;

extern "C" int tqr_factor_noalloc(double* A, int64_t m, int64_t n, int nb, int ib, const int32_t* list,
                                  int64_t count, int ts, double* tau_geqrt, double* tau_elim, int32_t* status,
                                  void* stream) {
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1 || n > m) return -3;
    if (nb < 8 || nb > 256 || nb % 4 != 0) return -4;
    if (ib < 1 || ib > 64 || nb % ib != 0) return -5;
    if (!list && count > 0) return -6;
    if (count < 0) return -7;
    if (ts != 0 && ts != 1) return -8;
    if (!tau_geqrt) return -9;
    if (!tau_elim) return -10;
    if (!status) return -11;
    const int64_t p64 = (m + nb - 1) / nb, q64 = (n + nb - 1) / nb;
    if (p64 * q64 > kMaxTiles) return TQR_ERR_TOO_LARGE;
    const int p = static_cast<int>(p64), q = static_cast<int>(q64);
    int G = 0, smem = 0;
    if (!choose_layout(nb, ib, &G, &smem)) return TQR_ERR_UNSUPPORTED;
    const int W = strip_width(G);
    if ((nb + W - 1) / W > kMaxStrips) return TQR_ERR_UNSUPPORTED;

    std::lock_guard<std::mutex> lk(g_mu);
    void* scratch = nullptr;
    int rc = setup(&scratch);
    if (rc != TQR_OK) return rc;
    rc = validate(p, q, list, count);
    if (rc != TQR_OK) return rc;
    Builder b(p, q, nb, W, static_cast<int>(n - static_cast<int64_t>(q - 1) * nb), ts != 0);
    rc = b.build(list, count);
    if (rc != TQR_OK) return rc;

    unsigned char* base = static_cast<unsigned char*>(scratch);
    DevGraph g;
    g.tasks = reinterpret_cast<DevTask*>(base + kOffTasks);
    g.succ_ptr = reinterpret_cast<int32_t*>(base + kOffSuccPtr);
    g.succ = reinterpret_cast<int32_t*>(base + kOffSucc);
    g.indeg = reinterpret_cast<int32_t*>(base + kOffIndeg);
    g.ready = reinterpret_cast<int32_t*>(base + kOffReady);
    g.ntasks = g_h.ntasks;
    g.nready = g_h.nready;
    g.nedges = g_h.nedges;
    ExecState st;
    st.deps = reinterpret_cast<int32_t*>(base + kOffDeps);
    st.queue = reinterpret_cast<int32_t*>(base + kOffQueue);
    st.ctr = reinterpret_cast<uint32_t*>(base + kOffCtr);
    st.status = status;
    st.capacity = kMaxTasks;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nt = static_cast<size_t>(g_h.ntasks);
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &capture) != cudaSuccess) return TQR_ERR_CUDA;
    if (capture == cudaStreamCaptureStatusInvalidated) return TQR_ERR_CUDA;
    const bool capturing = capture == cudaStreamCaptureStatusActive;
    auto upload = [&](void* dst, const void* src, size_t bytes) {
        return capturing ? put_words(dst, src, bytes, s) : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    if (upload(g.tasks, g_h.tasks, nt * sizeof(DevTask)) != cudaSuccess ||
        upload(g.succ_ptr, g_h.succ_ptr, (nt + 1) * sizeof(int32_t)) != cudaSuccess ||
        upload(g.succ, g_h.succ, static_cast<size_t>(g_h.nedges) * sizeof(int32_t)) != cudaSuccess ||
        upload(g.indeg, g_h.indeg, nt * sizeof(int32_t)) != cudaSuccess ||
        upload(g.ready, g_h.ready, static_cast<size_t>(g_h.nready) * sizeof(int32_t)) != cudaSuccess)
        return TQR_ERR_CUDA;

    ExecParams P{};
    P.A = A;
    P.lda = m;
    P.m = m;
    P.n = n;
    P.nb = nb;
    P.ib = ib;
    P.p = p;
    P.q = q;
    P.tau_ge = tau_geqrt;
    P.tau_el = tau_elim;
    P.trans = 1;
    P.timeout_ns = exec_timeout_ns(2.0 * static_cast<double>(n) * n * (m - n / 3.0));
    // The launch resets the counters, queue, head/tail and *status first.
    return launch_factor_exec(P, graph_for_launch(g), st, G, smem, true, s) == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

// The task graph tqr_factor_noalloc builds for this problem, built on the
// host with update strips of `strip` columns (no GPU, no allocation).
extern "C" int tqr_noalloc_graph(int64_t m, int64_t n, int nb, int ib, const int32_t* list, int64_t count, int ts,
                                 int strip, int32_t* tasks, int64_t task_cap, int64_t* ntasks, int32_t* src,
                                 int32_t* dst, int64_t edge_cap, int64_t* nedges) {
    if (m < 1) return -1;
    if (n < 1 || n > m) return -2;
    if (nb < 8 || nb > 256 || nb % 4 != 0) return -3;
    if (ib < 1 || ib > 64 || nb % ib != 0) return -4;
    if (!list && count > 0) return -5;
    if (count < 0) return -6;
    if (ts != 0 && ts != 1) return -7;
    if (strip != 16 && strip != 32 && strip != 64) return -8;
    if (!ntasks) return -11;
    if (!nedges) return -15;
    const int64_t p64 = (m + nb - 1) / nb, q64 = (n + nb - 1) / nb;
    if (p64 * q64 > kMaxTiles) return TQR_ERR_TOO_LARGE;
    if ((nb + strip - 1) / strip > kMaxStrips) return TQR_ERR_UNSUPPORTED;
    const int p = static_cast<int>(p64), q = static_cast<int>(q64);
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = validate(p, q, list, count);
    if (rc != TQR_OK) return rc;
    Builder b(p, q, nb, strip, static_cast<int>(n - static_cast<int64_t>(q - 1) * nb), ts != 0);
    rc = b.build(list, count);
    if (rc != TQR_OK) return rc;
    *ntasks = g_h.ntasks;
    *nedges = g_h.nedges;
    if (*ntasks > task_cap || *nedges > edge_cap) return TQR_ERR_CAPACITY;
    if ((!tasks && *ntasks) || ((!src || !dst) && *nedges)) return TQR_ERR_CAPACITY;
    for (int t = 0; t < g_h.ntasks; ++t) {
        const DevTask& d = g_h.tasks[t];
        int32_t* o = tasks + 6 * t;
        o[0] = d.kind & kKindMask;
        o[1] = d.i;
        o[2] = d.piv;
        o[3] = d.k;
        o[4] = d.j;
        o[5] = d.strip;
    }
    int64_t e = 0;
    for (int t = 0; t < g_h.ntasks; ++t)
        for (int32_t k = g_h.succ_ptr[t]; k < g_h.succ_ptr[t + 1]; ++k, ++e) {
            src[e] = t;
            dst[e] = g_h.succ[k];
        }
    return TQR_OK;
}
