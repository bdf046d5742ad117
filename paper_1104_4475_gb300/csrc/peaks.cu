// Peak-rate probes: the roofline denominators of the library's kernels,
// measured on the GPU that runs them.  Each probe keeps every SM's pipe of
// one kind busy with independent chains of one instruction and reports how
// many flops a launch performs; the caller times the launch.
//   TQR_PEAK_DFMA  FP64 fused multiply-add (the executor's arithmetic)
//   TQR_PEAK_DMMA  FP64 mma.sync m8n8k4 (the FP64 tensor path)
//   TQR_PEAK_FFMA  FP32 fused multiply-add (the FP32 batched kernel)
//   TQR_PEAK_TF32  TF32 mma.sync m16n8k8, FP32 accumulation (the low-precision updates)
#include "tqr_internal.h"
#include "../../include/tqr.h"

#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 256;

__global__ void dfma_probe(double* out, int64_t iters, double b, double d) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = threadIdx.x * 1e-3 + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678) out[0] = s;            // keeps the chains live; never true for these inputs
}

__global__ void ffma_probe(float* out, int64_t iters, float b, float d) {
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = threadIdx.x * 1e-3f + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678f) out[0] = s;
}

__global__ void dmma_probe(double* out, int64_t iters) {
    const int lane = threadIdx.x & 31;
    const double x = 1.0 + lane * 1e-9, y = 1.0 - lane * 1e-9;
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 0.0;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(x), "d"(y));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
    if (s == 12345.678) out[0] = s;
}

__global__ void tf32_probe(float* out, int64_t iters) {
    const int lane = threadIdx.x & 31;
    const uint32_t a = __float_as_uint(1.0f + lane * 1e-6f) & 0xffffe000u;
    const uint32_t b = __float_as_uint(1.0f - lane * 1e-6f) & 0xffffe000u;
    float d[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k][0] = d[k][1] = d[k][2] = d[k][3] = 0.0f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(d[k][0]), "+f"(d[k][1]), "+f"(d[k][2]), "+f"(d[k][3])
                : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1] + d[k][2] + d[k][3];
    if (s == 12345.678f) out[0] = s;
}

double* g_probe_sink[64] = {};                 // one word per device, for the never-taken stores

}  // namespace

extern "C" int tqr_peak_probe(int kind, int64_t iters, void* stream, double* flops) {
    if (kind < TQR_PEAK_DFMA || kind > TQR_PEAK_TF32) return -1;
    if (iters < 1) return -2;
    if (!flops) return -4;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ERR_CUDA;
    if (dev < 0 || dev >= 64) return TQR_ERR_UNSUPPORTED;
    if (!g_probe_sink[dev] && cudaMalloc(&g_probe_sink[dev], sizeof(double)) != cudaSuccess) return TQR_ERR_NOMEM;
    const int nsm = tqr::device_sm_count();
    if (nsm < 1) return TQR_ERR_CUDA;
    const int grid = 2 * nsm;                  // two CTAs of 8 warps per SM
    const double warps = static_cast<double>(grid) * (kProbeThreads / 32);
    const double it = static_cast<double>(iters);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case TQR_PEAK_DFMA:
            dfma_probe<<<grid, kProbeThreads, 0, s>>>(g_probe_sink[dev], iters, 0.9999999, 1e-9);
            *flops = 2.0 * 8 * 32 * warps * it;
            break;
        case TQR_PEAK_DMMA:
            dmma_probe<<<grid, kProbeThreads, 0, s>>>(g_probe_sink[dev], iters);
            *flops = 2.0 * 8 * 8 * 4 * 4 * warps * it;
            break;
        case TQR_PEAK_FFMA:
            ffma_probe<<<grid, kProbeThreads, 0, s>>>(reinterpret_cast<float*>(g_probe_sink[dev]), iters, 0.9999f,
                                                      1e-6f);
            *flops = 2.0 * 8 * 32 * warps * it;
            break;
        default:
            tf32_probe<<<grid, kProbeThreads, 0, s>>>(reinterpret_cast<float*>(g_probe_sink[dev]), iters);
            *flops = 2.0 * 16 * 8 * 8 * 4 * warps * it;
            break;
    }
    return cudaGetLastError() == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}
