// Cost-model network: a 3-layer perceptron in -> 64 -> 64 -> 1 with ReLU,
// FP32, trained with mean-squared error and Adam.  Used to predict the
// makespan of a factorization from its shape and configuration (the paper
// has no learned component).  Parameters form one flat device array:
//   W1 (64 x d, row-major) | b1 (64) | W2 (64 x 64) | b2 (64) | W3 (64) | b3 (1).
#include "../../include/tqr.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int H = 64;
constexpr int kMaxIn = TQR_MLP_MAX_IN;

__host__ __device__ inline int pcount(int d) { return H * d + H + H * H + H + H + 1; }

// Per sample: forward pass and the backward deltas.  Writes a1, a2 (ReLU
// outputs), dz1, dz2 (loss gradient w.r.t. the pre-activations), dy and the
// sample's share of the loss; with t == nullptr only y is produced.
__global__ void mlp_samples(const float* __restrict__ theta, int d, const float* __restrict__ X, int B,
                            const float* __restrict__ t, float* __restrict__ y, float* __restrict__ a1g,
                            float* __restrict__ a2g, float* __restrict__ dz1g, float* __restrict__ dz2g,
                            float* __restrict__ dyg, float* __restrict__ lossg) {
    extern __shared__ float sp[];
    const int P = pcount(d);
    for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = theta[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float* W1 = sp;
    const float* b1 = W1 + H * d;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float b3 = W3[H];
    float x[kMaxIn];
    for (int i = 0; i < d; ++i) x[i] = X[static_cast<int64_t>(s) * d + i];
    float z1[H], z2[H];
    for (int j = 0; j < H; ++j) {
        float acc = b1[j];
        for (int i = 0; i < d; ++i) acc = fmaf(W1[j * d + i], x[i], acc);
        z1[j] = acc;
    }
    for (int j = 0; j < H; ++j) {
        float acc = b2[j];
        for (int k = 0; k < H; ++k) acc = fmaf(W2[j * H + k], fmaxf(z1[k], 0.0f), acc);
        z2[j] = acc;
    }
    float out = b3;
    for (int k = 0; k < H; ++k) out = fmaf(W3[k], fmaxf(z2[k], 0.0f), out);
    if (y) y[s] = out;
    if (!t) return;
    const float r = out - t[s];
    const float dy = 2.0f * r / static_cast<float>(B);
    dyg[s] = dy;
    lossg[s] = r * r / static_cast<float>(B);
    float dz2[H];
    for (int j = 0; j < H; ++j) {
        dz2[j] = (z2[j] > 0.0f) ? dy * W3[j] : 0.0f;
        a2g[static_cast<int64_t>(s) * H + j] = fmaxf(z2[j], 0.0f);
        dz2g[static_cast<int64_t>(s) * H + j] = dz2[j];
    }
    for (int k = 0; k < H; ++k) {
        float acc = 0.0f;
        for (int j = 0; j < H; ++j) acc = fmaf(dz2[j], W2[j * H + k], acc);
        a1g[static_cast<int64_t>(s) * H + k] = fmaxf(z1[k], 0.0f);
        dz1g[static_cast<int64_t>(s) * H + k] = (z1[k] > 0.0f) ? acc : 0.0f;
    }
}

// One thread per parameter: its gradient summed over the samples in a fixed
// order (deterministic); the last thread also sums the loss.
__global__ void mlp_param_grads(int d, const float* __restrict__ X, int B, const float* __restrict__ a1,
                                const float* __restrict__ a2, const float* __restrict__ dz1,
                                const float* __restrict__ dz2, const float* __restrict__ dy,
                                const float* __restrict__ lossv, float* __restrict__ grad, float* __restrict__ loss) {
    const int P = pcount(d);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    float acc = 0.0f;
    if (p == P) {                                 // loss
        for (int s = 0; s < B; ++s) acc += lossv[s];
        *loss = acc;
        return;
    }
    int o = p;
    if (o < H * d) {                              // W1[j, i]
        const int j = o / d, i = o % d;
        for (int s = 0; s < B; ++s) acc = fmaf(dz1[static_cast<int64_t>(s) * H + j], X[static_cast<int64_t>(s) * d + i], acc);
    } else if ((o -= H * d) < H) {                // b1[j]
        for (int s = 0; s < B; ++s) acc += dz1[static_cast<int64_t>(s) * H + o];
    } else if ((o -= H) < H * H) {                // W2[j, k]
        const int j = o / H, k = o % H;
        for (int s = 0; s < B; ++s) acc = fmaf(dz2[static_cast<int64_t>(s) * H + j], a1[static_cast<int64_t>(s) * H + k], acc);
    } else if ((o -= H * H) < H) {                // b2[j]
        for (int s = 0; s < B; ++s) acc += dz2[static_cast<int64_t>(s) * H + o];
    } else if ((o -= H) < H) {                    // W3[k]
        for (int s = 0; s < B; ++s) acc = fmaf(dy[s], a2[static_cast<int64_t>(s) * H + o], acc);
    } else {                                      // b3
        for (int s = 0; s < B; ++s) acc += dy[s];
    }
    grad[p] = acc;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

extern "C" {

int tqr_mlp_param_count(int in_dim) {
    if (in_dim < 1 || in_dim > kMaxIn) return -1;
    return pcount(in_dim);
}

int tqr_mlp_forward(const float* params, int in_dim, const float* X, int B, float* y, void* stream) {
    if (!params) return -1;
    if (in_dim < 1 || in_dim > kMaxIn) return -2;
    if (!X && B > 0) return -3;
    if (B < 0) return -4;
    if (!y && B > 0) return -5;
    if (B == 0) return TQR_OK;
    const int smem = pcount(in_dim) * static_cast<int>(sizeof(float));
    if (cudaFuncSetAttribute(mlp_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TQR_ERR_CUDA;
    mlp_samples<<<(B + 127) / 128, 128, smem, static_cast<cudaStream_t>(stream)>>>(
        params, in_dim, X, B, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

int tqr_mlp_loss_grad(const float* params, int in_dim, const float* X, const float* t, int B, float* work,
                      float* grad, float* loss, void* stream) {
    if (!params) return -1;
    if (in_dim < 1 || in_dim > kMaxIn) return -2;
    if (!X) return -3;
    if (!t) return -4;
    if (B < 1) return -5;
    if (!work) return -6;
    if (!grad) return -7;
    if (!loss) return -8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* a1 = work;
    float* a2 = a1 + static_cast<int64_t>(B) * H;
    float* dz1 = a2 + static_cast<int64_t>(B) * H;
    float* dz2 = dz1 + static_cast<int64_t>(B) * H;
    float* dy = dz2 + static_cast<int64_t>(B) * H;
    float* lv = dy + B;
    const int smem = pcount(in_dim) * static_cast<int>(sizeof(float));
    if (cudaFuncSetAttribute(mlp_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TQR_ERR_CUDA;
    mlp_samples<<<(B + 127) / 128, 128, smem, s>>>(params, in_dim, X, B, t, nullptr, a1, a2, dz1, dz2, dy, lv);
    const int P = pcount(in_dim);
    mlp_param_grads<<<(P + 1 + 255) / 256, 256, 0, s>>>(in_dim, X, B, a1, a2, dz1, dz2, dy, lv, grad, loss);
    return cudaGetLastError() == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

int tqr_mlp_adam_step(float* params, const float* grad, float* m, float* v, int count, float lr, float beta1,
                      float beta2, float eps, int step, void* stream) {
    if (!params) return -1;
    if (!grad) return -2;
    if (!m) return -3;
    if (!v) return -4;
    if (count < 1) return -5;
    if (step < 1) return -10;
    const float c1 = 1.0f - powf(beta1, static_cast<float>(step));
    const float c2 = 1.0f - powf(beta2, static_cast<float>(step));
    adam_kernel<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, count, lr,
                                                                                    beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

}  // extern "C"
