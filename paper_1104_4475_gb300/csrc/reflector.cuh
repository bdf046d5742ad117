// Scalars of one Householder reflector, shared by the executor's panels and
// the one-column batched kernel.
//
// The reflector maps (alpha, x) to (beta, 0), LAPACK convention, with
// s = alpha^2 + ||x||^2:  beta = -sign(alpha) sqrt(s) (sign(0) = +1),
// tau = (beta - alpha) / beta,  scale = 1 / (alpha - beta)  (v = scale * x).
//
// On GB300 every FP64 operation shares a slow pipe with the other warps'
// updates, so the chain that forms a reflector -- on the critical path of
// every panel -- is kept short.  For FP64 it uses Newton's method:
//   r = 1 / sqrt(s): seed from the FP32 rsqrtf, then twice r <- r (3/2 - (s/2) r^2);
//   sqrt(s) = s r and 1 / beta = -sign(alpha) r, so tau = (beta - alpha) / beta
//   needs no division;
//   scale = 1 / d, d = alpha - beta: seed from the FP32 reciprocal, then twice
//   q <- q + q (1 - d q).
// Each Newton step squares the relative error (about 2^-22 for the FP32 seeds,
// 2^-44 after one step, below the FP64 rounding level after two), so the
// results are within a few ulp of the correctly rounded ones.  Where s lies
// outside the range in which the FP32 seeds are accurate the IEEE sqrt and
// divisions are used.
#pragma once

#include <cuda_runtime.h>

namespace tqr {

__device__ __forceinline__ void reflector_scalars(double alpha, double sig, double* beta, double* tau,
                                                  double* scale) {
    const double s = fma(alpha, alpha, sig);
    if (s > 1e-30 && s < 1e30) {
        const double h = 0.5 * s;
        double r = static_cast<double>(rsqrtf(static_cast<float>(s)));
        r = r * fma(-h, r * r, 1.5);
        r = r * fma(-h, r * r, 1.5);
        const double nrm = s * r;
        const double b = alpha >= 0.0 ? -nrm : nrm;
        const double rb = alpha >= 0.0 ? -r : r;               // 1 / beta
        const double d = alpha - b;                              // |d| = |alpha| + nrm > 0
        double q = static_cast<double>(__frcp_rn(static_cast<float>(d)));
        q = fma(q, fma(-d, q, 1.0), q);
        q = fma(q, fma(-d, q, 1.0), q);
        *beta = b;
        *tau = (b - alpha) * rb;
        *scale = q;
    } else {
        const double nrm = sqrt(s);
        const double b = alpha >= 0.0 ? -nrm : nrm;
        *beta = b;
        *tau = (b - alpha) / b;
        *scale = 1.0 / (alpha - b);
    }
}

// FP32: r = rsqrtf(s) (within 2 ulp) gives sqrt(s) = s r and 1/beta = -sign(alpha) r,
// and scale is the correctly rounded reciprocal; no IEEE square root or
// division sequence on the reflector's chain.  Outside (1e-30, 1e30) the IEEE
// operations are used.
__device__ __forceinline__ void reflector_scalars(float alpha, float sig, float* beta, float* tau, float* scale) {
    const float s = fmaf(alpha, alpha, sig);
    if (s > 1e-30f && s < 1e30f) {
        const float r = rsqrtf(s);
        const float nrm = s * r;
        const float b = alpha >= 0.0f ? -nrm : nrm;
        const float rb = alpha >= 0.0f ? -r : r;                  // 1 / beta
        *beta = b;
        *tau = (b - alpha) * rb;
        *scale = __frcp_rn(alpha - b);
    } else {
        const float nrm = sqrtf(s);
        const float b = alpha >= 0.0f ? -nrm : nrm;
        *beta = b;
        *tau = (b - alpha) / b;
        *scale = 1.0f / (alpha - b);
    }
}

}  // namespace tqr
