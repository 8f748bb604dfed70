// Per-state update of App. A in the TF32 and BF16 forms: the orthogonal step
// Gamma <- R Gamma R^T, R = exp(X), X = (ds/4)[Gamma, dGamma] (Eq. ExpStep), with
// its products on the tensor cores, followed by the FP64 canonical-form
// renormalisation (Newton-Schulz polar iteration).
//
// Only small quantities pass through the low-precision products, so their
// relative rounding (2^-11 for TF32) scales the step, not the state:
//   * E = R - I by scaling and squaring in increment form: with X_s = X 2^-s,
//     E_s = X_s P_2, P_j = I + (X_s / j) P_{j+1}, P_d = I + X_s / d (Horner), and
//     each squaring E <- 2E + E E.  The recurrences run on transposes, which the
//     tensor core reads directly (a K-major operand is a row-major transpose):
//     Q_j = P_j^T = I + (1/j) Q_{j+1} X_s^T, E^T = Q_2 X_s^T, E^T <- 2 E^T + E^T E^T,
//     each product also writing its transpose.
//   * Gamma' = Gamma + F - F^T + G, F = E Gamma, G = F E^T (= E Gamma E^T), summed
//     in FP64 onto the FP64 Gamma.
// The purification then removes the purity drift of order 2^-11 ||E|| in FP64.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace sgs {

#define EXP_LP_DEGREE 6        // Taylor degree: ||X_s|| <= 1/8 truncates below 1e-10 relative
#define LP_NS_ITERS 3          // purity drift ~1e-3 ||E|| reaches rounding in three Newton-Schulz steps

// X_s = 2^-s (ds/4)(Y - Y^T) with ||X_s||_F <= 1/8 and Q_d = I - X_s / d, one CTA per
// state; Y: [M][n][n] fp32; X_s, Q: [M][n][ldp] fp32 with zero padding columns.
__global__ void __launch_bounds__(1024) exp_prepare_lp_kernel(const float* Y, int n, int ldp, double ds, float* Xs,
                                                               float* Q, int* sq, int* err) {
    __shared__ double red[32];
    const int mu = blockIdx.x;
    const float* y = Y + (size_t)mu * n * n;
    double ss = 0.0;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        const double v = 0.25 * ds * ((double)y[e] - (double)y[(size_t)l * n + k]);
        ss += v * v;
    }
    ss = block_sum(ss, red);
    const double nrm = sqrt(ss);
    int s = 0;
    while (nrm * ldexp(1.0, -s) > EXP_THETA && s < 64) s++;
    if (s > EXP_MAX_SQUARINGS) {
        if (threadIdx.x == 0) atomicOr(err, SGS_DEV_EXPNORM);
        s = EXP_MAX_SQUARINGS;
    }
    if (threadIdx.x == 0) sq[mu] = s;
    const float sc = (float)(0.25 * ds * ldexp(1.0, -s));
    float* xs = Xs + (size_t)mu * n * ldp;
    float* q = Q + (size_t)mu * n * ldp;
    for (size_t e = threadIdx.x; e < (size_t)n * ldp; e += blockDim.x) {
        const int k = (int)(e / ldp), l = (int)(e % ldp);
        float v = 0.0f;
        if (l < n) v = sc * (y[(size_t)k * n + l] - y[(size_t)l * n + k]);
        xs[e] = v;
        q[e] = (k == l ? 1.0f : 0.0f) - v * (1.0f / EXP_LP_DEGREE);
    }
}

// fp32 [count] -> tensor-core operand: kind 0 tf32 (rounded to nearest), 1 bf16, 2 tf32
// split (hi, lo)
__global__ void lp_split_kernel(const float* src, void* hi, void* lo, size_t count, int kind) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const float x = src[e];
        if (kind == 0) {
            static_cast<float*>(hi)[e] = round_tf32(x);
        } else if (kind == 1) {
            static_cast<__nv_bfloat16*>(hi)[e] = __float2bfloat16_rn(x);
        } else {
            const float h = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
            static_cast<float*>(hi)[e] = h;
            static_cast<float*>(lo)[e] = x - h;
        }
    }
}

// FP64 [M][n][n] -> operand [M][n][ldp]: kind 0 tf32 (rounded), 1 bf16, 2 tf32 split (hi, lo)
__global__ void lp_from_f64_kernel(const double* src, int n, int ldp, void* hi, void* lo, int kind) {
    const int mu = blockIdx.y;
    const double* x = src + (size_t)mu * n * n;
    const size_t off = (size_t)mu * n * ldp;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)n * ldp; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / ldp), l = (int)(e % ldp);
        const double v = l < n ? x[(size_t)k * n + l] : 0.0;
        if (kind == 1) {
            static_cast<__nv_bfloat16*>(hi)[off + e] = __float2bfloat16_rn((float)v);
        } else if (kind == 2) {
            const float f = (float)v;
            const float h = __uint_as_float(__float_as_uint(f) & 0xffffe000u);
            static_cast<float*>(hi)[off + e] = h;
            static_cast<float*>(lo)[off + e] = (float)(v - (double)h);
        } else {
            static_cast<float*>(hi)[off + e] = round_tf32((float)v);
        }
    }
}

// Gamma' = Gamma + (F - F^T) + (G - G^T)/2 in FP64; F, G: [M][n][ldp] fp32
__global__ void assemble_lp_kernel(const double* gamma, const float* F, const float* G, int n, int ldp, double* out) {
    const int mu = blockIdx.y;
    const size_t nn = (size_t)n * n, np = (size_t)n * ldp;
    const double* g = gamma + mu * nn;
    const float* f = F + mu * np;
    const float* h = G + mu * np;
    double* o = out + mu * nn;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        const size_t a = (size_t)k * ldp + l, t = (size_t)l * ldp + k;
        o[e] = g[e] + ((double)f[a] - (double)f[t]) + 0.5 * ((double)h[a] - (double)h[t]);
    }
}

}  // namespace sgs
