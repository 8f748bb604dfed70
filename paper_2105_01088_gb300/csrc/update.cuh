// Per-state update of App. A: Gamma <- R Gamma R^T with R = exp(X),
// X = (ds/4)[Gamma, dGamma] (Eq. ExpStep; the factor 1/4 makes the step agree
// with Gamma + ds dGamma of Eq. RKstep to first order), followed by the
// canonical-form renormalisation (polar factor, Newton-Schulz in FP64).
//
// exp(X) by scaling and squaring: X_s = X / 2^s with ||X_s||_F <= 1/8, the Taylor
// polynomial of degree 10 (truncation < 3e-18) evaluated by Paterson-Stockmeyer in
// blocks of three, p = B0 + B1 Y + B2 Y^2 + B3 Y^3 with Y = X_s^3 and
// B_j = sum_i X_s^i / (3j + i)!, i < 3 (five products instead of Horner's nine), then s
// squarings.  The products run on the batched FP64 GEMM; this file holds the
// elementwise pieces.
#pragma once
#include "common.cuh"

namespace sgs {

#define EXP_TAYLOR_DEGREE 10
#define EXP_MAX_SQUARINGS 14
#define EXP_THETA 0.125
#define EULER_NS_ITERS 6       // Newton-Schulz steps after an Euler step: singular values 1 + d with
                               // |d| <= 0.3 reach 1 to rounding (d -> -1.5 d^2 per step)

// X = (ds/4)(Y - Y^T) with Y = Gamma dGamma (so [Gamma, dGamma] = Y - Y^T), its
// Frobenius norm -> squarings s (||X 2^-s||_F <= 1/8), and X_s = 2^-s X -> Xs.
__global__ void __launch_bounds__(1024) exp_prepare_kernel(const double* Y, double* Xs, int n, double ds, int* sq,
                                                            double* scale, int* err) {
    __shared__ double red[32];
    const int mu = blockIdx.x;
    const size_t nn = (size_t)n * n;
    const double* y = Y + mu * nn;
    double* x = Xs + mu * nn;
    double ss = 0.0;
    for (size_t e = threadIdx.x; e < nn; e += blockDim.x) {
        int k = (int)(e / n), l = (int)(e % n);
        double v = 0.25 * ds * (y[e] - y[(size_t)l * n + k]);
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
    const double sc = ldexp(1.0, -s);
    if (threadIdx.x == 0) { sq[mu] = s; scale[mu] = sc; }
    for (size_t e = threadIdx.x; e < nn; e += blockDim.x) {
        int k = (int)(e / n), l = (int)(e % n);
        x[e] = sc * 0.25 * ds * (y[e] - y[(size_t)l * n + k]);
    }
}

// out = a X + d I (the leading block of the Paterson-Stockmeyer evaluation)
__global__ void scaled_plus_identity_kernel(const double* X, double a, double d, int n, double* out, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const size_t w = e % ((size_t)n * n);
        const int k = (int)(w / n), l = (int)(w % n);
        out[e] = a * X[e] + (k == l ? d : 0.0);
    }
}

// health of an instance: out[0] = max |(Gamma^2)_kl + delta_kl| over the states (G2 holds
// Gamma^2), out[1] = number of non-finite entries of Gamma, out[2] = smallest / largest
// eigenvalue of G at the last amplitude solve (the diagonal of its Jacobi result, m x m
// real embedding), out[3] = the energy of that solve
__global__ void __launch_bounds__(1024) health_kernel(const double* G2, const double* gamma, size_t count, int n,
                                                       const double* eig, int m, const double* E, double* out) {
    __shared__ double red[32];
    double worst = 0.0, bad = 0.0;
    const size_t nn = (size_t)n * n;
    for (size_t e = threadIdx.x; e < count; e += blockDim.x) {
        const size_t w = e % nn;
        const double d = G2[e] + ((w / n) == (w % n) ? 1.0 : 0.0);
        worst = fmax(worst, fabs(d));
        if (!isfinite(gamma[e])) bad += 1.0;
        if (!isfinite(d)) worst = INFINITY;
    }
    // block max via a sum of per-warp maxima is not a max: reduce with shuffles, then shared memory
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_down_sync(0xffffffffu, worst, o));
    __shared__ double wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = worst;
    bad = block_sum(bad, red);
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, wmax[w]);
        double lo = INFINITY, hi = 0.0;
        for (int j = 0; j < m; j++) {
            const double v = eig[(size_t)j * m + j];
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
        out[0] = mx;
        out[1] = bad;
        out[2] = hi > 0.0 ? lo / hi : 0.0;
        out[3] = E[0];
    }
}

// out = x + a y (the Euler step of Eq. RKstep)
__global__ void axpy_kernel(const double* x, const double* y, double a, double* out, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        out[e] = x[e] + a * y[e];
}

__global__ void copy_kernel(const double* src, double* dst, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

}  // namespace sgs
