// Equation of motion of every covariance matrix (Eq. EOM-Gamma3), assembled
// per receiver state mu with a fixed summation order over beta:
//   dGamma^mu = sum_beta 2 Re{ a1 [Delta, F] + a2 (Delta F Delta + F) + a3 Delta }
// with Delta = Delta^{beta,mu}, F = F^{beta,mu} and the per-(mu, beta)
// coefficients a1..a3 of the amplitude kernel.  For beta = mu, Delta = Gamma_mu
// and Delta F Delta = Gamma F Gamma comes from a per-state product; for beta !=
// mu the pair (a, b) = (min, max) supplies Delta^{a,b} (receiver b) or its
// complex conjugate Delta^{b,a} (receiver a), and likewise F, [Delta, F], Q.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace sgs {

// R: arithmetic type of the assembly.  The FP64 form assembles in double; the mixed
// forms, whose dense products already carry tensor-core rounding, assemble in float
// (FP64 arithmetic is slow on this part and the assembly would otherwise be bound by it).
template <typename R>
__global__ void __launch_bounds__(256) eom_kernel(InstDev d, const double* si, const double* imd,
                                                  const double* qr, const double* qi, const double* fimp,
                                                  const double* fimp_state, const double* gfg,
                                                  const double* coef, const int* pair_index, double* dgamma) {
    const int mu = blockIdx.y;
    const int n = d.n, ni = d.nimp, M = d.M;
    const double* gm = d.gamma + (size_t)mu * nn(d);
    const double* fs = fimp_state + (size_t)mu * ni * ni;
    const double* gfgm = gfg + (size_t)mu * nn(d);
    double* out = dgamma + (size_t)mu * nn(d);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn(d); e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        const int sk = d.slot[k], sl = d.slot[l];
        // A_kl (row k of the CSR)
        R akl = 0;
        for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++)
            if (d.a_col[q] == l) akl = (R)d.a_val[q];
        R acc = 0;
        {   // beta = mu
            const double* co = coef + (size_t)(mu * M + mu) * 6;
            const R g = (R)gm[e];
            const R f = akl + ((sk >= 0 && sl >= 0) ? (R)fs[sk * ni + sl] : (R)0);
            R gf = 0, fg = 0;   // (Gamma F)_kl, (F Gamma)_kl
            for (int q = d.a_rowptr[l]; q < d.a_rowptr[l + 1]; q++) gf -= (R)gm[(size_t)k * n + d.a_col[q]] * (R)d.a_val[q];
            for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++) fg += (R)d.a_val[q] * (R)gm[(size_t)d.a_col[q] * n + l];
            if (sl >= 0) for (int m = 0; m < ni; m++) gf += (R)gm[(size_t)k * n + d.imp[m]] * (R)fs[m * ni + sl];
            if (sk >= 0) for (int m = 0; m < ni; m++) fg += (R)fs[sk * ni + m] * (R)gm[(size_t)d.imp[m] * n + l];
            acc += (R)2 * ((R)co[0] * (gf - fg) + (R)co[2] * ((R)gfgm[e] + f) + (R)co[4] * g);
        }
        for (int be = 0; be < M; be++) {
            if (be == mu) continue;
            const int p = pair_index[mu * M + be];
            const R sgn = (d.pa[p] == mu) ? (R)-1 : (R)1;    // receiver a: complex conjugate
            const double* s = si + (size_t)p * nn(d);
            const double* im = imd + (size_t)p * nn(d);
            const double* fp = fimp + (size_t)p * ni * ni * 2;
            // Delta = -2 S^{-1} + i sgn Im
            auto dre = [&](int r, int c) -> R { return (R)-2 * (R)s[(size_t)r * n + c]; };
            auto dim = [&](int r, int c) -> R { return sgn * (R)im[(size_t)r * n + c]; };
            const R Dx = dre(k, l), Dy = dim(k, l);
            R Fx = akl, Fy = 0;
            if (sk >= 0 && sl >= 0) { Fx += (R)fp[2 * (sk * ni + sl)]; Fy += sgn * (R)fp[2 * (sk * ni + sl) + 1]; }
            // C = Delta F - F Delta; the sparse (quadratic) part sums S^{-1} and Im against A
            // first and scales by -2 and sgn once
            R ss = 0, si_ = 0;
            for (int q = d.a_rowptr[l]; q < d.a_rowptr[l + 1]; q++) {
                const R a = (R)d.a_val[q];
                ss -= (R)s[(size_t)k * n + d.a_col[q]] * a;
                si_ -= (R)im[(size_t)k * n + d.a_col[q]] * a;
            }
            for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++) {
                const R a = (R)d.a_val[q];
                ss -= a * (R)s[(size_t)d.a_col[q] * n + l];
                si_ -= a * (R)im[(size_t)d.a_col[q] * n + l];
            }
            R dfx = (R)-2 * ss, dfy = sgn * si_, fdx = 0, fdy = 0;
            if (sl >= 0)
                for (int m = 0; m < ni; m++) {
                    const R ax = dre(k, d.imp[m]), ay = dim(k, d.imp[m]);
                    const R bx = (R)fp[2 * (m * ni + sl)], by = sgn * (R)fp[2 * (m * ni + sl) + 1];
                    dfx += ax * bx - ay * by;
                    dfy += ax * by + ay * bx;
                }
            if (sk >= 0)
                for (int m = 0; m < ni; m++) {
                    const R ax = (R)fp[2 * (sk * ni + m)], ay = sgn * (R)fp[2 * (sk * ni + m) + 1];
                    const R bx = dre(d.imp[m], l), by = dim(d.imp[m], l);
                    fdx += ax * bx - ay * by;
                    fdy += ax * by + ay * bx;
                }
            const R Cx = dfx - fdx, Cy = dfy - fdy;
            const R QFx = (R)qr[(size_t)p * nn(d) + e] + Fx, QFy = sgn * (R)qi[(size_t)p * nn(d) + e] + Fy;
            const double* co = coef + (size_t)(mu * M + be) * 6;
            // 2 Re{a1 C + a2 (Q + F) + a3 Delta}
            acc += (R)2 * ((R)co[0] * Cx - (R)co[1] * Cy + (R)co[2] * QFx - (R)co[3] * QFy + (R)co[4] * Dx -
                           (R)co[5] * Dy);
        }
        out[e] = (double)acc;
    }
}

// dGamma <- (dGamma - dGamma^T) / 2: the float assembly of the mixed forms computes each
// element on its own, so its rounding leaves a symmetric part of relative size 1e-7 that the
// exact dGamma (tangent to the pure states) does not have
__global__ void antisymmetrise_kernel(double* a, int n) {
    double* x = a + (size_t)blockIdx.y * n * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        if (k > l) continue;
        const double v = k == l ? 0.0 : 0.5 * (x[e] - x[(size_t)l * n + k]);
        x[e] = v;
        x[(size_t)l * n + k] = -v;
    }
}

}  // namespace sgs
