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
        double akl = 0.0;
        for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++)
            if (d.a_col[q] == l) akl = d.a_val[q];
        double acc = 0.0;
        {   // beta = mu
            const double* co = coef + (size_t)(mu * M + mu) * 6;
            double g = gm[e];
            double f = akl + ((sk >= 0 && sl >= 0) ? fs[sk * ni + sl] : 0.0);
            double gf = 0.0, fg = 0.0;   // (Gamma F)_kl, (F Gamma)_kl
            for (int q = d.a_rowptr[l]; q < d.a_rowptr[l + 1]; q++) gf -= gm[(size_t)k * n + d.a_col[q]] * d.a_val[q];
            for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++) fg += d.a_val[q] * gm[(size_t)d.a_col[q] * n + l];
            if (sl >= 0) for (int m = 0; m < ni; m++) gf += gm[(size_t)k * n + d.imp[m]] * fs[m * ni + sl];
            if (sk >= 0) for (int m = 0; m < ni; m++) fg += fs[sk * ni + m] * gm[(size_t)d.imp[m] * n + l];
            acc += 2.0 * (co[0] * (gf - fg) + co[2] * (gfgm[e] + f) + co[4] * g);
        }
        for (int be = 0; be < M; be++) {
            if (be == mu) continue;
            const int p = pair_index[mu * M + be];
            const double sgn = (d.pa[p] == mu) ? -1.0 : 1.0;   // receiver a: complex conjugate
            const double* s = si + (size_t)p * nn(d);
            const double* im = imd + (size_t)p * nn(d);
            const double* fp = fimp + (size_t)p * ni * ni * 2;
            auto dl = [&](int r, int c) -> cplx {
                size_t o = (size_t)r * n + c;
                return cmk(-2.0 * s[o], sgn * im[o]);
            };
            cplx D = dl(k, l);
            cplx F = cmk(akl, 0.0);
            if (sk >= 0 && sl >= 0) F = cadd(F, cmk(fp[2 * (sk * ni + sl)], sgn * fp[2 * (sk * ni + sl) + 1]));
            // C = Delta F - F Delta
            cplx df = cmk(0.0, 0.0), fd = cmk(0.0, 0.0);
            for (int q = d.a_rowptr[l]; q < d.a_rowptr[l + 1]; q++) df = csub(df, cscale(dl(k, d.a_col[q]), d.a_val[q]));
            for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++) fd = cadd(fd, cscale(dl(d.a_col[q], l), d.a_val[q]));
            if (sl >= 0)
                for (int m = 0; m < ni; m++)
                    df = cadd(df, cmul(dl(k, d.imp[m]), cmk(fp[2 * (m * ni + sl)], sgn * fp[2 * (m * ni + sl) + 1])));
            if (sk >= 0)
                for (int m = 0; m < ni; m++)
                    fd = cadd(fd, cmul(cmk(fp[2 * (sk * ni + m)], sgn * fp[2 * (sk * ni + m) + 1]), dl(d.imp[m], l)));
            cplx C = csub(df, fd);
            cplx Q = cmk(qr[(size_t)p * nn(d) + e], sgn * qi[(size_t)p * nn(d) + e]);
            const double* co = coef + (size_t)(mu * M + be) * 6;
            cplx QF = cadd(Q, F);
            // 2 Re{a1 C + a2 (Q + F) + a3 Delta}
            acc += 2.0 * (co[0] * C.x - co[1] * C.y + co[2] * QF.x - co[3] * QF.y + co[4] * D.x - co[5] * D.y);
        }
        out[e] = acc;
    }
}

}  // namespace sgs
