// Spin-spin correlators of the SGS state (Eq. Cr, Eq. K2CK).
//
// <psi|O|psi> = sum_ab conj(lambda_a) lambda_b G_ab t_ab, with t_ab the
// generalised-Wick value of O on Delta^{b,a}; O is Hermitian, so an unordered
// pair contributes 2 Re{conj(lambda_a) lambda_b G_ab t(Delta^{b,a})} and a
// state |lambda_a|^2 t(Gamma_a).
//
// For sites 0 and s != 0 (Majoranas 0..3 and 4s..4s+3), each spin component
// S^a = (i/8) sum_pq K^a_pq c_p c_q (K^z: (01) = 1, (23) = -1; K^x: (03) = 1,
// (12) = -1; K^y: (02) = -1, (13) = -1, antisymmetrised) gives, by Wick with
// two-point values i Delta,
//   <S^a(0) S^a(s)> = [ (K:B00)(K:Bss) - 2 tr(K^T B0s K B0s^T) ] / 64,
// where B00, Bss, B0s are the 4x4 blocks of Delta.  For s = 0,
// S(0).S(0) = 3/4 (n_up + n_dn - 2 n_up n_dn).
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace sgs {

__device__ __forceinline__ double kspin(int a, int p, int q) {
    // antisymmetric 4x4 K^a, a = 0 (x), 1 (y), 2 (z)
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    const double s = p < q ? 1.0 : -1.0;
    double v = 0.0;
    if (a == 2) v = (lo == 0 && hi == 1) ? 1.0 : (lo == 2 && hi == 3) ? -1.0 : 0.0;
    else if (a == 0) v = (lo == 0 && hi == 3) ? 1.0 : (lo == 1 && hi == 2) ? -1.0 : 0.0;
    else v = (lo == 0 && hi == 2) ? -1.0 : (lo == 1 && hi == 3) ? -1.0 : 0.0;
    return s * v;
}

template <class Acc>
__device__ cplx spin_dot_value(const Acc& D, int s) {
    if (s == 0) {
        cplx d01 = D(0, 1), d23 = D(2, 3), d02 = D(0, 2), d13 = D(1, 3), d03 = D(0, 3), d12 = D(1, 2);
        cplx nu = cscale(csub(cmk(1.0, 0.0), d01), 0.5);
        cplx nv = cscale(csub(cmk(1.0, 0.0), d23), 0.5);
        cplx pf = cadd(csub(cmul(d01, d23), cmul(d02, d13)), cmul(d03, d12));
        cplx nn = cscale(cadd(csub(csub(cmk(1.0, 0.0), d01), d23), pf), 0.25);
        return cscale(csub(cadd(nu, nv), cscale(nn, 2.0)), 0.75);
    }
    cplx B00[4][4], Bss[4][4], B0s[4][4];
    for (int p = 0; p < 4; p++)
        for (int q = 0; q < 4; q++) {
            B00[p][q] = D(p, q);
            Bss[p][q] = D(4 * s + p, 4 * s + q);
            B0s[p][q] = D(p, 4 * s + q);
        }
    cplx tot = cmk(0.0, 0.0);
    for (int a = 0; a < 3; a++) {
        cplx k0 = cmk(0.0, 0.0), ks = cmk(0.0, 0.0), tr = cmk(0.0, 0.0);
        for (int p = 0; p < 4; p++)
            for (int q = 0; q < 4; q++) {
                const double K = kspin(a, p, q);
                if (K == 0.0) continue;
                k0 = cadd(k0, cscale(B00[p][q], K));
                ks = cadd(ks, cscale(Bss[p][q], K));
                // tr(K^T B0s K B0s^T) = sum_pq K_pq sum_st B0s[p][s] K_st B0s[q][t]
                for (int u = 0; u < 4; u++)
                    for (int v = 0; v < 4; v++) {
                        const double K2 = kspin(a, u, v);
                        if (K2 != 0.0) tr = cadd(tr, cscale(cmul(B0s[p][u], B0s[q][v]), K * K2));
                    }
            }
        tot = cadd(tot, cscale(csub(cmul(k0, ks), cscale(tr, 2.0)), 1.0 / 64.0));
    }
    return tot;
}

// kind 0: out[i] = C(sites[i]); kind 1: out[i] = sum over n_ch channels of
// <S(0).S(1 + (r-1) n_ch + c)>, r = sites[i].  partial: [P + M][n_sites]
__global__ void spin_corr_kernel(InstDev d, const double* si, const double* imd, const double* Gm, const double* lam,
                                 const int* sites, int n_sites, int kind, int n_ch, double* partial) {
    const int blk = blockIdx.x;
    const bool diag = blk >= d.P;
    const int a = diag ? blk - d.P : d.pa[blk];
    const int b = diag ? a : d.pb[blk];
    const int n = d.n, M = d.M;
    const double* g = d.gamma + (size_t)a * nn(d);
    const double* s = diag ? nullptr : si + (size_t)blk * nn(d);
    const double* im = diag ? nullptr : imd + (size_t)blk * nn(d);
    // Delta^{b,a} = conj(Delta^{a,b}) = -2 Si - i Im ; Delta^{a,a} = Gamma_a
    auto D = [&](int r, int c) -> cplx {
        if (diag) return cmk(g[(size_t)r * n + c], 0.0);
        return cmk(-2.0 * s[(size_t)r * n + c], -im[(size_t)r * n + c]);
    };
    cplx w;
    const cplx la = cmk(lam[2 * a], lam[2 * a + 1]), lb = cmk(lam[2 * b], lam[2 * b + 1]);
    if (diag) w = cmk(cabs2(la), 0.0);
    else w = cscale(cmul(cmul(cconj(la), lb), cmk(Gm[2 * (a * M + b)], Gm[2 * (a * M + b) + 1])), 2.0);
    for (int i = threadIdx.x; i < n_sites; i += blockDim.x) {
        cplx t = cmk(0.0, 0.0);
        if (kind == 0) {
            t = spin_dot_value(D, sites[i]);
        } else {
            for (int ch = 0; ch < n_ch; ch++) t = cadd(t, spin_dot_value(D, 1 + (sites[i] - 1) * n_ch + ch));
        }
        partial[(size_t)blk * n_sites + i] = cmul(w, t).x;
    }
}

__global__ void column_sum_kernel(const double* partial, int rows, int cols, double* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cols; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < rows; r++) acc += partial[(size_t)r * cols + i];
        out[i] = acc;
    }
}

}  // namespace sgs
