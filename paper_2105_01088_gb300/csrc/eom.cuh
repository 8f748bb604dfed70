// Equation of motion of every covariance matrix (Eq. EOM-Gamma3), assembled
// per receiver state mu with a fixed summation order over beta:
//   dGamma^mu = sum_beta 2 Re{ a1 [Delta, F] + a2 (Delta F Delta + F) + a3 Delta }
// with Delta = Delta^{beta,mu}, F = F^{beta,mu} and the per-(mu, beta)
// coefficients a1..a3 of the amplitude kernel.  For beta = mu, Delta = Gamma_mu
// and Delta F Delta = Gamma F Gamma comes from a per-state product; for beta !=
// mu the pair (a, b) = (min, max) supplies Delta^{a,b} (receiver b) or its
// complex conjugate Delta^{b,a} (receiver a), and likewise F, [Delta, F], Q.
// The sum over beta runs in the order the two kernels below give it.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace sgs {

// R: arithmetic type of the assembly.  The FP64 form assembles in double; the mixed
// forms, whose dense products already carry tensor-core rounding, assemble in float
// (FP64 arithmetic is slow on this part and the assembly would otherwise be bound by it).
//
// Every beta != mu term is linear in the pair's S^{-1}, Im Delta, Qr and Qi, so with the
// per-(mu, beta) weights
//   w0 = -4 a1x, w1 = -2 sgn a1y, w2 = 2 a2x, w3 = -2 sgn a2y, w4 = -4 a3x, w5 = -2 sgn a3y
// (a_jx, a_jy = co[2j - 2], co[2j - 1]; sgn = -1 where mu is the pair's first state) the
// sum over beta splits into
//   D = sum_beta (w2 Qr + w3 Qi + w4 S^{-1} + w5 Im)          (elementwise)
//   T = sum_beta (w0 S^{-1} + w1 Im)                          (elementwise)
// and the beta != mu part of dGamma_kl is D_kl + A_kl sum_beta w2 - sum_q T[k][c_q] a_q (over
// row l of A) - sum_q a_q T[c_q][l] (over row k of A), plus, on the rows and columns of the
// impurity modes, the terms of the pairs' F_imp.
// eom_pairs_kernel forms D (into dGamma) and T, six FMAs per pair and element;
// eom_finish_kernel adds the sparse part, the beta = mu term and the impurity terms.
// D, T and dGamma are antisymmetric (every term is), so both kernels compute the
// strictly lower entries of a tile pair (K >= L) and store them with their mirror:
// grid (lower_tile_count(n), M), 256 threads.

// weights w0..w5 of one (mu, beta != mu) and the pair's index in the view, into shared
// memory; a pair outside the view (another chunk of pairs) or not held at all (index -1:
// another rank's share of a pair-sharded step) contributes nothing here
template <typename R>
__device__ __forceinline__ void eom_weights(const InstDev& d, const double* coef, const int* pair_index, int mu,
                                            R* sw, int* sp) {
    const int M = d.M;
    for (int be = threadIdx.x; be < M; be += blockDim.x) {
        if (be == mu) { sp[be] = -1; continue; }
        const int p = pair_index[mu * M + be] - d.p_off;
        if (p < 0 || p >= d.p_cnt) { sp[be] = -1; continue; }
        const double sgn = (d.pa[p] == mu) ? -1.0 : 1.0;     // receiver a: complex conjugate
        const double* co = coef + (size_t)(mu * M + be) * 6;
        sw[6 * be + 0] = (R)(-4.0 * co[0]);
        sw[6 * be + 1] = (R)(-2.0 * sgn * co[1]);
        sw[6 * be + 2] = (R)(2.0 * co[2]);
        sw[6 * be + 3] = (R)(-2.0 * sgn * co[3]);
        sw[6 * be + 4] = (R)(-4.0 * co[4]);
        sw[6 * be + 5] = (R)(-2.0 * sgn * co[5]);
        sp[be] = p;
    }
}

// dynamic shared memory of both assembly kernels: M x 6 weights and M pair indices
template <typename R> inline size_t eom_smem(int M) { return (size_t)M * 6 * sizeof(R) + (size_t)M * sizeof(int); }

// accumulate = 1 adds onto tsum and dgamma (the pairs in chunks), 0 overwrites them
template <typename R>
__global__ void __launch_bounds__(256) eom_pairs_kernel(InstDev d, const double* si, const double* imd,
                                                        const double* qr, const double* qi, const double* coef,
                                                        const int* pair_index, double* tsum, double* dgamma,
                                                        int accumulate) {
    extern __shared__ double eom_sraw[];
    __shared__ double st[2][32][33];
    const int mu = blockIdx.y, M = d.M, n = d.n;
    R* sw = reinterpret_cast<R*>(eom_sraw);
    int* sp = reinterpret_cast<int*>(sw + 6 * M);
    eom_weights<R>(d, coef, pair_index, mu, sw, sp);
    __syncthreads();
    int K, L;
    lower_tile(blockIdx.x, K, L);
    const int k0 = K * 32, l0 = L * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const size_t N = nn(d);
    double* T = tsum + (size_t)mu * N;
    double* out = dgamma + (size_t)mu * N;
    for (int j = ty; j < 32; j += 8) {
        const int k = k0 + j, l = l0 + tx;
        if (k >= n || l >= n || k <= l) continue;
        const size_t e = (size_t)k * n + l;
        R t = 0, acc = 0;
        for (int be = 0; be < M; be++) {
            const int p = sp[be];
            if (p < 0) continue;
            const size_t o = (size_t)p * N + e;
            const R sv = (R)si[o], iv = (R)imd[o], qrv = (R)qr[o], qiv = (R)qi[o];
            const R* w = sw + 6 * be;
            t = fma(w[0], sv, t);
            t = fma(w[1], iv, t);
            acc = fma(w[2], qrv, acc);
            acc = fma(w[3], qiv, acc);
            acc = fma(w[4], sv, acc);
            acc = fma(w[5], iv, acc);
        }
        st[0][j][tx] = accumulate ? T[e] + (double)t : (double)t;
        st[1][j][tx] = accumulate ? out[e] + (double)acc : (double)acc;
    }
    __syncthreads();
    store_antisym_tile(T, n, k0, l0, st[0]);
    store_antisym_tile(out, n, k0, l0, st[1]);
}

// parts of eom_finish_kernel: the pairs' impurity terms (per chunk of pairs), the rest (the
// sparse A terms on the summed T and sum w2 of every pair, and the beta = mu term), or both
enum { EOM_FINISH_PAIRS = 1, EOM_FINISH_REST = 2, EOM_FINISH_ALL = 3 };

// self_mask (may be nullptr): state mu's beta = mu term is added only where self_mask[mu] != 0
// (a pair-sharded step adds it on one rank, so that the ranks' partial sums add up to dGamma)
template <typename R>
__global__ void __launch_bounds__(256) eom_finish_kernel(InstDev d, const double* si, const double* imd,
                                                         const double* fimp, const double* fimp_state,
                                                         const double* gfg, const double* coef, const int* pair_index,
                                                         const double* tsum, double* dgamma, const int* self_mask,
                                                         int part) {
    extern __shared__ double eom_sraw[];
    __shared__ R s_w2;
    __shared__ double sf[32][33];
    __shared__ unsigned char sh[32][33];
    const int mu = blockIdx.y;
    const int n = d.n, ni = d.nimp, M = d.M;
    R* sw = reinterpret_cast<R*>(eom_sraw);
    int* sp = reinterpret_cast<int*>(sw + 6 * M);
    eom_weights<R>(d, coef, pair_index, mu, sw, sp);
    __syncthreads();
    if (threadIdx.x == 0) {
        R w = 0;
        for (int be = 0; be < M; be++)
            if (sp[be] >= 0) w += sw[6 * be + 2];
        s_w2 = w;
    }
    __syncthreads();
    const size_t N = nn(d);
    const bool rest = (part & EOM_FINISH_REST) != 0, pair_imp = (part & EOM_FINISH_PAIRS) != 0;
    const bool self_term = rest && (self_mask == nullptr || self_mask[mu] != 0);
    const double* gm = d.gamma + (size_t)mu * N;
    const double* fs = fimp_state + (size_t)mu * ni * ni;
    const double* gfgm = gfg + (size_t)mu * N;
    const double* T = tsum + (size_t)mu * N;
    double* out = dgamma + (size_t)mu * N;
    int K, L;
    lower_tile(blockIdx.x, K, L);
    const int k0 = K * 32, l0 = L * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int k = k0 + j, l = l0 + tx;
        sh[j][tx] = 0;
        if (k >= n || l >= n || k < l) continue;
        if (k == l) {                                       // the diagonal is zero
            sf[j][tx] = 0.0;
            sh[j][tx] = 1;
            continue;
        }
        const size_t e = (size_t)k * n + l;
        const int sk = d.slot[k], sl = d.slot[l];
        if (!rest && sk < 0 && sl < 0) continue;            // the pairs' impurity terms only
        // one pass over each of the CSR rows l and k of A (read-only loads) for A_kl, the pairs'
        // commutator terms against A, -(T A^T)_kl - (A T)_kl, and the beta = mu term's
        // (Gamma F)_kl, (F Gamma)_kl: the T and Gamma loads of a row entry issue together
        R akl = 0, ta = 0, at = 0, gf = 0, fg = 0;
        {
            const int q0 = __ldg(d.a_rowptr + l), q1 = __ldg(d.a_rowptr + l + 1);
            for (int q = q0; q < q1; q++) {
                const int cq = __ldg(d.a_col + q);
                const R v = (R)__ldg(d.a_val + q);
                if (rest) ta = fma((R)T[(size_t)k * n + cq], v, ta);
                if (self_term) gf = fma(-(R)gm[(size_t)k * n + cq], v, gf);
            }
        }
        {
            const int q0 = __ldg(d.a_rowptr + k), q1 = __ldg(d.a_rowptr + k + 1);
            for (int q = q0; q < q1; q++) {
                const int cq = __ldg(d.a_col + q);
                const R v = (R)__ldg(d.a_val + q);
                if (cq == l) akl = v;
                if (rest) at = fma(v, (R)T[(size_t)cq * n + l], at);
                if (self_term) fg = fma(v, (R)gm[(size_t)cq * n + l], fg);
            }
        }
        R acc = (R)out[e];
        if (rest) {
            acc = fma(akl, s_w2, acc);
            acc = acc - ta - at;
        }
        if (self_term) {   // beta = mu: Delta = Gamma_mu, Delta F Delta = Gamma F Gamma
            const double* co = coef + (size_t)(mu * M + mu) * 6;
            const R g = (R)gm[e];
            const R f = akl + ((sk >= 0 && sl >= 0) ? (R)fs[sk * ni + sl] : (R)0);
            if (sl >= 0) for (int m = 0; m < ni; m++) gf += (R)gm[(size_t)k * n + d.imp[m]] * (R)fs[m * ni + sl];
            if (sk >= 0) for (int m = 0; m < ni; m++) fg += (R)fs[sk * ni + m] * (R)gm[(size_t)d.imp[m] * n + l];
            acc += (R)2 * ((R)co[0] * (gf - fg) + (R)co[2] * ((R)gfgm[e] + f) + (R)co[4] * g);
        }
        if (pair_imp && (sk >= 0 || sl >= 0)) {
            // rows and columns of the impurity modes: the pairs' F_imp terms of [Delta, F] and Q + F
            for (int be = 0; be < M; be++) {
                const int p = sp[be];
                if (p < 0) continue;
                const R sgn = (d.pa[p] == mu) ? (R)-1 : (R)1;
                const double* s = si + (size_t)p * N;
                const double* im = imd + (size_t)p * N;
                const double* fp = fimp + (size_t)p * ni * ni * 2;
                R dfx = 0, dfy = 0, fdx = 0, fdy = 0, Fx = 0, Fy = 0;
                if (sl >= 0)
                    for (int m = 0; m < ni; m++) {
                        const R ax = (R)-2 * (R)s[(size_t)k * n + d.imp[m]], ay = sgn * (R)im[(size_t)k * n + d.imp[m]];
                        const R bx = (R)fp[2 * (m * ni + sl)], by = sgn * (R)fp[2 * (m * ni + sl) + 1];
                        dfx += ax * bx - ay * by;
                        dfy += ax * by + ay * bx;
                    }
                if (sk >= 0)
                    for (int m = 0; m < ni; m++) {
                        const R ax = (R)fp[2 * (sk * ni + m)], ay = sgn * (R)fp[2 * (sk * ni + m) + 1];
                        const R bx = (R)-2 * (R)s[(size_t)d.imp[m] * n + l], by = sgn * (R)im[(size_t)d.imp[m] * n + l];
                        fdx += ax * bx - ay * by;
                        fdy += ax * by + ay * bx;
                    }
                if (sk >= 0 && sl >= 0) {
                    Fx = (R)fp[2 * (sk * ni + sl)];
                    Fy = sgn * (R)fp[2 * (sk * ni + sl) + 1];
                }
                const double* co = coef + (size_t)(mu * M + be) * 6;
                acc += (R)2 * ((R)co[0] * (dfx - fdx) - (R)co[1] * (dfy - fdy) + (R)co[2] * Fx - (R)co[3] * Fy);
            }
        }
        sf[j][tx] = (double)acc;
        sh[j][tx] = 1;
    }
    __syncthreads();
    store_antisym_tile(out, n, k0, l0, sf, sh);
}

}  // namespace sgs
