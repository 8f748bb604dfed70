// Pair-level kernels of one imaginary-time step (Sec. II B-C, III B).
//
// For an unordered pair (a < b): S = Gamma_a + Gamma_b, D = Gamma_a - Gamma_b,
// Si = S^{-1}, Im = D Si, and the transition matrix of Eq. (def-delta-matrix)
//   Delta^{a,b} = (iD - 2) Si = -2 Si + i Im,   Delta^{b,a} = conj(Delta^{a,b}).
// Because D S = -S D for pure states, Delta^{a,b} = -Si (iD + 2) too, so
//   Q = Delta F Delta = -(iD - 2) W (iD + 2),  W = Si F Si,
//     = D W D - 2i (D W - W D) + 4 W,
// and with F = Fr + i Fi (Fi non-zero only on the impurity block) every
// dense product is real: Wr = (Si Fr) Si, V = D Wr, X = V D, W D = (D W)^T;
// the Fi parts are rank <= (#impurity Majoranas) corrections.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace sgs {

struct InstDev {
    int n, N, M, P, Ppf, nimp, nq;
    double e_const;
    double parity;
    const int* pa;          // [P] first state of pair p
    const int* pb;          // [P] second state
    const int* pf_pair;     // [Ppf] pair of each phase-Pfaffian entry (pairs with a >= 1)
    const int* pair_pf;     // [P] phase-Pfaffian entry of pair p, or -1 (a == 0)
    const double* gamma;    // [M][n][n]
    const int* a_rowptr;    // CSR of A (n+1)
    const int* a_row;       // row of each non-zero (COO view of the same entries)
    const int* a_col;
    int a_nnz;
    const double* a_val;
    const int* q_idx;       // [nq][4] antisymmetrised quartic entries
    const double* q_val;    // [nq]
    const int* imp;         // [nimp] impurity Majoranas
    const int* slot;        // [n] slot in imp, or -1
    int p_off, p_cnt;       // the pairs this view holds: global pair indices p_off .. p_off + p_cnt - 1
                            // (pair_index is global; pa, pb, pair_pf and the per-pair buffers are the view's)
    int nh;                 // interaction terms of more than four Majoranas
    const int* h_len;       // [nh] 6 or 8
    const int* h_off;       // [nh] offset of each term's indices in h_idx
    const int* h_idx;       // indices, each term in its own order
    const double* h_val;    // [nh] v (-1)^((r + r mod 2) / 2): the energy is h_val Pf(Delta_S)
};

#define SGS_MAX_TERM 8      // Majoranas in one interaction term

// Pfaffian of a small complex antisymmetric matrix X (m <= SGS_MAX_TERM, m even,
// row-major, destroyed) by Parlett-Reid elimination with pivoting; 0 for a zero pivot
__device__ inline cplx small_pf(cplx* X, int m) {
    cplx pf = cmk(1.0, 0.0);
    for (int k = 0; k + 1 < m; k += 2) {
        int p = k + 1;
        double best = cabs2(X[(k + 1) * m + k]);
        for (int j = k + 2; j < m; j++) {
            const double v = cabs2(X[j * m + k]);
            if (v > best) { best = v; p = j; }
        }
        if (p != k + 1) {
            for (int j = 0; j < m; j++) { cplx t = X[(k + 1) * m + j]; X[(k + 1) * m + j] = X[p * m + j]; X[p * m + j] = t; }
            for (int j = 0; j < m; j++) { cplx t = X[j * m + k + 1]; X[j * m + k + 1] = X[j * m + p]; X[j * m + p] = t; }
            pf = cscale(pf, -1.0);
        }
        const cplx piv = X[k * m + k + 1];
        const double pm2 = cabs2(piv);
        if (!(pm2 > 0.0)) return cmk(0.0, 0.0);
        pf = cmul(pf, piv);
        const cplx inv = cscale(cconj(piv), 1.0 / pm2);
        for (int i = k + 2; i < m; i++) {
            const cplx ti = cmul(X[k * m + i], inv), ui = X[i * m + k + 1];
            for (int j = k + 2; j < m; j++) {
                const cplx tj = cmul(X[k * m + j], inv), uj = X[j * m + k + 1];
                X[i * m + j] = cadd(X[i * m + j], cadd(cmul(ti, uj), cscale(cmul(ui, tj), -1.0)));
            }
        }
    }
    return pf;
}

__device__ __forceinline__ size_t nn(const InstDev& d) { return (size_t)d.n * d.n; }

// S_p = Gamma_a + Gamma_b into the Gauss-Jordan work matrix of pair p
__global__ void pair_sum_kernel(InstDev d, double* work) {
    const int p = blockIdx.y;
    const double* ga = d.gamma + (size_t)d.pa[p] * nn(d);
    const double* gb = d.gamma + (size_t)d.pb[p] * nn(d);
    double* w = work + (size_t)p * nn(d);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn(d); e += (size_t)gridDim.x * blockDim.x)
        w[e] = ga[e] + gb[e];
}

// Y_q = Gamma_0 + Delta^{a,b} = (Gamma_0 - 2 Si) + i Im for the phase Pfaffian
__global__ void pf_build_kernel(InstDev d, const double* si, const double* imd, double* work) {
    const int q = blockIdx.y;
    const int p = d.pf_pair[q];
    const double* g0 = d.gamma;
    const double* s = si + (size_t)p * nn(d);
    const double* im = imd + (size_t)p * nn(d);
    double* yr = work + (size_t)q * 2 * nn(d);
    double* yi = yr + nn(d);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn(d); e += (size_t)gridDim.x * blockDim.x) {
        yr[e] = g0[e] - 2.0 * s[e];
        yi[e] = im[e];
    }
}

// Gram matrix, Hamiltonian matrix and the impurity block of the generalised
// Fock matrices.  Blocks [0, P): pairs; blocks [P, P+M): diagonal states.
//   G_ab = |G_ab| e^{i phi}, log|G_ab| = (-N log 2 + log|det S|/2)/2,
//   phase from Pf(Gamma_0) Pf(Gamma_0 + Delta^{a,b}) (reference gauge), and
//   h_ba = G_ba (e_const + Tr(A Delta^{a,b}) - 3 sum U Delta Delta).
// parts: GH_FOCK (the impurity blocks of F and the energy density, into dens), GH_GRAM (G and h
// from dens, log|det S| and the phase Pfaffian), or both.  The equation of motion's products need
// only the first, so they may run while the phase Pfaffians are computed.
enum { GH_FOCK = 1, GH_GRAM = 2, GH_ALL = 3 };
__global__ void __launch_bounds__(256) pair_gh_kernel(InstDev d, const double* si, const double* imd,
                                                      const double* logdet, const double* pfphase,
                                                      double* Gm, double* hm, double* fimp, double* fimp_state,
                                                      int part, double* dens_buf) {
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const bool diag = blk >= d.P;
    const int p = diag ? -1 : blk;
    const int a = diag ? blk - d.P : d.pa[p];
    const int bq = diag ? a : d.pb[p];
    const int n = d.n;
    if (!(part & GH_FOCK)) {
        // G and h from the stored energy density
        if (threadIdx.x == 0) {
            const int M = d.M;
            const cplx dens = cmk(dens_buf[2 * blk], dens_buf[2 * blk + 1]);
            if (diag) {
                Gm[2 * (a * M + a)] = 1.0;
                Gm[2 * (a * M + a) + 1] = 0.0;
                hm[2 * (a * M + a)] = dens.x;
                hm[2 * (a * M + a) + 1] = 0.0;
            } else {
                double ld = logdet[p];
                double mag = (ld == -INFINITY || ld != ld) ? 0.0 : exp(0.5 * (-d.N * 0.6931471805599453 + 0.5 * ld));
                cplx ph = cmk(1.0, 0.0);
                int q2 = d.pair_pf[p];
                if (q2 >= 0) {
                    ph = cmk(d.parity * pfphase[2 * q2], d.parity * pfphase[2 * q2 + 1]);
                    double m2 = sqrt(cabs2(ph));
                    ph = m2 > 0.0 ? cscale(ph, 1.0 / m2) : cmk(0.0, 0.0);
                }
                cplx gab = cscale(ph, mag);
                cplx gba = cconj(gab);
                cplx hba = cmul(gba, dens);
                Gm[2 * (a * M + bq)] = gab.x;
                Gm[2 * (a * M + bq) + 1] = gab.y;
                Gm[2 * (bq * M + a)] = gba.x;
                Gm[2 * (bq * M + a) + 1] = gba.y;
                hm[2 * (bq * M + a)] = hba.x;
                hm[2 * (bq * M + a) + 1] = hba.y;
                hm[2 * (a * M + bq)] = hba.x;
                hm[2 * (a * M + bq) + 1] = -hba.y;
            }
        }
        return;
    }
    const double* dr = diag ? d.gamma + (size_t)a * nn(d) : si + (size_t)p * nn(d);
    const double* di = diag ? nullptr : imd + (size_t)p * nn(d);
    // Delta^{a,b}[k][l] = -2 Si[k][l] + i Im[k][l];  Delta^{a,a} = Gamma_a
    auto delta = [&](int k, int l) -> cplx {
        if (diag) return cmk(dr[(size_t)k * n + l], 0.0);
        return cmk(-2.0 * dr[(size_t)k * n + l], di[(size_t)k * n + l]);
    };
    // Tr(A Delta) = sum_kl A_kl Delta_lk over the non-zeros of A
    double tr_r = 0.0, tr_i = 0.0;
    for (int e = threadIdx.x; e < d.a_nnz; e += blockDim.x) {
        cplx v = delta(d.a_col[e], d.a_row[e]);
        tr_r += d.a_val[e] * v.x;
        tr_i += d.a_val[e] * v.y;
    }
    tr_r = block_sum(tr_r, red);
    tr_i = block_sum(tr_i, red);
    if (threadIdx.x == 0) {
        cplx q = cmk(0.0, 0.0);
        const int ni = d.nimp;
        cplx F[SGS_MAX_IMP * SGS_MAX_IMP];
        for (int e = 0; e < ni * ni; e++) F[e] = cmk(0.0, 0.0);
        for (int e = 0; e < d.nq; e++) {
            const int* ix = d.q_idx + 4 * e;
            const double v = d.q_val[e];
            cplx x = delta(ix[2], ix[3]);
            q = cadd(q, cscale(cmul(delta(ix[0], ix[1]), x), v));
            int s0 = d.slot[ix[0]], s1 = d.slot[ix[1]];
            F[s0 * ni + s1] = cadd(F[s0 * ni + s1], cscale(x, 6.0 * v));
        }
        // terms of six or eight Majoranas: energy h_val Pf(Delta_S); Fock entries
        // F_{s_a s_b} = -(1/2) h_val (-1)^(a + b + 1) Pf(Delta_S without a, b) (a < b), antisymmetric
        cplx qh = cmk(0.0, 0.0);
        for (int t = 0; t < d.nh; t++) {
            const int m = d.h_len[t];
            const int* ix = d.h_idx + d.h_off[t];
            const double v = d.h_val[t];
            cplx S[SGS_MAX_TERM * SGS_MAX_TERM], X[SGS_MAX_TERM * SGS_MAX_TERM];
            for (int i = 0; i < m; i++)
                for (int j = 0; j < m; j++) S[i * m + j] = (i == j) ? cmk(0.0, 0.0) : delta(ix[i], ix[j]);
            for (int e = 0; e < m * m; e++) X[e] = S[e];
            qh = cadd(qh, cscale(small_pf(X, m), v));
            const int mm = m - 2;
            for (int a = 0; a < m; a++)
                for (int b = a + 1; b < m; b++) {
                    int r = 0;
                    for (int i = 0; i < m; i++) {
                        if (i == a || i == b) continue;
                        int c = 0;
                        for (int j = 0; j < m; j++) {
                            if (j == a || j == b) continue;
                            X[r * mm + c++] = S[i * m + j];
                        }
                        r++;
                    }
                    const double sgn = ((a + b + 1) & 1) ? -1.0 : 1.0;
                    const cplx f = cscale(small_pf(X, mm), -0.5 * v * sgn);
                    const int s0 = d.slot[ix[a]], s1 = d.slot[ix[b]];
                    F[s0 * ni + s1] = cadd(F[s0 * ni + s1], f);
                    F[s1 * ni + s0] = cadd(F[s1 * ni + s0], cscale(f, -1.0));
                }
        }
        cplx dens = cmk(d.e_const + tr_r - 3.0 * q.x + qh.x, tr_i - 3.0 * q.y + qh.y);
        const int M = d.M;
        if (!(part & GH_GRAM)) {
            dens_buf[2 * blk] = dens.x;
            dens_buf[2 * blk + 1] = dens.y;
            if (diag) {
                for (int e = 0; e < ni * ni; e++) fimp_state[(size_t)a * ni * ni + e] = F[e].x;
            } else {
                double* fp = fimp + (size_t)p * ni * ni * 2;
                for (int e = 0; e < ni * ni; e++) { fp[2 * e] = F[e].x; fp[2 * e + 1] = F[e].y; }
            }
            return;
        }
        if (diag) {
            Gm[2 * (a * M + a)] = 1.0;
            Gm[2 * (a * M + a) + 1] = 0.0;
            hm[2 * (a * M + a)] = dens.x;
            hm[2 * (a * M + a) + 1] = 0.0;
            for (int e = 0; e < ni * ni; e++) fimp_state[(size_t)a * ni * ni + e] = F[e].x;
        } else {
            double ld = logdet[p];
            double mag = (ld == -INFINITY || ld != ld) ? 0.0 : exp(0.5 * (-d.N * 0.6931471805599453 + 0.5 * ld));
            cplx ph = cmk(1.0, 0.0);
            int q2 = d.pair_pf[p];
            if (q2 >= 0) {
                ph = cmk(d.parity * pfphase[2 * q2], d.parity * pfphase[2 * q2 + 1]);
                double m2 = sqrt(cabs2(ph));
                ph = m2 > 0.0 ? cscale(ph, 1.0 / m2) : cmk(0.0, 0.0);
            }
            cplx gab = cscale(ph, mag);
            cplx gba = cconj(gab);
            cplx hba = cmul(gba, dens);
            Gm[2 * (a * M + bq)] = gab.x;
            Gm[2 * (a * M + bq) + 1] = gab.y;
            Gm[2 * (bq * M + a)] = gba.x;
            Gm[2 * (bq * M + a) + 1] = gba.y;
            hm[2 * (bq * M + a)] = hba.x;
            hm[2 * (bq * M + a) + 1] = hba.y;
            hm[2 * (a * M + bq)] = hba.x;
            hm[2 * (a * M + bq) + 1] = -hba.y;
            double* fp = fimp + (size_t)p * ni * ni * 2;
            for (int e = 0; e < ni * ni; e++) { fp[2 * e] = F[e].x; fp[2 * e + 1] = F[e].y; }
        }
    }
}

// T1_p = Si (A + Re Fimp^{a,b}):  (Si A)[k][l] = -sum_{(m,v) in row l of A} Si[k][m] v
__global__ void pair_sparse_right_kernel(InstDev d, const double* si, const double* fimp, double* t1) {
    const int p = blockIdx.y;
    const int n = d.n, ni = d.nimp;
    const double* s = si + (size_t)p * nn(d);
    const double* fp = fimp + (size_t)p * ni * ni * 2;
    double* out = t1 + (size_t)p * nn(d);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn(d); e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        const double* srow = s + (size_t)k * n;
        double v = 0.0;
        for (int q = d.a_rowptr[l]; q < d.a_rowptr[l + 1]; q++) v -= srow[d.a_col[q]] * d.a_val[q];
        const int sl = d.slot[l];
        if (sl >= 0)
            for (int m = 0; m < ni; m++) v += srow[d.imp[m]] * fp[2 * (m * ni + sl)];
        out[e] = v;
    }
}

// T2_mu = F_mu Gamma_mu with F_mu = A + 6 U:Gamma_mu (real)
__global__ void state_sparse_left_kernel(InstDev d, const double* fimp_state, double* t2) {
    const int mu = blockIdx.y;
    const int n = d.n, ni = d.nimp;
    const double* g = d.gamma + (size_t)mu * nn(d);
    const double* fs = fimp_state + (size_t)mu * ni * ni;
    double* out = t2 + (size_t)mu * nn(d);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn(d); e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), l = (int)(e % n);
        double v = 0.0;
        for (int q = d.a_rowptr[k]; q < d.a_rowptr[k + 1]; q++) v += d.a_val[q] * g[(size_t)d.a_col[q] * n + l];
        const int sk = d.slot[k];
        if (sk >= 0)
            for (int m = 0; m < ni; m++) v += fs[sk * ni + m] * g[(size_t)d.imp[m] * n + l];
        out[e] = v;
    }
}

// L1 = Im[:, imp] Fi, L2 = 4 Si[:, imp] Fi  (n x nimp each), Fi = Im Fimp^{a,b}; the factor 4
// of L2's one use (Qi below) is applied here, exactly
__global__ void pair_lr_kernel(InstDev d, const double* si, const double* imd, const double* fimp, double* lr) {
    const int p = blockIdx.y;
    const int n = d.n, ni = d.nimp;
    const double* s = si + (size_t)p * nn(d);
    const double* im = imd + (size_t)p * nn(d);
    const double* fp = fimp + (size_t)p * ni * ni * 2;
    double* L1 = lr + (size_t)p * 2 * n * ni;
    double* L2 = L1 + (size_t)n * ni;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * ni; e += gridDim.x * blockDim.x) {
        const int k = e / ni, j = e % ni;
        double v1 = 0.0, v2 = 0.0;
        for (int m = 0; m < ni; m++) {
            double fi = fp[2 * (m * ni + j) + 1];
            v1 += im[(size_t)k * n + d.imp[m]] * fi;
            v2 += s[(size_t)k * n + d.imp[m]] * fi;
        }
        L1[e] = v1;
        L2[e] = 4.0 * v2;
    }
}

// Q = Delta F Delta (real and imaginary planes) from X = D Wr D, Wr and V = D Wr
// (T: double on the FP64 path, float on the tensor-core path):
//   Qr = X + 4 Wr + 2 (L1 Si[imp,:] + Si[:,imp] L1^T)
//   Qi = L2 Si[imp,:] - L1 Im[imp,:] - 2 (V - V^T)       (L2 carries its factor 4)
// as chains of FMAs (FP64 issues at a small fraction of the other pipes' rates on this
// part, so the count of FP64 instructions sets this kernel's time).  Both planes are
// antisymmetric (Delta and F are), so one CTA computes the strictly lower entries of a
// tile pair (K >= L) and stores them with their mirror: half the FP64 work of computing
// every entry.
// On the FP64 path the outputs alias the inputs (qr_out = xa_in, qi_out = wr_in): a CTA
// reads its tile (K, L) of X and Wr before it writes tiles (K, L) and (L, K), which no
// other CTA touches.
template <typename T>
__global__ void __launch_bounds__(256) pair_q_kernel(InstDev d, const double* si, const double* imd, const double* lr,
                                                     const T* va, const T* xa_in, const T* wr_in, double* qr_out,
                                                     double* qi_out) {
    // V^T is staged through shared memory so both reads of V coalesce
    __shared__ double vt[32][33];
    __shared__ double sq[2][32][33];
    const int p = blockIdx.y;
    const int n = d.n, ni = d.nimp;
    int K, L;
    lower_tile(blockIdx.x, K, L);
    const int k0 = K * 32, l0 = L * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const double* s = si + (size_t)p * nn(d);
    const double* im = imd + (size_t)p * nn(d);
    const double* L1 = lr + (size_t)p * 2 * n * ni;
    const double* L2 = L1 + (size_t)n * ni;
    const T* v = va + (size_t)p * nn(d);
    const T* X = xa_in + (size_t)p * nn(d);
    const T* W = wr_in + (size_t)p * nn(d);
    double* Qr = qr_out + (size_t)p * nn(d);
    double* Qi = qi_out + (size_t)p * nn(d);
    for (int j = ty; j < 32; j += 8) {            // vt[j][c] = V[l0 + j][k0 + c]
        const int r = l0 + j, c = k0 + tx;
        vt[j][tx] = (r < n && c < n) ? (double)v[(size_t)r * n + c] : 0.0;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int k = k0 + j, l = l0 + tx;
        if (k >= n || l >= n || k <= l) continue;
        const size_t e = (size_t)k * n + l;
        double a1 = 0.0, a2 = 0.0;
        for (int m = 0; m < ni; m++) {
            const int im_m = d.imp[m];
            const double s_ml = s[(size_t)im_m * n + l], l1 = L1[k * ni + m];
            a1 = fma(l1, s_ml, a1);
            a1 = fma(s[(size_t)k * n + im_m], L1[l * ni + m], a1);
            a2 = fma(L2[k * ni + m], s_ml, a2);
            a2 = fma(-l1, im[(size_t)im_m * n + l], a2);
        }
        sq[0][j][tx] = fma(2.0, a1, fma(4.0, (double)W[e], (double)X[e]));
        sq[1][j][tx] = fma(-2.0, (double)v[e] - vt[tx][j], a2);      // V[l][k] = vt[l - l0][k - k0]
    }
    __syncthreads();
    store_antisym_tile(Qr, n, k0, l0, sq[0]);
    store_antisym_tile(Qi, n, k0, l0, sq[1]);
}

// Tensor-core operands from FP64 (or fp32) data: x = src - src2 (src2 optional)
// to fp32 (TF32 kind), bf16, or an exact fp32 split hi + lo with hi on the
// tf32 grid (3xTF32).  Sources are n x n with leading dimension n; operands
// have leading dimension ldp >= n (a multiple of 8: a 16-byte chunk holds 8
// bf16 values), columns n..ldp-1 zero.
template <typename S>
__global__ void lp_convert_kernel(const S* const* src, const double* const* src2, void* const* hi, void* const* lo,
                                  int n, int ldp, int kind) {
    const int b = blockIdx.y;
    const S* x0 = src[b];
    const double* x1 = src2 ? src2[b] : nullptr;
    const size_t count = (size_t)n * ldp;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / ldp), q = (int)(e % ldp);
        double x = 0.0;
        if (q < n) {
            const size_t o = (size_t)r * n + q;
            x = (double)x0[o] - (x1 ? x1[o] : 0.0);
        }
        if (kind == 1) {
            static_cast<__nv_bfloat16*>(hi[b])[e] = __float2bfloat16_rn((float)x);
        } else if (kind == 2) {
            const float f = (float)x;
            const float h = __uint_as_float(__float_as_uint(f) & 0xffffe000u);
            static_cast<float*>(hi[b])[e] = h;
            static_cast<float*>(lo[b])[e] = (float)(x - (double)h);
        } else {
            static_cast<float*>(hi[b])[e] = round_tf32((float)x);
        }
    }
}

}  // namespace sgs
