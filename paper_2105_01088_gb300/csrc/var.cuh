// Hamiltonian variance delta_H^2 = <psi|H^2|psi> - <psi|H|psi>^2 (Eq. residual,
// Sec. IV A) of the SGS state, by Wick's theorem on each pair's transition matrix.
//
// H = e + H2 + H4 with H2 = i sum_kl A_kl c_k c_l and H4 = sum_m v_m c_m0 c_m1 c_m2 c_m3
// over monomials with increasing indices.  In the transition state of a pair
// (matrix Delta = Delta^{b,a}; Gamma_a for a state) the ordered contraction of c_x
// (left) with c_y (right) is g_xy = delta_xy + i Delta_xy, and a product of
// Majoranas, repeats allowed, is the Pfaffian of its ordered contractions.
// Summing the Wick terms over the quadratic indices in matrix form gives
//   <H2>         = T = Tr(A Delta)
//   <H2 H2>      = T^2 - 2 tr(A^2) - 2 tr(A Delta A Delta)
//   <H2 H4_m>    = T Pf4_m - i dPf4_m[C],   C  = B - B^T,   B  = g^T A g
//   <H4_m H2>    = T Pf4_m - i dPf4_m[C'],  C' = B' - B'^T, B' = g A g^T
//   <H4_m H4_m'> = Pf8 of the ordered contractions of (m, m'),
// where Pf4_m is the Pfaffian of g on the monomial's indices and dPf4_m[C] its
// derivative in the direction C.  With the sparse A (a few entries per row)
// everything is O(n^2) per pair: tr(A Delta A Delta) = sum_kl (A Delta)_kl
// (Delta A)_kl, and B, B' only on the Majoranas of the quartic terms.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace sgs {

#define VAR_MAX_MON 64           // canonical quartic monomials handled

// Pfaffian of a small complex antisymmetric matrix (m <= 8, row-major in X,
// destroyed) by Parlett-Reid elimination with pivoting.
__device__ cplx pf_small(cplx* X, int m) {
    cplx pf = cmk(1.0, 0.0);
    for (int k = 0; k + 1 < m; k += 2) {
        int piv = k + 1;
        double best = cabs2(X[k * m + k + 1]);
        for (int j = k + 2; j < m; j++) {
            const double v = cabs2(X[k * m + j]);
            if (v > best) { best = v; piv = j; }
        }
        if (piv != k + 1) {     // swap rows and columns k+1 <-> piv
            for (int j = 0; j < m; j++) { cplx t = X[(k + 1) * m + j]; X[(k + 1) * m + j] = X[piv * m + j]; X[piv * m + j] = t; }
            for (int j = 0; j < m; j++) { cplx t = X[j * m + k + 1]; X[j * m + k + 1] = X[j * m + piv]; X[j * m + piv] = t; }
            pf = cscale(pf, -1.0);
        }
        const cplx p = X[k * m + k + 1];
        pf = cmul(pf, p);
        if (best == 0.0) return cmk(0.0, 0.0);
        const cplx ip = cdiv(cmk(1.0, 0.0), p);
        // Schur complement of the 2x2 block [[0, p], [-p, 0]]:
        // X_ij += (X_ik X_{k+1,j} - X_{i,k+1} X_kj) / p for i, j > k+1
        for (int i = k + 2; i < m; i++)
            for (int j = k + 2; j < m; j++) {
                const cplx t = csub(cmul(X[i * m + k], X[(k + 1) * m + j]), cmul(X[i * m + k + 1], X[k * m + j]));
                X[i * m + j] = cadd(X[i * m + j], cmul(t, ip));
            }
    }
    return pf;
}

__device__ __forceinline__ cplx pf4v(const cplx x[4][4]) {
    return cadd(csub(cmul(x[0][1], x[2][3]), cmul(x[0][2], x[1][3])), cmul(x[0][3], x[1][2]));
}

__device__ __forceinline__ cplx dpf4v(const cplx x[4][4], const cplx c[4][4]) {
    cplx r = cadd(cmul(c[0][1], x[2][3]), cmul(x[0][1], c[2][3]));
    r = csub(r, cadd(cmul(c[0][2], x[1][3]), cmul(x[0][2], c[1][3])));
    return cadd(r, cadd(cmul(c[0][3], x[1][2]), cmul(x[0][3], c[1][2])));
}

__device__ __forceinline__ cplx block_csum(cplx v, double* red) {
    const double re = block_sum(v.x, red);
    __syncthreads();
    const double im = block_sum(v.y, red);
    __syncthreads();
    return cmk(re, im);
}

struct VarArgs {
    InstDev d;
    const double* si;        // per pair S^{-1}; Delta^{b,a} = -2 S^{-1} - i Im
    const double* imd;       // per pair Im Delta^{a,b}
    const double* Gm;        // [M][M] complex
    const double* lam;       // [M] complex
    const int* c_idx;        // [nc][4] canonical monomials (increasing indices)
    const double* c_val;
    int nc;
    double trA2;             // tr(A^2)
    double* partial;         // [P + M]: Re of the weighted <H^2> of each pair / state
};

// one CTA per unordered pair (blocks 0..P-1) and per state (P..P+M-1)
__global__ void __launch_bounds__(256) variance_kernel(VarArgs v) {
    __shared__ double red[32];
    __shared__ cplx Bs[2][SGS_MAX_IMP * SGS_MAX_IMP];
    const InstDev& d = v.d;
    const int blk = blockIdx.x;
    const bool diag = blk >= d.P;
    const int a = diag ? blk - d.P : d.pa[blk];
    const int b = diag ? a : d.pb[blk];
    const int n = d.n, M = d.M, ni = d.nimp;
    const double* gam = d.gamma + (size_t)a * nn(d);
    const double* s = diag ? nullptr : v.si + (size_t)blk * nn(d);
    const double* im = diag ? nullptr : v.imd + (size_t)blk * nn(d);
    auto D = [&](int r, int c) -> cplx {
        if (diag) return cmk(gam[(size_t)r * n + c], 0.0);
        return cmk(-2.0 * s[(size_t)r * n + c], -im[(size_t)r * n + c]);
    };
    // g = 1 + i Delta
    auto g = [&](int r, int c) -> cplx {
        const cplx x = D(r, c);
        return cmk((r == c ? 1.0 : 0.0) - x.y, x.x);
    };
    const int tid = threadIdx.x, nt = blockDim.x;

    // T = Tr(A Delta) = sum_kl A_kl Delta_lk
    cplx T = cmk(0.0, 0.0);
    for (int j = tid; j < d.a_nnz; j += nt) T = cadd(T, cscale(D(d.a_col[j], d.a_row[j]), d.a_val[j]));
    T = block_csum(T, red);

    // t2 = tr(A Delta A Delta) = sum_kl (A Delta)_kl (Delta A)_kl,
    // (Delta A)_kl = -sum_{j in row l} Delta_kj A_lj  (A antisymmetric)
    cplx t2 = cmk(0.0, 0.0);
    for (size_t e = tid; e < (size_t)n * n; e += nt) {
        const int k = (int)(e / n), l = (int)(e % n);
        cplx x = cmk(0.0, 0.0), y = cmk(0.0, 0.0);
        for (int p = d.a_rowptr[k]; p < d.a_rowptr[k + 1]; p++) x = cadd(x, cscale(D(d.a_col[p], l), d.a_val[p]));
        if (x.x == 0.0 && x.y == 0.0) continue;
        for (int p = d.a_rowptr[l]; p < d.a_rowptr[l + 1]; p++) y = csub(y, cscale(D(k, d.a_col[p]), d.a_val[p]));
        t2 = cadd(t2, cmul(x, y));
    }
    t2 = block_csum(t2, red);

    // B = g^T A g and B' = g A g^T on the Majoranas of the quartic terms
    const int tasks = 2 * ni * ni;
    for (int t = tid; t < tasks; t += nt) Bs[t / (ni * ni)][t % (ni * ni)] = cmk(0.0, 0.0);
    __syncthreads();
    if (tasks > 0) {
        const int chunks = max(1, nt / tasks);
        for (int t = tid; t < tasks * chunks; t += nt) {
            const int task = t % tasks, ch = t / tasks;
            const int mat = task / (ni * ni), x = d.imp[(task % (ni * ni)) / ni], y = d.imp[task % ni];
            cplx acc = cmk(0.0, 0.0);
            for (int j = ch; j < d.a_nnz; j += chunks) {
                const int k = d.a_row[j], l = d.a_col[j];
                const cplx u = mat == 0 ? cmul(g(k, x), g(l, y)) : cmul(g(x, k), g(y, l));
                acc = cadd(acc, cscale(u, d.a_val[j]));
            }
            atomicAdd(&Bs[mat][task % (ni * ni)].x, acc.x);
            atomicAdd(&Bs[mat][task % (ni * ni)].y, acc.y);
        }
    }
    __syncthreads();

    // quartic terms: <H4>, the cross terms, and <H4 H4>
    cplx Q = cmk(0.0, 0.0), h24 = cmk(0.0, 0.0), h42 = cmk(0.0, 0.0), h44 = cmk(0.0, 0.0);
    for (int m = tid; m < v.nc; m += nt) {
        const int* ix = v.c_idx + 4 * m;
        cplx X[4][4], C[4][4], Cp[4][4];
        for (int p = 0; p < 4; p++)
            for (int q = 0; q < 4; q++) {
                X[p][q] = p < q ? g(ix[p], ix[q]) : (p > q ? cscale(g(ix[q], ix[p]), -1.0) : cmk(0.0, 0.0));
                const int sp = d.slot[ix[p]], sq = d.slot[ix[q]];
                C[p][q] = csub(Bs[0][sp * ni + sq], Bs[0][sq * ni + sp]);
                Cp[p][q] = csub(Bs[1][sp * ni + sq], Bs[1][sq * ni + sp]);
            }
        const double vm = v.c_val[m];
        const cplx p4 = pf4v(X);
        const cplx mi = cmk(0.0, -1.0);
        Q = cadd(Q, cscale(p4, vm));
        h24 = cadd(h24, cscale(cadd(cmul(T, p4), cmul(mi, dpf4v(X, C))), vm));
        h42 = cadd(h42, cscale(cadd(cmul(T, p4), cmul(mi, dpf4v(X, Cp))), vm));
    }
    for (int t = tid; t < v.nc * v.nc; t += nt) {
        const int m1 = t / v.nc, m2 = t % v.nc;
        int ix[8];
        for (int p = 0; p < 4; p++) { ix[p] = v.c_idx[4 * m1 + p]; ix[4 + p] = v.c_idx[4 * m2 + p]; }
        cplx X[64];
        for (int p = 0; p < 8; p++)
            for (int q = 0; q < 8; q++)
                X[p * 8 + q] = p < q ? g(ix[p], ix[q]) : (p > q ? cscale(g(ix[q], ix[p]), -1.0) : cmk(0.0, 0.0));
        h44 = cadd(h44, cscale(pf_small(X, 8), v.c_val[m1] * v.c_val[m2]));
    }
    Q = block_csum(Q, red);
    h24 = block_csum(h24, red);
    h42 = block_csum(h42, red);
    h44 = block_csum(h44, red);

    if (tid == 0) {
        const double e = d.e_const;
        cplx h2 = cmk(e * e, 0.0);
        h2 = cadd(h2, cscale(cadd(T, Q), 2.0 * e));
        h2 = cadd(h2, csub(cmul(T, T), cadd(cmk(2.0 * v.trA2, 0.0), cscale(t2, 2.0))));
        h2 = cadd(h2, cadd(h24, cadd(h42, h44)));
        const cplx la = cmk(v.lam[2 * a], v.lam[2 * a + 1]), lb = cmk(v.lam[2 * b], v.lam[2 * b + 1]);
        cplx w;
        if (diag) w = cmk(cabs2(la), 0.0);
        else w = cscale(cmul(cmul(cconj(la), lb), cmk(v.Gm[2 * (a * M + b)], v.Gm[2 * (a * M + b) + 1])), 2.0);
        v.partial[blk] = cmul(w, h2).x;
    }
}

}  // namespace sgs
