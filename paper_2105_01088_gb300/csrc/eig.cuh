// Optimal amplitudes: lowest solution of h lambda = E G lambda (Eq. eigLambda)
// by canonical orthogonalisation, in FP64, one CTA per instance.
//
// The M x M Hermitian pair (G, h) is embedded as the real symmetric 2M x 2M
// pair [[Re, -Im], [Im, Re]] (every eigenvalue doubled; the eigenvector
// [x; y] maps to x + i y).  Both symmetric eigenproblems are solved with
// parallel cyclic Jacobi (round-robin pairing, disjoint rotations applied to
// all rows and then all columns).  Eigenvalues of G below cut * max are
// dropped (the paper assumes linearly independent states).
//
// The same kernel then forms lambda-tilde = G lambda, the decoupling
// constants c_mu (Sec. III A) and the per-(mu, beta) coefficients of
// Eq. (EOM-Gamma3): with z = conj(lt_mu) c_mu lambda_beta,
//   a1 = 2i z G_mu,beta,  a2 = 2 z G_mu,beta,  a3 = -z (h_mu,beta - E G_mu,beta).
#pragma once
#include "common.cuh"

namespace sgs {

struct AmpArgs {
    int M;
    const double* Gm;     // [M][M] complex
    const double* hm;     // [M][M] complex
    double* scratch;      // >= 6 (2M)^2 + 8 (2M) doubles
    double* E;            // [1] energy of this step
    double* lam;          // [M] complex
    double* lt;           // [M] complex
    double* coef;         // [M][M][6]
    int cmode;            // 0: c = 1/(lambda conj(lt)); 1: c = lt conj(lambda)/|lambda lt|
    double cut;
    int* err;
};

// Jacobi on the m x m symmetric A (row stride ld), accumulating V (= I on
// entry).  Returns the number of sweeps used (or -1 if not converged).
__device__ int jacobi_sym(double* A, double* V, int m, int ld, double* rc, double* rs, int* rp, int* rq,
                          double* red) {
    const int mm = (m + 1) & ~1;            // pad to even with one idle index
    const int npair = mm / 2;
    int sweeps = 0;
    for (; sweeps < 60; sweeps++) {
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = e / m, j = e % m;
            double v = A[i * ld + j];
            if (i == j) dg += v * v; else off += v * v;
        }
        off = block_sum(off, red);
        dg = block_sum(dg, red);
        if (off <= 1e-30 * dg || off < 1e-280) return sweeps;
        for (int r = 0; r < mm - 1; r++) {
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                auto pos = [&](int j) { return j == 0 ? 0 : ((j - 1 + r) % (mm - 1)) + 1; };
                int p = pos(i), q = pos(mm - 1 - i);
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < m) {
                    double apq = A[p * ld + q];
                    if (fabs(apq) > 1e-300) {
                        double th = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
                        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                } else {
                    q = -1;
                }
                rc[i] = c; rs[i] = s; rp[i] = p; rq[i] = q;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < npair * m; e += blockDim.x) {
                int i = e / m, j = e % m;
                int p = rp[i], q = rq[i];
                if (q < 0 || rs[i] == 0.0) continue;
                double c = rc[i], s = rs[i];
                double ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < npair * m; e += blockDim.x) {
                int i = e / m, j = e % m;
                int p = rp[i], q = rq[i];
                if (q < 0 || rs[i] == 0.0) continue;
                double c = rc[i], s = rs[i];
                double ap = A[j * ld + p], aq = A[j * ld + q];
                A[j * ld + p] = c * ap - s * aq;
                A[j * ld + q] = s * ap + c * aq;
                double vp = V[j * ld + p], vq = V[j * ld + q];
                V[j * ld + p] = c * vp - s * vq;
                V[j * ld + q] = s * vp + c * vq;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                int p = rp[i], q = rq[i];
                if (q >= 0 && rs[i] != 0.0) { A[p * ld + q] = 0.0; A[q * ld + p] = 0.0; }
            }
            __syncthreads();
        }
    }
    return -1;
}

__global__ void __launch_bounds__(256) amp_solve_kernel(AmpArgs a) {
    __shared__ double rc[SGS_MAX_RANK + 1], rs[SGS_MAX_RANK + 1];
    __shared__ int rp[SGS_MAX_RANK + 1], rq[SGS_MAX_RANK + 1];
    __shared__ double red[32];
    __shared__ int s_keep[2 * SGS_MAX_RANK];
    __shared__ int s_nkeep, s_jmin;
    __shared__ double s_E, s_nrm;

    const int M = a.M, m = 2 * M, ld = m;
    double* GR = a.scratch;
    double* V1 = GR + m * m;
    double* HR = V1 + m * m;
    double* XR = HR + m * m;
    double* TM = XR + m * m;
    double* V2 = TM + m * m;
    double* lr = V2 + m * m;    // 2M
    const double* G = a.Gm;
    const double* h = a.hm;

    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        int ib = i / M, jb = j / M, ii = i % M, jj = j % M;
        double gr = G[2 * (ii * M + jj)], gi = G[2 * (ii * M + jj) + 1];
        double hr = h[2 * (ii * M + jj)], hi = h[2 * (ii * M + jj) + 1];
        double gv, hv;
        if (ib == jb) { gv = gr; hv = hr; }
        else if (ib == 0) { gv = -gi; hv = -hi; }   // upper-right block: -Im
        else { gv = gi; hv = hi; }                  // lower-left block: +Im
        GR[e] = gv;
        HR[e] = hv;
        V1[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    int sw = jacobi_sym(GR, V1, m, ld, rc, rs, rp, rq, red);
    if (threadIdx.x == 0) {
        if (sw < 0) atomicOr(a.err, SGS_DEV_EIG);
        double wmax = 0.0;
        for (int j = 0; j < m; j++) wmax = fmax(wmax, GR[j * ld + j]);
        int nk = 0;
        for (int j = 0; j < m; j++)
            if (GR[j * ld + j] > a.cut * wmax) s_keep[nk++] = j;
        s_nkeep = nk;
        if (nk == 0) atomicOr(a.err, SGS_DEV_EIG);
    }
    __syncthreads();
    const int K = s_nkeep;
    if (K == 0) return;
    // XR = V1[:, keep] / sqrt(w)
    for (int e = threadIdx.x; e < m * K; e += blockDim.x) {
        int i = e / K, t = e % K;
        int j = s_keep[t];
        XR[i * ld + t] = V1[i * ld + j] / sqrt(GR[j * ld + j]);
    }
    __syncthreads();
    // TM = HR XR (m x K), then H' = XR^T TM (K x K) into V1's storage
    for (int e = threadIdx.x; e < m * K; e += blockDim.x) {
        int i = e / K, t = e % K;
        double v = 0.0;
        for (int j = 0; j < m; j++) v += HR[i * ld + j] * XR[j * ld + t];
        TM[i * ld + t] = v;
    }
    __syncthreads();
    double* Hp = V1;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        int s = e / K, t = e % K;
        double v = 0.0;
        for (int i = 0; i < m; i++) v += XR[i * ld + s] * TM[i * ld + t];
        Hp[s * ld + t] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        int s = e / K, t = e % K;
        if (s < t) {
            double v = 0.5 * (Hp[s * ld + t] + Hp[t * ld + s]);
            Hp[s * ld + t] = v;
            Hp[t * ld + s] = v;
        }
        V2[s * ld + t] = (s == t) ? 1.0 : 0.0;
    }
    __syncthreads();
    sw = jacobi_sym(Hp, V2, K, ld, rc, rs, rp, rq, red);
    if (threadIdx.x == 0) {
        if (sw < 0) atomicOr(a.err, SGS_DEV_EIG);
        int jm = 0;
        for (int j = 1; j < K; j++)
            if (Hp[j * ld + j] < Hp[jm * ld + jm]) jm = j;
        s_jmin = jm;
        s_E = Hp[jm * ld + jm];
    }
    __syncthreads();
    // lambda_R = XR u
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double v = 0.0;
        for (int t = 0; t < K; t++) v += XR[i * ld + t] * V2[t * ld + s_jmin];
        lr[i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // complex lambda, normalisation lambda^dag G lambda = 1, phase convention
        double nrm = 0.0;
        for (int i = 0; i < M; i++) {
            double xr = 0.0, xi = 0.0;
            for (int j = 0; j < M; j++) {
                double gr = G[2 * (i * M + j)], gi = G[2 * (i * M + j) + 1];
                xr += gr * lr[j] - gi * lr[M + j];
                xi += gr * lr[M + j] + gi * lr[j];
            }
            nrm += lr[i] * xr + lr[M + i] * xi;
        }
        s_nrm = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sc = 1.0 / sqrt(s_nrm);
        int jb = 0;
        double best = -1.0;
        for (int i = 0; i < M; i++) {
            double m2 = lr[i] * lr[i] + lr[M + i] * lr[M + i];
            if (m2 > best * (1.0 + 1e-12)) { best = m2; jb = i; }
        }
        double pr = lr[jb], pi = lr[M + jb];
        double pm = sqrt(pr * pr + pi * pi);
        cplx ph = cmk(pr / pm, -pi / pm);   // multiply by conj(lambda_j)/|lambda_j|
        for (int i = 0; i < M; i++) {
            cplx l = cmul(cmk(lr[i] * sc, lr[M + i] * sc), ph);
            a.lam[2 * i] = l.x;
            a.lam[2 * i + 1] = l.y;
        }
        a.E[0] = s_E;
    }
    __syncthreads();
    // lambda-tilde = G lambda
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        cplx v = cmk(0.0, 0.0);
        for (int j = 0; j < M; j++)
            v = cadd(v, cmul(cmk(G[2 * (i * M + j)], G[2 * (i * M + j) + 1]), cmk(a.lam[2 * j], a.lam[2 * j + 1])));
        a.lt[2 * i] = v.x;
        a.lt[2 * i + 1] = v.y;
    }
    __syncthreads();
    const double E = s_E;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int mu = e / M, be = e % M;
        cplx l = cmk(a.lam[2 * mu], a.lam[2 * mu + 1]);
        cplx t = cmk(a.lt[2 * mu], a.lt[2 * mu + 1]);
        cplx zz = cmul(l, cconj(t));                // lambda_mu conj(lt_mu)
        double az = sqrt(cabs2(zz));
        cplx c = cmk(0.0, 0.0);
        if (az >= 1e-300) c = (a.cmode == 0) ? cdiv(cmk(1.0, 0.0), zz) : cscale(cconj(zz), 1.0 / az);
        cplx w = cmul(cconj(t), c);
        cplx z = cmul(w, cmk(a.lam[2 * be], a.lam[2 * be + 1]));
        cplx g = cmk(G[2 * (mu * M + be)], G[2 * (mu * M + be) + 1]);
        cplx hh = cmk(h[2 * (mu * M + be)], h[2 * (mu * M + be) + 1]);
        cplx zg = cmul(z, g);
        cplx a1 = cmul(cmk(0.0, 2.0), zg);
        cplx a2 = cscale(zg, 2.0);
        cplx a3 = cscale(cmul(z, csub(hh, cscale(g, E))), -1.0);
        double* co = a.coef + (size_t)e * 6;
        co[0] = a1.x; co[1] = a1.y; co[2] = a2.x; co[3] = a2.y; co[4] = a3.x; co[5] = a3.y;
    }
}

}  // namespace sgs
