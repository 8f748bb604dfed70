// Renyi-2 entropy of the leading 2 N_A Majoranas (impurity + first l sites)
// of the SGS state (App. B).
//
// With the transition operator X_ab = |a><b| / <b|a>, whose two-point matrix is
// Delta^{a,b} (Sec. III B), rho_a rho_b = |G_ab|^2 X_ab, and the partial trace
// over B of an even Gaussian operator keeps the A block of its matrix.  The
// trace of two unit-trace Gaussian operators on A with matrices D1, D2 is
// 2^-N_A Pf([[D1, i 1], [-i 1, D2]]), so
//   T^{ab}_{cd} = lambda_a conj(lambda_b) lambda_c conj(lambda_d) G_ba G_dc 2^-N_A
//                 Pf([[Delta^{ab}_A, i 1], [-i 1, Delta^{cd}_A]]),
// which equals the paper's Eq. TrArho2_final term by term (checked against
// it and against Fock-space reduced density matrices) but needs no Pfaffian
// of the 4 N_B x 4 N_B matrix M_B: the pair pass already holds Delta.
// S_2 = -ln sum T (Eq. S2_SGS); T^{ab}_{cd} = T^{cd}_{ab}, so unordered pairs
// of ordered pairs (u <= v) are evaluated once.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace sgs {

#define RENYI_MAX_DIM 104     // 2 * 2 N_A <= 104 (impurity + up to 12 sites) in one CTA's shared memory

// blocks[u] = Delta^{ab}_A (complex, na2 x na2), w[u] = lambda_a conj(lambda_b) G_ba, u = a M + b
__global__ void renyi_blocks_kernel(InstDev d, const double* si, const double* imd, const double* Gm,
                                    const double* lam, const int* pair_index, int na2, double* blocks, double* w) {
    const int u = blockIdx.x;
    const int M = d.M, n = d.n;
    const int a = u / M, b = u % M;
    double* B = blocks + (size_t)u * na2 * na2 * 2;
    const double* g = d.gamma + (size_t)a * nn(d);
    int p = (a == b) ? -1 : pair_index[a * M + b];
    const double sgn = (a < b) ? 1.0 : -1.0;      // Delta^{ab} for a > b is conj(Delta^{ba})
    for (int e = threadIdx.x; e < na2 * na2; e += blockDim.x) {
        const int r = e / na2, c = e % na2;
        double re, im;
        if (p < 0) { re = g[(size_t)r * n + c]; im = 0.0; }
        else {
            re = -2.0 * si[(size_t)p * nn(d) + (size_t)r * n + c];
            im = sgn * imd[(size_t)p * nn(d) + (size_t)r * n + c];
        }
        B[2 * e] = re;
        B[2 * e + 1] = im;
    }
    if (threadIdx.x == 0) {
        cplx la = cmk(lam[2 * a], lam[2 * a + 1]), lb = cmk(lam[2 * b], lam[2 * b + 1]);
        cplx gba = cmk(Gm[2 * (b * M + a)], Gm[2 * (b * M + a) + 1]);
        cplx x = cmul(cmul(la, cconj(lb)), gba);
        w[2 * u] = x.x;
        w[2 * u + 1] = x.y;
    }
}

// one CTA per unordered pair (u <= v) of ordered pairs: complex Parlett-Reid in shared memory
__global__ void __launch_bounds__(256) renyi_pf_kernel(const double* blocks, const double* w, long long npairs,
                                                       int na2, double log_norm, double* partial) {
    extern __shared__ double sm[];
    const int m = 2 * na2;
    const int ld = m + 1;
    double* Zr = sm;
    double* Zi = sm + (size_t)m * ld;
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ double s_log, s_pr, s_pi;
    const long long q = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    if (q >= npairs) return;
    // decode q = v (v + 1) / 2 + u, u <= v
    long long v = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((v + 1) * (v + 2) / 2 <= q) ++v;
    while (v * (v + 1) / 2 > q) --v;
    const long long u = q - v * (v + 1) / 2;
    const double* Bu = blocks + (size_t)u * na2 * na2 * 2;
    const double* Bv = blocks + (size_t)v * na2 * na2 * 2;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        double zr = 0.0, zi = 0.0;
        if (r < na2 && c < na2) { zr = Bu[2 * (r * na2 + c)]; zi = Bu[2 * (r * na2 + c) + 1]; }
        else if (r >= na2 && c >= na2) { zr = Bv[2 * ((r - na2) * na2 + c - na2)]; zi = Bv[2 * ((r - na2) * na2 + c - na2) + 1]; }
        else if (c == r + na2) zi = 1.0;          // i 1
        else if (r == c + na2) zi = -1.0;         // -i 1
        Zr[r * ld + c] = zr;
        Zi[r * ld + c] = zi;
    }
    if (threadIdx.x == 0) { s_log = 0.0; s_pr = 1.0; s_pi = 0.0; }
    __syncthreads();
    bool zero = false;
    for (int k = 0; k < m - 1; k += 2) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) {
            const double x = Zr[i * ld + k] * Zr[i * ld + k] + Zi[i * ld + k] * Zi[i * ld + k];
            if (x > best) { best = x; bi = i; }
        }
        double mv;
        int p;
        block_argmax(best, bi, red_v, red_i, mv, p);
        if (!(mv > 0.0)) { zero = true; break; }
        if (p != k + 1) {
            const int a = k + 1;
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                double t = Zr[a * ld + j]; Zr[a * ld + j] = Zr[p * ld + j]; Zr[p * ld + j] = t;
                t = Zi[a * ld + j]; Zi[a * ld + j] = Zi[p * ld + j]; Zi[p * ld + j] = t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                double t = Zr[i * ld + a]; Zr[i * ld + a] = Zr[i * ld + p]; Zr[i * ld + p] = t;
                t = Zi[i * ld + a]; Zi[i * ld + a] = Zi[i * ld + p]; Zi[i * ld + p] = t;
            }
            if (threadIdx.x == 0) { s_pr = -s_pr; s_pi = -s_pi; }
            __syncthreads();
        }
        const double pr = Zr[k * ld + k + 1], pi = Zi[k * ld + k + 1];
        const double pm2 = pr * pr + pi * pi;
        if (threadIdx.x == 0) {
            const double am = sqrt(pm2);
            s_log += log(am);
            const double ur = pr / am, ui = pi / am;
            const double nr = s_pr * ur - s_pi * ui, ni = s_pr * ui + s_pi * ur;
            s_pr = nr; s_pi = ni;
        }
        // A[k+2:, k+2:] += tau u^T - u tau^T with tau = A[k, k+2:] / pivot, u = A[k+2:, k+1]
        const double ir = pr / pm2, ii = -pi / pm2;
        const int t0 = k + 2, mt = m - t0;
        for (int e = threadIdx.x; e < mt * mt; e += blockDim.x) {
            const int i = t0 + e / mt, j = t0 + e % mt;
            const double ti_r = Zr[k * ld + i] * ir - Zi[k * ld + i] * ii, ti_i = Zr[k * ld + i] * ii + Zi[k * ld + i] * ir;
            const double tj_r = Zr[k * ld + j] * ir - Zi[k * ld + j] * ii, tj_i = Zr[k * ld + j] * ii + Zi[k * ld + j] * ir;
            const double uj_r = Zr[j * ld + k + 1], uj_i = Zi[j * ld + k + 1];
            const double ui_r = Zr[i * ld + k + 1], ui_i = Zi[i * ld + k + 1];
            Zr[i * ld + j] += (ti_r * uj_r - ti_i * uj_i) - (ui_r * tj_r - ui_i * tj_i);
            Zi[i * ld + j] += (ti_r * uj_i + ti_i * uj_r) - (ui_r * tj_i + ui_i * tj_r);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        if (!zero) {
            const cplx wu = cmk(w[2 * u], w[2 * u + 1]), wv = cmk(w[2 * v], w[2 * v + 1]);
            cplx x = cmul(cmul(wu, wv), cmk(s_pr, s_pi));
            const double mag = exp(s_log + log_norm) * (u < v ? 2.0 : 1.0);
            tr = x.x * mag;
            ti = x.y * mag;
        }
        partial[2 * q] = tr;
        partial[2 * q + 1] = ti;
    }
}

// Subsystems too large for one CTA's shared memory: the Pfaffians of a chunk of
// pairs go through the batched blocked Pfaffian of the pair pass.  Z_q =
// [[Delta_u, i 1], [-i 1, Delta_v]] in planes (re, im) of m x m, m = 2 na2; entries past
// the last pair get the pairing matrix J (Pf = 1) and are ignored.
__global__ void renyi_build_kernel(const double* blocks, long long q0, long long npairs, int na2, double* Y) {
    const long long q = q0 + blockIdx.x;
    const int m = 2 * na2;
    const size_t mm = (size_t)m * m;
    double* zr = Y + (size_t)blockIdx.x * 2 * mm;
    double* zi = zr + mm;
    if (q >= npairs) {
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            const int r = (int)(e / m), c = (int)(e % m);
            zr[e] = (c == r + 1 && (r & 1) == 0) ? 1.0 : ((r == c + 1 && (c & 1) == 0) ? -1.0 : 0.0);
            zi[e] = 0.0;
        }
        return;
    }
    long long v = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((v + 1) * (v + 2) / 2 <= q) ++v;
    while (v * (v + 1) / 2 > q) --v;
    const long long u = q - v * (v + 1) / 2;
    const double* Bu = blocks + (size_t)u * na2 * na2 * 2;
    const double* Bv = blocks + (size_t)v * na2 * na2 * 2;
    for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
        const int r = (int)(e / m), c = (int)(e % m);
        double xr = 0.0, xi = 0.0;
        if (r < na2 && c < na2) { xr = Bu[2 * (r * na2 + c)]; xi = Bu[2 * (r * na2 + c) + 1]; }
        else if (r >= na2 && c >= na2) { xr = Bv[2 * ((r - na2) * na2 + c - na2)]; xi = Bv[2 * ((r - na2) * na2 + c - na2) + 1]; }
        else if (c == r + na2) xi = 1.0;
        else if (r == c + na2) xi = -1.0;
        zr[e] = xr;
        zi[e] = xi;
    }
}

// T of each pair of the chunk from the Pfaffian (phase, log|Pf|)
__global__ void renyi_combine_kernel(const double* logabs, const double* phase, const double* w, long long q0,
                                     long long cnt, long long npairs, double log_norm, double* partial) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (long long)gridDim.x * blockDim.x) {
        const long long q = q0 + j;
        if (q >= npairs) continue;
        long long v = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
        while ((v + 1) * (v + 2) / 2 <= q) ++v;
        while (v * (v + 1) / 2 > q) --v;
        const long long u = q - v * (v + 1) / 2;
        double tr = 0.0, ti = 0.0;
        const double la = logabs[j];
        if (la > -1e300) {
            const cplx x = cmul(cmul(cmk(w[2 * u], w[2 * u + 1]), cmk(w[2 * v], w[2 * v + 1])),
                                cmk(phase[2 * j], phase[2 * j + 1]));
            const double mag = exp(la + log_norm) * (u < v ? 2.0 : 1.0);
            tr = x.x * mag;
            ti = x.y * mag;
        }
        partial[2 * q] = tr;
        partial[2 * q + 1] = ti;
    }
}

// deterministic sum of count complex values: block partial sums, then one block
__global__ void complex_sum_kernel(const double* in, long long count, double* out) {
    __shared__ double red[32];
    double sr = 0.0, si = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
        sr += in[2 * e];
        si += in[2 * e + 1];
    }
    sr = block_sum(sr, red);
    si = block_sum(si, red);
    if (threadIdx.x == 0) { out[2 * blockIdx.x] = sr; out[2 * blockIdx.x + 1] = si; }
}

}  // namespace sgs
