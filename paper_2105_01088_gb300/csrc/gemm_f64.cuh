// Batched FP64 GEMM on the FP64 FMA pipe of the CUDA cores (the native FP64
// product path, SGS_FP64_FMA).  tcgen05 has no f64 kind.  On GB300 the FP64 FMA
// of the CUDA cores and the m8n8k4 FP64 MMA (mma.sync .f64) share one FP64 pipe,
// measured at 1.25 and 1.09 TFLOP/s, so the products issue FMAs.  Every FP64
// product of the step (pair products, the delayed updates of the blocked
// factorisations, the per-state exponential and purification) goes through it
// on that path; the emulated path (gemm_oz.cuh) shares its batch descriptor.
//
// C_b = alpha * alpha_b[b] * op(A_b) op(B_b) + beta * Cin_b + beta2 * Cin2_b + diag * I
// with A_b = A1_b + sA2 * A2_b (the pair difference Gamma_a - Gamma_b is
// fused into the operand load), likewise for B.
//
// Output modes: FULL; SKEW (only lower tiles computed, each written to
// C[r][c] and -C[c][r], zero diagonal: used where the product is skew by
// construction); GJ (Gauss-Jordan delayed update: rows inside the panel
// start from 0, and unless gj_cols = 0 columns inside the panel are not
// written).
#pragma once
#include "common.cuh"

namespace sgs {

enum GemmMode { GEMM_FULL = 0, GEMM_SKEW = 1, GEMM_GJ = 2 };

struct GemmBatch {
    int m, n, k;                         // op(A): m x k, op(B): k x n, C: m x n
    const double* const* A; long long offA; int lda; int transA;
    const double* const* A2; double sA2;  // optional (nullptr)
    const double* const* B; long long offB; int ldb; int transB;
    const double* const* B2; double sB2;  // optional (nullptr)
    const double* const* Cin; long long offCin; int ldcin; double beta;  // optional
    const double* const* Cin2; double beta2;   // optional second addend (same offset and stride as Cin)
    double* const* C; long long offC; int ldc;
    double alpha; double diag;
    const double* alpha_b;               // optional per-batch multiplier of alpha
    const int* active_flag;              // optional: batch b computes only if active_flag[b] > active_cmp
    int active_cmp;                      //   otherwise C = Cin (pass-through)
    int mode; int gj_k0; int gj_b;
    int gj_cols;                         // GJ: 1 = output columns gj_k0 .. gj_k0 + gj_b - 1 not written
    int gj_acc;                          // GJ: 1 = rows gj_k0 .. gj_k0 + gj_b - 1 add Cin like the others
                                         // (a later K chunk of a Gauss-Jordan update)
    int cin_trans;                       // 1: Cin element (r, c) is read at Cin[b][offCin + c ldcin + r]
                                         // (every batch entry active; the Pfaffian's updates read the
                                         // upper triangle, with beta = -1)
                                         //     (the panel's own), 0 = every output column written
    int batch;
    int b_antisym;                       // hint: B (and B2) antisymmetric, op(B)'s columns = -B's rows
    long long offBr;                     // (emulated products) offset of op(B)'s K range in B's rows
};

#define GBM 64
#define GBN 64
#define GBK 16
#define GAS 20   // padded row stride of the A tile
#define GBS 68   // padded row stride of the B tile

// Each thread accumulates a 4 x 8 register tile (rows 4*(t/8).., columns 8*(t%8)..).
template <int TA, int TB>
__global__ void __launch_bounds__(128) gemm_f64_kernel(GemmBatch g) {
    __shared__ __align__(16) double As[2][GBM * GAS];
    __shared__ __align__(16) double Bs[2][GBK * GBS];

    const int b = blockIdx.y;
    int tm, tn;
    const int ntn = (g.n + GBN - 1) / GBN;
    if (g.mode == GEMM_SKEW) {
        // linear index over lower-triangular tile pairs (tm >= tn)
        int t = blockIdx.x;
        tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
        while (tm * (tm + 1) / 2 > t) --tm;
        tn = t - tm * (tm + 1) / 2;
    } else {
        tm = blockIdx.x / ntn;
        tn = blockIdx.x % ntn;
    }
    const int m0 = tm * GBM, n0 = tn * GBN;
    const int tid = threadIdx.x;

    const bool active = (g.active_flag == nullptr) || (g.active_flag[b] > g.active_cmp);
    double alpha = g.alpha * (g.alpha_b ? g.alpha_b[b] : 1.0);

    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j][0] = acc[i][j][1] = 0.0;

    if (active && g.k > 0) {
        const double* Ab = g.A[b] + g.offA;
        const double* A2b = g.A2 ? g.A2[b] + g.offA : nullptr;
        const double* Bb = g.B[b] + g.offB;
        const double* B2b = g.B2 ? g.B2[b] + g.offB : nullptr;
        double ra[8], rb[8];

        auto load_tiles = [&](int k0) {
            // A tile: GBM x GBK of op(A)
#pragma unroll
            for (int e = 0; e < 8; e++) {
                int r, kk;
                if (!TA) { r = tid >> 1; kk = (tid & 1) * 8 + e; }
                else     { kk = tid >> 3; r = (tid & 7) * 8 + e; }
                int gr = m0 + r, gk = k0 + kk;
                double v = 0.0;
                if (gr < g.m && gk < g.k) {
                    long long off = TA ? (long long)gk * g.lda + gr : (long long)gr * g.lda + gk;
                    v = __ldg(Ab + off);
                    if (A2b) v += g.sA2 * __ldg(A2b + off);
                }
                ra[e] = v;
            }
            // B tile: GBK x GBN of op(B)
#pragma unroll
            for (int e = 0; e < 8; e++) {
                int kk, c;
                if (!TB) { kk = tid >> 3; c = (tid & 7) * 8 + e; }
                else     { c = tid >> 1; kk = (tid & 1) * 8 + e; }
                int gk = k0 + kk, gc = n0 + c;
                double v = 0.0;
                if (gk < g.k && gc < g.n) {
                    long long off = TB ? (long long)gc * g.ldb + gk : (long long)gk * g.ldb + gc;
                    v = __ldg(Bb + off);
                    if (B2b) v += g.sB2 * __ldg(B2b + off);
                }
                rb[e] = v;
            }
        };
        auto store_tiles = [&](int s) {
#pragma unroll
            for (int e = 0; e < 8; e++) {
                int r, kk;
                if (!TA) { r = tid >> 1; kk = (tid & 1) * 8 + e; }
                else     { kk = tid >> 3; r = (tid & 7) * 8 + e; }
                As[s][r * GAS + kk] = ra[e];
            }
#pragma unroll
            for (int e = 0; e < 8; e++) {
                int kk, c;
                if (!TB) { kk = tid >> 3; c = (tid & 7) * 8 + e; }
                else     { c = tid >> 1; kk = (tid & 1) * 8 + e; }
                Bs[s][kk * GBS + c] = rb[e];
            }
        };

        const int nk = (g.k + GBK - 1) / GBK;
        load_tiles(0);
        store_tiles(0);
        __syncthreads();
        for (int kt = 0; kt < nk; kt++) {
            const int s = kt & 1;
            if (kt + 1 < nk) load_tiles((kt + 1) * GBK);
            const int r0 = (tid >> 3) * 4, c0 = (tid & 7) * 8;
#pragma unroll
            for (int kk = 0; kk < GBK; kk++) {
                double af[4], bf[8];
#pragma unroll
                for (int i = 0; i < 4; i++) af[i] = As[s][(r0 + i) * GAS + kk];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    const double2 v = *reinterpret_cast<const double2*>(&Bs[s][kk * GBS + c0 + j]);
                    bf[j] = v.x;
                    bf[j + 1] = v.y;
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        acc[i][j][0] = fma(af[i], bf[2 * j], acc[i][j][0]);
                        acc[i][j][1] = fma(af[i], bf[2 * j + 1], acc[i][j][1]);
                    }
            }
            if (kt + 1 < nk) store_tiles(s ^ 1);
            __syncthreads();
        }
    }

    // epilogue
    const double* Cinb = g.Cin ? g.Cin[b] + g.offCin : nullptr;
    const double* Cin2b = g.Cin2 ? g.Cin2[b] + g.offCin : nullptr;
    double* Cb = g.C[b] + g.offC;
#pragma unroll
    for (int i = 0; i < 4; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int r = m0 + (tid >> 3) * 4 + i;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c = n0 + (tid & 7) * 8 + 2 * j + h;
                if (r >= g.m || c >= g.n) continue;
                double v;
                if (!active) {
                    v = Cinb ? Cinb[g.cin_trans ? (long long)c * g.ldcin + r : (long long)r * g.ldcin + c] : 0.0;
                    if (g.mode == GEMM_SKEW && r < c) continue;
                } else {
                    v = alpha * acc[i][j][h];
                    if (Cinb && g.beta != 0.0) {
                        bool use = true;
                        if (g.mode == GEMM_GJ && !g.gj_acc && r >= g.gj_k0 && r < g.gj_k0 + g.gj_b) use = false;
                        if (use) v += g.beta * Cinb[g.cin_trans ? (long long)c * g.ldcin + r : (long long)r * g.ldcin + c];
                    }
                    if (Cin2b) v += g.beta2 * Cin2b[(long long)r * g.ldcin + c];
                    if (r == c) v += g.diag;
                }
                if (g.mode == GEMM_FULL) {
                    Cb[(long long)r * g.ldc + c] = v;
                } else if (g.mode == GEMM_GJ) {
                    if (!g.gj_cols || c < g.gj_k0 || c >= g.gj_k0 + g.gj_b) Cb[(long long)r * g.ldc + c] = v;
                } else {  // SKEW
                    if (tm == tn && r <= c) {
                        if (r == c) Cb[(long long)r * g.ldc + c] = 0.0;
                        continue;
                    }
                    Cb[(long long)r * g.ldc + c] = v;
                    Cb[(long long)c * g.ldc + r] = -v;
                }
            }
        }
    }
}

inline cudaError_t gemm_f64(const GemmBatch& g, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
    const int tmn = (g.m + GBM - 1) / GBM, tnn = (g.n + GBN - 1) / GBN;
    unsigned gx = (g.mode == GEMM_SKEW) ? (unsigned)(tmn * (tmn + 1) / 2) : (unsigned)(tmn * tnn);
    dim3 grid(gx, g.batch);
    if (!g.transA && !g.transB) gemm_f64_kernel<0, 0><<<grid, 128, 0, st>>>(g);
    else if (!g.transA && g.transB) gemm_f64_kernel<0, 1><<<grid, 128, 0, st>>>(g);
    else if (g.transA && !g.transB) gemm_f64_kernel<1, 0><<<grid, 128, 0, st>>>(g);
    else gemm_f64_kernel<1, 1><<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

inline GemmBatch gemm_defaults() {
    GemmBatch g{};
    g.alpha = 1.0; g.beta = 0.0; g.diag = 0.0; g.sA2 = 0.0; g.sB2 = 0.0; g.Cin2 = nullptr; g.beta2 = 0.0;
    g.mode = GEMM_FULL; g.active_flag = nullptr; g.alpha_b = nullptr; g.active_cmp = 0; g.b_antisym = 0;
    g.gj_cols = 1;
    g.gj_acc = 0;
    g.cin_trans = 0;
    return g;
}

}  // namespace sgs
