// Batched FP64 factorisations of the pair matrices.
//
//  * Gauss-Jordan inverse with partial pivoting of S = Gamma_a + Gamma_b
//    (Eq. def-delta-matrix needs S^{-1}; |Pf S| = |det S|^{1/2} gives the
//    overlap magnitude of Sec. II B).  Blocked: a panel kernel eliminates b
//    columns of every matrix (one CTA per matrix, panel in shared memory),
//    then one batched product applies the delayed rank-b update to the
//    rest of each matrix.
//  * Complex Pfaffian of Y = Gamma_0 + Delta^{a,b} (the phase of the overlap
//    in the reference gauge of Sec. II B) by Parlett-Reid elimination with
//    pivoting, blocked the same way: the panel kernel performs b elimination
//    steps, materialising the two columns each step needs from the stored
//    matrix (its upper triangle, the only part kept current) plus the pending
//    rank-2 updates, and the rank-2b trailing update is a batch of two real
//    products per matrix (real and imaginary parts, k = 4b).
#pragma once
#include "common.cuh"
#include "oz_digits.cuh"

namespace sgs {

// ---------------------------------------------------------------- Gauss-Jordan

#define GJ_MAX_PANEL 64       // widest Gauss-Jordan panel

struct GJPanelArgs {
    double* const* W;        // [batch] n x n working matrices (row-major)
    double* const* T;        // [batch] bb x n copy of the panel rows (update operand)
    int* piv;                // [batch][n]
    double* logdet;          // [batch] log|det S|
    double* dsign;           // [batch] sign(det S)
    int* err;                // error word (SGS_DEV_SINGULAR)
    int n, k0, bb;
    double tiny;             // a pivot of magnitude <= tiny counts as singular
};

// bf16 digits of four values into w (w[i][0] | w[i][1] << 32: the four digits of slice i), zero
// where E = 0 or the value is absent (present[u] false)
__device__ __forceinline__ void oz_digits4(const double (&v)[4], const bool (&present)[4], int E, unsigned (&w)[OZ_S][2]) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
        float f[OZ_S];
        if (E > 0 && present[u]) oz_digit_floats((unsigned long long)__double_as_longlong(v[u]), E, f);
        else {
#pragma unroll
            for (int i = 0; i < OZ_S; i++) f[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < OZ_S; i++) {
            const unsigned h = __float_as_uint(f[i]) >> 16;
            if (u & 1) w[i][u >> 1] |= h << 16;
            else w[i][u >> 1] = h;
        }
    }
}

// The end of a Gauss-Jordan panel, after its columns are back in W: log |det| += the sum
// of log |pivot_j|; the panel's row interchanges (k0 + j <-> piv_j, in order) applied to the
// other columns of W as one permutation of the rows they touch (row rows[e] receives the old
// row src[e]), staged through stage[0 .. cap); the update operand T (the pivot rows, panel
// columns zeroed).
__device__ void gj_panel_finish(const GJPanelArgs& a, double* W, int b, double* stage, int cap, const int* s_piv,
                                const double* s_pabs, int* s_rows, int* s_src, int* s_nr, double* s_logdet,
                                double* s_sign) {
    const int n = a.n, k0 = a.k0, bb = a.bb;
    if (threadIdx.x < 32) {         // log |det| += sum_j log |pivot_j|
        double l = 0.0;
        for (int j = threadIdx.x; j < bb; j += 32) l += log(s_pabs[j]);
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (threadIdx.x == 0) *s_logdet += l;
    }
    // the panel's interchanges (k0 + j <-> piv_j, in order) on the other columns as one
    // permutation of the rows they touch: row rows[e] receives the old row src[e]
    __syncthreads();
    if (threadIdx.x < 32) {         // warp 0: the list searches as ballots
        const int lane = threadIdx.x;
        int nr = 0;
        for (int j = 0; j < bb; j++) {
            const int c = k0 + j, p = s_piv[j];
            if (p == c) continue;
            unsigned mc = 0, mp = 0;
            for (int e0 = 0; e0 < nr; e0 += 32) {
                const int e = e0 + lane;
                const int r = e < nr ? s_rows[e] : -1;
                const unsigned bc = __ballot_sync(0xffffffffu, r == c), bp = __ballot_sync(0xffffffffu, r == p);
                if (!mc && bc) mc = (unsigned)(e0 + __ffs(bc));       // 1 + index
                if (!mp && bp) mp = (unsigned)(e0 + __ffs(bp));
            }
            int ic = (int)mc - 1, ip = (int)mp - 1;
            if (ic < 0) { if (lane == 0) { s_rows[nr] = c; s_src[nr] = c; } ic = nr++; }
            if (ip < 0) { if (lane == 0) { s_rows[nr] = p; s_src[nr] = p; } ip = nr++; }
            __syncwarp();
            if (lane == 0) {
                const int t = s_src[ic];
                s_src[ic] = s_src[ip];
                s_src[ip] = t;
            }
            __syncwarp();
        }
        if (lane == 0) *s_nr = nr;
    }
    __syncthreads();
    const int nr = *s_nr;
    if (nr > 0) {
        // gather every touched row's new contents through the staging memory, a block of
        // columns at a time, then scatter
        const int qc = min(n, cap / nr);
        for (int q0 = 0; q0 < n; q0 += qc) {
            const int qn = min(qc, n - q0);
            for (int x = threadIdx.x; x < nr * qn; x += blockDim.x) {
                const int e = x / qn, q = q0 + x % qn;
                if (q < k0 || q >= k0 + bb) stage[x] = W[(size_t)s_src[e] * n + q];
            }
            __syncthreads();
            for (int x = threadIdx.x; x < nr * qn; x += blockDim.x) {
                const int e = x / qn, q = q0 + x % qn;
                if (q < k0 || q >= k0 + bb) W[(size_t)s_rows[e] * n + q] = stage[x];
            }
            __syncthreads();
        }
    }
    __syncthreads();
    double* T = a.T[b];
    for (int e = threadIdx.x; e < bb * n; e += blockDim.x) {
        int r = e / n, q = e % n;
        T[(size_t)r * n + q] = (q >= k0 && q < k0 + bb) ? 0.0 : W[(size_t)(k0 + r) * n + q];
    }
    if (threadIdx.x == 0) { a.logdet[b] = *s_logdet; a.dsign[b] = *s_sign; }
}

__global__ void __launch_bounds__(512) gj_panel_kernel(GJPanelArgs a) {
    extern __shared__ double sm[];
    const int ps = a.bb + 1;                   // odd row stride: column walks hit distinct banks
    double* panel = sm;                        // n x ps
    double* rowc = panel + (size_t)a.n * ps;   // bb
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ double s_logdet, s_sign;
    __shared__ int s_piv[GJ_MAX_PANEL], s_rows[2 * GJ_MAX_PANEL], s_src[2 * GJ_MAX_PANEL], s_nr;
    __shared__ double s_pabs[GJ_MAX_PANEL], s_inv;

    const int b = blockIdx.x, n = a.n, k0 = a.k0, bb = a.bb;
    double* W = a.W[b];
    int* piv = a.piv + (size_t)b * n;

    for (int e = threadIdx.x; e < n * bb; e += blockDim.x) {
        int r = e / bb, q = e % bb;
        panel[r * ps + q] = W[(size_t)r * n + k0 + q];
    }
    if (threadIdx.x == 0) {
        s_logdet = (k0 == 0) ? 0.0 : a.logdet[b];
        s_sign = (k0 == 0) ? 1.0 : a.dsign[b];
    }
    __syncthreads();

    for (int j = 0; j < bb; j++) {
        const int c = k0 + j;
        long long best = -1;
        int bi = 0x7fffffff;
        for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
            const long long v = abs_key(panel[r * ps + j]);
            if (v > best) { best = v; bi = r; }
        }
        double mv;
        int p;
        block_argmax(best < 0 ? -1.0 : __longlong_as_double(best), bi, red_v, red_i, mv, p);
        if (!(mv > a.tiny)) {          // singular (or NaN): flag, keep going with p = c
            if (threadIdx.x == 0) { atomicOr(a.err, SGS_DEV_SINGULAR); s_logdet = -INFINITY; }
            p = c;
        }
        // rows c and p: interchanged now in the panel; on the other columns of W the panel's
        // interchanges are applied together after the panel (nothing reads them before)
        if (p != c) {
            for (int q = threadIdx.x; q < bb; q += blockDim.x) {
                double t = panel[c * ps + q];
                panel[c * ps + q] = panel[p * ps + q];
                panel[p * ps + q] = t;
            }
        }
        if (threadIdx.x == 0) { piv[c] = p; s_piv[j] = p; }
        __syncthreads();
        // warp 0 forms the pivot's reciprocal once (an FP64 division is many instructions on this
        // part's FP64 pipe) and the scaled pivot row; |pivot| is kept and the logarithms are summed
        // after the panel
        if (threadIdx.x < 32) {
            double pv = panel[c * ps + j];
            const bool sing = !(mv > a.tiny);
            if (sing) pv = 1.0;
            double inv = 0.0;
            if (threadIdx.x == 0) {
                inv = 1.0 / pv;
                s_inv = inv;
                s_pabs[j] = sing ? 1.0 : fabs(pv);
                s_sign *= (pv < 0.0 ? -1.0 : 1.0) * (p != c ? -1.0 : 1.0);
            }
            inv = __shfl_sync(0xffffffffu, inv, 0);
            for (int q = threadIdx.x; q < bb; q += 32) rowc[q] = (q == j) ? inv : panel[c * ps + q] * inv;
        }
        __syncthreads();
        const double inv = s_inv;
        for (int q = threadIdx.x; q < bb; q += blockDim.x) panel[c * ps + q] = rowc[q];
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            if (r == c) continue;
            double f = panel[r * ps + j];
            if (abs_key(f) != 0) {               // an integer test: no FP64 compare
                for (int q = 0; q < bb; q++)
                    if (q != j) panel[r * ps + q] -= f * rowc[q];
            }
            panel[r * ps + j] = -f * inv;
        }
        __syncthreads();
    }

    for (int e = threadIdx.x; e < n * bb; e += blockDim.x) {
        int r = e / bb, q = e % bb;
        W[(size_t)r * n + k0 + q] = panel[r * ps + q];
    }
    gj_panel_finish(a, W, b, panel, n * ps, s_piv, s_pabs, s_rows, s_src, &s_nr, &s_logdet, &s_sign);
}

// Rows p0 .. p0 + K - 1, columns t0 .. t0 + w - 1 of every W into T (K x w, row stride w):
// the pivot rows of the target columns of a delayed Gauss-Jordan update, taken before the
// update overwrites them.  Reads and writes run along the rows.
__global__ void gj_gather_rows_kernel(double* const* W, double* const* T, int n, int p0, int K, int t0, int w) {
    const double* src = W[blockIdx.y];
    double* dst = T[blockIdx.y];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)K * w;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / w), q = (int)(e % w);
        dst[e] = src[(size_t)(p0 + k) * n + t0 + q];
    }
}

// Both operands of a Gauss-Jordan update of small K and w (both <= 64), written directly as the
// slices the emulated product reads: A = columns p0 .. p0 + K - 1 of W (rows of K values;
// [batch][OZ_S][mp][kp], planes in oz_plane order, exponent fields [batch][mp]) and B = rows
// p0 .. p0 + K - 1 of the target columns t0 .. t0 + w - 1, op(B) column j (the K entries of
// column t0 + j) as row j ([batch][OZ_S][np][kp], natural plane order, exponent fields
// [batch][np]).  Padding rows and columns K .. kp - 1 get zero digits, as the slicers write
// them.  Grid (mp / GJ_SLICE_ROWS + 1, batch): a block of A rows per CTA, four consecutive
// columns of one row per thread; the last CTA of each matrix takes B.  One launch instead of
// the pivot-row gather and two slicing launches.
#define GJ_SLICE_ROWS 64
__global__ void __launch_bounds__(256) gj_update_slice_kernel(double* const* W, int n, int p0, int K, int t0, int w,
                                                              uint16_t* sa, int* ea, int mp, uint16_t* sb, int* eb,
                                                              int np, int kp) {
    __shared__ double tile[64][65];              // B: tile[j][k]
    __shared__ int s_e[64];
    const int b = blockIdx.y;
    const double* src = W[b];
    const int c4 = kp >> 2;
    for (int j = threadIdx.x; j < 64; j += blockDim.x) s_e[j] = 0;
    if (blockIdx.x < gridDim.x - 1) {
        const int r0 = blockIdx.x * GJ_SLICE_ROWS;
        __syncthreads();
        for (int e = threadIdx.x; e < GJ_SLICE_ROWS * c4; e += blockDim.x) {
            const int rr = e / c4, c = 4 * (e % c4), r = r0 + rr;
            int ef = 0;
            if (r < n)
                for (int u = 0; u < 4 && c + u < K; u++)
                    ef = max(ef, oz_expo_field((unsigned long long)__double_as_longlong(src[(size_t)r * n + p0 + c + u])));
            if (ef) atomicMax(&s_e[rr], ef);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < GJ_SLICE_ROWS * c4; e += blockDim.x) {
            const int rr = e / c4, c = 4 * (e % c4), r = r0 + rr;
            if (r >= mp) continue;
            const int ef = s_e[rr];
            if (c == 0 && r < n) ea[(size_t)b * mp + r] = ef;
            double v[4];
            bool pr[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                pr[u] = r < n && c + u < K;
                v[u] = pr[u] ? src[(size_t)r * n + p0 + c + u] : 0.0;
            }
            unsigned wd[OZ_S][2];
            oz_digits4(v, pr, ef, wd);
#pragma unroll
            for (int i = 0; i < OZ_S; i++)
                *reinterpret_cast<unsigned long long*>(sa + (((size_t)b * OZ_S + oz_plane(i)) * mp + r) * kp + c) =
                    (unsigned long long)wd[i][0] | ((unsigned long long)wd[i][1] << 32);
        }
        return;
    }
    for (int e = threadIdx.x; e < K * w; e += blockDim.x) {
        const int k = e / w, j = e % w;           // along the rows of W
        tile[j][k] = src[(size_t)(p0 + k) * n + t0 + j];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        int ef = 0;
        for (int k = 0; k < K; k++) ef = max(ef, oz_expo_field((unsigned long long)__double_as_longlong(tile[j][k])));
        s_e[j] = ef;
        eb[(size_t)b * np + j] = ef;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np * c4; e += blockDim.x) {
        const int j = e / c4, c = 4 * (e % c4);
        double v[4];
        bool pr[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            pr[u] = j < w && c + u < K;
            v[u] = pr[u] ? tile[j][c + u] : 0.0;
        }
        unsigned wd[OZ_S][2];
        oz_digits4(v, pr, j < w ? s_e[j] : 0, wd);
#pragma unroll
        for (int i = 0; i < OZ_S; i++)
            *reinterpret_cast<unsigned long long*>(sb + (((size_t)b * OZ_S + i) * np + j) * kp + c) =
                (unsigned long long)wd[i][0] | ((unsigned long long)wd[i][1] << 32);
    }
}

// Undo the row interchanges of Gauss-Jordan: inverse = X P, i.e. the column
// interchanges applied in reverse order.  perm[c] = source column of column c.
// One block per matrix: the pivots and the permutation in shared memory (2 n ints of dynamic
// shared memory), the serial interchanges by one thread there.
__global__ void gj_perm_kernel(const int* piv, int* perm, int n, int batch) {
    extern __shared__ int gj_pm[];
    int* pm = gj_pm;
    int* pv = gj_pm + n;
    const int b = blockIdx.x;
    if (b >= batch) return;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        pm[c] = c;
        pv[c] = piv[(size_t)b * n + c];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = n - 1; j >= 0; j--) {
            const int p = pv[j];
            if (p != j) { const int t = pm[j]; pm[j] = pm[p]; pm[p] = t; }
        }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) perm[(size_t)b * n + c] = pm[c];
}

__global__ void gj_gather_kernel(double* const* W, double* const* out, const int* perm, int n) {
    const int b = blockIdx.y;
    const int* pm = perm + (size_t)b * n;
    const double* src = W[b];
    double* dst = out[b];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)n * n;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e / n), c = (int)(e % n);
        dst[e] = src[(size_t)r * n + pm[c]];
    }
}

// ---------------------------------------------------------------- Pfaffian

struct PfPanelArgs {
    double* const* Y;        // [batch] planes: Re (n x n) then Im (n x n), antisymmetric
    double* const* TU;       // [batch] 4 x bs x n scratch: Tr, Ti, Ur, Ui (row t = step, contiguous in i)
    double* const* PA;       // [batch] packs, 4 blocks n x 4*bsmax apart:
                             //   A_re=[Tr,-Ti,-Ur,Ui] B_re=[Ur,Ui,Tr,Ti] A_im=[Tr,Ti,-Ur,-Ui] B_im=[Ui,Ur,Ti,Tr]
    double* logabs;          // [batch]
    double* phase;           // [batch][2]
    int* err;
    int n, k0, bs;           // bs = elimination steps in this panel
    int bsmax;               // pack blocks are n x 4*bsmax apart (row stride 4*bs)
    // emulated trailing update: with sa set the panel writes the update's operands as the
    // slices and exponent fields the product reads (entries 2 b, 2 b + 1: the real and
    // imaginary parts of matrix b; m = n - k0 - 2 bs rows, K = 4 bs; A slices [entry][OZ_S]
    // [mp][4 bs] in oz_plane order, B slices [entry][OZ_S][np][4 bs], exponents [entry][mp]
    // and [entry][np]) instead of the FP64 packs
    uint16_t* sa;
    uint16_t* sb;
    int* ea;
    int* eb;
    int mp, np;
};

#define PF_MAX_PANEL 32       // widest Pfaffian panel (column pairs)

// four digits per plane (w[i][0] | w[i][1] << 32: columns col .. col + 3 of slice i) into a slice
// batch [entry][OZ_S][rp][kk], planes in oz_plane order (inter, A operands) or natural order
__device__ __forceinline__ void pf_put_digits(uint16_t* base, int rp, int entry, int row, int kk, int col, bool inter,
                                              const unsigned (&w)[OZ_S][2]) {
#pragma unroll
    for (int i = 0; i < OZ_S; i++) {
        const int pl = inter ? oz_plane(i) : i;
        __stcs(reinterpret_cast<unsigned long long*>(base + (((size_t)entry * OZ_S + pl) * rp + row) * kk + col),
               (unsigned long long)w[i][0] | ((unsigned long long)w[i][1] << 32));
    }
}

// One pending rank-2 term of the panel on element (i, k): v += T[i][t] U[k][t] - U[i][t] T[k][t]
// (complex), as four FMAs per component (FP64 issues at a small fraction of the other
// pipes' rates on this part, so the count of FP64 instructions sets the panel's time).
// rowTU holds row k's T and U entries: Tr, Ti, Ur, Ui at offsets 0, bs, 2 bs, 3 bs.
__device__ __forceinline__ void pf_pending(double& vr, double& vi, double tr, double ti, double ur, double ui,
                                           const double* rowTU, int bs, int t) {
    const double Tkr = rowTU[t], Tki = rowTU[bs + t], Ukr = rowTU[2 * bs + t], Uki = rowTU[3 * bs + t];
    vr = fma(tr, Ukr, vr);
    vr = fma(-ti, Uki, vr);
    vr = fma(-ur, Tkr, vr);
    vr = fma(ui, Tki, vr);
    vi = fma(tr, Uki, vi);
    vi = fma(ti, Ukr, vi);
    vi = fma(-ur, Tki, vi);
    vi = fma(-ui, Tkr, vi);
}

// Columns of the antisymmetric Y are read as negated rows (coalesced); the
// pending rank-2 updates of the panel are added on the fly.  Launched with
// PF_PANEL_THREADS threads: four CTAs fit an SM (registers and shared memory),
// so up to 608 matrices run in one wave on 152 SMs.
#define PF_PANEL_THREADS 256
__global__ void __launch_bounds__(PF_PANEL_THREADS, 4) pf_panel_kernel(PfPanelArgs a) {
    extern __shared__ double sm[];
    const int n = a.n, k0 = a.k0, bs = a.bs;
    double* ckr = sm;            // current column k (real)
    double* cki = ckr + n;
    double* c1r = cki + n;       // current column k+1
    double* c1i = c1r + n;
    double* rowTU = c1i + n;     // 4 x bs: T/U entries of the row being materialised
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ double s_log, s_pr, s_pi, s_ir, s_ii;
    __shared__ double s_pvr[PF_MAX_PANEL], s_pvi[PF_MAX_PANEL];
    __shared__ int s_pok[PF_MAX_PANEL], s_flip;

    const int b = blockIdx.x;
    double* Yr = a.Y[b];
    double* Yi = Yr + (size_t)n * n;
    double* Tr = a.TU[b];                  // Tr[t * n + i]
    double* Ti = Tr + (size_t)n * bs;
    double* Ur = Ti + (size_t)n * bs;
    double* Ui = Ur + (size_t)n * bs;

    if (threadIdx.x == 0) {
        s_log = (k0 == 0) ? 0.0 : a.logabs[b];
        s_pr = (k0 == 0) ? 1.0 : a.phase[2 * b];
        s_pi = (k0 == 0) ? 0.0 : a.phase[2 * b + 1];
        s_flip = 0;
    }

    for (int s = 0; s < bs; s++) {
        const int k = k0 + 2 * s;
        for (int t = threadIdx.x; t < s; t += blockDim.x) {
            rowTU[t] = Tr[(size_t)t * n + k];
            rowTU[bs + t] = Ti[(size_t)t * n + k];
            rowTU[2 * bs + t] = Ur[(size_t)t * n + k];
            rowTU[3 * bs + t] = Ui[(size_t)t * n + k];
        }
        __syncthreads();
        // current column k: -Y[k][i] + sum_t (T[i][t] U[k][t] - U[i][t] T[k][t])
        long long best = -1;
        int bi = 0x7fffffff;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double vr = -Yr[(size_t)k * n + i], vi = -Yi[(size_t)k * n + i];
            for (int t = 0; t < s; t++)
                pf_pending(vr, vi, Tr[(size_t)t * n + i], Ti[(size_t)t * n + i], Ur[(size_t)t * n + i],
                           Ui[(size_t)t * n + i], rowTU, bs, t);
            ckr[i] = vr;
            cki[i] = vi;
            const long long m2 = abs_key(fma(vr, vr, vi * vi));
            if (m2 > best) { best = m2; bi = i; }
        }
        double mv;
        int p;
        block_argmax(best < 0 ? -1.0 : __longlong_as_double(best), bi, red_v, red_i, mv, p);
        if (!(mv > 0.0)) {
            if (threadIdx.x == 0) { atomicOr(a.err, SGS_DEV_PF_ZERO); s_log = -INFINITY; }
            p = k + 1;
        }
        if (p != k + 1) {
            const int q = k + 1;
            // symmetric interchange q <-> p on the upper triangle of the live part, the only part the
            // panels read (row k is done: its entries are in ckr, cki); the trailing update reads its
            // Cin there too (cin_trans), so the lower triangle is left stale.  With q < p:
            //   row entries beyond p:    Y[q][j] <-> Y[p][j]                       (j > p)
            //   between q and p:         Y'[q][c] = -Y[c][p], Y'[c][p] = -Y[q][c]  (q < c < p)
            //   the pair:                Y'[q][p] = -Y[q][p]
            for (int j = p + 1 + threadIdx.x; j < n; j += blockDim.x) {
                double t;
                t = Yr[(size_t)q * n + j]; Yr[(size_t)q * n + j] = Yr[(size_t)p * n + j]; Yr[(size_t)p * n + j] = t;
                t = Yi[(size_t)q * n + j]; Yi[(size_t)q * n + j] = Yi[(size_t)p * n + j]; Yi[(size_t)p * n + j] = t;
            }
            for (int c = q + 1 + threadIdx.x; c < p; c += blockDim.x) {
                const double ar = Yr[(size_t)q * n + c], ai = Yi[(size_t)q * n + c];
                Yr[(size_t)q * n + c] = -Yr[(size_t)c * n + p];
                Yi[(size_t)q * n + c] = -Yi[(size_t)c * n + p];
                Yr[(size_t)c * n + p] = -ar;
                Yi[(size_t)c * n + p] = -ai;
            }
            if (threadIdx.x == 0) {
                Yr[(size_t)q * n + p] = -Yr[(size_t)q * n + p];
                Yi[(size_t)q * n + p] = -Yi[(size_t)q * n + p];
            }
            for (int t = threadIdx.x; t < s; t += blockDim.x) {
                double x;
                x = Tr[(size_t)t * n + q]; Tr[(size_t)t * n + q] = Tr[(size_t)t * n + p]; Tr[(size_t)t * n + p] = x;
                x = Ti[(size_t)t * n + q]; Ti[(size_t)t * n + q] = Ti[(size_t)t * n + p]; Ti[(size_t)t * n + p] = x;
                x = Ur[(size_t)t * n + q]; Ur[(size_t)t * n + q] = Ur[(size_t)t * n + p]; Ur[(size_t)t * n + p] = x;
                x = Ui[(size_t)t * n + q]; Ui[(size_t)t * n + q] = Ui[(size_t)t * n + p]; Ui[(size_t)t * n + p] = x;
            }
            if (threadIdx.x == 0) {
                double x = ckr[q]; ckr[q] = ckr[p]; ckr[p] = x;
                x = cki[q]; cki[q] = cki[p]; cki[p] = x;
                s_flip ^= 1;      // a row/column interchange flips the sign (applied after the panel)
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < s; t += blockDim.x) {
            rowTU[t] = Tr[(size_t)t * n + k + 1];
            rowTU[bs + t] = Ti[(size_t)t * n + k + 1];
            rowTU[2 * bs + t] = Ur[(size_t)t * n + k + 1];
            rowTU[3 * bs + t] = Ui[(size_t)t * n + k + 1];
        }
        __syncthreads();
        // current column k+1 (rows >= k+2): -Y[k+1][i] + pending
        for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) {
            double vr = -Yr[(size_t)(k + 1) * n + i], vi = -Yi[(size_t)(k + 1) * n + i];
            for (int t = 0; t < s; t++)
                pf_pending(vr, vi, Tr[(size_t)t * n + i], Ti[(size_t)t * n + i], Ur[(size_t)t * n + i],
                           Ui[(size_t)t * n + i], rowTU, bs, t);
            c1r[i] = vr;
            c1i[i] = vi;
        }
        // pivot Y[k][k+1] = -Y[k+1][k]: thread 0 forms 1/pivot once (an FP64 division is many
        // instructions on this part's FP64 pipe) and keeps the pivot, whose logarithm and unit
        // phase are accumulated after the panel in the same order
        if (threadIdx.x == 0) {
            double pr = -ckr[k + 1], pi = -cki[k + 1];
            const bool ok = mv > 0.0;
            if (!ok) { pr = 1.0; pi = 0.0; }
            const double pm2 = pr * pr + pi * pi;
            s_ir = pr / pm2;
            s_ii = -pi / pm2;
            s_pvr[s] = pr;
            s_pvi[s] = pi;
            s_pok[s] = ok ? 1 : 0;
        }
        __syncthreads();
        // tau = (row k)/pivot = -(column k)/pivot, u = column k+1; zero above k+2
        const double ir = s_ir, ii = s_ii;   // 1/pivot
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double tr = 0.0, ti = 0.0, ur = 0.0, ui = 0.0;
            if (i >= k + 2) {
                const double xr = -ckr[i], xi = -cki[i];
                tr = xr * ir - xi * ii;
                ti = xr * ii + xi * ir;
                ur = c1r[i];
                ui = c1i[i];
            }
            Tr[(size_t)s * n + i] = tr;
            Ti[(size_t)s * n + i] = ti;
            Ur[(size_t)s * n + i] = ur;
            Ui[(size_t)s * n + i] = ui;
        }
        __syncthreads();
    }

    // packs for the trailing update (rows >= k0 + 2 bs are the only ones used)
    const int e0 = k0 + 2 * bs;
    const int kk = 4 * bs;
    double* PAre = a.PA[b];
    const size_t blk = (size_t)n * 4 * a.bsmax;
    double* PBre = PAre + blk;
    double* PAim = PBre + blk;
    double* PBim = PAim + blk;
    // rows are staged through the column buffers (4 n doubles, free now), R rows at a time
    // with an odd row stride: T/U read along i and the packs written along their rows,
    // both coalesced, with streaming stores (the packs are read once, by the next kernel,
    // and should not push the T/U vectors of CTAs still in their panel out of L2)
    const bool sliced = a.sa != nullptr;
    __shared__ int s_E[32];
    int R = n / bs - 1;
    if (R < 1) R = 1;
    if (sliced && R > 32) R = 32;
    const int rs = R | 1;                       // 4 bs rs <= 4 n
    double* stg = sm;
    for (int i0 = e0; i0 < n; i0 += R) {
        const int rn = min(R, n - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < 4 * bs * rn; e += blockDim.x) {
            const int r = e % rn, qt = e / rn;  // qt = plane * bs + t; planes Tr, Ti, Ur, Ui
            stg[qt * rs + r] = Tr[(size_t)(qt / bs) * n * bs + (size_t)(qt % bs) * n + i0 + r];
        }
        __syncthreads();
        if (!sliced) {
            for (int e = threadIdx.x; e < rn * kk; e += blockDim.x) {
                const int r = e / kk, c = e % kk, blk = c / bs, t = c % bs;
                const double* v = stg + r;      // v[(plane * bs + t) * rs]: plane 0 Tr, 1 Ti, 2 Ur, 3 Ui
                const size_t o = (size_t)(i0 + r) * kk + c;
                // A_re = [Tr, -Ti, -Ur, Ui], B_re = [Ur, Ui, Tr, Ti], A_im = [Tr, Ti, -Ur, -Ui], B_im = [Ui, Ur, Ti, Tr]
                const double x = v[(blk * bs + t) * rs];
                __stcs(PAre + o, (blk == 1 || blk == 2) ? -x : x);
                __stcs(PAim + o, blk >= 2 ? -x : x);
                __stcs(PBre + o, v[(((blk + 2) & 3) * bs + t) * rs]);
                __stcs(PBim + o, v[((3 - blk) * bs + t) * rs]);
            }
            continue;
        }
        // slices: every pack row is a signed permutation of the same 4 bs values, so the four
        // packs share the row's exponent field (the largest of them), one warp per row
        for (int r = threadIdx.x >> 5; r < rn; r += blockDim.x >> 5) {
            int ef = 0;
            for (int q = threadIdx.x & 31; q < kk; q += 32)
                ef = max(ef, oz_expo_field((unsigned long long)__double_as_longlong(stg[q * rs + r])));
            for (int w = 16; w > 0; w >>= 1) ef = max(ef, __shfl_xor_sync(0xffffffffu, ef, w));
            if ((threadIdx.x & 31) == 0) {
                s_E[r] = ef;
                const int row = i0 + r - e0;
                a.ea[(size_t)(2 * b) * a.mp + row] = ef;
                a.ea[(size_t)(2 * b + 1) * a.mp + row] = ef;
                a.eb[(size_t)(2 * b) * a.np + row] = ef;
                a.eb[(size_t)(2 * b + 1) * a.np + row] = ef;
            }
        }
        __syncthreads();
        // digits of four consecutive values t .. t + 3 of one source plane (Tr, Ti, Ur, Ui) of one
        // row per thread, once per sign the packs take them with (as the slicers write them: one
        // 8-byte word of four bf16 per plane).  Plane src sits in block src of A_re = [Tr, -Ti,
        // -Ur, Ui] and A_im = [Tr, Ti, -Ur, -Ui], block (src + 2) & 3 of B_re = [Ur, Ui, Tr, Ti]
        // and block 3 - src of B_im = [Ui, Ur, Ti, Tr]
        const int t4n = bs >> 2;
        for (int e = threadIdx.x; e < rn * 4 * t4n; e += blockDim.x) {
            const int t = 4 * (e % t4n), src = (e / t4n) & 3, r = e / (4 * t4n);
            const int E = s_E[r], row = i0 + r - e0;
            const bool nre = src == 1 || src == 2, nim = src >= 2;
#pragma unroll 1
            for (int sg = 0; sg < 2; sg++) {
                if (sg == 1 && !nre && !nim) break;
                unsigned w[OZ_S][2];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const double x = stg[(src * bs + t + u) * rs + r];
                    float f[OZ_S];
                    if (E > 0) oz_digit_floats((unsigned long long)__double_as_longlong(sg ? -x : x), E, f);
                    else {
#pragma unroll
                        for (int i = 0; i < OZ_S; i++) f[i] = 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < OZ_S; i++) {
                        const unsigned h = __float_as_uint(f[i]) >> 16;
                        if (u & 1) w[i][u >> 1] |= h << 16;
                        else w[i][u >> 1] = h;
                    }
                }
                // pk 0, 1: A_re, A_im (block src, the sign they take); 2, 3: B_re, B_im (positive)
#pragma unroll 1
                for (int pk = 0; pk < 4; pk++) {
                    const bool take = pk == 0 ? nre == (sg == 1) : pk == 1 ? nim == (sg == 1) : sg == 0;
                    if (!take) continue;
                    const int blk = pk < 2 ? src : pk == 2 ? ((src + 2) & 3) : 3 - src;
                    pf_put_digits(pk < 2 ? a.sa : a.sb, pk < 2 ? a.mp : a.np, 2 * b + (pk & 1), row, kk, blk * bs + t,
                                  pk < 2, w);
                }
            }
        }
    }
    if (sliced && e0 < n) {
        // zero digits on the padding rows m .. mp - 1 (A) and m .. np - 1 (B), as the slicers write
        const int m = n - e0, c4n = kk >> 2;
        const int za = (a.mp - m) * c4n, zb = (a.np - m) * c4n;
        for (int e = threadIdx.x; e < 2 * OZ_S * (za + zb); e += blockDim.x) {
            const int ep = e / (OZ_S * (za + zb)), x = e % (OZ_S * (za + zb));
            const int pl = x / (za + zb), y = x % (za + zb);
            const bool isA = y < za;
            const int z = isA ? y : y - za, row = m + z / c4n, c = 4 * (z % c4n);
            uint16_t* base = isA ? a.sa : a.sb;
            const int rp = isA ? a.mp : a.np;
            __stcs(reinterpret_cast<unsigned long long*>(base + (((size_t)(2 * b + ep) * OZ_S + pl) * rp + row) * kk + c),
                   0ull);
        }
    }
    if (threadIdx.x == 0) {
        double lg = s_log, ph_r = s_pr, ph_i = s_pi;
        for (int t = 0; t < bs; t++) {
            if (!s_pok[t]) continue;
            const double pr = s_pvr[t], pi = s_pvi[t];
            const double am = sqrt(pr * pr + pi * pi);
            lg += log(am);
            const double ur = pr / am, ui = pi / am;
            const double nr = ph_r * ur - ph_i * ui, ni = ph_r * ui + ph_i * ur;
            ph_r = nr;
            ph_i = ni;
        }
        if (s_flip) { ph_r = -ph_r; ph_i = -ph_i; }
        a.logabs[b] = lg;
        a.phase[2 * b] = ph_r;
        a.phase[2 * b + 1] = ph_i;
    }
}

}  // namespace sgs
