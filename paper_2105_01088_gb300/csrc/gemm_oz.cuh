// Batched FP64 GEMM emulated on the bf16 tensor cores (tcgen05 kind::f16) by
// splitting both operands into integer slices (the Ozaki scheme: Ozaki, Ogita,
// Oishi and Rump, Numer. Algorithms 59 (2012); its tensor-core forms by Mukunoki
// et al. and Ootomo et al.).  GB300's FP64 pipe issues about 1.25 TFLOP/s while
// its bf16 tensor cores issue over 2 PFLOP/s, so the products of the step run
// here when the emulated path is selected.  The error bound is normwise per row
// of op(A) and column of op(B) (the error budget below), not elementwise like
// that of the FP64 FMA kernel.
//
// Slicing.  Every row r of op(A) (K-major) gets the exponent field E_r of its
// largest element, so |a_rk| < 2^(E_r - 1022).  The element is rounded to the
// signed integer X = a_rk 2^(56 - (E_r - 1022)) (|X| < 2^56) and written as
// eight balanced base-128 digits, most significant first:
//     X = sum_{i=0..7} t_i 2^(7 (7 - i)),  |t_0| <= 128, |t_i| <= 64 (i >= 1),
// so a_rk = 2^(E_r - 1022) sum_i t_i 2^(-7 (i + 1)) up to 2^-57 of the row's
// scale.  Each digit is a bf16 (at most 8 significant bits: exact).  Columns of
// op(B) are sliced the same way.  The digit extraction is integer arithmetic on
// the IEEE bit pattern (FP64 arithmetic is the scarce resource here).
//
// Products.  The slice products t_i(A) t_j(B) with i + j <= 7 (36 of the 64)
// are accumulated into eight fp32 TMEM accumulators, one per group G = i + j
// (weight 2^(-7 (G + 2))).  Each product term is an integer of magnitude at
// most 2^14 (i = j = 0), 2^13 (one index 0) or 2^12, so over a K chunk of 512
// the sums of groups G <= 5 stay within 2^24 and are exact in fp32; groups 6
// and 7 may round, by at most 2^-47 of the output scale, below FP64's own
// rounding of a 512-term dot product.  K beyond 512 runs as further launches
// that add onto the output (one FP64 rounding per chunk).  The dropped products
// (i + j >= 8) weigh at most 2^-63 per term.
//
// Combination.  The eight group sums are converted to integers and combined
// exactly, hi = sum_{G<4} v_G 2^(7 (3 - G)), lo = sum_{G>=4} v_G 2^(7 (7 - G)),
// V = hi 2^28 + lo = H 2^28 + L (0 <= L < 2^28); V is rounded once to 53 bits
// and given the exponent E_r + F_c - 2107 (plus that of alpha when alpha is a
// power of two, else one multiplication), all in straight-line integer
// arithmetic on the bit pattern.  The GemmBatch epilogue (beta Cin, beta2 Cin2,
// diag, FULL / SKEW / GJ modes, pass-through of inactive batch entries) is
// applied as in gemm_f64, with no FP64 instruction beyond the additions the
// epilogue terms need (FP64 issues at a small fraction of the integer rate).
//
// Kernels per batch chunk: exponents and slices of op(A) and op(B), one pass
// over each (a warp per row where the operand's K rows are contiguous and long,
// else a block of whole rows at a time through shared memory), then the product
// kernel.  It takes a 128 x 32 output tile per CTA of 10 warps (256 TMEM
// columns, 97 KB of shared memory), so two CTAs share an SM and one's epilogue
// overlaps the other's loads and MMAs.  In the kernel:
//   * one producer lane loads, per 64-element K slab, the eight B slices as one
//     TMA box (TMA issue costs about the same per box whatever its size, so
//     boxes are made large) and the A slices in pairs (one 32 KB box per pair of
//     adjacent planes) through a ring, 128-byte swizzle, zero fill beyond K;
//     the B buffer is reloaded once the previous slab's MMAs have released it;
//   * one MMA lane issues, per A slice and K16 step, one MMA of N up to 256
//     covering all the products of that slice (the B slices and the groups they
//     feed are adjacent) into the eight accumulators;
//   * the epilogue warps wait for the MMAs, issue the loads of the tile's Cin
//     terms (for in-place updates every Cin element is read before the CTA
//     stores any), drain TMEM and combine, and write the output through a
//     shared-memory tile (coalesced rows).
// Every mbarrier wait is bounded; on a timeout the launch records
// SGS_DEV_TC_TIMEOUT in the error word, waits (bounded) for its loads and MMAs
// in flight, frees TMEM and returns.
#pragma once
#include "gemm_f64.cuh"
#include "gemm_tma.cuh"
#include "oz_digits.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>

namespace sgs {

#define OZ_G 8                // accumulator groups G = i + j <= 7
#define OZ_BM 128
#define OZ_KS 64              // K elements of one 128-byte slab row
#define OZ_KC 512             // K per exactly accumulated chunk
#define OZ_UNIT 2             // A slices per TMA box (one ring slot)
#define OZ_SLAB_A (OZ_BM * 128)

// Kernel shapes: BN output columns per tile (TMEM: 8 BN columns), EPIW epilogue warps,
// RING A-ring depth (units), BDBL double-buffered B slabs.  The form launched (32, 8, 2,
// single) fits two CTAs per SM.  A 128 x 64 tile (64, 16, 3, double) takes all of an SM's
// TMEM and shared memory; with its epilogue serialised after the main loop it measured
// about half the throughput at K = 512, so it is not launched.
template <int BN, int EPIW, int RING, bool BDBL> struct OzCfg {
    static constexpr int SLAB_B = BN * 128;
    static constexpr int SMEM = (BDBL ? 2 : 1) * OZ_S * SLAB_B + RING * OZ_UNIT * OZ_SLAB_A + 1024;
    static constexpr int THREADS = 32 * (EPIW + 2);
};
#define OZ_NARROW 32, 8, 2, false
// 128 x 16 tiles for products of at most 16 output columns (the Gauss-Jordan leaf updates):
// half the epilogue of a 128 x 32 tile whose other half would be discarded
#define OZ_NARROW16 16, 8, 2, false

// device scratch of one owner (an instance, or a temporary context): slices and
// exponent fields of one batch chunk
struct OzBuf {
    uint8_t* base = nullptr;
    size_t bytes = 0;
};

// K-major operand rows as seen by the slicer: element (r, k) of op(X) is
// X[b][off + r * ld + k] (strided = 0) or X[b][off + k * ld + r] (strided = 1),
// plus s2 times the same element of X2 when X2 is given
struct OzOperand {
    const double* const* X;
    const double* const* X2;
    double s2;
    long long off;
    int ld, strided;
    int rows, k;              // K-major rows and K
    int rows_pad, kp;         // padded rows (a multiple of the tile) and row pitch (a multiple of 8)
    int b0;                   // first batch entry of the chunk
    const int* active; int active_cmp;
    int* expo;                // [chunk][rows_pad] exponent fields
    uint16_t* slices;         // [chunk][OZ_S][rows_pad][kp] bf16 digits (planes)
    int interleave;           // 1: slice i in plane oz_plane(i) (A operands), 0: plane i (B operands)
};



// element (r, k) of op(X) as its bit pattern (plus s2 times the same element of X2, the one
// FP64 operation of the slicers)
__device__ __forceinline__ unsigned long long oz_load(const OzOperand& o, const double* x, const double* x2, int r,
                                                      int k) {
    const long long off = o.strided ? (long long)k * o.ld + r : (long long)r * o.ld + k;
    if (x2) return (unsigned long long)__double_as_longlong(fma(o.s2, x2[off], x[off]));
    return reinterpret_cast<const unsigned long long*>(x)[off];
}

__device__ __forceinline__ bool oz_active(const int* flag, int cmp, int b) {
    return flag == nullptr || flag[b] > cmp;
}



// the eight planes of four consecutive k of row r starting at k (k + 3 < kp; entries at or
// beyond o.k are zero digits, which the tensor map never reads): per plane one 8-byte word
// of four bf16, the high halves of the digits' floats
__device__ __forceinline__ void oz_store4(const OzOperand& o, int bl, int r, int k, const unsigned long long (&v)[4],
                                          int E) {
    float f[4][OZ_S];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (E > 0 && k + u < o.k) oz_digit_floats(v[u], E, f[u]);
        else {
#pragma unroll
            for (int i = 0; i < OZ_S; i++) f[u][i] = 0.0f;
        }
    }
#pragma unroll
    for (int i = 0; i < OZ_S; i++) {
        const int pl = o.interleave ? oz_plane(i) : i;
        const unsigned lo = __byte_perm(__float_as_uint(f[0][i]), __float_as_uint(f[1][i]), 0x7632);
        const unsigned hi = __byte_perm(__float_as_uint(f[2][i]), __float_as_uint(f[3][i]), 0x7632);
        *reinterpret_cast<unsigned long long*>(o.slices + (((size_t)bl * OZ_S + pl) * o.rows_pad + r) * o.kp + k) =
            (unsigned long long)lo | ((unsigned long long)hi << 32);
    }
}

// Rows of a block of the one-pass slicer: rb K-major rows of kp doubles in shared memory
// (at most OZ_BLK_BYTES), rb a power of two in 16 .. 128
#define OZ_BLK_BYTES (68 * 1024)
__host__ __device__ __forceinline__ int oz_block_rows(int kp) {
    int rb = 128;
    while (rb > 16 && (size_t)rb * (kp + 1) * 8 > OZ_BLK_BYTES) rb >>= 1;
    return rb;
}

// Slices of an operand whose K-major rows are strided, or contiguous and short (K <= 512):
// a block takes rb rows whole into shared memory (loads coalesced along r for a strided
// operand, along k for a contiguous one), reduces every row's exponent field there and writes
// the digits, one pass over the operand; rows in [rows, rows_pad) get zero digits
__global__ void __launch_bounds__(256) oz_block_slice_kernel(OzOperand o) {
    extern __shared__ unsigned long long oz_blk[];
    __shared__ int s_e[128];
    const int bl = blockIdx.y, b = o.b0 + bl;
    if (!oz_active(o.active, o.active_cmp, b)) return;
    const double* x = o.X[b] + o.off;
    const double* x2 = o.X2 ? o.X2[b] + o.off : nullptr;
    const int kp = o.kp, ts = kp + 1, rb = oz_block_rows(kp), r0 = blockIdx.x * rb;
    const int total = rb * kp;
    if (o.strided) {
        // element idx: k = idx / rb, row idx % rb (rb consecutive doubles of one k)
        const int sh = __ffs(rb) - 1;
#pragma unroll 8
        for (int idx = threadIdx.x; idx < total; idx += 256) {
            const int k = idx >> sh, rr = idx & (rb - 1), r = r0 + rr;
            oz_blk[rr * ts + k] = (r < o.rows && k < o.k) ? oz_load(o, x, x2, r, k) : 0ull;
        }
    } else {
        // element idx: row idx / kp, k = idx % kp, stepped without divisions
        const int dr = 256 / kp, dk = 256 - dr * kp;
        int rr = threadIdx.x / kp, k = threadIdx.x - rr * kp;
#pragma unroll 8
        for (int idx = threadIdx.x; idx < total; idx += 256) {
            const int r = r0 + rr;
            oz_blk[rr * ts + k] = (r < o.rows && k < o.k) ? oz_load(o, x, x2, r, k) : 0ull;
            rr += dr;
            k += dk;
            if (k >= kp) { k -= kp; rr++; }
        }
    }
    __syncthreads();
    {   // exponent fields: 256 / rb consecutive threads per row, reduced by shuffles
        const int tpr = 256 / rb, rr = threadIdx.x / tpr, q = threadIdx.x - rr * tpr, r = r0 + rr;
        int e = 0;
        for (int k = q; k < o.k; k += tpr) e = max(e, oz_expo_field(oz_blk[rr * ts + k]));
        for (int w = tpr >> 1; w > 0; w >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, w));
        if (q == 0) {
            s_e[rr] = r < o.rows ? e : 0;
            if (r < o.rows) o.expo[(size_t)bl * o.rows_pad + r] = e;
        }
    }
    __syncthreads();
    // digits, four consecutive k per step (kp is a multiple of 8)
    const int cpr = kp >> 2;
    const int dr = 256 / cpr, dc = 256 - dr * cpr;
    int rr = threadIdx.x / cpr, c = threadIdx.x - rr * cpr;
    for (int idx = threadIdx.x; idx < rb * cpr; idx += 256) {
        const int r = r0 + rr, k = 4 * c;
        if (r < o.rows_pad) {
            const unsigned long long* t = oz_blk + rr * ts + k;
            const unsigned long long v[4] = {t[0], t[1], t[2], t[3]};
            oz_store4(o, bl, r, k, v, s_e[rr]);
        }
        rr += dr;
        c += dc;
        if (c >= cpr) { c -= cpr; rr++; }
    }
}

// contiguous rows (K <= 512): one warp per row takes the row into registers, reduces the
// exponent field and writes the digits, four k per lane per step (one pass over the operand)
__global__ void __launch_bounds__(256) oz_row_slice_kernel(OzOperand o) {
    const int bl = blockIdx.y, b = o.b0 + bl;
    if (!oz_active(o.active, o.active_cmp, b)) return;
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= o.rows_pad) return;
    const double* x = o.X[b] + o.off;
    const double* x2 = o.X2 ? o.X2[b] + o.off : nullptr;
    unsigned long long v[4][4];          // k = 4 lane + 128 s + u, s < 4 (K <= 512)
    int e = 0;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int k = 128 * s + 4 * lane + u;
            v[s][u] = (r < o.rows && k < o.k) ? oz_load(o, x, x2, r, k) : 0ull;
            e = max(e, oz_expo_field(v[s][u]));
        }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, sh));
    if (lane == 0 && r < o.rows) o.expo[(size_t)bl * o.rows_pad + r] = e;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const int k = 128 * s + 4 * lane;
        if (k < o.kp) oz_store4(o, bl, r, k, v[s], r < o.rows ? e : 0);
    }
}

struct OzGemm {
    CUtensorMap ta, tb;       // slices: 3-D [chunk * 8][rows_pad][k] bf16, box 64 x rows x 1
    GemmBatch g;              // sizes, output and epilogue fields (batch index = b0 + local)
    int b0;
    int m_pad, n_pad;
    const int* ea; const int* eb;
    int* err;
    int alpha_pow2;           // alpha = +-2^alpha_e (no per-batch factor): folded into the exponent
    int alpha_e, alpha_neg;
};

__device__ __forceinline__ void oz_tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}

// The eight group sums (integers held exactly in fp32, or rounded to even integers for
// the two lowest groups) of output column j, combined exactly into V = H 2^28 + L with
// 0 <= L < 2^28: hi = sum_{G<4} v_G 2^(7 (3 - G)) and lo = sum_{G>=4} v_G 2^(7 (7 - G))
// (|hi|, |lo| < 2^46, each a chain of 32 x 32 -> 64-bit multiply-adds), V = hi 2^28 + lo,
// H = hi + floor(lo / 2^28), L = lo mod 2^28.
__device__ __forceinline__ void oz_combine(const uint32_t (&u)[OZ_G][8], int j, long long& H, unsigned& L) {
    int v[OZ_G];
#pragma unroll
    for (int G = 0; G < OZ_G; G++) v[G] = __float2int_rn(__uint_as_float(u[G][j]));
    const long long hi = (long long)v[0] * (1 << 21) + (long long)v[1] * (1 << 14) + (long long)v[2] * 128 + v[3];
    const long long lo = (long long)v[4] * (1 << 21) + (long long)v[5] * (1 << 14) + (long long)v[6] * 128 + v[7];
    H = hi + (lo >> 28);
    L = (unsigned)lo & 0xFFFFFFFu;
}

// The bit pattern of (-1)^neg V 2^e as a double, V = H 2^28 + L (|H| < 2^47, 0 <= L < 2^28), rounded once to
// 53 bits (to nearest, ties to even) in integer arithmetic: |V| = Hm 2^28 + Lm is
// left-justified into one 64-bit word N (bits shifted out are kept as a sticky flag), N is
// rounded at its bit 11, and the biased exponent is added onto the rounded significand (a
// carry out of the significand moves into the exponent by itself).  Results beyond the
// normal range become infinities, and below it subnormals (q rounded once more).  The code
// is straight-line: both justifications of N (|V| of more or fewer than 64 bits), the case
// |V| < 2^28 and the range ends are computed with shift amounts kept in range and selected,
// with no branch and no FP64 instruction, so that the eight columns a thread combines
// interleave.
__device__ __forceinline__ unsigned long long oz_to_double_bits(long long H, unsigned L, int e, bool neg) {
    const bool sv = H < 0;
    const unsigned long long Hm = sv ? (unsigned long long)(L ? ~H : -H) : (unsigned long long)H;
    const unsigned Lm = sv ? ((0x10000000u - L) & 0xFFFFFFFu) : L;
    // |V| >= 2^28: from Hm's leading bit (lzh in 17 .. 63)
    const int lzh = __clzll((long long)Hm) & 63;               // Hm = 0: 0, and unused
    const bool right = lzh < 28;                               // Lm loses 28 - lzh bits
    const unsigned long long low = right ? (unsigned long long)(Lm >> (right ? 28 - lzh : 0))
                                         : (unsigned long long)Lm << (right ? 0 : lzh - 28);
    const unsigned long long NH = (Hm << lzh) | low;
    const unsigned stH = right ? (Lm << ((lzh + 4) & 31)) : 0u;
    // |V| < 2^28: from Lm's
    const int lzl = __clz((int)Lm);                            // Lm = 0: 32 (V = 0, handled below)
    const unsigned long long NL = (unsigned long long)Lm << ((lzl + 32) & 63);
    const bool hz = Hm == 0ull;
    const unsigned long long N = hz ? NL : NH;
    const unsigned sticky = hz ? 0u : stH;
    const int P = hz ? 31 - lzl : 91 - lzh;                    // leading bit of |V|
    unsigned long long q = N >> 11;
    const unsigned rest = (unsigned)(N & 0x3FFull) | sticky;
    q += ((N >> 10) & 1ull) & ((rest != 0u ? 1ull : 0ull) | (q & 1ull));
    const int be = P + e + 1023;
    const unsigned long long sbit = (unsigned long long)(sv != neg) << 63;
    unsigned long long bits = sbit + ((unsigned long long)(be - 1) << 52) + q;   // be <= 2046: a carry out of
    bits = be > 2046 ? (sbit | 0x7FF0000000000000ull) : bits;                  // q overflows to infinity
    // subnormal: q 2^(be - 1) in units of 2^-1074, q rounded once more to nearest even
    const int sh = min(max(1 - be, 1), 63);
    const unsigned long long ms = q >> sh, rem = q & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const unsigned long long msub = (1 - be < 64) ? ms + ((rem > half || (rem == half && (ms & 1ull))) ? 1ull : 0ull)
                                                  : 0ull;
    bits = be < 1 ? (sbit | msub) : bits;                      // msub = 2^52: the smallest normal, exactly
    return (Hm | Lm) ? bits : 0ull;
}

// oz_to_double_bits where the result is known to be a normal number (biased exponent P + e + 1023 in
// 1 .. 2046 for every leading-bit position P of |V| that can occur, 0 .. 74): the same bits, without
// the selects of the range ends
__device__ __forceinline__ unsigned long long oz_to_double_bits_normal(long long H, unsigned L, int e, bool neg) {
    const bool sv = H < 0;
    const unsigned long long Hm = sv ? (unsigned long long)(L ? ~H : -H) : (unsigned long long)H;
    const unsigned Lm = sv ? ((0x10000000u - L) & 0xFFFFFFFu) : L;
    const int lzh = __clzll((long long)Hm) & 63;
    const bool right = lzh < 28;
    const unsigned long long low = right ? (unsigned long long)(Lm >> (right ? 28 - lzh : 0))
                                         : (unsigned long long)Lm << (right ? 0 : lzh - 28);
    const unsigned long long NH = (Hm << lzh) | low;
    const unsigned stH = right ? (Lm << ((lzh + 4) & 31)) : 0u;
    const int lzl = __clz((int)Lm);
    const unsigned long long NL = (unsigned long long)Lm << ((lzl + 32) & 63);
    const bool hz = Hm == 0ull;
    const unsigned long long N = hz ? NL : NH;
    const unsigned sticky = hz ? 0u : stH;
    const int P = hz ? 31 - lzl : 91 - lzh;
    unsigned long long q = N >> 11;
    const unsigned rest = (unsigned)(N & 0x3FFull) | sticky;
    q += ((N >> 10) & 1ull) & ((rest != 0u ? 1ull : 0ull) | (q & 1ull));
    const unsigned long long sbit = (unsigned long long)(sv != neg) << 63;
    const unsigned long long bits = sbit + ((unsigned long long)(P + e + 1022) << 52) + q;
    return (Hm | Lm) ? bits : 0ull;
}

template <int BN, int EPIW, int RING, bool BDBL>
__global__ void __launch_bounds__(32 * (EPIW + 2), BDBL ? 1 : 2) oz_gemm_kernel(const __grid_constant__ OzGemm p) {
    constexpr int SLAB_B = BN * 128, TS = BN + 1, NB = BDBL ? 2 : 1;
    constexpr uint32_t TCOLS = 8u * BN;          // TMEM columns: eight groups of BN
    extern __shared__ uint8_t oz_smem_raw[];
    __shared__ uint64_t bfull[2], bempty[2], afull[RING], aempty[RING], tfull, done;
    __shared__ uint32_t tmem_base;
    __shared__ int skip, abort_flag, s_ok, s_fcmin, s_fcmax;
    __shared__ int col_e[BN];

    const GemmBatch& g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) skip = (*(volatile int*)p.err & SGS_DEV_TC_TIMEOUT) != 0;
    __syncthreads();
    if (skip) return;
    const int bl = blockIdx.y, b = p.b0 + bl;
    const int tnn = (g.n + BN - 1) / BN;
    int tm, tn;
    if (g.mode == GEMM_SKEW) {      // tiles holding an element on or below the diagonal
        int t = blockIdx.x;
        tm = 0;
        while (true) {
            const int cnt = min((tm + 1) * (OZ_BM / BN), tnn);
            if (t < cnt) break;
            t -= cnt;
            tm++;
        }
        tn = t;
    } else {
        tm = blockIdx.x / tnn;
        tn = blockIdx.x % tnn;
    }
    const int m0 = tm * OZ_BM, n0 = tn * BN;
    const bool active = oz_active(g.active_flag, g.active_cmp, b);
    const int nslab = active ? (g.k + OZ_KS - 1) / OZ_KS : 0;      // k <= OZ_KC (the host splits K)

    const uint32_t raw = smem_u32(oz_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    auto sB = [&](int bb, int j) { return sbase + (uint32_t)(bb * OZ_S + j) * SLAB_B; };
    auto sA = [&](int slot) { return sbase + (uint32_t)NB * OZ_S * SLAB_B + (uint32_t)slot * (OZ_UNIT * OZ_SLAB_A); };
    auto bslot = [&](int sb) { return BDBL ? (sb & 1) : 0; };
    auto bphase = [&](int sb) { return (uint32_t)((BDBL ? (sb >> 1) : sb) & 1); };

    if (warp == EPIW + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bempty[s])));
        }
        for (int s = 0; s < RING; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&afull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&aempty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&tfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    if (tid < BN) col_e[tid] = (active && n0 + tid < g.n) ? p.eb[(size_t)bl * p.n_pad + n0 + tid] : 0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == EPIW) {
        if (lane == 0) {            // producer
            // one TMA box per B slab (the eight slices, 8 BN rows) and per A unit (two slices, 32 KB).
            // Double-buffered B: B(0); then per slab s: A units 0 and 1, B(s + 1) (once slab s - 1 has
            // released its buffer), A units 2 and 3, so the next slab's B loads during slab s's MMAs.
            // Single buffer: B(s) once slab s - 1 has released it.
            constexpr int NU = OZ_S / OZ_UNIT;
            int nb = 0, q = 0;      // B slabs and A units issued
            bool ok = true;
            auto issue_b = [&](int sb) {
                const int bb = bslot(sb);
                mbar_expect_tx(smem_u32(&bfull[bb]), (uint32_t)(OZ_S * SLAB_B));
                oz_tma_load(sB(bb, 0), &p.tb, sb * OZ_KS, n0, bl * OZ_S, smem_u32(&bfull[bb]));
                nb = sb + 1;
            };
            if (nslab > 0) issue_b(0);
            for (int s = 0; s < nslab && ok; s++) {
                if (!BDBL && s > 0) {
                    if (!mbar_wait_or_abort(smem_u32(&bempty[0]), bphase(s - 1), p.err)) { ok = false; break; }
                    issue_b(s);
                }
                for (int u = 0; u < NU; u++) {
                    if (BDBL && u == NU / 2 && s + 1 < nslab) {
                        if (s >= 1 && !mbar_wait_or_abort(smem_u32(&bempty[(s + 1) & 1]), bphase(s - 1), p.err)) {
                            ok = false;
                            break;
                        }
                        issue_b(s + 1);
                    }
                    const int slot = q % RING;
                    if (q >= RING &&
                        !mbar_wait_or_abort(smem_u32(&aempty[slot]), (uint32_t)(((q / RING) - 1) & 1), p.err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(&afull[slot]), (uint32_t)(OZ_UNIT * OZ_SLAB_A));
                    oz_tma_load(sA(slot), &p.ta, s * OZ_KS, m0, bl * OZ_S + OZ_UNIT * u, smem_u32(&afull[slot]));
                    q++;
                }
                if (*(volatile int*)&abort_flag) ok = false;
            }
            if (!ok) abort_flag = 1;
            // every load issued has landed before the CTA can leave
            for (int x = (nb > NB ? nb - NB : 0); x < nb; x++)
                mbar_wait(smem_u32(&bfull[bslot(x)]), bphase(x), p.err);
            for (int x = (q > RING ? q - RING : 0); x < q; x++)
                mbar_wait(smem_u32(&afull[x % RING]), (uint32_t)((x / RING) & 1), p.err);
        }
    } else if (warp == EPIW + 1) {
        if (lane == 0) {            // MMA issuer
            constexpr int MAXB = 256 / BN;             // B slices per MMA (N <= 256)
            // descriptors of slot 0 / buffer 0 slice 0; other slabs offset the 16-byte address field
            const uint64_t dA0 = tma_smem_desc(sA(0)), dB0 = tma_smem_desc(sB(0, 0));
            int q = 0;
            bool ok = true;
            for (int s = 0; s < nslab && ok; s++) {
                const int bb = bslot(s);
                if (!mbar_wait_or_abort(smem_u32(&bfull[bb]), bphase(s), p.err)) {
                    ok = false;
                    break;
                }
                const int kv = min(OZ_KS, g.k - s * OZ_KS);
                const int nk16 = (kv + 15) / 16;
                const uint64_t dB = dB0 + (uint64_t)((bb * OZ_S * SLAB_B) >> 4);
                for (int u = 0; u < OZ_S / OZ_UNIT; u++, q++) {
                    const int slot = q % RING;
                    if (!mbar_wait_or_abort(smem_u32(&afull[slot]), (uint32_t)((q / RING) & 1), p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                    for (int h = 0; h < OZ_UNIT; h++) {
                        const int i = oz_order(OZ_UNIT * u + h);
                        const uint64_t da = dA0 + (uint64_t)(((slot * OZ_UNIT + h) * OZ_SLAB_A) >> 4);
                        // the first slice (i = 0, taken first) opens every group's accumulator
                        const uint32_t first = (s == 0 && u == 0 && h == 0) ? 1u : 0u;
                        // products (i, j), j = 0 .. 7 - i, land in groups i .. 7: adjacent 64-column
                        // accumulators, and the B slices j are adjacent 64-row blocks in shared
                        // memory, so one MMA of N = 64 (8 - i) (at most 256 per instruction) covers them
#pragma unroll
                        for (int kk = 0; kk < OZ_KS / 16; kk++) {
                            if (kk < nk16) {
#pragma unroll
                                for (int c = 0; c < OZ_S; c += MAXB) {
                                    const int nb = min(MAXB, OZ_S - i - c);
                                    if (nb > 0) {
                                        const uint32_t acc = tmem + (uint32_t)((i + c) * BN);
                                        const uint64_t db = dB + (uint64_t)((c * SLAB_B) >> 4) + 2 * kk;
                                        tc_mma(acc, da + 2 * kk, db, tc_idesc(TC_BF16, BN * nb),
                                               (first && kk == 0) ? 0u : 1u, TC_BF16);
                                    }
                                }
                            }
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&aempty[slot])) : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(&bempty[bb])) : "memory");
                if (s == nslab - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&tfull)) : "memory");
                if (*(volatile int*)&abort_flag) ok = false;
            }
            if (!ok) abort_flag = 1;
            // every MMA issued has completed before TMEM is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&done)) : "memory");
            mbar_wait(smem_u32(&done), 0u, p.err);
        }
    } else {
        // epilogue: warps 0 .. EPIW - 1.  Warp w drains TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 (output
        // rows) for the columns of part w / 4; the store pass gives thread tid the elements tid + 32 EPIW q.
        constexpr int NE = 32 * EPIW, PER = OZ_BM * BN / NE;
        const double* Cinb = g.Cin ? g.Cin[b] + g.offCin : nullptr;
        const double* Cin2b = g.Cin2 ? g.Cin2[b] + g.offCin : nullptr;
        double* Cb = g.C[b] + g.offC;
        const bool skew = g.mode == GEMM_SKEW, gj = g.mode == GEMM_GJ;
        bool ok = true;
        if (nslab > 0) {
            if (tid == 0) {
                // the range of the tile's nonzero column exponent fields (for the normal-range test)
                int lo = 4096, hi = 0;
                for (int c = 0; c < BN; c++)
                    if (col_e[c] > 0) { lo = min(lo, col_e[c]); hi = max(hi, col_e[c]); }
                s_fcmin = lo;
                s_fcmax = hi;
                s_ok = mbar_wait_or_abort(smem_u32(&tfull), 0u, p.err) ? 1 : 0;
            }
            asm volatile("bar.sync 1, %0;" :: "n"(NE) : "memory");
            ok = s_ok != 0;
        }
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // every MMA has completed, so every load has been consumed: the stage buffers
            // become the (padded) FP64 output tile
            double* tile = reinterpret_cast<double*>(oz_smem_raw + (sbase - raw));
            // Cin's tile is copied into the free stage memory after the output tile with cp.async,
            // overlapping the drain and combination (a barrier does not wait for these asynchronous
            // copies, unlike ordinary loads); rows must start on 16 bytes, else the store pass reads
            // Cin itself.  Cin may be C itself: every Cin element is read before this CTA stores any.
            double* cin_s = tile + OZ_BM * TS;
            const bool use_cin = Cinb && (!active || g.beta != 0.0);
            const bool ct = g.cin_trans != 0;
            const bool cin_async = use_cin && ((reinterpret_cast<uintptr_t>(Cinb) & 15) == 0) &&
                                   ((g.ldcin & 1) == 0);
            // transposed Cin: element (rr, cc) at cin_s[cc OZ_BM + (rr ^ 2 (cc & 7))], copied 16 bytes
            // (two rows) at a time along the memory rows; the swizzle spreads the reads of consecutive
            // cc over eight bank pairs
            // one load at an integer-selected index (a select between two loaded doubles would issue
            // on the FP64 pipe)
            auto cin_smem = [&](int rr, int cc) {
                return cin_s[ct ? cc * OZ_BM + (rr ^ ((cc & 7) << 1)) : rr * BN + cc];
            };
            if (cin_async && ct) {
                for (int x = tid; x < BN * (OZ_BM / 2); x += NE) {
                    const int cc = x / (OZ_BM / 2), rp = 2 * (x % (OZ_BM / 2)), r = m0 + rp, c = n0 + cc;
                    const uint32_t bytes = c < g.n ? (r + 1 < g.m ? 16u : (r < g.m ? 8u : 0u)) : 0u;
                    const double* src = bytes ? Cinb + (long long)c * g.ldcin + r : Cinb;
                    cp_async16(smem_u32(cin_s + cc * OZ_BM + (rp ^ ((cc & 7) << 1))), src, bytes);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            } else if (cin_async) {
                for (int x = tid; x < OZ_BM * (BN / 2); x += NE) {
                    const int rr = x / (BN / 2), c = n0 + 2 * (x % (BN / 2)), r = m0 + rr;
                    const uint32_t bytes = r < g.m ? (c + 1 < g.n ? 16u : (c < g.n ? 8u : 0u)) : 0u;
                    const double* src = bytes ? Cinb + (long long)r * g.ldcin + c : Cinb;
                    cp_async16(smem_u32(cin_s + rr * BN + (c - n0)), src, bytes);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            const double alpha = g.alpha * (g.alpha_b ? g.alpha_b[b] : 1.0);
            constexpr int PCOLS = BN / (EPIW / 4);                 // columns per warp
            static_assert(PCOLS % 8 == 0, "eight-column TMEM loads");
            const int lq = warp & 3, part = warp >> 2;          // lane quarter, column part
            const int rr0 = lq * 32 + lane, row = m0 + rr0;
            const int er = (active && row < g.m) ? p.ea[(size_t)bl * p.m_pad + row] : 0;
            const int ae = p.alpha_pow2 ? p.alpha_e : 0;
            const bool an = p.alpha_pow2 && p.alpha_neg;
            // every result of this warp's rows is a normal number: with e = er + fc - 2107 + ae and
            // the leading bit P of |V| in 0 .. 74, the biased exponent P + e + 1023 stays in 1 .. 2046
            // (rows or columns with a zero exponent field give zeros either way); then the
            // combination takes the form without the range-end selects (the same bits)
            const bool row_normal = er == 0 || s_fcmax == 0 ||
                                    (er + s_fcmin - 2107 + ae + 1023 >= 1 && er + s_fcmax - 2107 + ae + 1023 + 74 <= 2046);
            const bool fast = __all_sync(0xffffffffu, row_normal);
            if (nslab > 0) {
                // eight columns per pass: one 8-column TMEM load per group, then eight independent
                // combinations
#pragma unroll 1
                for (int cb = part * (PCOLS / 8); cb < (part + 1) * (PCOLS / 8); cb++) {
                    uint32_t u[OZ_G][8];
#pragma unroll
                    for (int G = 0; G < OZ_G; G++) {
                        const uint32_t ta = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(G * BN + cb * 8);
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(u[G][0]), "=r"(u[G][1]), "=r"(u[G][2]), "=r"(u[G][3]),
                                       "=r"(u[G][4]), "=r"(u[G][5]), "=r"(u[G][6]), "=r"(u[G][7])
                                     : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        // computed for every column and selected (no branch between the columns)
                        const int c = cb * 8 + j, fc = col_e[c];
                        long long H;
                        unsigned L;
                        oz_combine(u, j, H, L);
                        const unsigned long long v = fast ? oz_to_double_bits_normal(H, L, er + fc - 2107 + ae, an)
                                                          : oz_to_double_bits(H, L, er + fc - 2107 + ae, an);
                        reinterpret_cast<unsigned long long*>(tile)[rr0 * TS + c] = (er > 0 && fc > 0) ? v : 0ull;
                    }
                }
            }
            if (cin_async) asm volatile("cp.async.wait_all;" ::: "memory");
            asm volatile("bar.sync 1, %0;" :: "n"(NE) : "memory");
            const bool scale_cin = active && g.beta != 1.0;          // beta = 1 (the in-place updates): no product
            // Cin(r, c) = -Cin^T: the sign bit flipped by an integer XOR, then the one addition
            const unsigned long long cin_sign = (active && ct && g.beta == -1.0) ? 0x8000000000000000ull : 0ull;
            const bool cin_neg = cin_sign != 0ull;
            const bool keep_tile = skew || (active && g.diag != 0.0);
            // an element's final value: kept in the tile for the mirrored block and the diagonal,
            // stored unless its column is one of the Gauss-Jordan panel's
            auto emit = [&](int rr, int cc, int r, int c, double v) {
                if (skew && r == c) v = 0.0;
                if (keep_tile) tile[rr * TS + cc] = v;
                if (!gj || !g.gj_cols || c < g.gj_k0 || c >= g.gj_k0 + g.gj_b) Cb[(long long)r * g.ldc + c] = v;
            };
            // The common forms get loops of their own, so that no FP64 instruction is issued where
            // none is needed (FP64 issues at a small fraction of the integer rate on this part):
            // the plain product, and the in-place update C = Cin + A B.
            if (active && p.alpha_pow2 && !Cin2b && !use_cin) {
#pragma unroll 4
                for (int q = 0; q < PER; q++) {
                    const int e = tid + NE * q, rr = e / BN, cc = e % BN, r = m0 + rr, c = n0 + cc;
                    if (r >= g.m || c >= g.n || (skew && r < c)) continue;
                    emit(rr, cc, r, c, tile[rr * TS + cc]);
                }
            } else if (active && p.alpha_pow2 && !Cin2b && use_cin && (!scale_cin || cin_neg) && cin_async) {
#pragma unroll 4
                for (int q = 0; q < PER; q++) {
                    const int e = tid + NE * q, rr = e / BN, cc = e % BN, r = m0 + rr, c = n0 + cc;
                    if (r >= g.m || c >= g.n || (skew && r < c)) continue;
                    const double t = tile[rr * TS + cc];
                    const bool gj_row = gj && !g.gj_acc && r >= g.gj_k0 && r < g.gj_k0 + g.gj_b;
                    const double ci = __longlong_as_double(__double_as_longlong(cin_smem(rr, cc)) ^ (long long)cin_sign);
                    emit(rr, cc, r, c, gj_row ? t : ci + t);
                }
            } else {
#pragma unroll 4
                for (int q = 0; q < PER; q++) {
                    const int e = tid + NE * q, rr = e / BN, cc = e % BN, r = m0 + rr, c = n0 + cc;
                    if (r >= g.m || c >= g.n || (skew && r < c)) continue;
                    double v = 0.0;
                    if (use_cin && !(active && gj && !g.gj_acc && r >= g.gj_k0 && r < g.gj_k0 + g.gj_b)) {
                        v = cin_async ? cin_smem(rr, cc)
                                      : Cinb[ct ? (long long)c * g.ldcin + r : (long long)r * g.ldcin + c];
                        if (scale_cin) v *= g.beta;
                    }
                    if (active) {
                        if (Cin2b) v = fma(g.beta2, Cin2b[(long long)r * g.ldcin + c], v);
                        double t = tile[rr * TS + cc];
                        if (!p.alpha_pow2) t *= alpha;
                        v += t;
                    }
                    emit(rr, cc, r, c, v);
                }
            }
            if (active && g.diag != 0.0 && !skew) {
                // the diagonal term, added to the stored values of the tile's diagonal elements
                asm volatile("bar.sync 1, %0;" :: "n"(NE) : "memory");
                const int c = n0 + tid, rr = c - m0;
                if (tid < BN && rr >= 0 && rr < OZ_BM && c < g.m && c < g.n &&
                    (!gj || !g.gj_cols || c < g.gj_k0 || c >= g.gj_k0 + g.gj_b))
                    Cb[(long long)c * g.ldc + c] = tile[rr * TS + tid] + g.diag;
            }
            if (skew) {
                // mirrored block: C[c][r] = -C[r][c] below the diagonal, rows of the mirror coalesced
                asm volatile("bar.sync 1, %0;" :: "n"(NE) : "memory");
                for (int e = tid; e < OZ_BM * BN; e += NE) {
                    const int cc = e / OZ_BM, rr = e % OZ_BM;
                    const int r = m0 + rr, c = n0 + cc;
                    if (r >= g.m || c >= g.n || r <= c) continue;
                    Cb[(long long)c * g.ldc + r] = -tile[rr * TS + cc];
                }
            }
        } else if (tid == 0) {
            abort_flag = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == EPIW + 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS));
    }
}

// ---------------------------------------------------------------- host side

inline size_t oz_round(size_t x, size_t a) { return (x + a - 1) / a * a; }

// scratch bytes of one batch entry of an m x n x k product (slices and exponent fields)
inline size_t oz_entry_bytes(int m, int n, int k) {
    const size_t kp = oz_round((size_t)k, 8), mp = oz_round((size_t)m, OZ_BM), np = oz_round((size_t)n, 64);
    return (size_t)OZ_S * 2 * (mp + np) * kp + 4 * (mp + np);
}

// Tensor map of a slice batch [nmat][rows_pad][kp] bf16 with x extent k (zero fill beyond),
// box 64 x box_rows x 1 (128-byte rows, 128-byte swizzle)
inline bool make_slice_map(CUtensorMap* map, const void* base, int k, int kp, int rows_pad, int nmat, int box_rows,
                           int box_planes) {
    TmaEncodeFn fn = tma_encode_fn();
    if (!fn || !base || ((uintptr_t)base & 15) || (kp & 7)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows_pad, (cuuint64_t)nmat};
    const cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * rows_pad * 2};
    const cuuint32_t box[3] = {(cuuint32_t)OZ_KS, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// exponents and slices of one operand, one pass: long contiguous rows a warp per row in
// registers, the others (strided, or short) a block of rows at a time through shared memory
inline bool oz_row_pass(const OzOperand& o) { return !o.strided && o.k >= 256 && o.k <= OZ_KC; }
inline size_t oz_block_smem(int kp) { return (size_t)oz_block_rows(kp) * (kp + 1) * 8; }
inline void oz_prepare(const OzOperand& o, int bc, cudaStream_t st) {
    if (oz_row_pass(o)) {
        oz_row_slice_kernel<<<dim3((o.rows_pad + 7) / 8, bc), 256, 0, st>>>(o);
    } else {
        const int rb = oz_block_rows(o.kp);
        oz_block_slice_kernel<<<dim3((o.rows_pad + rb - 1) / rb, bc), 256, oz_block_smem(o.kp), st>>>(o);
    }
}

// number of output tiles of one batch entry (tile width bn)
inline int oz_tiles(const GemmBatch& g, int bn) {
    const int tmn = (g.m + OZ_BM - 1) / OZ_BM, tnn = (g.n + bn - 1) / bn;
    if (g.mode != GEMM_SKEW) return tmn * tnn;
    int t = 0;
    for (int tm = 0; tm < tmn; tm++) t += std::min((tm + 1) * (OZ_BM / bn), tnn);
    return t;
}

// launches of one product, for launch accounting
inline int oz_launches(const GemmBatch& g, const OzBuf& buf) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0 || g.k <= 0 || !buf.base) return 1;
    int total = 0;
    for (int k0 = 0; k0 < g.k; k0 += OZ_KC) {
        const size_t per = oz_entry_bytes(g.m, g.n, std::min(OZ_KC, g.k - k0));
        const size_t chunk = std::min<size_t>(g.batch, buf.bytes > 8192 ? (buf.bytes - 8192) / per : 0);
        if (chunk == 0) return 1;
        // per batch chunk: one slicing launch per operand and the product
        total += 3 * (int)((g.batch + chunk - 1) / chunk);
    }
    return total;
}

// where the slices and exponent fields of a batch chunk of bc entries of an m x n x k product
// lie in the scratch: A slices [bc][OZ_S][mp][kp] (planes in oz_plane order), B slices
// [bc][OZ_S][np][kp] (natural order), exponent fields [bc][mp] and [bc][np]
struct OzLayout {
    uint16_t* as;
    uint16_t* bs;
    int* ea;
    int* eb;
    int mp, np, kp;
};
inline OzLayout oz_layout(int m, int n, int k, const OzBuf& buf, int bc) {
    OzLayout L;
    L.kp = (int)oz_round(k, 8);
    L.mp = (int)oz_round(m, OZ_BM);
    L.np = (int)oz_round(n, 64);
    const size_t sa = (size_t)OZ_S * L.mp * L.kp * 2, sb = (size_t)OZ_S * L.np * L.kp * 2;
    L.as = reinterpret_cast<uint16_t*>(buf.base);
    L.bs = reinterpret_cast<uint16_t*>(buf.base + oz_round((size_t)bc * sa, 1024));
    L.ea = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(L.bs) + oz_round((size_t)bc * sb, 1024));
    L.eb = L.ea + oz_round((size_t)bc * L.mp, 64);
    return L;
}

// batch entries of one K chunk (k <= OZ_KC) whose slices fit the scratch at once
inline int oz_chunk_entries(const GemmBatch& g, const OzBuf& buf) {
    const size_t per = oz_entry_bytes(g.m, g.n, g.k);
    return (int)std::min<size_t>(g.batch, buf.bytes > 8192 ? (buf.bytes - 8192) / per : 0);
}

// the product kernel on slices in place (layout L) for batch entries b0 .. b0 + bc - 1;
// b_rows: B's slices are its rows (an antisymmetric B), so alpha changes sign
inline cudaError_t oz_product(const GemmBatch& g, const OzLayout& L, int b0, int bc, bool b_rows, int* err,
                              cudaStream_t st) {
    const int bn = g.n <= 16 ? 16 : 32;                  // OZ_NARROW16's or OZ_NARROW's tile width
    OzGemm p;
    std::memset(&p, 0, sizeof(p));
    if (!make_slice_map(&p.ta, L.as, g.k, L.kp, L.mp, bc * OZ_S, OZ_BM, OZ_UNIT) ||
        !make_slice_map(&p.tb, L.bs, g.k, L.kp, L.np, bc * OZ_S, bn, OZ_S))
        return cudaErrorInvalidValue;
    p.g = g; p.b0 = b0; p.m_pad = L.mp; p.n_pad = L.np; p.ea = L.ea; p.eb = L.eb; p.err = err;
    if (b_rows) p.g.alpha = -g.alpha;
    int ex = 0;
    const double fr = std::frexp(p.g.alpha, &ex);
    if (!g.alpha_b && (fr == 0.5 || fr == -0.5)) {
        p.alpha_pow2 = 1; p.alpha_e = ex - 1; p.alpha_neg = p.g.alpha < 0.0;
    }
    if (bn == 16)
        oz_gemm_kernel<OZ_NARROW16>
            <<<dim3(oz_tiles(g, bn), bc), OzCfg<OZ_NARROW16>::THREADS, OzCfg<OZ_NARROW16>::SMEM, st>>>(p);
    else
        oz_gemm_kernel<OZ_NARROW><<<dim3(oz_tiles(g, bn), bc), OzCfg<OZ_NARROW>::THREADS, OzCfg<OZ_NARROW>::SMEM, st>>>(p);
    return cudaGetLastError();
}

// one K chunk (k <= OZ_KC) of the emulated product, in batch chunks that fit the scratch
inline cudaError_t gemm_oz_chunk(const GemmBatch& g, const OzBuf& buf, int* err, cudaStream_t st) {
    const int chunk = oz_chunk_entries(g, buf);
    if (chunk <= 0) return gemm_f64(g, st);
    for (int b0 = 0; b0 < g.batch; b0 += chunk) {
        const int bc = std::min(chunk, g.batch - b0);
        const OzLayout L = oz_layout(g.m, g.n, g.k, buf, bc);
        OzOperand oa{g.A, g.A2, g.sA2, g.offA, g.lda, g.transA ? 1 : 0, g.m, g.k, L.mp, L.kp, b0,
                     g.active_flag, g.active_cmp, L.ea, L.as, 1};
        // an antisymmetric B (not transposed): its K-major columns are its rows negated, so the
        // rows are sliced (contiguous, one pass) and alpha changes sign
        const bool b_rows = g.b_antisym && !g.transB;
        OzOperand ob{g.B, g.B2, g.sB2, b_rows ? g.offBr : g.offB, g.ldb, (g.transB || b_rows) ? 0 : 1, g.n, g.k, L.np,
                     L.kp, b0, g.active_flag, g.active_cmp, L.eb, L.bs, 0};
        oz_prepare(oa, bc, st);
        oz_prepare(ob, bc, st);
        const cudaError_t e = oz_product(g, L, b0, bc, b_rows, err, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The product on operands a producer kernel has already sliced into buf (layout oz_layout of
// the whole batch): k <= OZ_KC, every entry in one chunk (oz_chunk_entries(g, buf) == batch)
inline cudaError_t gemm_oz_presliced(const GemmBatch& g, const OzBuf& buf, int* err, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
    if (g.k <= 0 || g.k > OZ_KC || !buf.base || !err || oz_chunk_entries(g, buf) < g.batch ||
        (g.mode == GEMM_SKEW && g.m != g.n))
        return cudaErrorInvalidValue;
    return oz_product(g, oz_layout(g.m, g.n, g.k, buf, g.batch), 0, g.batch, g.b_antisym && !g.transB, err, st);
}

// the emulated product; K beyond OZ_KC runs as further launches that add onto C (the
// chunks' sums are FP64 roundings).  Falls back to gemm_f64 where there is nothing to
// slice or no scratch for one batch entry.  err: the owner's device error word.
inline cudaError_t gemm_oz(const GemmBatch& g, const OzBuf& buf, int* err, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
    if (g.k <= 0 || !buf.base || !err) return gemm_f64(g, st);
    if (g.mode == GEMM_SKEW && g.m != g.n) return cudaErrorInvalidValue;
    if (oz_entry_bytes(g.m, g.n, std::min(g.k, OZ_KC)) + 8192 > buf.bytes) return gemm_f64(g, st);
    for (int k0 = 0; k0 < g.k; k0 += OZ_KC) {
        GemmBatch h = g;
        h.k = std::min(OZ_KC, g.k - k0);
        h.offA += g.transA ? (long long)k0 * g.lda : k0;
        h.offBr = g.offB + k0;                         // the K range within B's rows (antisymmetric B)
        h.offB += g.transB ? k0 : (long long)k0 * g.ldb;
        if (k0 > 0) {
            h.Cin = (const double* const*)g.C; h.offCin = g.offC; h.ldcin = g.ldc; h.beta = 1.0;
            h.Cin2 = nullptr; h.beta2 = 0.0; h.diag = 0.0;
            h.gj_acc = 1;          // a Gauss-Jordan update's pivot rows hold the first chunk's product now
        }
        const cudaError_t e = gemm_oz_chunk(h, buf, err, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sgs
