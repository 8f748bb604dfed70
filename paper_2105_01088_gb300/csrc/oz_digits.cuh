// Digits of the emulated FP64 products (the Ozaki scheme, gemm_oz.cuh): an FP64 value, taken
// as its bit pattern, scaled by its row's exponent field to a 57-bit integer and written as
// eight balanced base-128 digits, each exact in bf16.  Shared by the slicing kernels and by
// kernels that write the slices of their own outputs (the Pfaffian panel).
#pragma once
#include "common.cuh"

namespace sgs {

#define OZ_S 8                // slices per operand

// Order in which the A slices of a slab are taken: 0 first (it opens every accumulator),
// then long and short rows of the product triangle in pairs, (0, 7) (1, 6) (2, 5) (3, 4):
// every pair feeds nine 64-column groups.  A operands store slice oz_order(t) in plane t,
// so that each pair is two adjacent planes, one TMA box.
__host__ __device__ __forceinline__ int oz_order(int t) {
    return (t & 1) ? (OZ_S - 1 - (t >> 1)) : (t >> 1);       // 0 7 1 6 2 5 3 4
}
__host__ __device__ __forceinline__ int oz_plane(int i) {
    return i < OZ_S / 2 ? 2 * i : 2 * (OZ_S - 1 - i) + 1;     // inverse of oz_order
}

// The slicers carry the operand as 64-bit bit patterns: they only take its exponent field and
// significand apart, and double-typed selects and moves of the loaded values cost issue
// slots of the FP64 pipe, which issues at a small fraction of the integer rate on this part.
__device__ __forceinline__ int oz_expo_field(unsigned long long u) {
    int e = (int)((u >> 52) & 0x7ff);
    if (e == 0 && (u << 1) != 0ull) e = 1;       // subnormal: scale of the smallest normal
    return e;
}

// X = round(v 2^(1078 - E)) (E = the row's exponent field, E > 0), |X| <= 2^56, rounded half
// up on the magnitude, from the bit pattern
__device__ __forceinline__ long long oz_scaled(unsigned long long u, int E) {
    int f = (int)((u >> 52) & 0x7ff);
    unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    if (f == 0) f = 1;
    else m |= 1ull << 52;
    const int sh = f - E + 3;                     // v 2^(1078 - E) = m 2^sh, sh <= 3
    unsigned long long a;
    if (sh >= 0) a = m << sh;
    else if (sh <= -63) a = 0;
    else a = (m + (1ull << (-sh - 1))) >> (-sh);
    const long long X = (long long)a;
    return (u >> 63) ? -X : X;
}

// The eight balanced base-128 digits of X (|t_0| <= 128, t_i in [-64, 63] for i >= 1) as
// floats, most significant first.  Offset form: with Y = X + sum_{j<7} 64 2^(7 j), the
// fields u_j = (Y >> 7 j) & 127 are the low digits plus 64 (no carries cross them) and
// Y >> 49 (arithmetic) is the top digit; a low digit reaches float as the float 2^23 + u_j
// (built by OR-ing u_j into the pattern of 2^23) less 2^23 + 64, an exact FP32 subtraction.
// Each digit has at most 8 significant bits, so a float's high half is its exact bf16.
__device__ __forceinline__ void oz_digit_floats(unsigned long long v, int E, float f[OZ_S]) {
    const long long Y = oz_scaled(v, E) + 0x1020408102040ll;
    f[0] = (float)(int)(Y >> 49);
#pragma unroll
    for (int i = 1; i < OZ_S; i++) {
        const unsigned u = (unsigned)(Y >> (7 * (OZ_S - 1 - i))) & 127u;
        f[i] = __uint_as_float(0x4B000000u | u) - 8388672.0f;
    }
}

}  // namespace sgs
