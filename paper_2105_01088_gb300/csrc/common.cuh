// Shared device helpers for the SGS imaginary-time step (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#define SGS_MAX_IMP 16          // Majoranas touched by quartic terms (impurity block)
#define SGS_MAX_RANK 64         // largest ansatz rank M handled by the amplitude solver

// Device-side error word bits (one int per instance, read back by the host).
#define SGS_DEV_SINGULAR   1    // zero pivot in the Gauss-Jordan inverse (orthogonal pair)
#define SGS_DEV_PF_ZERO    2    // zero pivot in the phase Pfaffian
#define SGS_DEV_EIG        4    // amplitude solver failed to converge / empty subspace
#define SGS_DEV_EXPNORM    8    // exponential step needs more squarings than provisioned

// fp32 -> nearest TF32 value (10 explicit mantissa bits; ties away from zero): add half
// an ulp of TF32 to the magnitude bits, then clear the 13 dropped bits.  The tensor
// core reads a TF32 operand by dropping those bits, i.e. truncating toward zero, a
// bias that accumulates along product chains; operands rounded here carry none.
__device__ __forceinline__ float round_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

struct cplx { double x, y; };
__device__ __forceinline__ cplx cmk(double a, double b) { cplx r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    double d = b.x * b.x + b.y * b.y;
    return cmk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Block-wide argmax of v (value, index); ties resolve to the smaller index.  v is a
// magnitude (non-negative, or NaN with its sign bit clear) or the sentinel -1 of a thread
// without candidates; the values are compared as their bit patterns, which order
// non-negative doubles as the numbers do, in integer instructions (FP64 compares share
// the FP64 pipe, which issues at a small fraction of the integer rate on this part).
// red_v / red_i: shared arrays of at least blockDim.x/32 entries.
__device__ __forceinline__ void block_argmax(double v, int idx, double* red_v, int* red_i,
                                             double& out_v, int& out_i) {
    const unsigned full = 0xffffffffu;
    long long key = __double_as_longlong(v);
    if (key < 0) key = -1;
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_down_sync(full, key, o);
        const int oi = __shfl_down_sync(full, idx, o);
        if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red_v[w] = __longlong_as_double(key); red_i[w] = idx; }
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        key = lane < nw ? __double_as_longlong(red_v[lane]) : -1ll;
        idx = lane < nw ? red_i[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const long long ok = __shfl_down_sync(full, key, o);
            const int oi = __shfl_down_sync(full, idx, o);
            if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; }
        }
        if (lane == 0) { red_v[0] = key < 0 ? -1.0 : __longlong_as_double(key); red_i[0] = idx; }
    }
    __syncthreads();
    out_v = red_v[0];
    out_i = red_i[0];
    __syncthreads();
}

// the magnitude |x| as the bit pattern block_argmax compares (sign bit cleared)
__device__ __forceinline__ long long abs_key(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }

// Block-wide sum of doubles; red: shared array of >= 32 entries.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const unsigned full = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// 32 x 32 tiles on or below the diagonal of an n x n matrix, numbered row by row:
// tile t is (K, L) with K >= L.  The antisymmetric results of the equation of motion
// are computed on these tiles only and mirrored (X_lk = -X_kl, zero diagonal).
__host__ __device__ __forceinline__ int lower_tile_count(int n) {
    const int t = (n + 31) / 32;
    return t * (t + 1) / 2;
}
__device__ __forceinline__ void lower_tile(int t, int& K, int& L) {
    int k = 0;
    while ((k + 1) * (k + 2) / 2 <= t) k++;
    K = k;
    L = t - k * (k + 1) / 2;
}

// Store a 32 x 32 tile of an antisymmetric matrix x (n x n) and its mirror from the
// shared tile s[j][c] = x[k0 + j][l0 + c] (entries valid strictly below the diagonal):
// tile (K, L) directly and tile (L, K) as -s^T; on a diagonal tile (K = L) the upper
// part is the negated transpose and the diagonal zero.  256 threads; the caller
// synchronises before (s complete) and after (s reused).
__device__ __forceinline__ void store_antisym_tile(double* x, int n, int k0, int l0, const double (*s)[33],
                                                   const unsigned char (*have)[33] = nullptr) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int k = k0 + j, l = l0 + tx;
        if (k < n && l < n) {
            if (k0 != l0) {
                if (!have || have[j][tx]) x[(size_t)k * n + l] = s[j][tx];
            } else if (k > l) {
                if (!have || have[j][tx]) x[(size_t)k * n + l] = s[j][tx];
            } else if (k < l) {
                if (!have || have[tx][j]) x[(size_t)k * n + l] = -s[tx][j];
            } else {
                if (!have || have[j][tx]) x[(size_t)k * n + l] = 0.0;
            }
        }
        if (k0 != l0) {
            const int r = l0 + j, c = k0 + tx;       // mirror: x[r][c] = -x[c][r] = -s[tx][j]
            if (r < n && c < n && (!have || have[tx][j])) x[(size_t)r * n + c] = -s[tx][j];
        }
    }
}
