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
