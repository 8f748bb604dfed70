// Throughput probes of the FP64 pipes, so that the FP64 roofline is measured
// on the device at hand: the m8n8k4 FP64 MMA and plain FP64 FMA (the pipe of
// the FMA-path products and of the factorisations' panels).  Fixed-length
// loops, one store each.
#pragma once
#include "common.cuh"

namespace sgs {

#define PROBE_ITERS 4096

__global__ void __launch_bounds__(256) probe_dmma_kernel(double* out, double s) {
    // 16 independent accumulators per warp (as in the GEMM's 32x32 warp tile), distinct
    // operands per chain: identical chains could be folded by the compiler
    double a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; j++) { a[j] = s + j * 1e-3 + threadIdx.x * 1e-9; b[j] = 1.0 - s - j * 1e-4; }
    double c[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) c[i][j][0] = c[i][j][1] = 0.0;
    for (int it = 0; it < PROBE_ITERS / 16; it++) {
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                             : "+d"(c[i][j][0]), "+d"(c[i][j][1]) : "d"(a[i]), "d"(b[j]));
    }
    double t = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) t += c[i][j][0] + c[i][j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(256) probe_dfma_kernel(double* out, double s) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = threadIdx.x * 1e-9 + j;
    const double b = s, c = 1.0 - s;
    for (int i = 0; i < PROBE_ITERS; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
    }
    double t = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) t += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// half the MMA work of probe_dmma_kernel interleaved with half the FMA work of
// probe_dfma_kernel; distinct operands per chain so nothing folds
__global__ void __launch_bounds__(256) probe_mixed_kernel(double* out, double s) {
    double a[2], b[2], f[8];
#pragma unroll
    for (int j = 0; j < 2; j++) { a[j] = s + j * 1e-3 + threadIdx.x * 1e-9; b[j] = 1.0 - s - j * 1e-4; }
#pragma unroll
    for (int j = 0; j < 8; j++) f[j] = threadIdx.x * 1e-9 + j;
    double c[2][2] = {{0, 0}, {0, 0}};
    for (int i = 0; i < PROBE_ITERS / 4; i++) {
#pragma unroll
        for (int j = 0; j < 2; j++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a[j]), "d"(b[j]));
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) f[j] = fma(f[j], s, 1.0 - s);
    }
    double t = c[0][0] + c[0][1] + c[1][0] + c[1][1];
#pragma unroll
    for (int j = 0; j < 8; j++) t += f[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace sgs
