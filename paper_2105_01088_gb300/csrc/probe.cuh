// Throughput probes of the FP64 pipes, so that the FP64 roofline is measured
// on the device at hand: the m8n8k4 FP64 MMA (the path every FP64 product of
// the step takes) and plain FP64 FMA.  Fixed-length loops, one store each.
#pragma once
#include "common.cuh"

namespace sgs {

#define PROBE_ITERS 4096

__global__ void __launch_bounds__(256) probe_dmma_kernel(double* out, double s) {
    double a = s + threadIdx.x * 1e-9, b = 1.0 - s;
    double c[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int i = 0; i < PROBE_ITERS / 4; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a), "d"(b));
    }
    double t = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) t += c[j][0] + c[j][1];
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

}  // namespace sgs
