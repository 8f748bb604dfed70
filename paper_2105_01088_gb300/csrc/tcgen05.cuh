// Shared pieces of the 5th-generation tensor-core (tcgen05, sm_103a) kernels:
// the operand kinds, the instruction descriptor (fp32 accumulator, K-major A and
// B, M = 128), the MMA issue, cp.async and the bounded mbarrier wait that every
// pipeline wait goes through (2 s of wall time, then the error word).
//
// Operand precision: kind::tf32 reads fp32 operands (10-bit mantissa), kind::f16
// with bf16 operands; accumulation is fp32 in TMEM.  The 3xTF32 form issues
// hi*hi, hi*lo, lo*hi products from split operand arrays into one accumulator.
#pragma once
#include <cuda_bf16.h>
#include <type_traits>
#include "common.cuh"

namespace sgs {

#define TC_BM 128
#define SGS_DEV_TC_TIMEOUT 16

enum TcKind { TC_TF32 = 0, TC_BF16 = 1, TC_3XTF32 = 2 };



__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// instruction descriptor: fp32 accumulator, A/B K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t tc_idesc(int kind, int bn) {
    return (1u << 4)                                              // D format f32
         | ((kind == TC_BF16 ? 1u : 2u) << 7)                      // A format: bf16 (f16 kind) / tf32
         | ((kind == TC_BF16 ? 1u : 2u) << 10)                     // B format
         | ((uint32_t)(bn >> 3) << 17)                             // N >> 3
         | ((uint32_t)(TC_BM >> 4) << 24);                         // M >> 4
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum,
                                       int kind) {
    if (kind == TC_BF16) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                     :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                     :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(dst), "l"(src), "r"(bytes));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every wait of the library's device code is bounded: `done()` is polled until it holds or
// limit_ns of wall time (the global timer) have passed; then SGS_DEV_TC_TIMEOUT is set in the
// error word and the wait returns false, and the caller drains its own work and returns.
// With abort_on_flag, a wait also gives up once another thread of the launch has recorded a
// timeout (checked every 256 polls).
constexpr uint64_t SGS_WAIT_LIMIT_NS = 2000000000ull;     // pipeline waits: 2 s

template <class Done>
__device__ __forceinline__ bool bounded_wait(Done done, uint64_t limit_ns, int* err, bool abort_on_flag) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; it++) {
        if (done()) return true;
        if ((it & 255u) == 255u) {
            if (abort_on_flag && (*(volatile int*)err & SGS_DEV_TC_TIMEOUT)) return false;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    atomicOr(err, SGS_DEV_TC_TIMEOUT);
    return false;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

// bounded wait on an mbarrier phase (2 s); returns false and sets the error word on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    return bounded_wait([&] { return mbar_try_wait(bar, parity); }, SGS_WAIT_LIMIT_NS, err, false);
}

// A wait on a flag in global memory that nothing sets, bounded by limit_ns: the failure
// path every pipeline wait takes, run on its own (sgs_probe_wait).  One thread waits and
// records the timeout; the launch then returns like a timed-out pipeline.
__global__ void wait_probe_kernel(const int* flag, unsigned long long limit_ns, int* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bounded_wait([&] { return *(const volatile int*)flag != 0; }, limit_ns, err, false);
}

}  // namespace sgs
