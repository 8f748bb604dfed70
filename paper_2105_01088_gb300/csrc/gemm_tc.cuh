// Batched GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) for the
// mixed-precision equation of motion: C_b = alpha * A_b B_b with A_b row-major
// (M x K, K contiguous) and B_b given K-major, i.e. as the row-major N x K
// matrix B_b^T.  Every B of the equation of motion is antisymmetric, so its
// K-major form is -B itself and the sign is folded into alpha by the caller.
//
// Tile 128 x BN x 32 (TF32: four K=8 MMAs; BF16: two K=16 MMAs per 32-element
// slab), one CTA of 4 warps.  Operands are staged by cp.async into the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices, leading
// byte offset 128 between core matrices along K, stride byte offset 1024
// between 8-row groups), two stages.  Thread 0 issues tcgen05.mma into a TMEM
// accumulator (128 lanes x BN fp32 columns) and commits each stage to an
// mbarrier; all mbarrier waits are bounded and report through the error word.
// The epilogue drains TMEM with tcgen05.ld (warp w owns lanes 32w..32w+31).
//
// Operand precision: kind::tf32 reads fp32 operands (10-bit mantissa), kind::f16
// with bf16 operands; accumulation is fp32 in TMEM.  The 3xTF32 variant issues
// hi*hi, hi*lo, lo*hi products from split operand arrays into one accumulator.
#pragma once
#include <cuda_bf16.h>
#include <type_traits>
#include "common.cuh"

namespace sgs {

#define TC_BM 128
#define TC_BK 32                     // elements of K per stage (fp32: 128 B per row)
#define SGS_DEV_TC_TIMEOUT 16

enum TcKind { TC_TF32 = 0, TC_BF16 = 1, TC_3XTF32 = 2 };

struct TcBatch {
    int m, n, k;
    const void* const* A;  int lda;      // fp32 (or bf16) row-major m x k
    const void* const* B;  int ldb;      // K-major: row-major n x k
    const void* const* A2;               // 3xTF32: lo parts (nullptr otherwise)
    const void* const* B2;
    void* const* C; int ldc;             // output (fp32 or fp64), row-major m x n
    double alpha;
    int out_f64;                         // 1: write doubles, 0: floats
    int skew;                            // 1: compute lower tiles, write C and -C^T, zero diagonal
    int* err;
    int batch;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                 // descriptor version (sm_100 family)
    return d;                                // base offset 0, relative LBO, no swizzle
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait on an mbarrier phase (2 s of wall time); returns false and sets the
// error word on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > 2000000000ull) break;
    }
    atomicOr(err, SGS_DEV_TC_TIMEOUT);
    return false;
}

// One 128 x 32 (or BN x 32) fp32-equivalent slab in core-matrix order:
// element (r, q): group g = r/8, row-in-group rr = r%8, chunk c = q/E (E = 16B / elem size)
//   byte offset = g*1024 + c*128 + rr*16 + (q%E)*elem
template <int ROWS, typename T>
__device__ __forceinline__ void tc_load_slab(uint32_t dst, const T* src, int ld, int row0, int rows, int k0, int kdim,
                                             int tid) {
    constexpr int E = 16 / sizeof(T);          // elements per 16-byte chunk
    constexpr int CH = TC_BK * 4 / 16;         // 16-byte chunks per row of a 128-byte slab = 8
    constexpr int KE = CH * E;                 // elements of K per slab row
    for (int e = tid; e < ROWS * CH; e += 128) {
        const int r = e / CH, c = e % CH;
        const int gr = row0 + r, gk = k0 + c * E;
        const bool ok = gr < rows && gk < kdim;
        const T* s = ok ? src + (size_t)gr * ld + gk : src;
        const uint32_t d = dst + (r >> 3) * 1024 + c * 128 + (r & 7) * 16;
        cp_async16(d, s, ok ? 16u : 0u);
    }
    (void)KE;
}

template <int BN, int KIND>
__global__ void __launch_bounds__(128) gemm_tc_kernel(TcBatch g) {
    using T = typename std::conditional<KIND == TC_BF16, __nv_bfloat16, float>::type;
    constexpr int SLAB_A = TC_BM * 128;          // bytes of one 128-row slab (32 fp32 or 64 bf16 of K)
    constexpr int SLAB_B = BN * 128;
    constexpr int NS = (KIND == TC_3XTF32) ? 2 : 1;   // operand pairs per stage (hi, lo)
    constexpr int STAGE = NS * (SLAB_A + SLAB_B);
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.y;
    int tm, tn;
    const int ntn = (g.n + BN - 1) / BN;
    if (g.skew) {
        // lower-triangular tile pairs of a square product (BN == TC_BM)
        int t = blockIdx.x;
        tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
        while (tm * (tm + 1) / 2 > t) --tm;
        tn = t - tm * (tm + 1) / 2;
    } else {
        tm = blockIdx.x / ntn;
        tn = blockIdx.x % ntn;
    }
    const int m0 = tm * TC_BM, n0 = tn * BN;
    uint8_t* base = tc_smem;
    const uint32_t sbase = smem_u32(base);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"((uint32_t)BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    const T* A = static_cast<const T*>(g.A[b]);
    const T* B = static_cast<const T*>(g.B[b]);
    const T* A2 = (KIND == TC_3XTF32) ? static_cast<const T*>(g.A2[b]) : nullptr;
    const T* B2 = (KIND == TC_3XTF32) ? static_cast<const T*>(g.B2[b]) : nullptr;
    constexpr int KSLAB = 128 / sizeof(T);                 // K elements per slab row (32 fp32, 64 bf16)
    const int nk = (g.k + KSLAB - 1) / KSLAB;
    constexpr uint32_t IDESC = tc_idesc(KIND, BN);
    constexpr int KMMA = (KIND == TC_BF16) ? 16 : 8;       // K per instruction
    constexpr int NMMA = KSLAB / KMMA;                     // 4 per slab
    uint32_t phase[2] = {0, 0};
    bool ok = true;

    for (int kt = 0; kt < nk && ok; kt++) {
        const int s = kt & 1;
        if (kt >= 2) {   // stage s is free once the MMAs of slab kt-2 completed
            ok = mbar_wait(smem_u32(&bars[s]), phase[s], g.err);
            phase[s] ^= 1;
            if (!ok) break;
        }
        const uint32_t st = sbase + s * STAGE;
        tc_load_slab<TC_BM, T>(st, A, g.lda, m0, g.m, kt * KSLAB, g.k, tid);
        tc_load_slab<BN, T>(st + NS * SLAB_A, B, g.ldb, n0, g.n, kt * KSLAB, g.k, tid);
        if (KIND == TC_3XTF32) {
            tc_load_slab<TC_BM, T>(st + SLAB_A, A2, g.lda, m0, g.m, kt * KSLAB, g.k, tid);
            tc_load_slab<BN, T>(st + NS * SLAB_A + SLAB_B, B2, g.ldb, n0, g.n, kt * KSLAB, g.k, tid);
        }
        asm volatile("cp.async.commit_group;");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int j = 0; j < NMMA; j++) {
                // advance 2 core matrices (32 bytes of K) per instruction
                const uint32_t koff = j * 2 * 128;
                const uint64_t da = tc_smem_desc(st + koff, 128, 1024);
                const uint64_t db = tc_smem_desc(st + NS * SLAB_A + koff, 128, 1024);
                tc_mma(tmem, da, db, IDESC, (kt > 0 || j > 0) ? 1u : 0u, KIND);
                if (KIND == TC_3XTF32) {
                    const uint64_t da2 = tc_smem_desc(st + SLAB_A + koff, 128, 1024);
                    const uint64_t db2 = tc_smem_desc(st + NS * SLAB_A + SLAB_B + koff, 128, 1024);
                    tc_mma(tmem, da, db2, IDESC, 1u, KIND);     // hi * lo
                    tc_mma(tmem, da2, db, IDESC, 1u, KIND);     // lo * hi
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&bars[s])) : "memory");
        }
        __syncthreads();
    }
    // wait for the last (up to two) commits
    for (int kt = (nk >= 2 ? nk - 2 : 0); kt < nk; kt++) {
        const int s = kt & 1;
        if (!mbar_wait(smem_u32(&bars[s]), phase[s], g.err)) ok = false;
        phase[s] ^= 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok);   // every warp must agree before the warp-collective loads

    // epilogue: warp w drains lanes 32w..32w+31 (tile rows), 32 columns at a time
    if (ok && nk > 0) {
        const int r = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                           "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                           "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                           "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                           "=r"(v[31])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < g.m) {
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const int c = n0 + c0 + j;
                    if (c >= g.n) continue;
                    const float x = (float)g.alpha * __uint_as_float(v[j]);   // alpha is +-1 here
                    if (g.skew) {
                        if (tm == tn && r <= c) {
                            if (r == c) {
                                if (g.out_f64) static_cast<double*>(g.C[b])[(size_t)r * g.ldc + c] = 0.0;
                                else static_cast<float*>(g.C[b])[(size_t)r * g.ldc + c] = 0.0f;
                            }
                            continue;
                        }
                        if (g.out_f64) {
                            static_cast<double*>(g.C[b])[(size_t)r * g.ldc + c] = (double)x;
                            static_cast<double*>(g.C[b])[(size_t)c * g.ldc + r] = -(double)x;
                        } else {
                            static_cast<float*>(g.C[b])[(size_t)r * g.ldc + c] = x;
                            static_cast<float*>(g.C[b])[(size_t)c * g.ldc + r] = -x;
                        }
                    } else {
                        if (g.out_f64) static_cast<double*>(g.C[b])[(size_t)r * g.ldc + c] = (double)x;
                        else static_cast<float*>(g.C[b])[(size_t)r * g.ldc + c] = x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)BN));
    }
}

template <int BN, int KIND>
inline cudaError_t gemm_tc_launch(const TcBatch& g, cudaStream_t st) {
    constexpr int NS = (KIND == TC_3XTF32) ? 2 : 1;
    // the dynamic shared-memory limit is raised once per process by the library, outside stream capture
    constexpr int smem = 2 * NS * (TC_BM * 128 + BN * 128) + 1024;
    const int tmn = (g.m + TC_BM - 1) / TC_BM, tnn = (g.n + BN - 1) / BN;
    const unsigned gx = g.skew ? (unsigned)(tmn * (tmn + 1) / 2) : (unsigned)(tmn * tnn);
    gemm_tc_kernel<BN, KIND><<<dim3(gx, g.batch), 128, smem, st>>>(g);
    return cudaGetLastError();
}

inline cudaError_t gemm_tc(const TcBatch& g, int kind, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
    if (g.skew && g.m != g.n) return cudaErrorInvalidValue;
    switch (kind) {
        case TC_TF32: return gemm_tc_launch<128, TC_TF32>(g, st);
        case TC_BF16: return gemm_tc_launch<128, TC_BF16>(g, st);
        default: return gemm_tc_launch<128, TC_3XTF32>(g, st);
    }
}

}  // namespace sgs
