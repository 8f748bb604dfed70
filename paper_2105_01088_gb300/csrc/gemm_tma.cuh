// Batched tensor-core GEMM fed by the Tensor Memory Accelerator (sm_103a):
// C_b = alpha * A_b B_b for the mixed-precision equation of motion, A_b row-major
// (m x k) and B_b given K-major (the row-major n x k matrix B_b^T; every B of the
// equation of motion is antisymmetric, so its K-major form is -B and the sign goes
// into alpha).
//
// Operands live in contiguous batches [batch][rows][ld] (ld a multiple of 8
// elements, so every row starts on a 16-byte boundary) and are described by one
// 3-D tensor map each.  A CTA owns a 128 x 128 output tile:
//   * thread 0 (warp 0) is the producer: per 128-byte slab of K it arms the
//     stage's "full" mbarrier with the stage's byte count and issues
//     cp.async.bulk.tensor loads of the A and B boxes (128 rows x 128 bytes,
//     128-byte swizzle, zero fill outside the matrix);
//   * thread 32 (warp 1) issues tcgen05.mma on the landed stage (K-major
//     128B-swizzled shared-memory descriptors, accumulator in TMEM) and commits
//     the stage's "empty" mbarrier, so the producer can refill it;
//   * all four warps drain TMEM with tcgen05.ld into a padded shared tile and
//     store it with coalesced rows (and, for an antisymmetric result, the
//     mirrored -C^T rows).
// Every mbarrier wait is bounded (2 s); on a timeout the kernel records
// SGS_DEV_TC_TIMEOUT, waits (bounded) for its own loads in flight and for its
// MMAs, frees TMEM and returns.
#pragma once
#include <cuda.h>
#include <mutex>
#include "tcgen05.cuh"

namespace sgs {

#define TMA_BM 128
#define TMA_BN 128

struct TmaBatch {
    CUtensorMap ta, tb, ta2, tb2;   // A, B^T (and lo parts for 3xTF32): [batch][rows][ld]
    int m, n, k;
    double alpha;
    void* C;                        // output base; batch b at C + b * c_stride elements
    long long c_stride;
    int ldc;
    int out_f64;                    // 1: doubles, 0: floats
    int skew;                       // 1: lower tiles only, write C and -C^T, zero diagonal
    int* err;
    int batch;
    // optional epilogue terms (fp32 output, skew = 0): C = alpha A B + beta Cin + diag I,
    // and a transposed copy CT = C^T
    const float* Cin; long long cin_stride; int ldcin; float beta; float diag;
    float* CT; long long ct_stride; int ldct;
    // optional pass-through: batch b with pass_flag[b] <= pass_cmp skips the product and
    // copies Cin (C = Cin, CT = Cin^T)
    const int* pass_flag; int pass_cmp;
};

template <int KIND> struct TmaCfg {
    static constexpr int NS = (KIND == TC_3XTF32) ? 2 : 1;          // operand pairs per stage
    static constexpr int SLAB = 128 * 128;                           // bytes of one 128 x 128-byte box
    static constexpr int STAGE = NS * 2 * SLAB;
    static constexpr int NST = (KIND == TC_3XTF32) ? 2 : 3;          // pipeline depth
    static constexpr int SMEM = NST * STAGE + 1024;                  // + alignment slack
};

// K-major operand in the canonical 128-byte-swizzle layout: rows of 128 bytes,
// 8-row atoms of 1024 bytes (stride byte offset), leading byte offset unused.
__device__ __forceinline__ uint64_t tma_smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (ignored for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                  // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}

// bounded wait that also gives up as soon as another CTA has recorded a timeout (so a
// failing launch drains quickly); used only where giving up leaves nothing in flight
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, int* err) {
    return bounded_wait([&] { return mbar_try_wait(bar, parity); }, SGS_WAIT_LIMIT_NS, err, true);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(128) gemm_tma_kernel(const __grid_constant__ TmaBatch g) {
    using Cfg = TmaCfg<KIND>;
    using T = typename std::conditional<KIND == TC_BF16, __nv_bfloat16, float>::type;
    constexpr int NST = Cfg::NST, SLAB = Cfg::SLAB, STAGE = Cfg::STAGE, NS = Cfg::NS;
    constexpr int KSLAB = 128 / sizeof(T);                  // K elements per 128-byte row
    constexpr int KMMA = (KIND == TC_BF16) ? 16 : 8;        // K per instruction (32 bytes)
    constexpr int NMMA = KSLAB / KMMA;                      // 4
    constexpr uint32_t IDESC = tc_idesc(KIND, TMA_BN);
    extern __shared__ uint8_t tma_smem_raw[];
    __shared__ uint64_t full[NST], empty[NST], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    __shared__ int skip;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a launch that already recorded a timeout does no further work (decided once, uniformly)
    if (tid == 0) skip = (*(volatile int*)g.err & SGS_DEV_TC_TIMEOUT) != 0;
    __syncthreads();
    if (skip) return;
    const int b = blockIdx.y;
    int tm, tn;
    if (g.skew) {
        const int t = blockIdx.x;
        tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
        while (tm * (tm + 1) / 2 > t) --tm;
        tn = t - tm * (tm + 1) / 2;
    } else {
        const int ntn = (g.n + TMA_BN - 1) / TMA_BN;
        tm = blockIdx.x / ntn;
        tn = blockIdx.x % ntn;
    }
    const int m0 = tm * TMA_BM, n0 = tn * TMA_BN;
    const uint32_t raw = smem_u32(tma_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;           // 1024-byte atoms of the swizzle
    uint8_t* gbase = tma_smem_raw + (sbase - raw);
    auto sA = [&](int s, int part) { return sbase + s * STAGE + part * SLAB; };
    auto sB = [&](int s, int part) { return sbase + s * STAGE + (NS + part) * SLAB; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"((uint32_t)TMA_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const bool pass = g.pass_flag && g.pass_flag[b] <= g.pass_cmp;     // uniform in the CTA
    const int nk = pass ? 0 : (g.k + KSLAB - 1) / KSLAB;

    if (tid == 0) {
        // producer
        int issued = 0;
        for (int kt = 0; kt < nk; kt++) {
            const int s = kt % NST;
            if (kt >= NST && !mbar_wait_or_abort(smem_u32(&empty[s]), (uint32_t)((kt / NST - 1) & 1), g.err)) {
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            mbar_expect_tx(smem_u32(&full[s]), (uint32_t)STAGE);
            const int kx = kt * KSLAB;
            tma_load_3d(sA(s, 0), &g.ta, kx, m0, b, smem_u32(&full[s]));
            tma_load_3d(sB(s, 0), &g.tb, kx, n0, b, smem_u32(&full[s]));
            if (KIND == TC_3XTF32) {
                tma_load_3d(sA(s, 1), &g.ta2, kx, m0, b, smem_u32(&full[s]));
                tma_load_3d(sB(s, 1), &g.tb2, kx, n0, b, smem_u32(&full[s]));
            }
            issued = kt + 1;
        }
        // every load this thread issued has landed before the CTA can leave
        for (int kt = (issued > NST ? issued - NST : 0); kt < issued; kt++)
            mbar_wait(smem_u32(&full[kt % NST]), (uint32_t)((kt / NST) & 1), g.err);
    } else if (tid == 32) {
        // MMA issuer
        for (int kt = 0; kt < nk; kt++) {
            const int s = kt % NST;
            if (!mbar_wait_or_abort(smem_u32(&full[s]), (uint32_t)((kt / NST) & 1), g.err)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int j = 0; j < NMMA; j++) {
                const uint32_t koff = j * 32;                 // 32 bytes of K per instruction
                const uint64_t da = tma_smem_desc(sA(s, 0) + koff);
                const uint64_t db = tma_smem_desc(sB(s, 0) + koff);
                tc_mma(tmem, da, db, IDESC, (kt > 0 || j > 0) ? 1u : 0u, KIND);
                if (KIND == TC_3XTF32) {
                    tc_mma(tmem, da, tma_smem_desc(sB(s, 1) + koff), IDESC, 1u, KIND);   // hi * lo
                    tc_mma(tmem, tma_smem_desc(sA(s, 1) + koff), db, IDESC, 1u, KIND);   // lo * hi
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[s])) : "memory");
        }
        // arrives once every MMA issued above has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&done)) : "memory");
    }
    __syncthreads();
    bool ok = mbar_wait(smem_u32(&done), 0u, g.err);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok && abort_flag == 0 && (nk > 0 || pass));

    if (ok) {
        // TMEM (or, passing through, Cin) -> padded shared tile (row stride 129 floats:
        // conflict-free both ways)
        float* tile = reinterpret_cast<float*>(gbase);
        constexpr int TS = TMA_BN + 1;
        const int r = warp * 32 + lane;
        if (pass) {
            for (int e = tid; e < TMA_BM * TMA_BN; e += 128) {
                const int rr = e / TMA_BN, cc = e % TMA_BN;
                const int row = m0 + rr, col = n0 + cc;
                tile[rr * TS + cc] = (row < g.m && col < g.n)
                                         ? g.Cin[(size_t)b * g.cin_stride + (size_t)row * g.ldcin + col] : 0.0f;
            }
        }
        for (int c0 = 0; c0 < TMA_BN && !pass; c0 += 32) {
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
#pragma unroll
            for (int j = 0; j < 32; j++) tile[r * TS + c0 + j] = __uint_as_float(v[j]);
        }
        __syncthreads();
        // fp32 epilogue (FP64 arithmetic is slow on this part)
        const float alpha = pass ? 1.0f : (float)g.alpha;
        const bool extra = !pass && (g.Cin || g.diag != 0.0f);
        auto put = [&](int row, int col, float x) {
            if (g.out_f64) static_cast<double*>(g.C)[(size_t)b * g.c_stride + (size_t)row * g.ldc + col] = (double)x;
            else static_cast<float*>(g.C)[(size_t)b * g.c_stride + (size_t)row * g.ldc + col] = x;
        };
        for (int e = tid; e < TMA_BM * TMA_BN; e += 128) {
            const int rr = e / TMA_BN, cc = e % TMA_BN;
            const int row = m0 + rr, col = n0 + cc;
            if (row >= g.m || col >= g.n) continue;
            if (!g.skew || tm != tn) {
                float x = alpha * tile[rr * TS + cc];
                if (extra) {
                    if (g.Cin) x += g.beta * g.Cin[(size_t)b * g.cin_stride + (size_t)row * g.ldcin + col];
                    if (row == col) x += g.diag;
                    tile[rr * TS + cc] = x;            // kept for the transposed copy
                }
                put(row, col, x);
            } else {       // diagonal tile: lower part from the tile, upper part mirrored, zero diagonal
                put(row, col, rr > cc ? alpha * tile[rr * TS + cc] : (rr < cc ? -alpha * tile[cc * TS + rr] : 0.0f));
            }
        }
        if (g.CT) {
            // CT[n0 + cc][m0 + rr] = C[m0 + rr][n0 + cc], rows of CT coalesced
            __syncthreads();
            const float a2 = extra ? 1.0f : alpha;
            for (int e = tid; e < TMA_BM * TMA_BN; e += 128) {
                const int cc = e / TMA_BM, rr = e % TMA_BM;
                const int row = n0 + cc, col = m0 + rr;
                if (row >= g.n || col >= g.m) continue;
                g.CT[(size_t)b * g.ct_stride + (size_t)row * g.ldct + col] = a2 * tile[rr * TS + cc];
            }
        }
        if (g.skew && tm != tn) {
            // mirrored block: C[n0 + cc][m0 + rr] = -C[m0 + rr][n0 + cc], rows of the mirror coalesced
            for (int e = tid; e < TMA_BM * TMA_BN; e += 128) {
                const int cc = e / TMA_BM, rr = e % TMA_BM;
                const int row = n0 + cc, col = m0 + rr;
                if (row >= g.n || col >= g.m) continue;
                put(row, col, -alpha * tile[rr * TS + cc]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)TMA_BN));
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*TmaEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline TmaEncodeFn tma_encode_fn() {
    static TmaEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TmaEncodeFn>(p);
    });
    return fn;
}

// Tensor map of a contiguous operand batch [batch][rows][ld] (ld in elements, a multiple
// of 8; rows start on 16-byte boundaries), box = 128 bytes of K x 128 rows, 128-byte swizzle.
inline bool make_operand_map(CUtensorMap* map, const void* base, bool bf16, int ld, int rows, int batch) {
    TmaEncodeFn fn = tma_encode_fn();
    if (!fn || !base || (ld & 7) || ((uintptr_t)base & 15)) return false;
    const cuuint64_t esz = bf16 ? 2 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * esz, (cuuint64_t)ld * rows * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(128 / esz), 128u, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND>
inline cudaError_t gemm_tma_launch(const TmaBatch& g, cudaStream_t st) {
    const int tmn = (g.m + TMA_BM - 1) / TMA_BM, tnn = (g.n + TMA_BN - 1) / TMA_BN;
    const unsigned gx = g.skew ? (unsigned)(tmn * (tmn + 1) / 2) : (unsigned)(tmn * tnn);
    gemm_tma_kernel<KIND><<<dim3(gx, g.batch), 128, TmaCfg<KIND>::SMEM, st>>>(g);
    return cudaGetLastError();
}

inline cudaError_t gemm_tma(const TmaBatch& g, int kind, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
    if (g.skew && g.m != g.n) return cudaErrorInvalidValue;
    switch (kind) {
        case TC_TF32: return gemm_tma_launch<TC_TF32>(g, st);
        case TC_BF16: return gemm_tma_launch<TC_BF16>(g, st);
        default: return gemm_tma_launch<TC_3XTF32>(g, st);
    }
}

}  // namespace sgs
