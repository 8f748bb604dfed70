// Host side of the SGS imaginary-time step library: context, device
// buffers, the per-step launch sequence and the C ABI of include/sgs.h.
//
// One step (Sec. III C) per instance, all on one CUDA stream:
//   pairs:   S = G_a + G_b -> blocked Gauss-Jordan (S^{-1}, log|det S|)
//            Im = (G_a - G_b) S^{-1}                        [Eq. def-delta-matrix]
//            Y = G_0 + Delta^{a,b} -> blocked complex Pfaffian (overlap phase)
//            G_ab, h_ab, impurity block of F^{a,b}          [Sec. II B-C, III B]
//   amplitudes: h lambda = E G lambda                        [Eq. eigLambda]
//   EOM:     W = S^{-1} F S^{-1}, V = D W, X = V D, Q = Delta F Delta,
//            dGamma^mu = sum_beta ...                        [Eq. EOM-Gamma3]
//   update:  R = exp{(ds/4)[G, dG]}, G <- R G R^T, Newton-Schulz polar factor
//                                                            [App. A]
#include "../../include/sgs.h"
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "gemm_f64.cuh"
#include "factor.cuh"
#include "pair.cuh"
#include "eig.cuh"
#include "eom.cuh"
#include "update.cuh"
#include "update_lp.cuh"
#include "probe.cuh"
#include "gemm_oz.cuh"
#include "gemm_tma.cuh"
#include "corr.cuh"
#include "renyi.cuh"
#include "var.cuh"
#include "host_init.hpp"

using namespace sgs;

namespace {

// kernels launched by this library (host-side count; sgs_get_profile reports
// the share of each context)
long long g_launches = 0;
inline void counted() { ++g_launches; }

sgs_alloc_fn g_alloc = nullptr;
sgs_free_fn g_release = nullptr;
void* g_user = nullptr;

struct Instance {
    bool live = true;                   // false once retired (slot ids stay stable)
    std::vector<void*> allocs;          // device memory owned by this instance
    size_t bytes = 0;
    cudaStream_t st = nullptr;          // branch stream of the captured step
    cudaEvent_t join = nullptr;
    // the equation of motion's products run on a side stream while the phase Pfaffians run, and
    // the second half of the pairs' Gauss-Jordan inverses before them
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double* dens = nullptr;             // [P + M] complex energy densities (between the two parts of pair_gh)
    int N = 0, n = 0, M = 0, P = 0, Ppf = 0, nimp = 0, nq = 0, a_nnz = 0;
    double dtau = 0.0, e_const = 0.0;
    int prec = 0, cmode = 0, parity = 1, integrator = 0;
    int fp64_path = SGS_FP64_EMULATED;  // arithmetic of the FP64 products (sgs_fp64_path)
    int shard_rank = 0, shard_world = 1; // pair sharding: this instance holds pairs p % world == rank
    // pairs in chunks (bounded memory): per-pair buffers hold Pc pairs; the step runs the pair pass
    // chunk by chunk for (G, h), then again for the equation of motion (recomputing S^-1, Im Delta)
    int Pc = 0, Ppfc = 0;               // pairs and phase-Pfaffian entries the per-pair buffers hold
    std::vector<int> ch_off, ch_cnt, ch_pfoff, ch_pfcnt;
    int cur = 0;                        // the chunk the pair kernels see (view)
    int nch() const { return (int)ch_off.size(); }
    int coff() const { return ch_off.empty() ? 0 : ch_off[cur]; }
    int ccnt() const { return ch_cnt.empty() ? 0 : ch_cnt[cur]; }
    int cpfoff() const { return ch_pfoff.empty() ? 0 : ch_pfoff[cur]; }
    int cpfcnt() const { return ch_pfcnt.empty() ? 0 : ch_pfcnt[cur]; }
    int* self_mask = nullptr;           // sharded: [M], 1 where this rank adds state mu's own term
    size_t oz_cap = 0;                  // emulated products: slice scratch cap (bytes)
    int gj_b = 32, pf_bs = 16;          // panel widths of the Gauss-Jordan inverse and the Pfaffian
    int gj_cap = 32, pf_cap = 16;       // widest widths the scratch holds
    int tuned_from_cache = -1;          // -1 not tuned, 0 timed, 1 cached
    std::vector<int> h_pa, h_pb;
    std::vector<double> hA, hq_val;     // host copy of the model: rank growth rebuilds the instance
    std::vector<int> hq_idx;
    std::vector<int> hh_len, hh_idx;    // terms of more than four Majoranas (host copy)
    std::vector<double> hh_val;
    int nh = 0;
    int *h_len = nullptr, *h_off = nullptr, *h_idx = nullptr;
    double* h_val = nullptr;

    double *gamma = nullptr, *dgamma = nullptr;
    int *pa = nullptr, *pb = nullptr, *pf_pair = nullptr, *pair_pf = nullptr, *pair_index = nullptr;
    int *a_rowptr = nullptr, *a_row = nullptr, *a_col = nullptr;
    double* a_val = nullptr;
    int* q_idx = nullptr;
    double* q_val = nullptr;
    int nc = 0;                         // quartic part as monomials with increasing indices
    int* c_idx = nullptr;
    double* c_val = nullptr;
    double trA2 = 0.0;                  // tr(A^2)
    int *imp = nullptr, *slot = nullptr;

    double *work = nullptr, *si = nullptr, *imd = nullptr, *wr = nullptr, *va = nullptr, *xa = nullptr;
    double* tbuf = nullptr;
    int *piv = nullptr, *perm = nullptr;
    double *logdet = nullptr, *dsign = nullptr;
    double *pfTU = nullptr, *pfpack = nullptr, *pflog = nullptr, *pfphase = nullptr;
    double *fimp = nullptr, *fimp_state = nullptr, *lr = nullptr;
    double* s[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int* sq = nullptr;
    double* scale = nullptr;
    double *Gm = nullptr, *hm = nullptr, *lam = nullptr, *lt = nullptr, *coef = nullptr;
    double* Ehist = nullptr;
    int Ecap = 0;
    double* Ecur = nullptr;             // energy slot written by the captured step
    int steps_since_profile = 0;
    double* corr_scratch = nullptr;     // observables: partial sums, sites, outputs
    size_t corr_cap = 0;
    double* renyi_scratch = nullptr;    // large Renyi subsystems: chunk of Pfaffian operands
    size_t renyi_cap = 0;
    long long renyi_chunk = 0;
    int renyi_m = 0;
    int* renyi_err = nullptr;
    double **r_Y = nullptr, **r_TU = nullptr, **r_PK = nullptr, **r_upA = nullptr, **r_upB = nullptr, **r_upC = nullptr;
    double* eigscratch = nullptr;
    int* err = nullptr;
    OzBuf oz;                           // emulated FP64 products: slice scratch (SGS_FP64_EMULATED only)
    OzBuf oz2;                          // the side stream's slice scratch (unchunked instances)
    int oz_side = 0;                    // 1 while the side stream's products are enqueued

    // tensor-core (mixed precision) operands of the equation of motion, per pair:
    // low-precision hi (fp32 or bf16) and lo (3xTF32) parts of S^{-1}, T1 = S^{-1} F,
    // D = G_a - G_b, W and V, fp32 results W, V, X
    int tc_kind = -1;
    int ldp = 0;          // leading dimension of the low-precision operands (multiple of 8)
    void *si_hi = nullptr, *si_lo = nullptr, *t1_hi = nullptr, *t1_lo = nullptr, *d_hi = nullptr, *d_lo = nullptr;
    void *wr_hi = nullptr, *wr_lo = nullptr, *va_hi = nullptr, *va_lo = nullptr;
    float *wr32 = nullptr, *va32 = nullptr, *xa32 = nullptr;
    TmaBatch tma_w{}, tma_v{}, tma_x{};   // TMA-fed products W = T1 S^{-1}, V = D W, X = V D
    bool tma_ok = false;
    // mixed-precision state update: fp32 masters [M][n][ldp] (0 X_s, 1-2 Q, 3 E^T, 4 E, 5 E^T,
    // 6 E, 7 F, 8 G) and tensor-core operands (0 Gamma, 1 dGamma, 2 + j = master j, j < 8)
    bool u_ok = false;
    float* u_y = nullptr;
    float* u_f32[9] = {};
    void* u_hi[10] = {};
    void* u_lo[10] = {};
    CUtensorMap u_map_hi[10], u_map_lo[10];
    void **q_si_hi = nullptr, **q_si_lo = nullptr, **q_t1_hi = nullptr, **q_t1_lo = nullptr, **q_d_hi = nullptr,
         **q_d_lo = nullptr, **q_wr_hi = nullptr, **q_wr_lo = nullptr, **q_va_hi = nullptr, **q_va_lo = nullptr,
         **q_wr32 = nullptr, **q_va32 = nullptr, **q_xa32 = nullptr;

    // pointer arrays (device)
    double **p_tup = nullptr;           // recursive Gauss-Jordan: pivot rows of an update (second half of work)
    double **p_work = nullptr, **p_tbuf = nullptr, **p_si = nullptr, **p_imd = nullptr, **p_wr = nullptr,
           **p_va = nullptr, **p_xa = nullptr, **p_ga = nullptr, **p_gb = nullptr;
    double **p_Y = nullptr, **p_TU = nullptr, **p_pack = nullptr;
    double **p_upA = nullptr, **p_upB = nullptr, **p_upC = nullptr;   // Pfaffian update (2 Ppf)
    double **p_gamma = nullptr, **p_dgamma = nullptr, **p_s[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    // the current chunk's view of the pairs (all pairs when unchunked)
    InstDev dev() const {
        InstDev d{};
        d.n = n; d.N = N; d.M = M; d.P = ccnt(); d.Ppf = cpfcnt(); d.nimp = nimp; d.nq = nq;
        d.e_const = e_const; d.parity = (double)parity;
        d.pa = pa + coff(); d.pb = pb + coff(); d.pf_pair = pf_pair + cpfoff(); d.pair_pf = pair_pf + coff();
        d.p_off = coff(); d.p_cnt = ccnt(); d.gamma = gamma;
        d.a_rowptr = a_rowptr; d.a_row = a_row; d.a_col = a_col; d.a_nnz = a_nnz; d.a_val = a_val;
        d.q_idx = q_idx; d.q_val = q_val; d.imp = imp; d.slot = slot;
        d.nh = nh; d.h_len = h_len; d.h_off = h_off; d.h_idx = h_idx; d.h_val = h_val;
        return d;
    }
    // every pair (the sums over all pairs of the assembly's last part; no per-pair buffer is read)
    InstDev dev_all() const {
        InstDev d = dev();
        d.P = P; d.Ppf = Ppf; d.pa = pa; d.pb = pb; d.pair_pf = pair_pf; d.p_off = 0; d.p_cnt = P;
        return d;
    }
};

}  // namespace

struct sgs_ctx {
    std::vector<Instance> inst;
    // one captured step of every live instance (a branch each), replayed by sgs_step
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int failed = -1;                    // first instance whose device error ended the last call
    std::vector<int> failed_list;       // every instance whose device error ended the last call
    std::vector<void*> allocs;
    int device = 0;
    Instance* owner = nullptr;          // instance being set up: its allocations are its own
    size_t bytes_in_use = 0, budget = 0;  // budget 0 = unlimited
    bool autotune = false;              // time the factorisation panel widths of new shapes
    cudaEvent_t fork = nullptr;

    void* dalloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        void* p = nullptr;
        if (g_alloc) {
            p = g_alloc(bytes, (void*)stream, g_user);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            p = nullptr;
        }
        if (p) {
            if (owner) { owner->allocs.push_back(p); owner->bytes += bytes; }
            else allocs.push_back(p);
            bytes_in_use += bytes;
        }
        return p;
    }
    void release_instance(Instance& I) {
        for (void* p : I.allocs) {
            if (release) release(p, release_user);
            else cudaFree(p);
        }
        I.allocs.clear();
        bytes_in_use -= I.bytes;
        I.bytes = 0;
    }
    void drop_graph() {
        if (graph_exec) { cudaGraphExecDestroy(graph_exec); graph_exec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    }
    template <class T>
    T* alloc(size_t count) { return static_cast<T*>(dalloc(count * sizeof(T))); }
    sgs_free_fn release = nullptr;   // hook captured at creation, used for every free
    void* release_user = nullptr;
    void release_all() {
        for (void* p : allocs) {
            if (release) release(p, release_user);
            else cudaFree(p);
        }
        allocs.clear();
    }
    sgs_ctx() : release(g_alloc ? g_release : nullptr), release_user(g_user) {}

    // stage timing (CUDA events on the context stream) and algorithmic work
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    int open_stage = -1;
    cudaEvent_t open_ev = nullptr;
    double stage_ms[SGS_N_STAGES] = {0};
    double stage_flops[SGS_N_STAGES] = {0};
    double stage_bytes[SGS_N_STAGES] = {0};
    long long launches = 0;
    // every FP64 GEMM launch (except the pass-through squarings) timed on its own
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gmarks;
    double gemm_ms = 0.0, gemm_flops = 0.0;
    long long gemm_count = 0;

    cudaEvent_t next_event() {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }
    // close the open stage, open stage s (-1: none); in profiling mode the stages are
    // CUDA-event intervals and NVTX ranges (named as sgs_stage)
    void stage(int s) {
        if (!prof) return;
        cudaEvent_t e = next_event();
        cudaEventRecord(e, stream);
        if (open_stage >= 0) {
            marks.push_back({open_stage, open_ev, e});
            nvtxRangePop();
        }
        if (s >= 0) {
            static const char* names[SGS_N_STAGES] = {"pair_inverse", "pair_delta", "phase_pfaffian", "amplitudes",
                                                      "eom_w", "eom_v", "eom_x", "eom_assembly", "update"};
            nvtxRangePushA(names[s]);
        }
        open_stage = s;
        open_ev = e;
    }
    void collect() {               // after a stream synchronisation
        for (auto& m : marks) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, m.a, m.b);
            stage_ms[m.stage] += ms;
        }
        marks.clear();
        for (auto& m : gmarks) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, m.first, m.second);
            gemm_ms += ms;
        }
        gmarks.clear();
        ev_used = 0;
        open_stage = -1;
    }
};

#define CUDA_TRY(ctx, call)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return SGS_ECUDA;                                                               \
        }                                                                                   \
    } while (0)

namespace {

template <class T>
T** upload_ptrs(sgs_ctx* c, const std::vector<T*>& v) {
    T** d = c->alloc<T*>(v.size());
    if (!d) return nullptr;
    cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T*), cudaMemcpyHostToDevice, c->stream);
    return d;
}

int perm_sign4(const int* p) {
    int s = 1;
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++)
            if (p[i] > p[j]) s = -s;
    return s;
}

unsigned grid_chunks(size_t work, int threads, unsigned cap) {
    size_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// device bytes one instance holds (the allocations of setup_instance, up to small terms)
// emulated FP64 products (path 2): slice scratch of one instance, enough for its widest
// batch (pairs, Pfaffian halves or states) of n x n x n products, capped per instance (the
// products then run in batch chunks)
constexpr size_t OZ_DEFAULT_CAP = (size_t)2 << 30;
size_t oz_cap_of(size_t requested) {
    return requested ? std::max<size_t>(requested, (size_t)1 << 20) : OZ_DEFAULT_CAP;
}
size_t oz_scratch_bytes(int n, int M, size_t cap, size_t pair_cap) {
    const size_t P = std::min<size_t>((size_t)M * (M - 1) / 2, pair_cap), Ppf = P;
    const size_t batch = std::max<size_t>(std::max<size_t>(P, 2 * Ppf), std::max<size_t>((size_t)M, 1));
    return std::min(batch * oz_entry_bytes(n, n, std::min(n, OZ_KC)) + 16384, cap);
}

size_t instance_bytes(int n, int M, int prec, int nimp, bool tune, int fp64_path, size_t oz_cap, int pair_chunk) {
    const size_t Pall = (size_t)M * (M - 1) / 2;
    const size_t nn = (size_t)n * n, P = pair_chunk > 0 ? std::min<size_t>(Pall, pair_chunk) : Pall, Ppf = P;
    const size_t gj_b = tune ? 64 : 32, bs = tune ? 32 : 16;
    const size_t ni = std::max(nimp, 1);
    size_t d = 7 * (size_t)M * nn + std::max<size_t>(P, 1) * nn * 7 + P * gj_b * n + Ppf * 20 * n * bs +
               P * ni * ni * 2 + P * 2 * n * ni + 6 * (size_t)(2 * M) * (2 * M) + 16 * (size_t)M * M;
    size_t bytes = 8 * d + 8 * P * n;   // + pivots and permutations
    if (prec != SGS_FP64 && P > 0) {
        const size_t ldp = (n + 7) & ~7, esz = (prec == SGS_MIXED_BF16) ? 2 : 4;
        const size_t ops = (prec == SGS_FP32_3XTF32) ? 10 : 5;
        bytes += P * n * ldp * esz * ops + 3 * P * nn * 4;
        if (prec != SGS_FP32_3XTF32)
            bytes += (size_t)M * nn * 4 + (size_t)M * n * ldp * (9 * 4 + 10 * esz);   // mixed update
    }
    if (fp64_path == SGS_FP64_EMULATED) bytes += oz_scratch_bytes(n, M, oz_cap, P) * (P == Pall ? 2 : 1);
    return bytes + (1 << 20);
}

// Candidate panel widths (the factorisations' tile shapes).  Gauss-Jordan: the panel
// kernel keeps n x (b + 1) doubles in shared memory; Pfaffian: 2 b <= n.
std::vector<int> gj_candidates(int n) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, gj_panel_kernel);
    const int limit = optin - (int)fa.sharedSizeBytes;
    std::vector<int> v;
    // between the powers of two: at n = 512 a panel of 12 columns fits four panel CTAs per SM
    // (one wave for up to 608 matrices), 20 three, 24 two
    for (int b : {8, 12, 16, 20, 24, 32, 48, 64})
        if (b <= n && (size_t)n * (b + 1) * sizeof(double) + b * sizeof(double) <= (size_t)limit) v.push_back(b);
    return v;
}
// leaf of the recursive form: 16 columns, or the widest candidate below it whose panel
// fits shared memory (large n)
int default_gj_width(int n) {
    int w = std::min(8, n);
    for (int b : gj_candidates(n))
        if (b <= 16) w = std::max(w, b);
    return std::min(w, n);
}
std::vector<int> pf_candidates(int n) {
    std::vector<int> v;
    for (int b : {8, 12, 16, 24, 32})
        if (2 * b <= n) v.push_back(b);
    return v;
}

int default_pf_width(int n) { return (2 * 16 > n) ? n / 2 : 16; }

// Pointer arrays of the Gauss-Jordan panel rows and the Pfaffian panel vectors and
// packed update operands for panel widths (gj_b, pf_bs); the scratch they point into is
// sized for the widest candidate the instance may use.
sgs_status set_panel_pointers(sgs_ctx* c, Instance& I, int gj_b, int pf_bs) {
    const int n = I.n, P = I.Pc, Ppf = I.Ppfc;    // one chunk of pairs
    const size_t nn = (size_t)n * n;
    I.gj_b = gj_b;
    I.pf_bs = pf_bs;
    Instance* prev = c->owner;          // allocations belong to the instance
    c->owner = &I;
    std::vector<double*> t;
    for (int p = 0; p < P; p++) t.push_back(I.tbuf + (size_t)p * gj_b * n);
    if (P > 0 && !(I.p_tbuf = upload_ptrs(c, t))) { c->owner = prev; return SGS_ENOMEM; }
    std::vector<double*> Y, TU, PK, upA, upB, upC;
    const size_t blk = (size_t)n * 4 * pf_bs;
    for (int q = 0; q < Ppf; q++) {
        Y.push_back(I.work + (size_t)q * 2 * nn);
        TU.push_back(I.pfTU + (size_t)q * 4 * n * pf_bs);
        PK.push_back(I.pfpack + (size_t)q * 4 * blk);
    }
    // the trailing updates' operands, real and imaginary planes of each entry next to each other, so
    // that the first 2 k entries serve a chunk of k phase Pfaffians
    for (int q = 0; q < Ppf; q++) {
        upA.push_back(PK[q]); upB.push_back(PK[q] + blk); upC.push_back(Y[q]);
        upA.push_back(PK[q] + 2 * blk); upB.push_back(PK[q] + 3 * blk); upC.push_back(Y[q] + nn);
    }
    if (Ppf > 0) {
        I.p_Y = upload_ptrs(c, Y); I.p_TU = upload_ptrs(c, TU); I.p_pack = upload_ptrs(c, PK);
        I.p_upA = upload_ptrs(c, upA); I.p_upB = upload_ptrs(c, upB); I.p_upC = upload_ptrs(c, upC);
        if (!I.p_Y || !I.p_TU || !I.p_pack || !I.p_upA || !I.p_upB || !I.p_upC) { c->owner = prev; return SGS_ENOMEM; }
    }
    c->owner = prev;
    return SGS_OK;
}

sgs_status setup_instance(sgs_ctx* c, Instance& I, const sgs_model& m, const sgs_options& o) {
    const int n = 2 * m.n_modes;
    I.N = m.n_modes;
    I.n = n;
    I.M = o.rank;
    I.dtau = o.dtau;
    I.prec = o.precision;
    I.cmode = o.cmode;
    I.parity = o.parity;
    I.integrator = o.integrator;
    I.fp64_path = o.fp64_path;
    I.oz_cap = oz_cap_of(o.emulation_scratch);
    I.shard_world = o.shard_world > 1 ? o.shard_world : 1;
    I.shard_rank = I.shard_world > 1 ? o.shard_rank : 0;
    I.e_const = m.e_const;
    I.hA.assign(m.A, m.A + (size_t)n * n);
    I.hq_idx.assign(m.quartic_idx, m.quartic_idx + (m.n_quartic > 0 ? 4 * m.n_quartic : 0));
    I.hq_val.assign(m.quartic_val, m.quartic_val + (m.n_quartic > 0 ? m.n_quartic : 0));
    I.gj_b = default_gj_width(n);
    I.pf_bs = default_pf_width(n);
    I.gj_cap = I.gj_b;
    I.pf_cap = I.pf_bs;
    if (c->autotune) {          // scratch for the widest candidate
        for (int b : gj_candidates(n)) I.gj_cap = std::max(I.gj_cap, b);
        for (int b : pf_candidates(n)) I.pf_cap = std::max(I.pf_cap, b);
    }

    // sparse A
    std::vector<int> rowptr(n + 1, 0), rows, cols;
    std::vector<double> vals;
    for (int k = 0; k < n; k++) {
        for (int l = 0; l < n; l++) {
            double v = m.A[(size_t)k * n + l];
            if (v != 0.0) { rows.push_back(k); cols.push_back(l); vals.push_back(v); }
        }
        rowptr[k + 1] = (int)cols.size();
    }
    I.a_nnz = (int)cols.size();
    // quartic: antisymmetrise
    std::map<std::vector<int>, double> U;
    for (int j = 0; j < m.n_quartic; j++) {
        const int* ix = m.quartic_idx + 4 * j;
        for (int a = 0; a < 4; a++) {
            if (ix[a] < 0 || ix[a] >= n) { c->err = "quartic index out of range"; return SGS_EINVAL; }
            for (int b = a + 1; b < 4; b++)
                if (ix[a] == ix[b]) { c->err = "quartic monomial needs four distinct Majoranas"; return SGS_EINVAL; }
        }
        int p[4] = {0, 1, 2, 3};
        do {
            std::vector<int> key = {ix[p[0]], ix[p[1]], ix[p[2]], ix[p[3]]};
            U[key] += perm_sign4(p) * m.quartic_val[j] / 24.0;
        } while (std::next_permutation(p, p + 4));
    }
    std::vector<int> qidx;
    std::vector<double> qval;
    std::vector<int> impv;
    for (auto& kv : U) {
        if (kv.second == 0.0) continue;
        for (int a = 0; a < 4; a++) {
            qidx.push_back(kv.first[a]);
            if (std::find(impv.begin(), impv.end(), kv.first[a]) == impv.end()) impv.push_back(kv.first[a]);
        }
        qval.push_back(kv.second);
    }
    // terms of more than four Majoranas: 6 or 8 distinct indices each, energy v (-1)^((r + r mod 2)/2)
    // Pf(Delta_S) for the term v i^(r mod 2) c_s1 ... c_s2r
    std::vector<int> hoff;
    std::vector<double> hval;
    I.hh_len.clear(); I.hh_idx.clear(); I.hh_val.clear();
    if (m.n_higher < 0 || m.n_higher > SGS_MAX_HIGHER ||
        (m.n_higher > 0 && (!m.higher_len || !m.higher_idx || !m.higher_val))) {
        c->err = "bad higher interaction terms";
        return SGS_EINVAL;
    }
    for (int j = 0, off = 0; j < m.n_higher; j++) {
        const int len = m.higher_len[j];
        if (len != 6 && len != 8) { c->err = "a higher interaction term has 6 or 8 Majoranas"; return SGS_EINVAL; }
        const int* ix = m.higher_idx + off;
        for (int a = 0; a < len; a++) {
            if (ix[a] < 0 || ix[a] >= n) { c->err = "higher term index out of range"; return SGS_EINVAL; }
            for (int b = a + 1; b < len; b++)
                if (ix[a] == ix[b]) { c->err = "a higher term needs distinct Majoranas"; return SGS_EINVAL; }
            if (std::find(impv.begin(), impv.end(), ix[a]) == impv.end()) impv.push_back(ix[a]);
        }
        const int r = len / 2;
        hoff.push_back((int)I.hh_idx.size());
        I.hh_len.push_back(len);
        I.hh_idx.insert(I.hh_idx.end(), ix, ix + len);
        I.hh_val.push_back(m.higher_val[j]);
        hval.push_back((((r + r % 2) / 2) % 2 ? -1.0 : 1.0) * m.higher_val[j]);
        off += len;
    }
    I.nh = m.n_higher;
    std::sort(impv.begin(), impv.end());
    if ((int)impv.size() > SGS_MAX_IMP) { c->err = "more than 16 Majoranas in interaction terms"; return SGS_EINVAL; }
    // canonical monomials: coefficient of c_k c_l c_p c_q (k < l < p < q) = 24 U_klpq
    std::vector<int> cidx;
    std::vector<double> cval;
    for (auto& kv : U) {
        const auto& k = kv.first;
        if (kv.second != 0.0 && k[0] < k[1] && k[1] < k[2] && k[2] < k[3]) {
            cidx.insert(cidx.end(), k.begin(), k.end());
            cval.push_back(24.0 * kv.second);
        }
    }
    I.nc = (int)cval.size();
    I.trA2 = 0.0;
    for (size_t e = 0; e < (size_t)n * n; e++) I.trA2 -= m.A[e] * m.A[e];   // tr(A^2) = -||A||_F^2
    I.nq = (int)qval.size();
    I.nimp = (int)impv.size();
    std::vector<int> slot(n, -1);
    for (int j = 0; j < I.nimp; j++) slot[impv[j]] = j;

    // pairs (a, b), a < b, in the order (0, 1), (0, 2), ..., (M - 2, M - 1); a sharded instance
    // holds the pairs whose index in that order is rank modulo world
    const int M = I.M;
    std::vector<int> pa, pb, pair_pf, pf_pair, pidx((size_t)M * M, -1);
    int gp = 0;
    for (int a = 0; a < M; a++)
        for (int b = a + 1; b < M; b++, gp++) {
            if (gp % I.shard_world != I.shard_rank) continue;
            int p = (int)pa.size();
            pa.push_back(a); pb.push_back(b);
            pidx[a * M + b] = pidx[b * M + a] = p;
            pair_pf.push_back(-1);
            if (a >= 1) { pair_pf[p] = (int)pf_pair.size(); pf_pair.push_back(p); }
        }
    I.P = (int)pa.size();
    const int P = I.P;
    I.Ppf = (int)pf_pair.size();
    I.h_pa = pa;
    I.h_pb = pb;
    // chunks of at most Pc consecutive pairs; the phase-Pfaffian entries (pairs with a >= 1) of each
    // chunk are listed by their index in the chunk, and pair_pf maps a pair to its chunk's entry
    I.Pc = (o.pair_chunk > 0 && o.pair_chunk < P) ? o.pair_chunk : P;
    I.ch_off.clear(); I.ch_cnt.clear(); I.ch_pfoff.clear(); I.ch_pfcnt.clear();
    pf_pair.clear();
    I.Ppfc = 0;
    for (int off = 0; off < std::max(P, 1); off += std::max(I.Pc, 1)) {
        const int cnt = std::min(I.Pc, P - off);
        I.ch_off.push_back(off); I.ch_cnt.push_back(std::max(cnt, 0)); I.ch_pfoff.push_back((int)pf_pair.size());
        int k = 0;
        for (int j = 0; j < cnt; j++) {
            pair_pf[off + j] = -1;
            if (pa[off + j] >= 1) { pair_pf[off + j] = k++; pf_pair.push_back(j); }
        }
        I.ch_pfcnt.push_back(k);
        I.Ppfc = std::max(I.Ppfc, k);
    }
    I.cur = 0;
    if (pair_pf.empty()) pair_pf.push_back(-1);
    const int Pc = I.Pc;

    const size_t nn = (size_t)n * n;
    const size_t Pm = std::max(P, 1), Pcm = std::max(Pc, 1);
    const size_t Pf = std::max(I.Ppf, 1), Pfc = std::max(I.Ppfc, 1);
    const int ni = std::max(I.nimp, 1);
    I.gamma = c->alloc<double>(M * nn);
    I.dgamma = c->alloc<double>(M * nn);
    I.pa = c->alloc<int>(Pm); I.pb = c->alloc<int>(Pm);
    I.pf_pair = c->alloc<int>(Pf); I.pair_pf = c->alloc<int>(Pm); I.pair_index = c->alloc<int>((size_t)M * M);
    I.a_rowptr = c->alloc<int>(n + 1); I.a_row = c->alloc<int>(std::max(I.a_nnz, 1));
    I.a_col = c->alloc<int>(std::max(I.a_nnz, 1)); I.a_val = c->alloc<double>(std::max(I.a_nnz, 1));
    I.q_idx = c->alloc<int>(std::max(4 * I.nq, 4)); I.q_val = c->alloc<double>(std::max(I.nq, 1));
    I.c_idx = c->alloc<int>(std::max(4 * I.nc, 4)); I.c_val = c->alloc<double>(std::max(I.nc, 1));
    I.imp = c->alloc<int>(ni); I.slot = c->alloc<int>(n);
    if (I.nh > 0) {
        I.h_len = c->alloc<int>(I.nh); I.h_off = c->alloc<int>(I.nh); I.h_idx = c->alloc<int>(I.hh_idx.size());
        I.h_val = c->alloc<double>(I.nh);
        if (!I.h_len || !I.h_off || !I.h_idx || !I.h_val) { c->err = "device allocation failed"; return SGS_ENOMEM; }
    }
    // per-pair buffers hold one chunk; the impurity blocks of F are kept for every pair (the
    // equation-of-motion pass of a chunked step reads the amplitude pass's)
    I.work = c->alloc<double>(Pcm * 2 * nn);
    I.si = c->alloc<double>(Pcm * nn); I.imd = c->alloc<double>(Pcm * nn);
    I.wr = c->alloc<double>(Pcm * nn); I.va = c->alloc<double>(Pcm * nn); I.xa = c->alloc<double>(Pcm * nn);
    I.tbuf = c->alloc<double>(Pcm * I.gj_cap * n);
    I.piv = c->alloc<int>(Pcm * n); I.perm = c->alloc<int>(Pcm * n);
    I.logdet = c->alloc<double>(Pcm); I.dsign = c->alloc<double>(Pcm);
    I.pfTU = c->alloc<double>(Pfc * 4 * n * I.pf_cap);
    I.pfpack = c->alloc<double>(Pfc * 4 * n * 4 * I.pf_cap);
    I.pflog = c->alloc<double>(Pfc); I.pfphase = c->alloc<double>(2 * Pfc);
    I.fimp = c->alloc<double>(Pm * ni * ni * 2); I.fimp_state = c->alloc<double>((size_t)M * ni * ni);
    I.lr = c->alloc<double>(Pcm * 2 * n * ni);
    for (int j = 0; j < 5; j++) I.s[j] = c->alloc<double>(M * nn);
    I.sq = c->alloc<int>(M); I.scale = c->alloc<double>(M);
    I.Gm = c->alloc<double>(2 * M * M); I.hm = c->alloc<double>(2 * M * M);
    I.lam = c->alloc<double>(2 * M); I.lt = c->alloc<double>(2 * M); I.coef = c->alloc<double>(6 * M * M);
    I.Ecap = 1;
    I.Ehist = c->alloc<double>(1);
    I.Ecur = c->alloc<double>(1);
    I.eigscratch = c->alloc<double>(6 * (size_t)(2 * M) * (2 * M) + 8 * 2 * M);
    I.err = c->alloc<int>(1);
    I.dens = c->alloc<double>(2 * ((size_t)Pcm + M));
    if (I.shard_world > 1) {
        I.self_mask = c->alloc<int>(M);
        if (!I.self_mask) { c->err = "device allocation failed"; return SGS_ENOMEM; }
        std::vector<int> mask(M);
        for (int mu = 0; mu < M; mu++) mask[mu] = (mu % I.shard_world == I.shard_rank) ? 1 : 0;
        CUDA_TRY(c, cudaMemcpyAsync(I.self_mask, mask.data(), M * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    }
    void* check[] = {I.gamma, I.dgamma, I.work, I.si, I.imd, I.wr, I.va, I.xa, I.tbuf, I.pfTU, I.pfpack, I.s[0],
                     I.s[1], I.s[2], I.s[3], I.s[4], I.eigscratch, I.err, I.lr, I.fimp};
    for (void* p : check)
        if (!p) { c->err = "device allocation failed"; return SGS_ENOMEM; }

    cudaStream_t st = c->stream;
    // gamma0 == nullptr: the caller fills the states on the device (rank growth)
    if (o.gamma0)
        CUDA_TRY(c, cudaMemcpyAsync(I.gamma, o.gamma0, M * nn * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemsetAsync(I.dgamma, 0, M * nn * sizeof(double), st));
    CUDA_TRY(c, cudaMemsetAsync(I.sq, 0, M * sizeof(int), st));
    if (P > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(I.pa, pa.data(), P * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.pb, pb.data(), P * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.pair_pf, pair_pf.data(), P * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    if (!pf_pair.empty())
        CUDA_TRY(c, cudaMemcpyAsync(I.pf_pair, pf_pair.data(), pf_pair.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(I.pair_index, pidx.data(), (size_t)M * M * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(I.a_rowptr, rowptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    if (I.a_nnz > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(I.a_row, rows.data(), I.a_nnz * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.a_col, cols.data(), I.a_nnz * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.a_val, vals.data(), I.a_nnz * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (I.nq > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(I.q_idx, qidx.data(), 4 * I.nq * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.q_val, qval.data(), I.nq * sizeof(double), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.imp, impv.data(), I.nimp * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    if (I.nc > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(I.c_idx, cidx.data(), 4 * I.nc * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.c_val, cval.data(), I.nc * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    CUDA_TRY(c, cudaMemcpyAsync(I.slot, slot.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    if (I.nh > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(I.h_len, I.hh_len.data(), I.nh * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.h_off, hoff.data(), I.nh * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.h_idx, I.hh_idx.data(), I.hh_idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(I.h_val, hval.data(), I.nh * sizeof(double), cudaMemcpyHostToDevice, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));     // hoff and hval are host temporaries
    }
    std::vector<double> lam0(2 * M, 0.0);
    if (o.lambda0) std::memcpy(lam0.data(), o.lambda0, 2 * M * sizeof(double));
    CUDA_TRY(c, cudaMemcpyAsync(I.lam, lam0.data(), 2 * M * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemsetAsync(I.err, 0, sizeof(int), st));

    // pointer arrays: the per-pair buffers of one chunk (index in the chunk), the states of every pair
    std::vector<double*> w, s_, im, wr, va, xa, ga, gb;
    for (int p = 0; p < Pc; p++) {
        w.push_back(I.work + p * nn);
        s_.push_back(I.si + p * nn);
        im.push_back(I.imd + p * nn);
        wr.push_back(I.wr + p * nn);
        va.push_back(I.va + p * nn);
        xa.push_back(I.xa + p * nn);
    }
    for (int p = 0; p < P; p++) {
        ga.push_back(I.gamma + pa[p] * nn);
        gb.push_back(I.gamma + pb[p] * nn);
    }
    if (P > 0) {
        std::vector<double*> tup;
        for (int p = 0; p < Pc; p++) tup.push_back(I.work + (size_t)Pc * nn + (size_t)p * nn);
        I.p_tup = upload_ptrs(c, tup);
        I.p_work = upload_ptrs(c, w); I.p_si = upload_ptrs(c, s_);
        I.p_imd = upload_ptrs(c, im); I.p_wr = upload_ptrs(c, wr); I.p_va = upload_ptrs(c, va);
        I.p_xa = upload_ptrs(c, xa); I.p_ga = upload_ptrs(c, ga); I.p_gb = upload_ptrs(c, gb);
    }
    if (set_panel_pointers(c, I, I.gj_b, I.pf_bs) != SGS_OK) { c->err = "device allocation failed"; return SGS_ENOMEM; }
    std::vector<double*> g, dg, ss[5];
    for (int mu = 0; mu < M; mu++) {
        g.push_back(I.gamma + mu * nn);
        dg.push_back(I.dgamma + mu * nn);
        for (int j = 0; j < 5; j++) ss[j].push_back(I.s[j] + mu * nn);
    }
    I.p_gamma = upload_ptrs(c, g);
    I.p_dgamma = upload_ptrs(c, dg);
    for (int j = 0; j < 5; j++) I.p_s[j] = upload_ptrs(c, ss[j]);

    if (I.prec != SGS_FP64 && P > 0) {
        I.tc_kind = (I.prec == SGS_MIXED_TF32) ? TC_TF32 : (I.prec == SGS_MIXED_BF16) ? TC_BF16 : TC_3XTF32;
        const size_t esz = (I.tc_kind == TC_BF16) ? 2 : 4;
        const bool split = I.tc_kind == TC_3XTF32;
        I.ldp = (n + 7) & ~7;
        const size_t lpn = (size_t)n * I.ldp;           // elements of one padded operand
        const size_t bytes = (size_t)Pc * lpn * esz;
        I.si_hi = c->dalloc(bytes); I.t1_hi = c->dalloc(bytes); I.d_hi = c->dalloc(bytes);
        I.wr32 = c->alloc<float>(Pc * nn); I.va32 = c->alloc<float>(Pc * nn); I.xa32 = c->alloc<float>(Pc * nn);
        // fp32 results become operands through a rounding conversion (TF32: to nearest)
        I.wr_hi = c->dalloc(bytes);
        I.va_hi = c->dalloc(bytes);
        if (split) {
            I.si_lo = c->dalloc(bytes); I.t1_lo = c->dalloc(bytes); I.d_lo = c->dalloc(bytes);
            I.wr_lo = c->dalloc(bytes); I.va_lo = c->dalloc(bytes);
        }
        if (!I.si_hi || !I.t1_hi || !I.d_hi || !I.wr32 || !I.va32 || !I.xa32 || !I.wr_hi || !I.va_hi ||
            (split && (!I.si_lo || !I.t1_lo || !I.d_lo || !I.wr_lo || !I.va_lo))) {
            c->err = "device allocation failed (tensor-core operands)";
            return SGS_ENOMEM;
        }
        auto arr = [&](void* base, size_t stride) {
            std::vector<void*> v;
            for (int p = 0; p < Pc; p++) v.push_back(base ? (uint8_t*)base + p * stride : nullptr);
            return upload_ptrs(c, v);
        };
        const size_t lp = lpn * esz, f4 = nn * 4;
        I.q_si_hi = arr(I.si_hi, lp); I.q_t1_hi = arr(I.t1_hi, lp); I.q_d_hi = arr(I.d_hi, lp);
        I.q_wr_hi = arr(I.wr_hi, lp);
        I.q_va_hi = arr(I.va_hi, lp);
        I.q_wr32 = arr(I.wr32, f4); I.q_va32 = arr(I.va32, f4); I.q_xa32 = arr(I.xa32, f4);
        I.q_si_lo = arr(I.si_lo, lp); I.q_t1_lo = arr(I.t1_lo, lp); I.q_d_lo = arr(I.d_lo, lp);
        I.q_wr_lo = arr(I.wr_lo, lp); I.q_va_lo = arr(I.va_lo, lp);
        // tensor maps of the contiguous operand batches [Pc][n][ldp] (one chunk of pairs)
        const bool bf = I.tc_kind == TC_BF16;
        auto prod = [&](TmaBatch& t, void* A, void* A2, void* B, void* B2, float* C, int skew) {
            bool ok = make_operand_map(&t.ta, A, bf, I.ldp, n, Pc) && make_operand_map(&t.tb, B, bf, I.ldp, n, Pc);
            if (split) ok = ok && make_operand_map(&t.ta2, A2, bf, I.ldp, n, Pc) && make_operand_map(&t.tb2, B2, bf, I.ldp, n, Pc);
            t.m = n; t.n = n; t.k = n; t.alpha = -1.0; t.C = C; t.c_stride = (long long)nn; t.ldc = n;
            t.out_f64 = 0; t.skew = skew; t.err = I.err; t.batch = Pc;
            return ok;
        };
        I.tma_ok = prod(I.tma_w, I.t1_hi, I.t1_lo, I.si_hi, I.si_lo, I.wr32, 1) &&
                   prod(I.tma_v, I.d_hi, I.d_lo, I.wr_hi, I.wr_lo, I.va32, 0) &&
                   prod(I.tma_x, I.va_hi, I.va_lo, I.d_hi, I.d_lo, I.xa32, 1);
        if (!I.tma_ok) { c->err = "tensor map encoding failed"; return SGS_ECUDA; }

        // mixed-precision state update (TMA-fed products; TF32 and BF16 forms): 3xTF32 keeps
        // the FP64 update, since its products accumulate in fp32 and would hold the step to
        // ~1e-6 relative, below the form's purpose
        if (I.tma_ok && I.tc_kind != TC_3XTF32) {
            const size_t mp = (size_t)M * n * I.ldp;
            I.u_y = c->alloc<float>((size_t)M * nn);
            bool ok = I.u_y != nullptr;
            for (int j = 0; j < 9 && ok; j++) {
                I.u_f32[j] = c->alloc<float>(mp);
                ok = I.u_f32[j] != nullptr && cudaMemsetAsync(I.u_f32[j], 0, mp * sizeof(float), c->stream) == cudaSuccess;
            }
            for (int i = 0; i < 10 && ok; i++) {
                I.u_hi[i] = c->dalloc(mp * esz);       // rounded operand copies of the fp32 results
                ok = I.u_hi[i] != nullptr;
                if (ok && split) ok = (I.u_lo[i] = c->dalloc(mp * esz)) != nullptr;
                if (ok) ok = make_operand_map(&I.u_map_hi[i], I.u_hi[i], bf, I.ldp, n, M);
                if (ok && split) ok = make_operand_map(&I.u_map_lo[i], I.u_lo[i], bf, I.ldp, n, M);
            }
            if (!ok) { c->err = "device allocation failed (mixed-precision update)"; return SGS_ENOMEM; }
            I.u_ok = true;
        }
    }
    if (I.fp64_path == SGS_FP64_EMULATED) {
        // emulated FP64 products: slice scratch for one batch chunk, and one for the side stream
        const size_t b = oz_scratch_bytes(n, M, I.oz_cap, Pc);
        I.oz.base = static_cast<uint8_t*>(c->dalloc(b));
        if (!I.oz.base) { c->err = "device allocation failed (emulated-product scratch)"; return SGS_ENOMEM; }
        I.oz.bytes = b;
        if (I.nch() == 1 && P > 0) {
            I.oz2.base = static_cast<uint8_t*>(c->dalloc(b));
            if (!I.oz2.base) { c->err = "device allocation failed (emulated-product scratch)"; return SGS_ENOMEM; }
            I.oz2.bytes = b;
        }
    }
    return SGS_OK;
}

// ------------------------------------------------------------------ launches

// Kernels with large dynamic shared memory: raise their limit (227 KB, the per-block
// maximum of sm_100-class GPUs) once per device, with that device current and outside
// any stream capture.  The attribute belongs to the device's context, so each device
// the library runs on is set up on its first use.
template <class K>
void raise_smem_limit(K kernel, int optin) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    // the limit applies to dynamic shared memory on top of the kernel's static shared memory
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
constexpr int SGS_MAX_DEVICES = 64;
std::mutex g_attr_mutex;
bool g_attr_done[SGS_MAX_DEVICES] = {};
void set_kernel_attributes() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SGS_MAX_DEVICES) return;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (g_attr_done[dev]) return;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    raise_smem_limit(gj_panel_kernel, optin);
    raise_smem_limit(pf_panel_kernel, optin);
    raise_smem_limit(renyi_pf_kernel, optin);
    raise_smem_limit(gemm_tma_kernel<TC_TF32>, optin);
    raise_smem_limit(gemm_tma_kernel<TC_BF16>, optin);
    raise_smem_limit(gemm_tma_kernel<TC_3XTF32>, optin);
    raise_smem_limit(oz_gemm_kernel<OZ_NARROW>, optin);
    raise_smem_limit(oz_gemm_kernel<OZ_NARROW16>, optin);
    raise_smem_limit(oz_block_slice_kernel, optin);
    cudaGetLastError();
    g_attr_done[dev] = true;
}

inline cudaError_t tma_product(const TmaBatch& t, int kind, cudaStream_t st) { return gemm_tma(t, kind, st); }

// every FP64 product of the library goes through here; flops = algorithmic work of
// the launch (antisymmetric outputs count half), < 0 = not profiled.  With slice
// scratch (an instance or call on the emulated path) the product runs emulated on
// the bf16 tensor cores, otherwise on the FP64 FMA pipe.
// presliced: the operands' slices are already in *oz (gemm_oz_presliced; their producer sliced
// them, so the product's time below excludes the slicing)
inline cudaError_t gemm(sgs_ctx* c, const GemmBatch& g, cudaStream_t st, double flops, const OzBuf* oz = nullptr,
                        int* oz_err = nullptr, bool presliced = false) {
    const bool emulate = oz && oz->base && oz_err;
    if (emulate) set_kernel_attributes();             // the kernels' shared-memory limits (once)
    if (emulate && !presliced) for (int i = oz_launches(g, *oz); i > 0; i--) counted();
    else counted();
    auto run = [&]() {
        if (emulate && presliced) return gemm_oz_presliced(g, *oz, oz_err, st);
        return emulate ? gemm_oz(g, *oz, oz_err, st) : gemm_f64(g, st);
    };
    if (c && c->prof && flops >= 0.0) {
        cudaEvent_t a = c->next_event(), b = c->next_event();
        cudaEventRecord(a, st);
        cudaError_t e = run();
        cudaEventRecord(b, st);
        c->gmarks.push_back({a, b});
        c->gemm_flops += flops;
        c->gemm_count++;
        return e;
    }
    return run();
}
inline cudaError_t gemm(sgs_ctx* c, Instance& I, const GemmBatch& g, cudaStream_t st, double flops) {
    return gemm(c, g, st, flops, I.oz_side ? &I.oz2 : &I.oz, I.err);
}

GemmBatch gb_basic(int m, int n, int k, double** A, int lda, double** B, int ldb, double** C, int ldc, int batch) {
    GemmBatch g = gemm_defaults();
    g.m = m; g.n = n; g.k = k;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.batch = batch;
    return g;
}

cudaError_t launch_gj(sgs_ctx* c, int n, int batch, int bsz, double** W, double** T, int* piv, double* logdet,
                      double* dsign, int* err, double tiny, cudaStream_t st, const OzBuf* oz = nullptr) {
    set_kernel_attributes();
    for (int k0 = 0; k0 < n; k0 += bsz) {
        const int bb = std::min(bsz, n - k0);
        GJPanelArgs a{W, T, piv, logdet, dsign, err, n, k0, bb, tiny};
        gj_panel_kernel<<<batch, 512, (size_t)n * (bb + 1) * sizeof(double) + bb * sizeof(double), st>>>(a);
        counted();
        GemmBatch g = gb_basic(n, n, bb, W, n, T, n, W, n, batch);
        g.offA = k0;
        g.Cin = (const double* const*)W; g.ldcin = n; g.beta = 1.0;
        g.mode = GEMM_GJ; g.gj_k0 = k0; g.gj_b = bb;
        cudaError_t e = gemm(c, g, st, 2.0 * n * (double)(n - bb) * bb * batch, oz, err);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// The delayed Gauss-Jordan update of target columns t0 .. t0 + w - 1 by the eliminated columns
// p0 .. p0 + K - 1 (their pivot rows p0 .. p0 + K - 1): W[:, t] <- W[:, p] T + W[:, t] with the
// pivot rows replaced rather than added to, T = the target columns' pivot rows before the update.
GemmBatch gj_update_batch(int n, int batch, double** W, double** Tup, int p0, int K, int t0, int w) {
    GemmBatch g = gb_basic(n, w, K, W, n, Tup, w, W, n, batch);
    g.offA = p0;
    g.offC = t0;
    g.Cin = (const double* const*)W; g.offCin = t0; g.ldcin = n; g.beta = 1.0;
    g.mode = GEMM_GJ; g.gj_k0 = p0; g.gj_b = K; g.gj_cols = 0;
    return g;
}

// whether an emulated update of w target columns by K eliminated columns takes both operands'
// slices from one kernel (gj_update_slice_kernel): small K and w, the whole batch in the slice
// scratch
bool gj_presliced(const OzBuf* oz, const int* err, int n, int batch, int K, int w) {
    if (!oz || !oz->base || !err || K > 64 || w > 64 || K < 1 || w < 1) return false;
    return oz_chunk_entries(gj_update_batch(n, batch, nullptr, nullptr, 0, K, 0, w), *oz) >= batch;
}

// columns t0 .. t0 + w - 1 of every W updated by the eliminated columns p0 .. p0 + K - 1
cudaError_t gj_update(sgs_ctx* c, int n, int batch, double** W, double** Tup, int p0, int K, int t0, int w,
                      cudaStream_t st, const OzBuf* oz, int* err) {
    const GemmBatch g = gj_update_batch(n, batch, W, Tup, p0, K, t0, w);
    const bool presliced = gj_presliced(oz, err, n, batch, K, w);
    if (presliced) {
        const OzLayout L = oz_layout(n, w, K, *oz, batch);
        gj_update_slice_kernel<<<dim3((L.mp + GJ_SLICE_ROWS - 1) / GJ_SLICE_ROWS + 1, batch), 256, 0, st>>>(
            W, n, p0, K, t0, w, L.as, L.ea, L.mp, L.bs, L.eb, L.np, L.kp);
        counted();
    } else {
        gj_gather_rows_kernel<<<dim3(grid_chunks((size_t)K * w, 256, 64), batch), 256, 0, st>>>(W, Tup, n, p0, K, t0,
                                                                                               w);
        counted();
    }
    return gemm(c, g, st, 2.0 * n * (double)w * K * batch, oz, err, presliced);
}

// Recursive blocked Gauss-Jordan of columns c0 .. c1 - 1: the left half, its transformation
// applied to the right half's columns (one product of K = the left half's width), the right
// half, its transformation applied to the left half's columns; columns of at most `leaf` are a
// panel (gj_panel_kernel).  Columns outside c0 .. c1 - 1 receive only the row interchanges
// (the panels apply them to every other column); their update by this range is the caller's.
// Every level updates n x n / 2 elements per matrix, about log2(n / leaf) levels in all,
// against n / leaf full n x n updates of the one-level blocked form.
cudaError_t gj_recurse(sgs_ctx* c, int n, int batch, int leaf, int c0, int c1, double** W, double** T, double** Tup,
                       int* piv, double* logdet, double* dsign, int* err, double tiny, cudaStream_t st,
                       const OzBuf* oz) {
    if (c1 - c0 <= leaf) {
        const int bb = c1 - c0;
        GJPanelArgs a{W, T, piv, logdet, dsign, err, n, c0, bb, tiny};
        gj_panel_kernel<<<batch, 512, (size_t)n * (bb + 1) * sizeof(double) + bb * sizeof(double), st>>>(a);
        counted();
        return cudaGetLastError();
    }
    const int leaves = (c1 - c0 + leaf - 1) / leaf;
    const int m = c0 + ((leaves + 1) / 2) * leaf;
    cudaError_t e = gj_recurse(c, n, batch, leaf, c0, m, W, T, Tup, piv, logdet, dsign, err, tiny, st, oz);
    if (e == cudaSuccess) e = gj_update(c, n, batch, W, Tup, c0, m - c0, m, c1 - m, st, oz, err);
    if (e == cudaSuccess) e = gj_recurse(c, n, batch, leaf, m, c1, W, T, Tup, piv, logdet, dsign, err, tiny, st, oz);
    if (e == cudaSuccess) e = gj_update(c, n, batch, W, Tup, m, c1 - m, c0, m - c0, st, oz, err);
    return e;
}

// S^{-1} in place in W by the recursive form; Tup: per matrix n * n / 4 doubles of scratch
cudaError_t launch_gj_recursive(sgs_ctx* c, int n, int batch, int leaf, double** W, double** T, double** Tup,
                                int* piv, double* logdet, double* dsign, int* err, double tiny, cudaStream_t st,
                                const OzBuf* oz) {
    set_kernel_attributes();
    return gj_recurse(c, n, batch, leaf, 0, n, W, T, Tup, piv, logdet, dsign, err, tiny, st, oz);
}

// upA, upB, upC: 2 batch entries, 2 b and 2 b + 1 the real and imaginary parts of matrix b's update
cudaError_t launch_pf(sgs_ctx* c, int n, int batch, int bsmax, double** Y, double** TU, double** PK, double** upA,
                      double** upB, double** upC, double* logabs, double* phase, int* err, cudaStream_t st,
                      const OzBuf* oz = nullptr) {
    const size_t smem = (4 * (size_t)n + 4 * bsmax) * sizeof(double);
    set_kernel_attributes();
    for (int k0 = 0; k0 < n; k0 += 2 * bsmax) {
        const int bs = std::min(bsmax, (n - k0) / 2);
        const int e0 = k0 + 2 * bs;
        PfPanelArgs a{Y, TU, PK, logabs, phase, err, n, k0, bs, bsmax, nullptr, nullptr, nullptr, nullptr, 0, 0};
        GemmBatch g = gb_basic(n - e0, n - e0, 4 * bs, upA, 4 * bs, upB, 4 * bs, upC, n, 2 * batch);
        // emulated update: the panel writes the operands' slices itself when the whole batch
        // fits the slice scratch (no FP64 packs, no slicing launches)
        const bool sliced = e0 < n && oz && oz->base && err && bs % 4 == 0 && oz_chunk_entries(g, *oz) >= g.batch;
        if (sliced) {
            const OzLayout L = oz_layout(g.m, g.n, g.k, *oz, g.batch);
            a.sa = L.as; a.sb = L.bs; a.ea = L.ea; a.eb = L.eb; a.mp = L.mp; a.np = L.np;
        }
        pf_panel_kernel<<<batch, PF_PANEL_THREADS, smem, st>>>(a);
        counted();
        if (e0 >= n) break;
        g.offA = (long long)e0 * 4 * bs;
        g.offB = (long long)e0 * 4 * bs;
        g.transB = 1;
        g.offC = (long long)e0 * n + e0;
        // the rank-2b complex update T U^T - U T^T is antisymmetric, as is the trailing
        // block it updates: compute the lower tiles and mirror them.  The panels keep only the
        // upper triangle current, so Cin(r, c) = -Y[c][r]: read transposed with beta = -1
        g.Cin = (const double* const*)upC; g.offCin = g.offC; g.ldcin = n; g.beta = -1.0;
        g.cin_trans = 1;
        g.mode = GEMM_SKEW;
        const double m2 = (double)(n - e0) * (n - e0);
        const cudaError_t e = gemm(c, g, st, m2 * 4.0 * bs * 2 * batch, oz, err, sliced);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Gauss-Jordan inverses (pivoted, FP64) of pairs p0 .. p0 + cnt - 1 of the current chunk, whose
// S = Gamma_a + Gamma_b is in the work matrices, with log|det S| and its sign; S^{-1} gathered out
// of the pivoted form.  S has entries of magnitude <= 2; two states of opposite parity give a
// pivot at rounding level (~1e-15), same-parity pairs O(0.1).
cudaError_t inverse_range(sgs_ctx* c, Instance& I, int p0, int cnt, cudaStream_t st, const OzBuf* oz) {
    const int n = I.n;
    const size_t nn = (size_t)n * n, po = (size_t)p0 * n;
    cudaError_t e = launch_gj_recursive(c, n, cnt, I.gj_b, I.p_work + p0, I.p_tbuf + p0, I.p_tup + p0, I.piv + po,
                                        I.logdet + p0, I.dsign + p0, I.err, 1e-12, st, oz);
    if (e != cudaSuccess) return e;
    gj_perm_kernel<<<cnt, 128, 2 * (size_t)n * sizeof(int), st>>>(I.piv + po, I.perm + po, n, cnt);
    gj_gather_kernel<<<dim3(grid_chunks(nn, 256, 64), cnt), 256, 0, st>>>(I.p_work + p0, I.p_si + p0, I.perm + po, n);
    counted(); counted();
    return cudaGetLastError();
}

// S = Gamma_a + Gamma_b and S^{-1} for every pair of the current chunk
cudaError_t pair_inverse(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const size_t nn = (size_t)I.n * I.n;
    pair_sum_kernel<<<dim3(grid_chunks(nn, 256, 64), I.ccnt()), 256, 0, st>>>(I.dev(), I.work);
    counted();
    return inverse_range(c, I, 0, I.ccnt(), st, &I.oz);
}

// Im Delta^{a,b} = (G_a - G_b) S^{-1} of pairs p0 .. p0 + cnt - 1 of the current chunk (side: with
// the side stream's slice scratch)
cudaError_t delta_range(sgs_ctx* c, Instance& I, int p0, int cnt, cudaStream_t st, int side) {
    const int n = I.n;
    GemmBatch g = gb_basic(n, n, n, I.p_ga + I.coff() + p0, n, I.p_si + p0, n, I.p_imd + p0, n, cnt);
    g.A2 = (const double* const*)(I.p_gb + I.coff() + p0); g.sA2 = -1.0;
    g.mode = GEMM_SKEW;
    g.b_antisym = 1;        // S^{-1} (antisymmetric up to the inversion's rounding)
    I.oz_side = side;
    const cudaError_t e = gemm(c, I, g, st, (double)n * n * n * cnt);   // antisymmetric product: half of 2 n^3
    I.oz_side = 0;
    return e;
}

// phase Pfaffians Pf(Gamma_0 + Delta^{a,b}) of the pairs without the reference state
cudaError_t pair_phase(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n;
    const size_t nn = (size_t)n * n;
    pf_build_kernel<<<dim3(grid_chunks(nn, 256, 64), I.cpfcnt()), 256, 0, st>>>(I.dev(), I.si, I.imd, I.work);
    counted();
    return launch_pf(c, n, I.cpfcnt(), I.pf_bs, I.p_Y, I.p_TU, I.p_pack, I.p_upA, I.p_upB, I.p_upC, I.pflog,
                     I.pfphase, I.err, st, &I.oz);
}

// S^{-1} and Im Delta of the current chunk's pairs (A1, A2, A4).  split: the pairs in two halves,
// the second on the instance's side stream with the side slice scratch, so that one half's
// Gauss-Jordan panels (FP64 pipe) run beside the other half's emulated products (tensor and
// integer pipes)
cudaError_t pair_factors(sgs_ctx* c, Instance& I, cudaStream_t st, bool split = false) {
    const double n3 = (double)I.n * I.n * I.n;
    const int P = I.ccnt();
    if (P == 0) return cudaSuccess;
    c->stage(SGS_STAGE_PAIR_INVERSE);
    c->stage_flops[SGS_STAGE_PAIR_INVERSE] += 2.0 * n3 * P;
    cudaError_t e;
    if (!(split && P >= 2 && I.st2 && I.oz2.base)) {
        if ((e = pair_inverse(c, I, st)) != cudaSuccess) return e;
        c->stage(SGS_STAGE_PAIR_DELTA);
        c->stage_flops[SGS_STAGE_PAIR_DELTA] += n3 * P;
        return delta_range(c, I, 0, P, st, 0);
    }
    c->stage_flops[SGS_STAGE_PAIR_DELTA] += n3 * P;
    const int PA = (P + 1) / 2, PB = P - PA;
    pair_sum_kernel<<<dim3(grid_chunks((size_t)I.n * I.n, 256, 64), P), 256, 0, st>>>(I.dev(), I.work);
    counted();
    if ((e = cudaEventRecord(I.ev_fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(I.st2, I.ev_fork, 0)) != cudaSuccess) return e;
    if ((e = inverse_range(c, I, 0, PA, st, &I.oz)) != cudaSuccess) return e;
    if ((e = inverse_range(c, I, PA, PB, I.st2, &I.oz2)) != cudaSuccess) return e;
    if ((e = delta_range(c, I, 0, PA, st, 0)) != cudaSuccess) return e;
    if ((e = delta_range(c, I, PA, PB, I.st2, 1)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(I.ev_join, I.st2)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(st, I.ev_join, 0);
}

// pair pass (A1-A5) of one instance, chunk by chunk: S^{-1}, Im Delta, phase Pfaffians, then G, h
// and the impurity blocks of F for its pairs (and, with the first chunk, for its states)
cudaError_t pair_products(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n, M = I.M;
    const double n3 = (double)n * n * n;
    const int ni = std::max(I.nimp, 1);
    for (int ch = 0; ch < I.nch(); ch++) {
        I.cur = ch;
        const int P = I.ccnt();
        cudaError_t e = pair_factors(c, I, st);
        if (e != cudaSuccess) return e;
        if (I.cpfcnt() > 0) {
            c->stage(SGS_STAGE_PHASE_PFAFFIAN);
            c->stage_flops[SGS_STAGE_PHASE_PFAFFIAN] += 4.0 / 3.0 * n3 * I.cpfcnt();
            if ((e = pair_phase(c, I, st)) != cudaSuccess) return e;
        }
        c->stage(SGS_STAGE_AMPLITUDES);
        pair_gh_kernel<<<P + (ch == 0 ? M : 0), 256, 0, st>>>(I.dev(), I.si, I.imd, I.logdet, I.pfphase, I.Gm, I.hm,
                                                              I.fimp + (size_t)I.coff() * ni * ni * 2, I.fimp_state,
                                                              GH_ALL, I.dens);
        counted();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    I.cur = 0;
    return cudaSuccess;
}

// amplitude solve (A6) on the instance's G, h; E -> Eout
cudaError_t amplitudes(Instance& I, double* Eout, cudaStream_t st) {
    AmpArgs aa{I.M, I.Gm, I.hm, I.eigscratch, Eout, I.lam, I.lt, I.coef, I.cmode, 1e-12, I.err};
    amp_solve_kernel<<<1, 256, 0, st>>>(aa);
    counted();
    return cudaGetLastError();
}

// pair pass + amplitude solve for one instance; E -> Eout
cudaError_t pair_pass(sgs_ctx* c, Instance& I, double* Eout, cudaStream_t st) {
    cudaError_t e = pair_products(c, I, st);
    if (e != cudaSuccess) return e;
    return amplitudes(I, Eout, st);
}

// a pair-sharded instance's share of (G, h) for the sum over ranks: out = [G | h], each
// [M][M] complex; entries of pairs this rank does not hold are zero (memset before the pair
// pass), the diagonal (state mu's own G_mu,mu = 1 and h_mu,mu) is kept on the rank that adds
// state mu's own terms and zeroed elsewhere
__global__ void shard_export_gh_kernel(const double* Gm, const double* hm, int M, const int* self_mask,
                                       double* out) {
    const int MM = M * M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MM; e += gridDim.x * blockDim.x) {
        const int a = e / M, b = e % M;
        const bool keep = a != b || self_mask[a] != 0;
        out[2 * e] = keep ? Gm[2 * e] : 0.0;
        out[2 * e + 1] = keep ? Gm[2 * e + 1] : 0.0;
        out[2 * MM + 2 * e] = keep ? hm[2 * e] : 0.0;
        out[2 * MM + 2 * e + 1] = keep ? hm[2 * e + 1] : 0.0;
    }
}

// ------------------------------------------------------------------ autotuning

std::mutex g_tune_mu;
std::map<std::array<int, 3>, std::array<int, 2>> g_tune_cache;   // (n, rank, precision) -> widths

// Time the candidate widths on the instance's own pairs (CUDA events on the context
// stream, best of two), keep the fastest; a shape already timed in this process reuses
// its widths.  Results change only by rounding.
sgs_status autotune_instance(sgs_ctx* c, Instance& I) {
    if (I.P == 0) return SGS_OK;
    const std::array<int, 3> key{I.n, I.M, I.prec};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            I.tuned_from_cache = 1;
            return set_panel_pointers(c, I, it->second[0], it->second[1]);
        }
    }
    cudaStream_t st = c->stream;
    const bool prof = c->prof;
    c->prof = false;
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    sgs_status status = SGS_OK;
    auto timed = [&](auto&& prep, auto&& work) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 2 && status == SGS_OK; rep++) {
            cudaError_t e = prep();
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = work();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                c->err = std::string("autotune: ") + cudaGetErrorString(e);
                status = SGS_ECUDA;
            } else {
                best = std::min(best, ms);
            }
        }
        return best;
    };
    int gj = I.gj_b, pf = I.pf_bs;
    float best = 1e30f;
    for (int b : gj_candidates(I.n)) {
        if (b > I.gj_cap) continue;
        if ((status = set_panel_pointers(c, I, b, pf)) != SGS_OK) break;
        const float t = timed([&] { return cudaSuccess; }, [&] { return pair_inverse(c, I, st); });
        if (t < best) { best = t; gj = b; }
    }
    if (status == SGS_OK && I.Ppf > 0) {
        status = set_panel_pointers(c, I, gj, pf);
        cudaError_t e = cudaSuccess;
        if (status == SGS_OK) e = pair_inverse(c, I, st);
        if (e == cudaSuccess) e = delta_range(c, I, 0, I.ccnt(), st, 0);
        if (e != cudaSuccess) { c->err = std::string("autotune: ") + cudaGetErrorString(e); status = SGS_ECUDA; }
        best = 1e30f;
        for (int b : pf_candidates(I.n)) {
            if (status != SGS_OK || b > I.pf_cap) continue;
            if ((status = set_panel_pointers(c, I, gj, b)) != SGS_OK) break;
            const float t = timed([&] { return cudaSuccess; }, [&] { return pair_phase(c, I, st); });
            if (t < best) { best = t; pf = b; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = prof;
    if (status != SGS_OK) return status;
    if ((status = set_panel_pointers(c, I, gj, pf)) != SGS_OK) return status;
    CUDA_TRY(c, cudaMemsetAsync(I.err, 0, sizeof(int), st));      // trial runs leave no error state
    CUDA_TRY(c, cudaStreamSynchronize(st));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {gj, pf};
    I.tuned_from_cache = 0;
    return SGS_OK;
}

// the pair part of the equation of motion for the current chunk's pairs: the dense products W, V,
// X, the low-rank impurity terms and the Delta F Delta planes Q (into xa, wr)
cudaError_t eom_pair_chunk(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n, P = I.ccnt();
    const size_t nn = (size_t)n * n;
    const double n3 = (double)n * n * n;
    const int ni = std::max(I.nimp, 1);
    const double* fimp = I.fimp + (size_t)I.coff() * ni * ni * 2;
    double** ga = I.p_ga + I.coff();
    double** gb = I.p_gb + I.coff();
    InstDev d = I.dev();
    cudaError_t e;
    c->stage(SGS_STAGE_EOM_W);
    c->stage_flops[SGS_STAGE_EOM_W] += n3 * P;   // Wr: antisymmetric
    if (I.tc_kind >= 0) {
        // tensor-core path: W = T1 S^{-1}, V = D W, X = V D, every B antisymmetric, so its
        // K-major form is -B and alpha = -1
        const int kind = I.tc_kind;
        const unsigned gch = grid_chunks(nn, 256, 64);
        pair_sparse_right_kernel<<<dim3(gch, P), 256, 0, st>>>(d, I.si, fimp, I.va);   // T1 (V later)
        const int ldp = I.ldp;
        lp_convert_kernel<double><<<dim3(gch, P), 256, 0, st>>>((const double* const*)I.p_si, nullptr, I.q_si_hi,
                                                                  I.q_si_lo, n, ldp, kind);
        lp_convert_kernel<double><<<dim3(gch, P), 256, 0, st>>>((const double* const*)I.p_va, nullptr, I.q_t1_hi,
                                                                  I.q_t1_lo, n, ldp, kind);
        lp_convert_kernel<double><<<dim3(gch, P), 256, 0, st>>>((const double* const*)ga, (const double* const*)gb,
                                                                  I.q_d_hi, I.q_d_lo, n, ldp, kind);
        counted(); counted(); counted(); counted();
        TmaBatch tw = I.tma_w, tv = I.tma_v, tx = I.tma_x;
        tw.batch = tv.batch = tx.batch = P;
        if ((e = tma_product(tw, kind, st)) != cudaSuccess) return e;
        counted();
        lp_convert_kernel<float><<<dim3(gch, P), 256, 0, st>>>((const float* const*)I.q_wr32, nullptr, I.q_wr_hi,
                                                                 I.q_wr_lo, n, ldp, kind);
        counted();
        c->stage(SGS_STAGE_EOM_V);
        c->stage_flops[SGS_STAGE_EOM_V] += 2.0 * n3 * P;
        if ((e = tma_product(tv, kind, st)) != cudaSuccess) return e;
        counted();
        c->stage(SGS_STAGE_EOM_X);
        c->stage_flops[SGS_STAGE_EOM_X] += n3 * P;
        lp_convert_kernel<float><<<dim3(gch, P), 256, 0, st>>>((const float* const*)I.q_va32, nullptr, I.q_va_hi,
                                                                 I.q_va_lo, n, ldp, kind);
        counted();
        if ((e = tma_product(tx, kind, st)) != cudaSuccess) return e;
        counted();
        c->stage(SGS_STAGE_EOM_ASSEMBLY);
        if (I.nimp > 0) {
            pair_lr_kernel<<<dim3(grid_chunks((size_t)n * I.nimp, 256, 64), P), 256, 0, st>>>(d, I.si, I.imd, fimp, I.lr);
            counted();
        }
        pair_q_kernel<float><<<dim3(lower_tile_count(n), P), 256, 0, st>>>(d, I.si, I.imd, I.lr, I.va32, I.xa32, I.wr32, I.xa, I.wr);
        counted();
    } else {
        // T1 = S^{-1} (A + Re Fimp)  (into va; V later), Wr = T1 S^{-1}
        pair_sparse_right_kernel<<<dim3(grid_chunks(nn, 256, 64), P), 256, 0, st>>>(d, I.si, fimp, I.va);
        counted();
        GemmBatch g = gb_basic(n, n, n, I.p_va, n, I.p_si, n, I.p_wr, n, P);
        g.mode = GEMM_SKEW;
        g.b_antisym = 1;    // S^{-1}
        if ((e = gemm(c, I, g, st, n3 * P)) != cudaSuccess) return e;
        // V = D Wr
        c->stage(SGS_STAGE_EOM_V);
        c->stage_flops[SGS_STAGE_EOM_V] += 2.0 * n3 * P;
        c->stage_bytes[SGS_STAGE_EOM_V] += 8.0 * nn * (2.0 * P + I.M);   // read Wr, write V; Gamma once
        g = gb_basic(n, n, n, ga, n, I.p_wr, n, I.p_va, n, P);
        g.A2 = (const double* const*)gb; g.sA2 = -1.0;
        g.b_antisym = 1;    // Wr (an antisymmetric product)
        if ((e = gemm(c, I, g, st, 2.0 * n3 * P)) != cudaSuccess) return e;
        // X = V D
        c->stage(SGS_STAGE_EOM_X);
        c->stage_flops[SGS_STAGE_EOM_X] += n3 * P;
        g = gb_basic(n, n, n, I.p_va, n, ga, n, I.p_xa, n, P);
        g.B2 = (const double* const*)gb; g.sB2 = -1.0;
        g.mode = GEMM_SKEW;
        g.b_antisym = 1;    // Gamma_a - Gamma_b
        if ((e = gemm(c, I, g, st, n3 * P)) != cudaSuccess) return e;
        c->stage(SGS_STAGE_EOM_ASSEMBLY);
        if (I.nimp > 0) {
            pair_lr_kernel<<<dim3(grid_chunks((size_t)n * I.nimp, 256, 64), P), 256, 0, st>>>(d, I.si, I.imd, fimp, I.lr);
            counted();
        }
        pair_q_kernel<double><<<dim3(lower_tile_count(n), P), 256, 0, st>>>(d, I.si, I.imd, I.lr, I.va, I.xa, I.wr,
                                                                            I.xa, I.wr);
        counted();
    }
    return cudaGetLastError();
}

// the states' part of the equation of motion: T2 = F Gamma (s0), GFG = Gamma T2 (s4)
cudaError_t eom_states(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n, M = I.M;
    const size_t nn = (size_t)n * n;
    const double n3 = (double)n * n * n;
    c->stage(SGS_STAGE_EOM_W);
    c->stage_flops[SGS_STAGE_EOM_W] += n3 * M;   // Gamma F Gamma: antisymmetric
    state_sparse_left_kernel<<<dim3(grid_chunks(nn, 256, 256), M), 256, 0, st>>>(I.dev(), I.fimp_state, I.s[0]);
    counted();
    GemmBatch g = gb_basic(n, n, n, I.p_gamma, n, I.p_s[0], n, I.p_s[4], n, M);
    g.mode = GEMM_SKEW;
    return gemm(c, I, g, st, n3 * M);
}

// the sums over beta of the current chunk's pairs: D into dGamma, T into s1 (accumulate: add onto
// them), and the finish part given
void eom_sums(sgs_ctx* c, Instance& I, cudaStream_t st, int accumulate, int part, const InstDev& d) {
    const int n = I.n, M = I.M;
    const int ni = std::max(I.nimp, 1);
    const dim3 eg(lower_tile_count(n), M);
    const double* fimp = I.fimp + (size_t)d.p_off * ni * ni * 2;
    double* tsum = I.s[1];
    if (part & EOM_FINISH_PAIRS) {
        if (I.tc_kind >= 0)
            eom_pairs_kernel<float><<<eg, 256, eom_smem<float>(M), st>>>(d, I.si, I.imd, I.xa, I.wr, I.coef,
                                                                         I.pair_index, tsum, I.dgamma, accumulate);
        else
            eom_pairs_kernel<double><<<eg, 256, eom_smem<double>(M), st>>>(d, I.si, I.imd, I.xa, I.wr, I.coef,
                                                                           I.pair_index, tsum, I.dgamma, accumulate);
        counted();
    }
    if (I.tc_kind >= 0)
        eom_finish_kernel<float><<<eg, 256, eom_smem<float>(M), st>>>(d, I.si, I.imd, fimp, I.fimp_state, I.s[4],
                                                                      I.coef, I.pair_index, tsum, I.dgamma,
                                                                      I.self_mask, part);
    else
        eom_finish_kernel<double><<<eg, 256, eom_smem<double>(M), st>>>(d, I.si, I.imd, fimp, I.fimp_state, I.s[4],
                                                                        I.coef, I.pair_index, tsum, I.dgamma,
                                                                        I.self_mask, part);
    counted();
}

// the end of the assembly: byte accounting (the assembly kernels store dGamma exactly
// antisymmetric, the float forms included)
cudaError_t eom_close(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n, M = I.M;
    const size_t nn = (size_t)n * n;
    // algorithmic bytes: pair_q reads Si, Im, V (twice), X, Wr and writes Qr, Qi; the EOM
    // reads Si, Im, Qr, Qi once per receiver of each pair plus Gamma, GFG and writes dGamma
    c->stage_bytes[SGS_STAGE_EOM_ASSEMBLY] += 8.0 * nn * (7.0 * I.P + 8.0 * I.P + 3.0 * M);
    return cudaGetLastError();
}

// Equation of motion of every state (A7).  The pairs' part runs chunk by chunk, last chunk first:
// its S^{-1} and Im Delta are still those of the pair pass; the other chunks recompute theirs.
// The pair sums D (into dGamma) and T (into s1) accumulate over the chunks; the last part of the
// assembly (sparse terms on T, the beta = mu terms) runs once.
cudaError_t eom_pass(sgs_ctx* c, Instance& I, cudaStream_t st) {
    cudaError_t e = eom_states(c, I, st);
    if (e != cudaSuccess) return e;
    const int nch = I.nch();
    const bool chunked = nch > 1;
    for (int ch = nch - 1; ch >= 0; ch--) {
        I.cur = ch;
        if (chunked && ch != nch - 1 && (e = pair_factors(c, I, st)) != cudaSuccess) return e;
        if (I.ccnt() > 0 && (e = eom_pair_chunk(c, I, st)) != cudaSuccess) return e;
        c->stage(SGS_STAGE_EOM_ASSEMBLY);
        eom_sums(c, I, st, ch != nch - 1, chunked ? EOM_FINISH_PAIRS : EOM_FINISH_ALL, I.dev());
    }
    I.cur = 0;
    if (chunked) eom_sums(c, I, st, 0, EOM_FINISH_REST, I.dev_all());
    return eom_close(c, I, st);
}

// exp(X_s) for the first `batch` states (App. A), X_s = 2^-s X in s1 as exp_prepare_kernel
// leaves it: the degree-10 Taylor polynomial by Paterson-Stockmeyer in blocks of three,
//   X2 = X_s^2 (s0), Y = X_s^3 (s2, antisymmetric), P = B3 (s3),
//   P <- P Y + B_j for j = 2, 1, 0, B_j = c_{3j} I + c_{3j+1} X_s + c_{3j+2} X2, c_k = 1/k!
// (the addends fused into the products' epilogue), then the squarings each state needs
// (states with fewer pass their matrix through).  *cur_out <- the s buffer (3 or 4) that holds R.
cudaError_t exp_products(sgs_ctx* c, Instance& I, int batch, cudaStream_t st, int* cur_out) {
    const int n = I.n;
    const size_t nn = (size_t)n * n;
    const double n3 = (double)n * n * n;
    static_assert(EXP_TAYLOR_DEGREE == 10, "blocks of three cover degrees 0..11");
    double cf[12];
    cf[0] = 1.0;
    for (int k = 1; k < 12; k++) cf[k] = cf[k - 1] / k;
    cf[11] = 0.0;                                         // degree 10
    cudaError_t e;
    GemmBatch g = gb_basic(n, n, n, I.p_s[1], n, I.p_s[1], n, I.p_s[0], n, batch);
    if ((e = gemm(c, I, g, st, 2.0 * n3 * batch)) != cudaSuccess) return e;         // X2
    g = gb_basic(n, n, n, I.p_s[0], n, I.p_s[1], n, I.p_s[2], n, batch);
    g.mode = GEMM_SKEW;                                                            // Y = X2 X_s
    if ((e = gemm(c, I, g, st, n3 * batch)) != cudaSuccess) return e;
    scaled_plus_identity_kernel<<<grid_chunks(batch * nn, 256, 4096), 256, 0, st>>>(I.s[1], cf[10], cf[9], n, I.s[3],
                                                                                   batch * nn);
    counted();
    int cur = 3;
    for (int j = 2; j >= 0; j--) {
        const int nxt = (cur == 3) ? 4 : 3;
        g = gb_basic(n, n, n, I.p_s[cur], n, I.p_s[2], n, I.p_s[nxt], n, batch);
        g.Cin = (const double* const*)I.p_s[0]; g.ldcin = n; g.beta = cf[3 * j + 2];
        g.Cin2 = (const double* const*)I.p_s[1]; g.beta2 = cf[3 * j + 1];
        g.diag = cf[3 * j];
        if ((e = gemm(c, I, g, st, 2.0 * n3 * batch)) != cudaSuccess) return e;
        cur = nxt;
    }
    for (int j = 0; j < EXP_MAX_SQUARINGS; j++) {
        const int nxt = (cur == 3) ? 4 : 3;
        g = gb_basic(n, n, n, I.p_s[cur], n, I.p_s[cur], n, I.p_s[nxt], n, batch);
        g.active_flag = I.sq; g.active_cmp = j;
        g.Cin = (const double* const*)I.p_s[cur]; g.ldcin = n; g.beta = 0.0;
        if ((e = gemm(c, I, g, st, -1.0)) != cudaSuccess) return e;
        cur = nxt;
    }
    *cur_out = cur;
    return cudaSuccess;
}

// Canonical-form renormalisation (App. A, Eq. CM-normal-form with every lambda_j = 1): the polar
// factor of the matrices in s4 by `iters` Newton-Schulz steps X <- 1.5 X + 0.5 X (X X); the result
// goes to gamma.
cudaError_t polar_pass(sgs_ctx* c, Instance& I, int iters, cudaStream_t st, int from = 4) {
    const int n = I.n, M = I.M;
    const size_t nn = (size_t)n * n;
    const double n3 = (double)n * n * n;
    cudaError_t e;
    double** src = I.p_s[from];
    double** dst = I.p_gamma;
    for (int it = 0; it < iters; it++) {
        GemmBatch g = gb_basic(n, n, n, src, n, src, n, I.p_s[0], n, M);
        if ((e = gemm(c, I, g, st, n3 * M)) != cudaSuccess) return e;     // X X: symmetric, half counted
        g = gb_basic(n, n, n, src, n, I.p_s[0], n, dst, n, M);
        g.alpha = 0.5; g.Cin = (const double* const*)src; g.ldcin = n; g.beta = 1.5; g.mode = GEMM_SKEW;
        if ((e = gemm(c, I, g, st, n3 * M)) != cudaSuccess) return e;
        std::swap(src, dst);
    }
    if (src == I.p_s[from]) {  // an even number of iterations ends in the source buffer
        copy_kernel<<<grid_chunks(M * nn, 256, 4096), 256, 0, st>>>(I.s[from], I.gamma, M * nn);
        counted();
    }
    return cudaGetLastError();
}

// the mixed forms' state update: products on the tensor cores, sums and purification in FP64
TmaBatch lp_product(const Instance& I, int a_op, int b_op, double alpha, float* C, int ldc, long long cstride) {
    TmaBatch t{};
    t.ta = I.u_map_hi[a_op];
    t.tb = I.u_map_hi[b_op];
    if (I.tc_kind == TC_3XTF32) { t.ta2 = I.u_map_lo[a_op]; t.tb2 = I.u_map_lo[b_op]; }
    t.m = t.n = t.k = I.n;
    t.alpha = alpha;
    t.C = C; t.ldc = ldc; t.c_stride = cstride;
    t.out_f64 = 0; t.skew = 0; t.err = I.err; t.batch = I.M;
    return t;
}

cudaError_t update_pass_lp(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const int n = I.n, M = I.M, ldp = I.ldp, kind = I.tc_kind;
    const size_t nn = (size_t)n * n, np = (size_t)n * ldp, mp = (size_t)M * np;
    const double n3 = (double)n * n * n;
    cudaError_t e;
    c->stage(SGS_STAGE_UPDATE);
    // Gamma dGamma 2, four Horner products 8, E^T 2, F 2, G 2, purification 2 per iteration
    // (squarings are added when profiles are read)
    c->stage_flops[SGS_STAGE_UPDATE] += (16.0 + 2.0 * LP_NS_ITERS) * n3 * M;
    const unsigned gch = grid_chunks(np, 256, 256);
    auto split = [&](int f32, int op) {
        lp_split_kernel<<<grid_chunks(mp, 256, 4096), 256, 0, st>>>(I.u_f32[f32], I.u_hi[op], I.u_lo[op], mp, kind);
        counted();
    };
    auto run = [&](const TmaBatch& t) { counted(); return tma_product(t, kind, st); };
    lp_from_f64_kernel<<<dim3(gch, M), 256, 0, st>>>(I.gamma, n, ldp, I.u_hi[0], I.u_lo[0], kind);
    lp_from_f64_kernel<<<dim3(gch, M), 256, 0, st>>>(I.dgamma, n, ldp, I.u_hi[1], I.u_lo[1], kind);
    counted(); counted();
    // Y = Gamma dGamma (dGamma antisymmetric: its K-major form is -dGamma)
    if ((e = run(lp_product(I, 0, 1, -1.0, I.u_y, n, (long long)nn))) != cudaSuccess) return e;
    exp_prepare_lp_kernel<<<M, 1024, 0, st>>>(I.u_y, n, ldp, I.dtau, I.u_f32[0], I.u_f32[1], I.sq, I.err);
    counted();
    split(0, 2);
    split(1, 3);
    // Horner on transposes: Q_j = I + (1/j) Q_{j+1} X_s^T (X_s^T's K-major form is X_s)
    int cur = 1, nxt = 2;
    for (int j = EXP_LP_DEGREE - 1; j >= 2; j--) {
        TmaBatch t = lp_product(I, 2 + cur, 2, 1.0 / j, I.u_f32[nxt], ldp, (long long)np);
        t.diag = 1.0f;
        if ((e = run(t)) != cudaSuccess) return e;
        split(nxt, 2 + nxt);
        std::swap(cur, nxt);
    }
    // E^T = Q_2 X_s^T, and E
    {
        TmaBatch t = lp_product(I, 2 + cur, 2, 1.0, I.u_f32[3], ldp, (long long)np);
        t.CT = I.u_f32[4]; t.ldct = ldp; t.ct_stride = (long long)np;
        if ((e = run(t)) != cudaSuccess) return e;
        split(3, 5);
        split(4, 6);
    }
    // squarings E^T <- E^T E^T + 2 E^T (K-major form of E^T is E); states that need
    // fewer pass theirs through
    int et = 3, ee = 4, et2 = 5, ee2 = 6;
    for (int j = 0; j < EXP_MAX_SQUARINGS; j++) {
        TmaBatch t = lp_product(I, 2 + et, 2 + ee, 1.0, I.u_f32[et2], ldp, (long long)np);
        t.Cin = I.u_f32[et]; t.ldcin = ldp; t.cin_stride = (long long)np; t.beta = 2.0f;
        t.CT = I.u_f32[ee2]; t.ldct = ldp; t.ct_stride = (long long)np;
        t.pass_flag = I.sq; t.pass_cmp = j;
        if ((e = run(t)) != cudaSuccess) return e;
        split(et2, 2 + et2);
        split(ee2, 2 + ee2);
        std::swap(et, et2);
        std::swap(ee, ee2);
    }
    // F = E Gamma (Gamma's K-major form is -Gamma), G = F E^T (K-major form E)
    if ((e = run(lp_product(I, 2 + ee, 0, -1.0, I.u_f32[7], ldp, (long long)np))) != cudaSuccess) return e;
    split(7, 9);
    if ((e = run(lp_product(I, 9, 2 + ee, 1.0, I.u_f32[8], ldp, (long long)np))) != cudaSuccess) return e;
    assemble_lp_kernel<<<dim3(grid_chunks(nn, 256, 256), M), 256, 0, st>>>(I.gamma, I.u_f32[7], I.u_f32[8], n, ldp,
                                                                          I.s[4]);
    counted();
    if ((e = polar_pass(c, I, LP_NS_ITERS, st)) != cudaSuccess) return e;
    I.steps_since_profile++;
    return cudaGetLastError();
}

cudaError_t update_pass(sgs_ctx* c, Instance& I, cudaStream_t st) {
    if (I.u_ok && I.integrator == SGS_INTEGRATOR_EXP) return update_pass_lp(c, I, st);
    const int n = I.n, M = I.M;
    const size_t nn = (size_t)n * n;
    const double n3 = (double)n * n * n;
    cudaError_t e;
    c->stage(SGS_STAGE_UPDATE);
    if (I.integrator == SGS_INTEGRATOR_EULER) {
        // Eq. RKstep: Gamma + ds dGamma -> s4, then the polar factor
        c->stage_flops[SGS_STAGE_UPDATE] += 2.0 * EULER_NS_ITERS * n3 * M;
        axpy_kernel<<<grid_chunks(M * nn, 256, 4096), 256, 0, st>>>(I.gamma, I.dgamma, I.dtau, I.s[4], M * nn);
        counted();
        if ((e = polar_pass(c, I, EULER_NS_ITERS, st)) != cudaSuccess) return e;
        I.steps_since_profile++;
        return cudaGetLastError();
    }
    // Gamma dGamma 2, the exponential's X^2 2, X^3 1 (antisymmetric) and three block products 6,
    // R Gamma 2, (R Gamma) R^T 1 (antisymmetric), one Newton-Schulz iteration (X X and X (X X),
    // half each) 2; squarings are added when profiles are read
    c->stage_flops[SGS_STAGE_UPDATE] += (2.0 + 9.0 + 2.0 + 1.0 + 2.0) * n3 * M;
    // Y = Gamma dGamma -> s0 ; X_s -> s1
    GemmBatch g = gb_basic(n, n, n, I.p_gamma, n, I.p_dgamma, n, I.p_s[0], n, M);
    if ((e = gemm(c, I, g, st, 2.0 * n3 * M)) != cudaSuccess) return e;
    exp_prepare_kernel<<<M, 1024, 0, st>>>(I.s[0], I.s[1], n, I.dtau, I.sq, I.scale, I.err);
    counted();
    int cur = 3;
    if ((e = exp_products(c, I, M, st, &cur)) != cudaSuccess) return e;
    // T = R Gamma -> s0 ; Gamma' = T R^T -> s2
    g = gb_basic(n, n, n, I.p_s[cur], n, I.p_gamma, n, I.p_s[0], n, M);
    if ((e = gemm(c, I, g, st, 2.0 * n3 * M)) != cudaSuccess) return e;
    g = gb_basic(n, n, n, I.p_s[0], n, I.p_s[cur], n, I.p_s[2], n, M);
    g.transB = 1; g.mode = GEMM_SKEW;
    if ((e = gemm(c, I, g, st, n3 * M)) != cudaSuccess) return e;
    // R is orthogonal to rounding, so R Gamma R^T leaves purity only at rounding level, which one
    // Newton-Schulz iteration (error -> 1.5 error^2) removes
    if ((e = polar_pass(c, I, 1, st, 2)) != cudaSuccess) return e;
    I.steps_since_profile++;
    return cudaGetLastError();
}

// One step of an instance.  Unchunked instances fork after S^{-1} and Im Delta: the equation of
// motion's products (they need the pairs' Fock blocks, not the overlaps or the amplitudes) run on a
// side stream with their own slice scratch while the main stream computes the phase Pfaffians, G, h
// and the amplitudes; the assembly waits for both.  Before the fork the Gauss-Jordan inverses run as
// two halves of the pairs on the two streams.  In both places the FP64 panels of one stream share
// the GPU with the tensor-core products of the other (a third stream that split the Pfaffians too
// measured no faster: the Pfaffian phase already overlaps the products).  Chunked instances, and every
// instance while stage profiles are taken (their stage events are on one stream), run the stages
// in order.  E -> Ecur.
cudaError_t step_instance(sgs_ctx* c, Instance& I, cudaStream_t st) {
    const bool overlap = I.nch() == 1 && I.P > 0 && !c->prof;
    if (!overlap) {
        cudaError_t e = pair_pass(c, I, I.Ecur, st);
        if (e == cudaSuccess) e = eom_pass(c, I, st);
        if (e == cudaSuccess) e = update_pass(c, I, st);
        return e;
    }
    cudaError_t e = cudaSuccess;
    if (!I.st2) e = cudaStreamCreateWithFlags(&I.st2, cudaStreamNonBlocking);
    if (e == cudaSuccess && !I.ev_fork) e = cudaEventCreateWithFlags(&I.ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !I.ev_join) e = cudaEventCreateWithFlags(&I.ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    I.cur = 0;
    const int M = I.M, ni = std::max(I.nimp, 1);
    (void)ni;
    if ((e = pair_factors(c, I, st, true)) != cudaSuccess) return e;
    pair_gh_kernel<<<I.P + M, 256, 0, st>>>(I.dev(), I.si, I.imd, I.logdet, I.pfphase, I.Gm, I.hm, I.fimp,
                                            I.fimp_state, GH_FOCK, I.dens);
    counted();
    if ((e = cudaEventRecord(I.ev_fork, st)) != cudaSuccess) return e;
    // side stream: the products of the equation of motion
    if ((e = cudaStreamWaitEvent(I.st2, I.ev_fork, 0)) != cudaSuccess) return e;
    I.oz_side = 1;
    e = eom_states(c, I, I.st2);
    if (e == cudaSuccess) e = eom_pair_chunk(c, I, I.st2);
    I.oz_side = 0;
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(I.ev_join, I.st2)) != cudaSuccess) return e;
    // main stream: overlaps, amplitudes
    if (I.Ppf > 0) {
        c->stage(SGS_STAGE_PHASE_PFAFFIAN);
        c->stage_flops[SGS_STAGE_PHASE_PFAFFIAN] += 4.0 / 3.0 * (double)I.n * I.n * I.n * I.Ppf;
        if ((e = pair_phase(c, I, st)) != cudaSuccess) return e;
    }
    c->stage(SGS_STAGE_AMPLITUDES);
    pair_gh_kernel<<<I.P + M, 256, 0, st>>>(I.dev(), I.si, I.imd, I.logdet, I.pfphase, I.Gm, I.hm, I.fimp,
                                            I.fimp_state, GH_GRAM, I.dens);
    counted();
    if ((e = amplitudes(I, I.Ecur, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, I.ev_join, 0)) != cudaSuccess) return e;
    c->stage(SGS_STAGE_EOM_ASSEMBLY);
    eom_sums(c, I, st, 0, EOM_FINISH_ALL, I.dev());
    if ((e = eom_close(c, I, st)) != cudaSuccess) return e;
    return update_pass(c, I, st);
}

// Reads and clears the device error word of every live instance.  Every instance whose
// word was set is listed in c->failed_list (c->failed is the first); the status and
// message are those of the first, and the message counts the others.
sgs_status check_device_error(sgs_ctx* c) {
    c->failed = -1;
    c->failed_list.clear();
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    sgs_status first = SGS_OK;
    for (size_t i = 0; i < c->inst.size(); i++) {
        if (!c->inst[i].live) continue;
        int e = 0;
        CUDA_TRY(c, cudaMemcpy(&e, c->inst[i].err, sizeof(int), cudaMemcpyDeviceToHost));
        if (!e) continue;
        CUDA_TRY(c, cudaMemset(c->inst[i].err, 0, sizeof(int)));
        c->failed_list.push_back((int)i);
        if (first != SGS_OK) continue;
        c->failed = (int)i;
        char buf[160];
        if (e & SGS_DEV_SINGULAR) {
            snprintf(buf, sizeof buf, "instance %zu: two ansatz states have a singular Gamma_a + Gamma_b", i);
            first = SGS_ESINGULAR;
        } else if (e & SGS_DEV_TC_TIMEOUT) {
            snprintf(buf, sizeof buf, "instance %zu: a bounded tensor-core pipeline wait ran out", i);
            first = SGS_ETIMEOUT;
        } else if (e & SGS_DEV_PF_ZERO) {
            snprintf(buf, sizeof buf, "instance %zu: a state is orthogonal to the reference state", i);
            first = SGS_ESINGULAR;
        } else {
            snprintf(buf, sizeof buf, "instance %zu: %s", i,
                     (e & SGS_DEV_EIG) ? "amplitude solver did not converge" : "exponential step out of range");
            first = SGS_ENOTCONV;
        }
        c->err = buf;
    }
    if (c->failed_list.size() > 1)
        c->err += " (and " + std::to_string(c->failed_list.size() - 1) + " more failed instance(s))";
    return first;
}

bool any_sharded(const sgs_ctx* c) {
    for (const auto& I : c->inst)
        if (I.live && I.shard_world > 1) return true;
    return false;
}

sgs_status ensure_ehist(sgs_ctx* c, Instance& I, int n) {
    if (I.Ecap >= n) return SGS_OK;
    double* p = c->alloc<double>(n);
    if (!p) { c->err = "device allocation failed"; return SGS_ENOMEM; }
    I.Ehist = p;
    I.Ecap = n;
    return SGS_OK;
}

// Renyi-2 terms of subsystems too large for the shared-memory Pfaffian: chunks of pairs
// through the batched blocked Pfaffian (the phase Pfaffians' kernels), scratch owned by
// the instance and reused
sgs_status renyi_large(sgs_ctx* c, Instance& I, const double* blocks, const double* wts, long long npairs, int na2,
                       double log_norm, double* partial) {
    cudaStream_t st = c->stream;
    const int m = 2 * na2, bs = std::min(16, m / 2);
    const size_t mm = (size_t)m * m;
    const size_t per = 2 * mm + 4 * (size_t)m * bs + 16 * (size_t)m * bs + 3;     // doubles per chunk entry
    const long long chunk = std::max<long long>(1, std::min<long long>(npairs, (long long)((1ull << 30) / (per * 8))));
    const size_t need = (size_t)chunk * per + 8;
    if (I.renyi_cap < need || I.renyi_chunk != chunk || I.renyi_m != m) {
        c->owner = &I;
        I.renyi_scratch = c->alloc<double>(need);
        if (!I.renyi_scratch) { c->owner = nullptr; c->err = "device allocation failed"; return SGS_ENOMEM; }
        double* Y = I.renyi_scratch;
        double* TU = Y + (size_t)chunk * 2 * mm;
        double* PK = TU + (size_t)chunk * 4 * m * bs;
        const size_t blk = (size_t)m * 4 * bs;
        std::vector<double*> y, tu, pk, upA, upB, upC;
        for (long long q = 0; q < chunk; q++) {
            y.push_back(Y + (size_t)q * 2 * mm);
            tu.push_back(TU + (size_t)q * 4 * m * bs);
            pk.push_back(PK + (size_t)q * 4 * blk);
        }
        for (long long q = 0; q < chunk; q++) {     // entries 2 q, 2 q + 1: real and imaginary parts
            upA.push_back(pk[q]); upB.push_back(pk[q] + blk); upC.push_back(y[q]);
            upA.push_back(pk[q] + 2 * blk); upB.push_back(pk[q] + 3 * blk); upC.push_back(y[q] + mm);
        }
        I.r_Y = upload_ptrs(c, y); I.r_TU = upload_ptrs(c, tu); I.r_PK = upload_ptrs(c, pk);
        I.r_upA = upload_ptrs(c, upA); I.r_upB = upload_ptrs(c, upB); I.r_upC = upload_ptrs(c, upC);
        I.renyi_err = c->alloc<int>(1);
        c->owner = nullptr;
        if (!I.r_Y || !I.r_TU || !I.r_PK || !I.r_upA || !I.r_upB || !I.r_upC || !I.renyi_err) {
            c->err = "device allocation failed";
            return SGS_ENOMEM;
        }
        I.renyi_cap = need;
        I.renyi_chunk = chunk;
        I.renyi_m = m;
    }
    double* Y = I.renyi_scratch;
    double* logabs = Y + (size_t)chunk * (2 * mm + 20 * (size_t)m * bs);
    double* phase = logabs + chunk;
    for (long long q0 = 0; q0 < npairs; q0 += chunk) {
        renyi_build_kernel<<<(unsigned)chunk, 256, 0, st>>>(blocks, q0, npairs, na2, Y);
        counted();
        cudaError_t e = launch_pf(c, m, (int)chunk, bs, I.r_Y, I.r_TU, I.r_PK, I.r_upA, I.r_upB, I.r_upC, logabs,
                                  phase, I.renyi_err, st);
        if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return SGS_ECUDA; }
        renyi_combine_kernel<<<(unsigned)((chunk + 255) / 256), 256, 0, st>>>(logabs, phase, wts, q0, chunk, npairs,
                                                                             log_norm, partial);
        counted();
    }
    // a zero Pfaffian is a zero term here, not an error
    CUDA_TRY(c, cudaMemsetAsync(I.renyi_err, 0, sizeof(int), st));
    return SGS_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

void sgs_set_allocator(sgs_alloc_fn alloc, sgs_free_fn release, void* user) {
    g_alloc = alloc;
    g_release = release;
    g_user = user;
}

namespace {
sgs_status check_args(const sgs_model& m, const sgs_options& o) {
    if (m.n_modes < 1 || !m.A || (m.n_quartic > 0 && (!m.quartic_idx || !m.quartic_val))) return SGS_EINVAL;
    if (o.rank < 1 || o.rank > SGS_MAX_RANK || (o.parity != 1 && o.parity != -1)) return SGS_EINVAL;
    if (o.precision < 0 || o.precision > 3 || (o.cmode != 0 && o.cmode != 1)) return SGS_EINVAL;
    if (o.integrator != SGS_INTEGRATOR_EXP && o.integrator != SGS_INTEGRATOR_EULER) return SGS_EINVAL;
    if (o.fp64_path != SGS_FP64_EMULATED && o.fp64_path != SGS_FP64_FMA) return SGS_EINVAL;
    if (o.shard_world < 0 || (o.shard_world > 1 && (o.shard_rank < 0 || o.shard_rank >= o.shard_world)))
        return SGS_EINVAL;
    if (o.pair_chunk < 0) return SGS_EINVAL;
    if (o.gamma0) {           // finite and antisymmetric (purity is reported by sgs_health)
        const int n = 2 * m.n_modes;
        for (int mu = 0; mu < o.rank; mu++) {
            const double* g = o.gamma0 + (size_t)mu * n * n;
            for (int i = 0; i < n; i++)
                for (int j = i; j < n; j++) {
                    const double a = g[(size_t)i * n + j], b = g[(size_t)j * n + i];
                    if (!std::isfinite(a) || !std::isfinite(b) || std::fabs(a + b) > 1e-8) return SGS_EINVAL;
                }
        }
    }
    return SGS_OK;
}
}  // namespace

sgs_status sgs_create(void* stream, size_t hbm_budget, sgs_ctx** out) {
    if (!out) return SGS_EINVAL;
    *out = nullptr;
    set_kernel_attributes();
    sgs_ctx* c = new sgs_ctx();
    cudaGetDevice(&c->device);
    c->budget = hbm_budget;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SGS_ECUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return SGS_OK;
}

sgs_status sgs_admit(sgs_ctx* c, const sgs_model* model, const sgs_options* opt, int* slot) {
    if (!c || !model || !opt || !slot) return SGS_EINVAL;
    *slot = -1;
    sgs_status s = check_args(*model, *opt);
    if (s != SGS_OK) { c->err = "invalid model, options or initial states (non-finite or not antisymmetric)"; return s; }
    const size_t need = instance_bytes(2 * model->n_modes, opt->rank, opt->precision, 16, c->autotune,
                                       opt->fp64_path, oz_cap_of(opt->emulation_scratch), opt->pair_chunk);
    if (c->budget && c->bytes_in_use + need > c->budget) {
        c->err = "over the HBM budget: " + std::to_string(c->bytes_in_use + need) + " > " + std::to_string(c->budget);
        return SGS_ENOMEM;
    }
    // no initial states: seeded Haar states and phases generated here
    std::vector<double> g0, l0;
    sgs_options o = *opt;
    if (!o.gamma0) {
        const int n = 2 * model->n_modes;
        g0.resize((size_t)o.rank * n * n);
        l0.resize(2 * (size_t)o.rank);
        seeded_states(n, o.rank, o.seed, o.parity, g0.data(), l0.data());
        o.gamma0 = g0.data();
        if (!o.lambda0) o.lambda0 = l0.data();
    }
    c->inst.emplace_back();
    Instance& I = c->inst.back();
    c->owner = &I;
    s = setup_instance(c, I, *model, o);
    c->owner = nullptr;
    if (s == SGS_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) s = SGS_ECUDA;
    if (s == SGS_OK && c->autotune) s = autotune_instance(c, I);
    if (s != SGS_OK) {
        cudaStreamSynchronize(c->stream);
        c->release_instance(I);
        c->inst.pop_back();
        return s;
    }
    c->drop_graph();     // the captured step no longer covers every live instance
    *slot = (int)c->inst.size() - 1;
    return SGS_OK;
}

sgs_status sgs_retire(sgs_ctx* c, int slot) {
    if (!c || slot < 0 || slot >= (int)c->inst.size() || !c->inst[slot].live) return SGS_EINVAL;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    Instance& I = c->inst[slot];
    c->release_instance(I);
    I.live = false;
    c->drop_graph();
    return SGS_OK;
}

size_t sgs_bytes_in_use(const sgs_ctx* c) { return c ? c->bytes_in_use : 0; }

int sgs_failed_instance(const sgs_ctx* c) { return c ? c->failed : -1; }

int sgs_failed_instances(const sgs_ctx* c, int* slots, int capacity) {
    if (!c) return 0;
    const int n = (int)c->failed_list.size();
    if (slots)
        for (int i = 0; i < std::min(n, capacity); i++) slots[i] = c->failed_list[i];
    return n;
}

sgs_status sgs_health(sgs_ctx* c, int instance, double* out) {
    if (!c || !out || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    Instance& I = c->inst[instance];
    const int n = I.n, M = I.M;
    const size_t nn = (size_t)n * n;
    cudaStream_t st = c->stream;
    CUDA_TRY(c, cudaStreamSynchronize(st));
    // Gamma_mu^2 -> s0, then max |Gamma^2 + 1|, non-finite entries of Gamma, and the extreme eigenvalues of G
    // of the last amplitude solve (diagonal of its Jacobi result)
    GemmBatch g = gb_basic(n, n, n, I.p_gamma, n, I.p_gamma, n, I.p_s[0], n, M);
    const bool prof = c->prof;
    c->prof = false;
    cudaError_t e = gemm(c, I, g, st, -1.0);
    c->prof = prof;
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return SGS_ECUDA; }
    if (I.corr_cap < 8) {
        c->owner = &I;
        I.corr_scratch = c->alloc<double>(8);
        c->owner = nullptr;
        if (!I.corr_scratch) { c->err = "device allocation failed"; return SGS_ENOMEM; }
        I.corr_cap = 8;
    }
    health_kernel<<<1, 1024, 0, st>>>(I.s[0], I.gamma, M * nn, n, I.eigscratch, 2 * M, I.Ecur, I.corr_scratch);
    counted();
    CUDA_TRY(c, cudaMemcpyAsync(out, I.corr_scratch, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    return SGS_OK;
}

sgs_status sgs_seeded_states(int n_modes, int rank, unsigned long long seed, int parity, double* gamma, double* lambda) {
    if (n_modes < 1 || rank < 1 || (parity != 1 && parity != -1) || !gamma || !lambda) return SGS_EINVAL;
    seeded_states(2 * n_modes, rank, seed, parity, gamma, lambda);
    return SGS_OK;
}

sgs_status sgs_set_autotune(sgs_ctx* c, int enable) {
    if (!c) return SGS_EINVAL;
    c->autotune = enable != 0;
    return SGS_OK;
}

sgs_status sgs_get_tuning(const sgs_ctx* c, int instance, int* gj_width, int* pf_width, int* from_cache) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    const Instance& I = c->inst[instance];
    if (gj_width) *gj_width = I.gj_b;
    if (pf_width) *pf_width = I.pf_bs;
    if (from_cache) *from_cache = I.tuned_from_cache;
    return SGS_OK;
}

sgs_status sgs_set_panel_widths(sgs_ctx* c, int instance, int gj_width, int pf_width) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    Instance& I = c->inst[instance];
    const std::vector<int> gj = gj_candidates(I.n), pf = pf_candidates(I.n);
    if (std::find(gj.begin(), gj.end(), gj_width) == gj.end() || gj_width > I.gj_cap ||
        std::find(pf.begin(), pf.end(), pf_width) == pf.end() || pf_width > I.pf_cap) {
        c->err = "panel width not a candidate, or wider than the instance's scratch";
        return SGS_EINVAL;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const sgs_status s = set_panel_pointers(c, I, gj_width, pf_width);
    if (s != SGS_OK) return s;
    I.tuned_from_cache = 2;
    c->drop_graph();     // the captured step launches the old panels
    return SGS_OK;
}

sgs_status sgs_add_state(sgs_ctx* c, int slot, const double* K, int src) {
    if (!c || slot < 0 || slot >= (int)c->inst.size() || !c->inst[slot].live || !K) return SGS_EINVAL;
    if (c->inst[slot].shard_world > 1 || c->inst[slot].nch() > 1) {
        c->err = "rank growth is not available on a pair-sharded or pair-chunked instance";
        return SGS_EINVAL;
    }
    const int n = c->inst[slot].n, M = c->inst[slot].M;
    if (M + 1 > SGS_MAX_RANK) { c->err = "the rank is already at its maximum"; return SGS_EINVAL; }
    if (src < -1 || src >= M) { c->err = "src out of range"; return SGS_EINVAL; }
    double fro = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            const double v = K[(size_t)i * n + j];
            if (!std::isfinite(v) || v != -K[(size_t)j * n + i]) { c->err = "K is not antisymmetric"; return SGS_EINVAL; }
            fro += v * v;
        }
    if (std::sqrt(fro) > 8.0) { c->err = "||K||_F > 8"; return SGS_EINVAL; }
    cudaStream_t st = c->stream;
    CUDA_TRY(c, cudaStreamSynchronize(st));
    Instance& I = c->inst[slot];
    if (src < 0) {
        std::vector<double> lam(2 * (size_t)M);
        CUDA_TRY(c, cudaMemcpy(lam.data(), I.lam, 2 * M * sizeof(double), cudaMemcpyDeviceToHost));
        double best = -1.0;
        for (int mu = 0; mu < M; mu++) {
            const double a = std::hypot(lam[2 * mu], lam[2 * mu + 1]);
            if (a > best) { best = a; src = mu; }
        }
    }
    const size_t need = instance_bytes(n, M + 1, I.prec, 16, c->autotune, I.fp64_path, I.oz_cap, 0);
    if (c->budget && c->bytes_in_use - I.bytes + need > c->budget) {
        c->err = "over the HBM budget: " + std::to_string(c->bytes_in_use - I.bytes + need) + " > " +
                 std::to_string(c->budget);
        return SGS_ENOMEM;
    }
    // the grown instance: same model and options, rank M + 1, states filled on the device
    Instance J;
    sgs_model m{I.N, I.hA.data(), (int)I.hq_val.size(), I.hq_idx.data(), I.hq_val.data(), I.e_const,
                I.nh, I.hh_len.data(), I.hh_idx.data(), I.hh_val.data()};
    sgs_options o{M + 1, I.dtau, I.prec, I.cmode, I.parity, nullptr, nullptr, nullptr, I.integrator, 0,
                  I.fp64_path, I.oz_cap, 0, 1, 0};
    c->owner = &J;
    sgs_status s = setup_instance(c, J, m, o);
    c->owner = nullptr;
    const size_t nn = (size_t)n * n;
    cudaError_t e = cudaSuccess;
    if (s == SGS_OK) {
        e = cudaMemcpyAsync(J.gamma, I.gamma, M * nn * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(J.lam, I.lam, 2 * M * sizeof(double), cudaMemcpyDeviceToDevice, st);
        // X = K: exp_prepare_kernel forms (ds/4)(Y - Y^T), which is K for Y = K and ds = 2
        if (e == cudaSuccess) e = cudaMemcpyAsync(J.s[0], K, nn * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            exp_prepare_kernel<<<1, 1024, 0, st>>>(J.s[0], J.s[1], n, 2.0, J.sq, J.scale, J.err);
            counted();
            e = cudaGetLastError();
        }
        int cur = 3;
        if (e == cudaSuccess) e = exp_products(c, J, 1, st, &cur);
        // Q Gamma_src -> s0 ; (Q Gamma_src) Q^T -> Gamma_M
        if (e == cudaSuccess) {
            GemmBatch g = gb_basic(n, n, n, J.p_s[cur], n, J.p_gamma + src, n, J.p_s[0], n, 1);
            e = gemm(c, J, g, st, -1.0);
        }
        if (e == cudaSuccess) {
            GemmBatch g = gb_basic(n, n, n, J.p_s[0], n, J.p_s[cur], n, J.p_gamma + M, n, 1);
            g.transB = 1; g.mode = GEMM_SKEW;
            e = gemm(c, J, g, st, -1.0);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(J.sq, 0, (M + 1) * sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        int derr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&derr, J.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            c->err = std::string("rank growth: ") + cudaGetErrorString(e);
            s = SGS_ECUDA;
        } else if (derr) {
            c->err = "rank growth: exponential out of range";
            s = SGS_ENOTCONV;
        }
        if (s == SGS_OK && c->autotune) s = autotune_instance(c, J);
    }
    if (s != SGS_OK) {
        cudaStreamSynchronize(st);
        c->release_instance(J);
        return s;
    }
    J.st = I.st; J.join = I.join;        // the slot keeps its branch stream and event
    I.st = nullptr; I.join = nullptr;
    J.st2 = I.st2; J.ev_fork = I.ev_fork; J.ev_join = I.ev_join;
    I.st2 = nullptr; I.ev_fork = nullptr; I.ev_join = nullptr;
    c->release_instance(I);
    c->inst[slot] = std::move(J);
    c->drop_graph();
    return SGS_OK;
}

sgs_status sgs_init(const sgs_model* models, const sgs_options* opts, int n_instances, sgs_ctx** out) {
    if (!out) return SGS_EINVAL;
    *out = nullptr;
    if (!models || !opts || n_instances < 1) return SGS_EINVAL;
    for (int i = 0; i < n_instances; i++)
        if (check_args(models[i], opts[i]) != SGS_OK) return SGS_EINVAL;
    sgs_ctx* c = nullptr;
    sgs_status s = sgs_create(opts[0].stream, 0, &c);
    if (s != SGS_OK) return s;
    c->inst.reserve(n_instances);
    for (int i = 0; i < n_instances; i++) {
        int slot;
        s = sgs_admit(c, &models[i], &opts[i], &slot);
        if (s != SGS_OK) {
            sgs_free(c);
            return s;
        }
    }
    *out = c;
    return SGS_OK;
}

sgs_status sgs_step(sgs_ctx* c, int n_steps, double* energies) {
    if (!c || n_steps < 0) return SGS_EINVAL;
    if (any_sharded(c)) { c->err = "a pair-sharded instance steps through sgs_shard_pairs/eom/update"; return SGS_EINVAL; }
    for (auto& I : c->inst) {
        if (!I.live) continue;
        c->owner = &I;
        sgs_status s = ensure_ehist(c, I, std::max(n_steps, 1));
        c->owner = nullptr;
        if (s != SGS_OK) return s;
    }
    const long long l0 = g_launches;
    // graph replay needs a capturable stream (not the legacy default stream) and no profiling
    const bool graph = c->use_graph && !c->prof && c->stream != nullptr && n_steps > 0;
    if (graph && !c->graph_exec) {
        if (!c->fork) CUDA_TRY(c, cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
        for (auto& I : c->inst) {
            if (!I.live) continue;
            if (!I.st) CUDA_TRY(c, cudaStreamCreateWithFlags(&I.st, cudaStreamNonBlocking));
            if (!I.join) CUDA_TRY(c, cudaEventCreateWithFlags(&I.join, cudaEventDisableTiming));
        }
        const long long g0 = g_launches;
        CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaEventRecord(c->fork, c->stream);
        // independent instances are independent branches of the graph: their kernels overlap
        for (auto& I : c->inst) {
            if (!I.live) continue;
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(I.st, c->fork, 0);
            if (ce == cudaSuccess) ce = step_instance(c, I, I.st);
            if (ce == cudaSuccess) ce = cudaEventRecord(I.join, I.st);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(c->stream, I.join, 0);
        }
        cudaError_t ee = cudaStreamEndCapture(c->stream, &c->graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            c->err = std::string("graph capture failed: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee);
            c->drop_graph();
            return SGS_ECUDA;
        }
        CUDA_TRY(c, cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
        c->graph_launches = g_launches - g0;
        g_launches = g0;   // captured, not launched
    }
    for (int step = 0; step < n_steps; step++) {
        if (graph) {
            CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->stream));
            g_launches += c->graph_launches;
            for (auto& I : c->inst)
                if (I.live)
                    CUDA_TRY(c, cudaMemcpyAsync(I.Ehist + step, I.Ecur, sizeof(double), cudaMemcpyDeviceToDevice,
                                                c->stream));
        } else {
            for (auto& I : c->inst) {
                if (!I.live) continue;
                CUDA_TRY(c, step_instance(c, I, c->stream));
                CUDA_TRY(c, cudaMemcpyAsync(I.Ehist + step, I.Ecur, sizeof(double), cudaMemcpyDeviceToDevice,
                                            c->stream));
            }
        }
    }
    c->stage(-1);
    c->launches += g_launches - l0;
    sgs_status s = check_device_error(c);
    c->collect();
    // the energies of the instances that completed every step, also when others failed
    if (energies) {
        for (size_t i = 0; i < c->inst.size(); i++)
            if (c->inst[i].live &&
                std::find(c->failed_list.begin(), c->failed_list.end(), (int)i) == c->failed_list.end())
                CUDA_TRY(c, cudaMemcpy(energies + i * n_steps, c->inst[i].Ehist, n_steps * sizeof(double),
                                       cudaMemcpyDeviceToHost));
    }
    return s;
}

sgs_status sgs_energy(sgs_ctx* c, double* energies) {
    if (!c) return SGS_EINVAL;
    if (any_sharded(c)) { c->err = "a pair-sharded instance steps through sgs_shard_pairs/eom/update"; return SGS_EINVAL; }
    const long long l0 = g_launches;
    for (auto& I : c->inst)
        if (I.live) CUDA_TRY(c, pair_pass(c, I, I.Ecur, c->stream));
    c->stage(-1);
    c->launches += g_launches - l0;
    sgs_status s = check_device_error(c);
    c->collect();
    if (s != SGS_OK) return s;
    if (energies)
        for (size_t i = 0; i < c->inst.size(); i++)
            if (c->inst[i].live)
                CUDA_TRY(c, cudaMemcpy(energies + i, c->inst[i].Ecur, sizeof(double), cudaMemcpyDeviceToHost));
    return SGS_OK;
}

// ---------------------------------------------------------------- pair-sharded step

namespace {
sgs_status shard_instance(sgs_ctx* c, int instance, Instance** out) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    if (c->inst[instance].shard_world <= 1) { c->err = "not a pair-sharded instance"; return SGS_EINVAL; }
    *out = &c->inst[instance];
    return SGS_OK;
}
}  // namespace

sgs_status sgs_shard_pairs(sgs_ctx* c, int instance, double* gh) {
    Instance* Ip = nullptr;
    sgs_status s = shard_instance(c, instance, &Ip);
    if (s != SGS_OK) return s;
    if (!gh) return SGS_EINVAL;
    Instance& I = *Ip;
    cudaStream_t st = c->stream;
    const long long l0 = g_launches;
    CUDA_TRY(c, cudaMemsetAsync(I.Gm, 0, 2 * (size_t)I.M * I.M * sizeof(double), st));
    CUDA_TRY(c, cudaMemsetAsync(I.hm, 0, 2 * (size_t)I.M * I.M * sizeof(double), st));
    CUDA_TRY(c, pair_products(c, I, st));
    shard_export_gh_kernel<<<grid_chunks((size_t)I.M * I.M, 256, 64), 256, 0, st>>>(I.Gm, I.hm, I.M, I.self_mask, gh);
    counted();
    CUDA_TRY(c, cudaGetLastError());
    c->stage(-1);
    c->launches += g_launches - l0;
    s = check_device_error(c);
    c->collect();
    return s;
}

sgs_status sgs_shard_eom(sgs_ctx* c, int instance, const double* gh, double* dgamma, double* energy) {
    Instance* Ip = nullptr;
    sgs_status s = shard_instance(c, instance, &Ip);
    if (s != SGS_OK) return s;
    if (!gh || !dgamma) return SGS_EINVAL;
    Instance& I = *Ip;
    cudaStream_t st = c->stream;
    const long long l0 = g_launches;
    const size_t mm2 = 2 * (size_t)I.M * I.M, nn = (size_t)I.n * I.n;
    CUDA_TRY(c, cudaMemcpyAsync(I.Gm, gh, mm2 * sizeof(double), cudaMemcpyDefault, st));
    CUDA_TRY(c, cudaMemcpyAsync(I.hm, gh + mm2, mm2 * sizeof(double), cudaMemcpyDefault, st));
    c->stage(SGS_STAGE_AMPLITUDES);
    CUDA_TRY(c, amplitudes(I, I.Ecur, st));
    CUDA_TRY(c, eom_pass(c, I, st));
    c->stage(-1);
    CUDA_TRY(c, cudaMemcpyAsync(dgamma, I.dgamma, (size_t)I.M * nn * sizeof(double), cudaMemcpyDefault, st));
    c->launches += g_launches - l0;
    s = check_device_error(c);
    c->collect();
    if (s != SGS_OK) return s;
    if (energy) CUDA_TRY(c, cudaMemcpy(energy, I.Ecur, sizeof(double), cudaMemcpyDeviceToHost));
    return SGS_OK;
}

sgs_status sgs_shard_update(sgs_ctx* c, int instance, const double* dgamma) {
    Instance* Ip = nullptr;
    sgs_status s = shard_instance(c, instance, &Ip);
    if (s != SGS_OK) return s;
    if (!dgamma) return SGS_EINVAL;
    Instance& I = *Ip;
    cudaStream_t st = c->stream;
    const long long l0 = g_launches;
    CUDA_TRY(c, cudaMemcpyAsync(I.dgamma, dgamma, (size_t)I.M * I.n * I.n * sizeof(double), cudaMemcpyDefault, st));
    CUDA_TRY(c, update_pass(c, I, st));
    c->stage(-1);
    c->launches += g_launches - l0;
    s = check_device_error(c);
    c->collect();
    return s;
}

sgs_status sgs_correlator(sgs_ctx* c, int instance, sgs_corr_kind kind, const int* sites, int n_sites, double* out) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live || !sites || !out || n_sites < 0) return SGS_EINVAL;
    if (c->inst[instance].shard_world > 1 || c->inst[instance].nch() > 1) {
        c->err = "observables need every pair at once: not on a pair-sharded or pair-chunked instance";
        return SGS_EINVAL;
    }
    if (n_sites == 0) return SGS_OK;
    Instance& I = c->inst[instance];
    const int nsite_tot = I.n / 4;          // spinful sites: modes 2s, 2s+1 -> Majoranas 4s..4s+3
    if (kind == SGS_CORR_SPIN_SPIN || kind == SGS_CORR_TWO_CHANNEL_K) {
        const int nch = (kind == SGS_CORR_TWO_CHANNEL_K) ? 2 : 1;
        for (int i = 0; i < n_sites; i++) {
            const int s = sites[i];
            const bool ok = (kind == SGS_CORR_SPIN_SPIN) ? (s >= 0 && s < nsite_tot)
                                                         : (s >= 1 && 1 + (s - 1) * nch + nch - 1 < nsite_tot);
            if (!ok) { c->err = "correlator site out of range"; return SGS_EINVAL; }
        }
        // current states: pair pass and amplitudes (the states are not changed)
        CUDA_TRY(c, pair_pass(c, I, I.Ecur, c->stream));
        c->stage(-1);
        const size_t rows = (size_t)I.P + I.M;
        const size_t need = rows * n_sites + 2 * (size_t)n_sites + 8;
        if (I.corr_cap < need) {
            c->owner = &I;
            I.corr_scratch = c->alloc<double>(need);
            c->owner = nullptr;
            if (!I.corr_scratch) { c->err = "device allocation failed"; return SGS_ENOMEM; }
            I.corr_cap = need;
        }
        double* partial = I.corr_scratch;
        double* dout = partial + rows * n_sites;
        int* dsites = reinterpret_cast<int*>(dout + n_sites);
        CUDA_TRY(c, cudaMemcpyAsync(dsites, sites, n_sites * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        spin_corr_kernel<<<(unsigned)rows, 128, 0, c->stream>>>(I.dev(), I.si, I.imd, I.Gm, I.lam, dsites, n_sites,
                                                               kind == SGS_CORR_SPIN_SPIN ? 0 : 1, nch, partial);
        column_sum_kernel<<<(n_sites + 127) / 128, 128, 0, c->stream>>>(partial, (int)rows, n_sites, dout);
        counted(); counted();
        sgs_status st = check_device_error(c);
        c->collect();
        if (st != SGS_OK) return st;
        CUDA_TRY(c, cudaMemcpy(out, dout, n_sites * sizeof(double), cudaMemcpyDeviceToHost));
        return SGS_OK;
    }
    if (kind == SGS_CORR_RENYI2) {
        for (int i = 0; i < n_sites; i++) {
            const int na2 = 4 * (1 + sites[i]);
            if (sites[i] < 0 || na2 > I.n) {
                c->err = "Renyi-2 subsystem out of range (impurity + l sites, 4(1+l) <= 2N)";
                return SGS_EINVAL;
            }
        }
        CUDA_TRY(c, pair_pass(c, I, I.Ecur, c->stream));
        c->stage(-1);
        const long long M2 = (long long)I.M * I.M;
        const long long npairs = M2 * (M2 + 1) / 2;
        const int nred = 1024;
        int maxna2 = 0;
        for (int i = 0; i < n_sites; i++) maxna2 = std::max(maxna2, 4 * (1 + sites[i]));
        const size_t need = (size_t)M2 * maxna2 * maxna2 * 2 + 2 * M2 + 2 * (size_t)npairs + 2 * nred + 8;
        if (I.corr_cap < need) {
            c->owner = &I;
            I.corr_scratch = c->alloc<double>(need);
            c->owner = nullptr;
            if (!I.corr_scratch) { c->err = "device allocation failed"; return SGS_ENOMEM; }
            I.corr_cap = need;
        }
        double* blocks = I.corr_scratch;
        double* wts = blocks + (size_t)M2 * maxna2 * maxna2 * 2;
        double* partial = wts + 2 * M2;
        double* sums = partial + 2 * (size_t)npairs;
        for (int i = 0; i < n_sites; i++) {
            const int na2 = 4 * (1 + sites[i]);
            const int m = 2 * na2;
            renyi_blocks_kernel<<<(unsigned)M2, 128, 0, c->stream>>>(I.dev(), I.si, I.imd, I.Gm, I.lam, I.pair_index,
                                                                     na2, blocks, wts);
            counted();
            const double log_norm = -(na2 / 2) * 0.6931471805599453;
            if (m <= RENYI_MAX_DIM) {
                const size_t smem = 2 * (size_t)m * (m + 1) * sizeof(double);
                set_kernel_attributes();
                const unsigned gx = (unsigned)std::min<long long>(npairs, 65535);
                const unsigned gy = (unsigned)((npairs + gx - 1) / gx);
                renyi_pf_kernel<<<dim3(gx, gy), 256, smem, c->stream>>>(blocks, wts, npairs, na2, log_norm, partial);
                counted();
            } else {
                sgs_status rs = renyi_large(c, I, blocks, wts, npairs, na2, log_norm, partial);
                if (rs != SGS_OK) return rs;
            }
            complex_sum_kernel<<<nred, 256, 0, c->stream>>>(partial, npairs, sums);
            complex_sum_kernel<<<1, 256, 0, c->stream>>>(sums, nred, sums + 2 * nred);
            counted(); counted();
            double tr[2];
            CUDA_TRY(c, cudaMemcpyAsync(tr, sums + 2 * nred, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            out[i] = -std::log(tr[0]);
        }
        sgs_status st = check_device_error(c);
        c->collect();
        return st;
    }
    c->err = "unknown correlator kind";
    return SGS_EINVAL;
}

sgs_status sgs_variance(sgs_ctx* c, int instance, double* energy, double* variance) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    Instance& I = c->inst[instance];
    if (I.shard_world > 1 || I.nch() > 1) {
        c->err = "observables need every pair at once: not on a pair-sharded or pair-chunked instance";
        return SGS_EINVAL;
    }
    if (I.nc > VAR_MAX_MON) { c->err = "more quartic monomials than the variance kernel handles"; return SGS_EINVAL; }
    if (I.nh > 0) { c->err = "the variance covers quadratic and quartic terms"; return SGS_EINVAL; }
    CUDA_TRY(c, pair_pass(c, I, I.Ecur, c->stream));
    c->stage(-1);
    const size_t rows = (size_t)I.P + I.M;
    const size_t need = rows + 8;
    if (I.corr_cap < need) {
        c->owner = &I;
        I.corr_scratch = c->alloc<double>(need);
        c->owner = nullptr;
        if (!I.corr_scratch) { c->err = "device allocation failed"; return SGS_ENOMEM; }
        I.corr_cap = need;
    }
    double* partial = I.corr_scratch;
    double* dout = partial + rows;
    VarArgs va{I.dev(), I.si, I.imd, I.Gm, I.lam, I.c_idx, I.c_val, I.nc, I.trA2, partial};
    variance_kernel<<<(unsigned)rows, 256, 0, c->stream>>>(va);
    column_sum_kernel<<<1, 32, 0, c->stream>>>(partial, (int)rows, 1, dout);
    counted(); counted();
    sgs_status st = check_device_error(c);
    c->collect();
    if (st != SGS_OK) return st;
    double h[2];
    CUDA_TRY(c, cudaMemcpy(h, dout, sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(h + 1, I.Ecur, sizeof(double), cudaMemcpyDeviceToHost));
    if (energy) *energy = h[1];
    if (variance) *variance = h[0] - h[1] * h[1];
    return SGS_OK;
}

void sgs_free(sgs_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    c->drop_graph();
    for (auto& I : c->inst) {
        c->release_instance(I);
        if (I.st) cudaStreamDestroy(I.st);
        if (I.join) cudaEventDestroy(I.join);
        if (I.st2) cudaStreamDestroy(I.st2);
        if (I.ev_fork) cudaEventDestroy(I.ev_fork);
        if (I.ev_join) cudaEventDestroy(I.ev_join);
    }
    if (c->fork) cudaEventDestroy(c->fork);
    c->release_all();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* sgs_last_error(const sgs_ctx* c) { return c ? c->err.c_str() : "no context"; }

sgs_status sgs_get_state(const sgs_ctx* cc, int instance, double* gamma, double* lambda) {
    sgs_ctx* c = const_cast<sgs_ctx*>(cc);
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    const Instance& I = c->inst[instance];
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (gamma)
        CUDA_TRY(c, cudaMemcpy(gamma, I.gamma, (size_t)I.M * I.n * I.n * sizeof(double), cudaMemcpyDeviceToHost));
    if (lambda) CUDA_TRY(c, cudaMemcpy(lambda, I.lam, 2 * I.M * sizeof(double), cudaMemcpyDeviceToHost));
    return SGS_OK;
}

sgs_status sgs_set_state(sgs_ctx* c, int instance, const double* gamma, const double* lambda) {
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    Instance& I = c->inst[instance];
    if (gamma)
        CUDA_TRY(c, cudaMemcpyAsync(I.gamma, gamma, (size_t)I.M * I.n * I.n * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
    if (lambda)
        CUDA_TRY(c, cudaMemcpyAsync(I.lam, lambda, 2 * I.M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SGS_OK;
}

sgs_status sgs_get_pair_matrices(const sgs_ctx* cc, int instance, double* G, double* h) {
    sgs_ctx* c = const_cast<sgs_ctx*>(cc);
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live) return SGS_EINVAL;
    const Instance& I = c->inst[instance];
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (G) CUDA_TRY(c, cudaMemcpy(G, I.Gm, 2 * I.M * I.M * sizeof(double), cudaMemcpyDeviceToHost));
    if (h) CUDA_TRY(c, cudaMemcpy(h, I.hm, 2 * I.M * I.M * sizeof(double), cudaMemcpyDeviceToHost));
    return SGS_OK;
}

sgs_status sgs_get_derivative(const sgs_ctx* cc, int instance, double* dgamma) {
    sgs_ctx* c = const_cast<sgs_ctx*>(cc);
    if (!c || instance < 0 || instance >= (int)c->inst.size() || !c->inst[instance].live || !dgamma) return SGS_EINVAL;
    const Instance& I = c->inst[instance];
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(dgamma, I.dgamma, (size_t)I.M * I.n * I.n * sizeof(double), cudaMemcpyDeviceToHost));
    return SGS_OK;
}

sgs_status sgs_set_profiling(sgs_ctx* c, int enable) {
    if (!c) return SGS_EINVAL;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->collect();
    c->prof = enable != 0;
    for (int j = 0; j < SGS_N_STAGES; j++) c->stage_ms[j] = c->stage_flops[j] = c->stage_bytes[j] = 0.0;
    c->launches = 0;
    c->gemm_ms = c->gemm_flops = 0.0;
    c->gemm_count = 0;
    for (auto& I : c->inst) I.steps_since_profile = 0;
    return SGS_OK;
}

sgs_status sgs_get_profile(const sgs_ctx* cc, double* ms, double* flops, double* bytes, long long* launches,
                           double* gemm_f64) {
    sgs_ctx* c = const_cast<sgs_ctx*>(cc);
    if (!c) return SGS_EINVAL;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->collect();
    // squarings of the exponential step: 2 n^3 per squaring actually applied (last step's counts)
    double sq_flops = 0.0;
    for (auto& I : c->inst) {
        std::vector<int> sq(I.M);
        CUDA_TRY(c, cudaMemcpy(sq.data(), I.sq, I.M * sizeof(int), cudaMemcpyDeviceToHost));
        double tot = 0;
        for (int v : sq) tot += v;
        sq_flops += 2.0 * (double)I.n * I.n * I.n * tot * I.steps_since_profile;
    }
    for (int j = 0; j < SGS_N_STAGES; j++) {
        if (ms) ms[j] = c->stage_ms[j];
        if (flops) flops[j] = c->stage_flops[j] + (j == SGS_STAGE_UPDATE ? sq_flops : 0.0);
        if (bytes) bytes[j] = c->stage_bytes[j];
    }
    if (launches) *launches = c->launches;
    if (gemm_f64) {
        gemm_f64[0] = c->gemm_ms;
        gemm_f64[1] = c->gemm_flops;
        gemm_f64[2] = (double)c->gemm_count;
    }
    return SGS_OK;
}

sgs_status sgs_probe_wait(unsigned long long limit_ns, double* elapsed_ms) {
    if (limit_ns < 1000ull || limit_ns > 10000000000ull) return SGS_EINVAL;
    int* buf = nullptr;
    if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return SGS_ENOMEM;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sgs_status s = SGS_OK;
    int err = 0;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMemsetAsync(buf, 0, 2 * sizeof(int), st) != cudaSuccess) {
        s = SGS_ECUDA;
    } else {
        cudaEventRecord(e0, st);
        wait_probe_kernel<<<1, 32, 0, st>>>(buf, limit_ns, buf + 1);      // the flag buf[0] stays 0
        counted();
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&err, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            s = SGS_ECUDA;
        } else {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (elapsed_ms) *elapsed_ms = ms;
            s = (err & SGS_DEV_TC_TIMEOUT) ? SGS_ETIMEOUT : SGS_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    return s;
}

sgs_status sgs_kernel_smem_limits(int n_out, int* limit, int* expected) {
    const void* k[] = {(const void*)gj_panel_kernel, (const void*)pf_panel_kernel, (const void*)renyi_pf_kernel,
                       (const void*)gemm_tma_kernel<TC_TF32>, (const void*)gemm_tma_kernel<TC_BF16>,
                       (const void*)gemm_tma_kernel<TC_3XTF32>, (const void*)oz_gemm_kernel<OZ_NARROW>,
                       (const void*)oz_block_slice_kernel, (const void*)oz_gemm_kernel<OZ_NARROW16>};
    const int nk = (int)(sizeof(k) / sizeof(k[0]));
    if (!limit || !expected || n_out < 1 || n_out > nk) return SGS_EINVAL;
    set_kernel_attributes();
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SGS_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return SGS_ECUDA;
    for (int i = 0; i < n_out; i++) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, k[i]) != cudaSuccess) return SGS_ECUDA;
        limit[i] = fa.maxDynamicSharedSizeBytes;
        expected[i] = optin - (int)fa.sharedSizeBytes;
    }
    return SGS_OK;
}

sgs_status sgs_set_graphs(sgs_ctx* c, int enable) {
    if (!c) return SGS_EINVAL;
    c->use_graph = enable != 0;
    return SGS_OK;
}

sgs_status sgs_probe_peak(int kind, double* tflops) {
    if (!tflops || kind < 0 || kind > 2) return SGS_EINVAL;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, thr = 256;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * thr) != cudaSuccess) return SGS_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0);
        if (kind == 0) probe_dmma_kernel<<<blocks, thr>>>(out, 0.999);
        else if (kind == 1) probe_dfma_kernel<<<blocks, thr>>>(out, 0.999);
        else probe_mixed_kernel<<<blocks, thr>>>(out, 0.999);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return SGS_ECUDA;
    // m8n8k4: 512 flops per warp-instruction; FMA: 2 flops per thread-instruction
    const double fmma = (double)blocks * (thr / 32) * PROBE_ITERS * 512.0;
    const double ffma = (double)blocks * thr * PROBE_ITERS * 8 * 2.0;
    const double fl = (kind == 0) ? fmma : (kind == 1) ? ffma : 0.5 * fmma + 0.5 * ffma;
    *tflops = fl / (best * 1e-3) / 1e12;
    return SGS_OK;
}

int sgs_build_anderson(int n_bath, int n_channels, double U, double eps_d, double V, double t, double mu, double* A,
                       int* quartic_idx, double* quartic_val, double* e_const) {
    if (n_bath < 1 || n_channels < 1 || !A || !quartic_idx || !quartic_val || !e_const) return -1;
    const int n_sites = 1 + n_channels * n_bath;
    const int nm = 2 * n_sites;
    const int n = 2 * nm;
    std::vector<double> h((size_t)nm * nm, 0.0);
    auto site = [&](int ch, int r) { return 1 + (r - 1) * n_channels + ch; };
    for (int sp = 0; sp < 2; sp++) {
        h[(size_t)sp * nm + sp] = eps_d;
        for (int ch = 0; ch < n_channels; ch++) {
            int b = 2 * site(ch, 1) + sp;
            h[(size_t)sp * nm + b] = h[(size_t)b * nm + sp] = -V;
            for (int r = 1; r <= n_bath; r++) {
                int m = 2 * site(ch, r) + sp;
                h[(size_t)m * nm + m] = -mu;
                if (r >= 2) {
                    int q = 2 * site(ch, r - 1) + sp;
                    h[(size_t)q * nm + m] = h[(size_t)m * nm + q] = -t;
                }
            }
        }
    }
    // sum_ij h_ij a_i^dag a_j = tr(h)/2 + i sum_kl A_kl c_k c_l with A_{2i,2j+1} = h_ij/4
    std::fill(A, A + (size_t)n * n, 0.0);
    double ec = 0.0;
    for (int i = 0; i < nm; i++) {
        ec += 0.5 * h[(size_t)i * nm + i];
        for (int j = 0; j < nm; j++) {
            double v = h[(size_t)i * nm + j];
            if (v == 0.0) continue;
            A[(size_t)(2 * i) * n + 2 * j + 1] += 0.25 * v;
            A[(size_t)(2 * j + 1) * n + 2 * i] -= 0.25 * v;
        }
    }
    // U n_0up n_0dn = U/4 + (U/4)(i c0 c1 + i c2 c3) - (U/4) c0 c1 c2 c3
    ec += 0.25 * U;
    for (int m = 0; m < 2; m++) {
        A[(size_t)(2 * m) * n + 2 * m + 1] += 0.125 * U;
        A[(size_t)(2 * m + 1) * n + 2 * m] -= 0.125 * U;
    }
    quartic_idx[0] = 0; quartic_idx[1] = 1; quartic_idx[2] = 2; quartic_idx[3] = 3;
    quartic_val[0] = -0.25 * U;
    *e_const = ec;
    return nm;
}

int sgs_build_2ck(int L, double J, double t, double* A, int* quartic_idx, double* quartic_val, double* e_const) {
    if (L < 2 || !A || !quartic_idx || !quartic_val || !e_const) return -1;
    const int n_sites = 2 * L;
    const int nm = 2 * n_sites;
    const int n = 2 * nm;
    auto site = [](int ch, int r) { return 1 + 2 * (r - 1) + ch; };
    std::fill(A, A + (size_t)n * n, 0.0);
    // hopping -t (a_p^dag a_q + h.c.): A_{2p,2q+1} = A_{2q,2p+1} = -t/4 (and the antisymmetric partners)
    auto hop = [&](int sp, int sq) {
        for (int s = 0; s < 2; s++) {
            const int p = 2 * sp + s, q = 2 * sq + s;
            A[(size_t)(2 * p) * n + 2 * q + 1] -= 0.25 * t;
            A[(size_t)(2 * q + 1) * n + 2 * p] += 0.25 * t;
            A[(size_t)(2 * q) * n + 2 * p + 1] -= 0.25 * t;
            A[(size_t)(2 * p + 1) * n + 2 * q] += 0.25 * t;
        }
    };
    for (int ch = 0; ch < 2; ch++) {
        for (int r = 2; r < L; r++) hop(site(ch, r - 1), site(ch, r));
        hop(site(ch, L - 1), n_sites - 1);          // H_BC: the boundary site joins the two channels
    }
    *e_const = 0.0;                                   // hopping has no diagonal
    // H_J = J sum_alpha S_imp . S_alpha(1); S^a of a site = (i/4) sum_{p<q} K^a_pq c_p c_q on its four
    // Majoranas (K^x: (03) +1, (12) -1; K^y: (02) -1, (13) -1; K^z: (01) +1, (23) -1), so
    // S^a_imp S^a_r = -(1/16) sum K^a_pq K^a_uv c_p c_q c_{4r+u} c_{4r+v}
    const int kp[3][2][2] = {{{0, 3}, {1, 2}}, {{0, 2}, {1, 3}}, {{0, 1}, {2, 3}}};
    const double kv[3][2] = {{1.0, -1.0}, {-1.0, -1.0}, {1.0, -1.0}};
    int q = 0;
    for (int ch = 0; ch < 2; ch++) {
        const int r0 = 4 * site(ch, 1);
        for (int a = 0; a < 3; a++)
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++) {
                    quartic_idx[4 * q + 0] = kp[a][i][0];
                    quartic_idx[4 * q + 1] = kp[a][i][1];
                    quartic_idx[4 * q + 2] = r0 + kp[a][j][0];
                    quartic_idx[4 * q + 3] = r0 + kp[a][j][1];
                    quartic_val[q] = -J / 16.0 * kv[a][i] * kv[a][j];
                    q++;
                }
    }
    return nm;
}

// ------------------------------------------------------------ building blocks

}  // extern "C"

// slice scratch of a temporary context for the emulated FP64 path (empty on the FMA path)
static OzBuf tmp_oz(sgs_ctx& tmp, size_t need, int fp64_path, size_t cap) {
    OzBuf o;
    if (fp64_path != SGS_FP64_EMULATED) return o;
    const size_t b = std::min(need + 16384, oz_cap_of(cap));
    o.base = static_cast<uint8_t*>(tmp.dalloc(b));
    o.bytes = o.base ? b : 0;
    return o;
}

extern "C" {

sgs_status sgs_kernel_gemm_tc(const double* A, const double* Bt, int m, int n, int k, int batch, int kind,
                              double* C) {
    if (!A || !Bt || !C || m < 1 || n < 1 || k < 1 || batch < 1 || kind < 0 || kind > 2 || (k & 7)) return SGS_EINVAL;
    set_kernel_attributes();
    sgs_ctx tmp;
    cudaStreamCreateWithFlags(&tmp.stream, cudaStreamNonBlocking);
    const size_t na = (size_t)m * k, nb = (size_t)n * k, nc = (size_t)m * n;
    const size_t esz = (kind == TC_BF16) ? 2 : 4;
    const int parts = (kind == TC_3XTF32) ? 2 : 1;
    void* dA = tmp.dalloc(parts * batch * na * esz);
    void* dB = tmp.dalloc(parts * batch * nb * esz);
    double* dC = tmp.alloc<double>(batch * nc);
    int* err = tmp.alloc<int>(1);
    sgs_status st = SGS_OK;
    if (!dA || !dB || !dC || !err) st = SGS_ENOMEM;
    if (st == SGS_OK) {
        // operand conversion on the host (building block only): fp32 / bf16, hi + lo for 3xTF32
        std::vector<uint8_t> ha(parts * batch * na * esz), hb(parts * batch * nb * esz);
        auto conv = [&](const double* src, size_t cnt, uint8_t* hi, uint8_t* lo) {
            for (size_t e = 0; e < cnt; e++) {
                if (kind == TC_BF16) {
                    __nv_bfloat16 v = __float2bfloat16_rn((float)src[e]);
                    std::memcpy(hi + 2 * e, &v, 2);
                } else {
                    float h = (float)src[e];
                    if (kind == TC_3XTF32) {
                        // hi keeps the top 10 mantissa bits (tf32), lo the remainder
                        uint32_t u;
                        std::memcpy(&u, &h, 4);
                        u &= 0xffffe000u;
                        float th;
                        std::memcpy(&th, &u, 4);
                        float tl = (float)(src[e] - (double)th);
                        std::memcpy(hi + 4 * e, &th, 4);
                        std::memcpy(lo + 4 * e, &tl, 4);
                    } else {
                        // nearest TF32 value, as the device-side conversions round
                        uint32_t u;
                        std::memcpy(&u, &h, 4);
                        u = (u + 0x1000u) & 0xffffe000u;
                        std::memcpy(hi + 4 * e, &u, 4);
                    }
                }
            }
        };
        conv(A, batch * na, ha.data(), ha.data() + batch * na * esz);
        conv(Bt, batch * nb, hb.data(), hb.data() + batch * nb * esz);
        cudaMemcpyAsync(dA, ha.data(), ha.size(), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemcpyAsync(dB, hb.data(), hb.size(), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemsetAsync(err, 0, sizeof(int), tmp.stream);
        {
            TmaBatch t{};
            const bool bf = kind == TC_BF16, split = kind == TC_3XTF32;
            bool ok = make_operand_map(&t.ta, dA, bf, k, m, batch) && make_operand_map(&t.tb, dB, bf, k, n, batch);
            if (split)
                ok = ok && make_operand_map(&t.ta2, (const uint8_t*)dA + batch * na * esz, bf, k, m, batch) &&
                     make_operand_map(&t.tb2, (const uint8_t*)dB + batch * nb * esz, bf, k, n, batch);
            t.m = m; t.n = n; t.k = k; t.alpha = 1.0; t.C = dC; t.c_stride = (long long)nc; t.ldc = n;
            t.out_f64 = 1; t.skew = 0; t.err = err; t.batch = batch;
            if (!ok || tma_product(t, kind, tmp.stream) != cudaSuccess) st = SGS_ECUDA;
        }
        counted();
        int herr = 0;
        cudaMemcpyAsync(C, dC, batch * nc * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, tmp.stream);
        if (cudaStreamSynchronize(tmp.stream) != cudaSuccess) st = SGS_ECUDA;
        else if (herr) st = SGS_ETIMEOUT;
    }
    cudaStreamSynchronize(tmp.stream);
    tmp.release_all();
    cudaStreamDestroy(tmp.stream);
    tmp.stream = nullptr;
    return st;
}

sgs_status sgs_kernel_gemm(const double* A, const double* B, const double* Cin, int m, int n, int k, int trans_a,
                           int trans_b, double alpha, double beta, double diag, int mode, int gj_k0, int gj_b,
                           int batch, int fp64_path, size_t emulation_scratch, double* C) {
    if (!A || !B || !C || m < 1 || n < 1 || k < 1 || batch < 1 || mode < 0 || mode > 6 || (mode & 3) > 2)
        return SGS_EINVAL;
    if (fp64_path != SGS_FP64_EMULATED && fp64_path != SGS_FP64_FMA) return SGS_EINVAL;
    const int b_antisym = mode >> 2;            // + 4: B antisymmetric (k = n)
    mode &= 3;
    if (b_antisym && (k != n || trans_b)) return SGS_EINVAL;
    if (mode == GEMM_SKEW && m != n) return SGS_EINVAL;
    if (mode == GEMM_GJ && (m != n || gj_k0 < 0 || gj_b < 1 || gj_k0 + gj_b > n)) return SGS_EINVAL;
    sgs_ctx tmp;
    cudaStreamCreateWithFlags(&tmp.stream, cudaStreamNonBlocking);
    tmp.own_stream = true;
    const size_t na = (size_t)m * k, nb = (size_t)k * n, nc = (size_t)m * n;
    double *dA = tmp.alloc<double>(batch * na), *dB = tmp.alloc<double>(batch * nb), *dC = tmp.alloc<double>(batch * nc);
    double* dI = Cin ? tmp.alloc<double>(batch * nc) : nullptr;
    int* err = tmp.alloc<int>(1);
    sgs_status st = SGS_OK;
    if (!dA || !dB || !dC || !err || (Cin && !dI)) st = SGS_ENOMEM;
    if (st == SGS_OK) {
        std::vector<double*> pa, pb, pc, pi;
        for (int b = 0; b < batch; b++) {
            pa.push_back(dA + b * na); pb.push_back(dB + b * nb); pc.push_back(dC + b * nc);
            pi.push_back(dI ? dI + b * nc : nullptr);
        }
        double **PA = upload_ptrs(&tmp, pa), **PB = upload_ptrs(&tmp, pb), **PC = upload_ptrs(&tmp, pc);
        double** PI = dI ? upload_ptrs(&tmp, pi) : nullptr;
        cudaMemcpyAsync(dA, A, batch * na * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemcpyAsync(dB, B, batch * nb * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemcpyAsync(dC, C, batch * nc * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        if (dI) cudaMemcpyAsync(dI, Cin, batch * nc * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemsetAsync(err, 0, sizeof(int), tmp.stream);
        GemmBatch g = gb_basic(m, n, k, PA, trans_a ? m : k, PB, trans_b ? k : n, PC, n, batch);
        g.transA = trans_a ? 1 : 0; g.transB = trans_b ? 1 : 0;
        g.alpha = alpha; g.diag = diag; g.mode = mode; g.gj_k0 = gj_k0; g.gj_b = gj_b; g.b_antisym = b_antisym;
        if (PI) { g.Cin = (const double* const*)PI; g.ldcin = n; g.beta = beta; }
        set_kernel_attributes();
        const OzBuf oz = tmp_oz(tmp, (size_t)batch * oz_entry_bytes(m, n, k), fp64_path, emulation_scratch);
        if (gemm(nullptr, g, tmp.stream, -1.0, &oz, err) != cudaSuccess) st = SGS_ECUDA;
        int herr = 0;
        cudaMemcpyAsync(C, dC, batch * nc * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, tmp.stream);
        if (cudaStreamSynchronize(tmp.stream) != cudaSuccess) st = SGS_ECUDA;
        else if (st == SGS_OK && herr) st = SGS_ETIMEOUT;
    }
    cudaStreamSynchronize(tmp.stream);
    tmp.release_all();
    cudaStreamDestroy(tmp.stream);
    tmp.stream = nullptr;
    return st;
}

sgs_status sgs_kernel_inverse(const double* S, int n, int batch, int fp64_path, double* inv, double* logabsdet) {
    if (!S || !inv || n < 1 || batch < 1) return SGS_EINVAL;
    if (fp64_path != SGS_FP64_EMULATED && fp64_path != SGS_FP64_FMA) return SGS_EINVAL;
    sgs_ctx tmp;
    cudaStreamCreateWithFlags(&tmp.stream, cudaStreamNonBlocking);
    const size_t nn = (size_t)n * n;
    const int bsz = (n <= 640) ? std::min(32, n) : 16;
    const size_t qn = (size_t)n * n / 4 + n;             // recursive form: pivot rows of the widest update
    double *W = tmp.alloc<double>(batch * nn), *O = tmp.alloc<double>(batch * nn), *T = tmp.alloc<double>((size_t)batch * bsz * n);
    double* U = tmp.alloc<double>(batch * qn);
    int *piv = tmp.alloc<int>((size_t)batch * n), *perm = tmp.alloc<int>((size_t)batch * n), *err = tmp.alloc<int>(1);
    double *ld = tmp.alloc<double>(batch), *ds = tmp.alloc<double>(batch);
    sgs_status st = SGS_OK;
    if (!W || !O || !T || !U || !piv || !perm || !err || !ld || !ds) st = SGS_ENOMEM;
    if (st == SGS_OK) {
        std::vector<double*> pw, pt, po, pu;
        for (int b = 0; b < batch; b++) {
            pw.push_back(W + b * nn); pt.push_back(T + (size_t)b * bsz * n); po.push_back(O + b * nn);
            pu.push_back(U + b * qn);
        }
        double **PW = upload_ptrs(&tmp, pw), **PT = upload_ptrs(&tmp, pt), **PO = upload_ptrs(&tmp, po);
        double** PU = upload_ptrs(&tmp, pu);
        cudaMemcpyAsync(W, S, batch * nn * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemsetAsync(err, 0, sizeof(int), tmp.stream);
        const OzBuf oz = tmp_oz(tmp, (size_t)batch * oz_entry_bytes(n, n, std::min(n, n / 2 + bsz)), fp64_path, 0);
        if (launch_gj_recursive(nullptr, n, batch, bsz, PW, PT, PU, piv, ld, ds, err, 0.0, tmp.stream, &oz) !=
            cudaSuccess)
            st = SGS_ECUDA;
        gj_perm_kernel<<<batch, 128, 2 * (size_t)n * sizeof(int), tmp.stream>>>(piv, perm, n, batch);
        gj_gather_kernel<<<dim3(grid_chunks(nn, 256, 64), batch), 256, 0, tmp.stream>>>(PW, PO, perm, n);
        cudaMemcpyAsync(inv, O, batch * nn * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        if (logabsdet) cudaMemcpyAsync(logabsdet, ld, batch * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        int herr = 0;
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, tmp.stream);
        if (cudaStreamSynchronize(tmp.stream) != cudaSuccess) st = SGS_ECUDA;
        else if (herr & SGS_DEV_TC_TIMEOUT) st = SGS_ETIMEOUT;
        else if (herr) st = SGS_ESINGULAR;
    }
    cudaStreamSynchronize(tmp.stream);
    tmp.release_all();
    cudaStreamDestroy(tmp.stream);
    tmp.stream = nullptr;
    return st;
}

sgs_status sgs_kernel_pfaffian(const double* Y, int n, int batch, int fp64_path, double* phase, double* logabs) {
    if (!Y || !phase || !logabs || n < 2 || (n & 1) || batch < 1) return SGS_EINVAL;
    if (fp64_path != SGS_FP64_EMULATED && fp64_path != SGS_FP64_FMA) return SGS_EINVAL;
    sgs_ctx tmp;
    cudaStreamCreateWithFlags(&tmp.stream, cudaStreamNonBlocking);
    const size_t nn = (size_t)n * n;
    const int bs = std::min(16, n / 2);
    double* W = tmp.alloc<double>(batch * 2 * nn);
    double* TU = tmp.alloc<double>((size_t)batch * 4 * n * bs);
    double* PK = tmp.alloc<double>((size_t)batch * 16 * n * bs);
    double *la = tmp.alloc<double>(batch), *ph = tmp.alloc<double>(2 * batch);
    int* err = tmp.alloc<int>(1);
    sgs_status st = SGS_OK;
    if (!W || !TU || !PK || !la || !ph || !err) st = SGS_ENOMEM;
    if (st == SGS_OK) {
        // de-interleave (re, im) into planes on the host
        std::vector<double> planes(batch * 2 * nn);
        for (int b = 0; b < batch; b++)
            for (size_t e = 0; e < nn; e++) {
                planes[b * 2 * nn + e] = Y[(b * nn + e) * 2];
                planes[b * 2 * nn + nn + e] = Y[(b * nn + e) * 2 + 1];
            }
        const size_t blk = (size_t)n * 4 * bs;
        std::vector<double*> py, ptu, ppk, ua, ub, uc;
        for (int b = 0; b < batch; b++) {
            py.push_back(W + b * 2 * nn); ptu.push_back(TU + (size_t)b * 4 * n * bs); ppk.push_back(PK + (size_t)b * 4 * blk);
        }
        for (int b = 0; b < batch; b++) {           // entries 2 b, 2 b + 1: real and imaginary parts
            ua.push_back(ppk[b]); ub.push_back(ppk[b] + blk); uc.push_back(py[b]);
            ua.push_back(ppk[b] + 2 * blk); ub.push_back(ppk[b] + 3 * blk); uc.push_back(py[b] + nn);
        }
        double **PY = upload_ptrs(&tmp, py), **PTU = upload_ptrs(&tmp, ptu), **PPK = upload_ptrs(&tmp, ppk);
        double **UA = upload_ptrs(&tmp, ua), **UB = upload_ptrs(&tmp, ub), **UC = upload_ptrs(&tmp, uc);
        cudaMemcpyAsync(W, planes.data(), planes.size() * sizeof(double), cudaMemcpyHostToDevice, tmp.stream);
        cudaMemsetAsync(err, 0, sizeof(int), tmp.stream);
        const OzBuf oz = tmp_oz(tmp, (size_t)2 * batch * oz_entry_bytes(n, n, 4 * bs), fp64_path, 0);
        if (launch_pf(nullptr, n, batch, bs, PY, PTU, PPK, UA, UB, UC, la, ph, err, tmp.stream, &oz) != cudaSuccess)
            st = SGS_ECUDA;
        int herr = 0;
        cudaMemcpyAsync(phase, ph, 2 * batch * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        cudaMemcpyAsync(logabs, la, batch * sizeof(double), cudaMemcpyDeviceToHost, tmp.stream);
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, tmp.stream);
        if (cudaStreamSynchronize(tmp.stream) != cudaSuccess) st = SGS_ECUDA;
        else if (herr & SGS_DEV_TC_TIMEOUT) st = SGS_ETIMEOUT;
    }
    cudaStreamSynchronize(tmp.stream);
    tmp.release_all();
    cudaStreamDestroy(tmp.stream);
    tmp.stream = nullptr;
    return st;
}

}  // extern "C"

// ====================================================== allocation-free inverse
//
// sgs_kernel_inverse_static: the batched Gauss-Jordan inverse for callers that
// must not allocate device memory during the call.  Its scratch lives in one
// file-scope device array; host code reaches it through the address that
// cudaGetSymbolAddress returns for the current device (the array's name in
// host code is only a stand-in, not a device address).

#define SGS_STATIC_MAX_N 1024
#define SGS_STATIC_MAX_BATCH_N 32768   // batch * n
#define SGS_STATIC_PANEL 16
// carve-up of the array (offsets in doubles, each a multiple of 32 = 256 bytes)
#define SGS_STATIC_OFF_T 0                                                        // batch*n*16 doubles
#define SGS_STATIC_OFF_PIV (SGS_STATIC_OFF_T + SGS_STATIC_MAX_BATCH_N * SGS_STATIC_PANEL)   // batch*n ints
#define SGS_STATIC_OFF_PERM (SGS_STATIC_OFF_PIV + SGS_STATIC_MAX_BATCH_N / 2)              // batch*n ints
#define SGS_STATIC_OFF_SIGN (SGS_STATIC_OFF_PERM + SGS_STATIC_MAX_BATCH_N / 2)             // batch doubles
#define SGS_STATIC_OFF_PTR (SGS_STATIC_OFF_SIGN + SGS_STATIC_MAX_BATCH_N)                  // 2*batch pointers
#define SGS_STATIC_OFF_ERR (SGS_STATIC_OFF_PTR + 2 * SGS_STATIC_MAX_BATCH_N)               // one int
#define SGS_STATIC_DOUBLES (SGS_STATIC_OFF_ERR + 32)                                       // ~4.9 MiB

static __device__ __align__(256) double g_inverse_scratch[SGS_STATIC_DOUBLES];

namespace {

// pointer arrays for the batched panel and update kernels
__global__ void static_fill_ptrs_kernel(double* inv, double* scratch, int n, int batch) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double** W = reinterpret_cast<double**>(scratch + SGS_STATIC_OFF_PTR);
    double** T = W + batch;
    W[b] = inv + (size_t)b * n * n;
    T[b] = scratch + SGS_STATIC_OFF_T + (size_t)b * SGS_STATIC_PANEL * n;
}

// undo the Gauss-Jordan row interchanges in place: with perm from gj_perm_kernel (the
// column swaps applied in reverse order to the identity), row r of the inverse is
// row r of the eliminated matrix gathered through perm.  Each block owns whole rows
// (blockIdx.x, blockIdx.x + gridDim.x, ...) of matrix blockIdx.y: a row is read into
// shared memory (n doubles) and written back permuted, both coalesced.
__global__ void static_unpermute_kernel(double* inv, const int* perm, int n) {
    extern __shared__ double row[];
    const int b = blockIdx.y;
    const int* pm = perm + (size_t)b * n;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        double* A = inv + ((size_t)b * n + r) * n;
        for (int c = threadIdx.x; c < n; c += blockDim.x) row[c] = A[c];
        __syncthreads();
        for (int c = threadIdx.x; c < n; c += blockDim.x) A[c] = row[pm[c]];
        __syncthreads();
    }
}

struct StaticSlot { bool ready = false; double* base = nullptr; };
StaticSlot g_static_slots[64];
std::mutex g_static_mutex;

}  // namespace

extern "C" sgs_status sgs_kernel_inverse_static(const double* S, double* inv, double* logabsdet, int n, int batch,
                                                void* stream) {
    if (!S || !inv || !logabsdet || n < 1 || batch < 1) return SGS_EINVAL;
    if (n > SGS_STATIC_MAX_N || (long long)batch * n > SGS_STATIC_MAX_BATCH_N) return SGS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SGS_ECUDA;
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_slots[dev].ready) {
            if (cudaGetSymbolAddress((void**)&g_static_slots[dev].base, g_inverse_scratch) != cudaSuccess)
                return SGS_ECUDA;
            g_static_slots[dev].ready = true;
        }
        base = g_static_slots[dev].base;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = (size_t)n * n;
    double** W = reinterpret_cast<double**>(base + SGS_STATIC_OFF_PTR);
    double** T = W + batch;
    int* piv = reinterpret_cast<int*>(base + SGS_STATIC_OFF_PIV);
    int* perm = reinterpret_cast<int*>(base + SGS_STATIC_OFF_PERM);
    double* dsign = base + SGS_STATIC_OFF_SIGN;
    int* err = reinterpret_cast<int*>(base + SGS_STATIC_OFF_ERR);
    // the array keeps the previous call's contents: the error word must start at 0
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return SGS_ECUDA;
    if (cudaMemcpyAsync(inv, S, batch * nn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SGS_ECUDA;
    static_fill_ptrs_kernel<<<(batch + 127) / 128, 128, 0, st>>>(inv, base, n, batch);
    counted();
    if (launch_gj(nullptr, n, batch, SGS_STATIC_PANEL, W, T, piv, logabsdet, dsign, err, 0.0, st) != cudaSuccess)
        return SGS_ECUDA;
    gj_perm_kernel<<<batch, 128, 2 * (size_t)n * sizeof(int), st>>>(piv, perm, n, batch);   // 8 KB at n = 1024
    static_unpermute_kernel<<<dim3((unsigned)std::min(n, 64), batch), 256, (size_t)n * sizeof(double), st>>>(inv, perm,
                                                                                                      n);
    counted(); counted();
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SGS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SGS_ECUDA;
    return herr ? SGS_ESINGULAR : SGS_OK;
}
