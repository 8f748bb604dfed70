/*
 * sgs.h -- C ABI of the GB300 (sm_103a) imaginary-time step of the
 * superposition-of-Gaussian-states (SGS) variational method for quantum
 * impurity models (Boutin & Bauer, arXiv:2105.01088).
 *
 * Problem statement (Sec. II): a fermion Hamiltonian in Majorana form
 *   H = e_const + i sum_kl A_kl c_k c_l + sum_klpq U_klpq c_k c_l c_p c_q
 * (Sec. II A), and a rank-M ansatz |psi> = sum_mu lambda_mu |phi_mu> of
 * Gaussian states, each described by its real antisymmetric 2N x 2N
 * covariance matrix Gamma^mu with (Gamma^mu)^2 = -1 (Sec. II B-C).
 *
 * One step (Sec. III C): all pair overlaps with phase, transition matrices
 * and Hamiltonian matrix elements (Sec. II B-C, III B); the amplitudes from
 * h lambda = E G lambda (Eq. eigLambda); the decoupled equation of motion of
 * every Gamma^mu (Eq. EOM-Gamma3); the orthogonal update and the
 * re-purification of App. A.
 *
 * Conventions for every call:
 *   - All array arguments are HOST pointers owned by the caller; inputs are
 *     copied during the call, outputs are written before the call returns.
 *   - Matrices are row-major FP64.  Complex numbers are stored as (re, im)
 *     pairs of doubles.
 *   - Majoranas c_{2m}, c_{2m+1} of fermion mode m (0-based) are a_m + a_m^dag
 *     and -i (a_m - a_m^dag); the vacuum has Gamma = (+)_m [[0,1],[-1,0]] and
 *     the fermion parity of a Gaussian state is Pf(Gamma).
 *   - The overlap gauge (Sec. II B) takes the first ansatz state as the
 *     reference: <phi_0|phi_mu> is real and positive.
 *   - Every call returns an sgs_status; nothing aborts or throws across the
 *     ABI.  sgs_last_error() describes the last failure of a context.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Device memory is owned by the context and released by sgs_free().
 */
#ifndef SGS_H
#define SGS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgs_ctx sgs_ctx;

typedef enum {
    SGS_OK = 0,
    SGS_EINVAL = 1,      /* bad argument (sizes, NULL pointers, rank, parity) */
    SGS_ENOMEM = 2,      /* device allocation failed, or over the HBM budget */
    SGS_ESINGULAR = 3,   /* two ansatz states orthogonal (Gamma_a + Gamma_b singular) */
    SGS_ENOTCONV = 4,    /* amplitude solver or exponential step out of range */
    SGS_ETIMEOUT = 5,    /* a bounded device wait ran out */
    SGS_ECUDA = 6        /* CUDA runtime error (message in sgs_last_error) */
} sgs_status;

typedef enum {
    SGS_FP64 = 0,        /* every product in FP64 (on the path sgs_options.fp64_path selects) */
    SGS_MIXED_TF32 = 1,  /* pair GEMMs of the equation of motion in TF32, FP32 accumulate */
    SGS_MIXED_BF16 = 2,  /* same in BF16 */
    SGS_FP32_3XTF32 = 3  /* same with the 3xTF32 split (about FP32 accuracy) */
} sgs_precision;

typedef enum {
    SGS_C_INVERSE = 0,   /* c_mu = [lambda_mu conj(lt_mu)]^{-1}           (Sec. III A) */
    SGS_C_PHASE = 1      /* c_mu = lt_mu conj(lambda_mu) / |lambda_mu lt_mu|  (Sec. III A) */
} sgs_cmode;

/* Arithmetic of the FP64 products (every product of the step in SGS_FP64, the
 * factorisations, Im Delta and the re-purification in the mixed forms), chosen
 * per instance.  Both are FP64 products; they differ in how they round.
 *  - SGS_FP64_EMULATED (default): on the bf16 tensor cores.  Each K-major row
 *    of op(A) and column of op(B) is scaled by the power of two of its largest
 *    entry and split into eight signed 7-bit integer slices (57 bits); the 36
 *    slice products of combined weight above 2^-63 are summed exactly in fp32
 *    TMEM accumulators (K in chunks of 512) and combined in 64-bit integers
 *    with one final rounding.  Error of one product, per element:
 *      |C_ij - (AB)_ij| <= u |(AB)_ij| + K 2^-52 max_k|A_ik| max_k|B_kj|
 *    (u = 2^-53), plus u times any added terms (beta Cin, diag): normwise in
 *    row i of A and column j of B, so an element whose terms are all far below
 *    those maxima is less accurate than the K u sum_k |A_ik||B_kj| of a native
 *    FP64 dot product.
 *  - SGS_FP64_FMA: FP64 fused multiply-adds on the CUDA cores (the error of a
 *    native FP64 dot product), about 8x slower on GB300 at 2N = 512. */
typedef enum {
    SGS_FP64_EMULATED = 0,
    SGS_FP64_FMA = 1
} sgs_fp64_path;

/* Model, Sec. II A.  A: n x n row-major real antisymmetric, n = 2 * n_modes.
 * Quartic part: n_quartic monomials value[j] * c_i0 c_i1 c_i2 c_i3 with four
 * distinct indices idx[4j..4j+3]; the library antisymmetrises them into U
 * (U_{pi(i)} = sgn(pi) value / 24).  Interaction terms of more than four
 * Majoranas (Sec. II A allows them; Sec. III C estimates their cost): term j
 * is v_j i^(r mod 2) c_s1 ... c_s(2r) with 2r = higher_len[j] (6 or 8)
 * distinct indices taken in order from higher_idx (concatenated) and
 * v_j = higher_val[j] real (the factor i^(r mod 2) makes it Hermitian).
 * Their expectation is the Pfaffian of the 2r x 2r sub-block of the
 * transition matrix, their share of the Fock matrix its derivative.  At most
 * 16 distinct Majoranas may appear in interaction terms (the impurity block),
 * and at most SGS_MAX_HIGHER higher terms.  A zero-initialised tail
 * (n_higher = 0) means none. */
#define SGS_MAX_HIGHER 64
typedef struct {
    int n_modes;
    const double* A;
    int n_quartic;
    const int* quartic_idx;
    const double* quartic_val;
    double e_const;
    int n_higher;
    const int* higher_len;
    const int* higher_idx;
    const double* higher_val;
} sgs_model;

typedef enum {
    SGS_INTEGRATOR_EXP = 0,    /* Gamma <- R Gamma R^T, R = exp{(ds/4)[Gamma, dGamma]} (App. A, Eq. ExpStep),
                                  then the canonical-form renormalisation */
    SGS_INTEGRATOR_EULER = 1   /* Gamma <- Gamma + ds dGamma (Eq. RKstep), then the canonical-form
                                  renormalisation (App. A): the polar factor, by six Newton-Schulz
                                  iterations (enough while ds ||dGamma||_2 <= 0.5) */
} sgs_integrator;

/* Per-instance options.  gamma0: [rank][n][n] pure states of one parity
 * (Pf Gamma = parity), or NULL for seeded random states: Gamma = O J O^T with O
 * Haar on O(2N) (QR of a standard-normal matrix, signs of diag R folded in, first
 * column negated to reach det O = parity), drawn from Philox4x32-10 keyed by
 * `seed` (state mu's matrix entries 2j, 2j+1 from counter (j, mu, 0, 0) by
 * Box-Muller on the first two words; the phase of lambda_mu, 2 pi x0 / 2^32,
 * from counter (0, mu, 1, 0)).  lambda0: [rank] complex, may be NULL (the first
 * solve replaces the amplitudes).  stream: a cudaStream_t, or NULL for the
 * context's own stream (the first instance's stream is used for all). */
typedef struct {
    int rank;
    double dtau;             /* step ds of App. A */
    int precision;           /* sgs_precision */
    int cmode;               /* sgs_cmode */
    int parity;              /* +1 or -1 */
    const double* gamma0;
    const double* lambda0;
    void* stream;
    int integrator;          /* sgs_integrator (0: the exponential step) */
    unsigned long long seed; /* initial states when gamma0 is NULL */
    int fp64_path;           /* sgs_fp64_path of this instance's FP64 products (0: emulated) */
    size_t emulation_scratch;/* SGS_FP64_EMULATED: bytes of operand-slice scratch this instance
                                owns (0: 2 GiB; at least 1 MiB); larger batches run in chunks */
    int shard_rank;          /* pair sharding (sgs_shard_pairs): this rank of shard_world; */
    int shard_world;         /*   shard_world <= 1: not sharded */
    int pair_chunk;          /* bounded memory: the per-pair buffers hold this many pairs and a step
                                runs the pairs in chunks of that size (0: all pairs at once) */
} sgs_options;

/* Create a context holding n_instances independent problems (models[i],
 * opts[i]); uploads the model and the initial states to device memory.
 * Errors: SGS_EINVAL (n_modes < 1, rank < 1 or > 64, parity not +-1),
 * SGS_ENOMEM, SGS_ECUDA.  On error *out is NULL. */
sgs_status sgs_init(const sgs_model* models, const sgs_options* opts, int n_instances, sgs_ctx** out);

/* Continuous batching.  sgs_create makes an empty context on `stream` (NULL:
 * a stream of its own) whose live instances may not hold more than
 * hbm_budget bytes of device memory (0: no budget).  sgs_admit adds one
 * instance (a solve request) while others are live: it returns its slot, or
 * SGS_ENOMEM without allocating if the instance's estimated footprint would
 * exceed the budget.  sgs_retire releases a slot's device memory for later
 * admissions.  Slot ids are stable; retired slots are skipped by sgs_step /
 * sgs_energy (their rows of `energies` are left untouched) and rejected by
 * the per-instance calls.  Instances never interact: a slot's results are the
 * same whatever else is live.  sgs_init = sgs_create + one sgs_admit each. */
sgs_status sgs_create(void* stream, size_t hbm_budget, sgs_ctx** out);
sgs_status sgs_admit(sgs_ctx* ctx, const sgs_model* model, const sgs_options* opts, int* slot);
sgs_status sgs_retire(sgs_ctx* ctx, int slot);
size_t sgs_bytes_in_use(const sgs_ctx* ctx);

/* The seeded initial states sgs_admit generates when gamma0 is NULL (host only,
 * no device work): gamma [rank][2N][2N], lambda [rank] complex (re, im). */
sgs_status sgs_seeded_states(int n_modes, int rank, unsigned long long seed, int parity, double* gamma,
                             double* lambda);

/* Health of one instance's current states (a per-step check a caller may run):
 * out[0] = max over states of max_kl |(Gamma^2)_kl + delta_kl| (purity residual),
 * out[1] = number of non-finite entries of Gamma, out[2] = smallest / largest
 * eigenvalue of the Gram matrix G at the last amplitude solve (1 for orthonormal
 * states, near 0 for nearly dependent ones), out[3] = the energy of that solve.
 * Admission itself rejects initial states that are not finite or not
 * antisymmetric (SGS_EINVAL); a wrong parity shows as SGS_ESINGULAR at the first
 * step. */
sgs_status sgs_health(sgs_ctx* ctx, int instance, double* out);

/* Instances whose device-side error (SGS_ESINGULAR, SGS_ENOTCONV,
 * SGS_ETIMEOUT) ended the last call.  sgs_failed_instance returns the first
 * (the one sgs_last_error describes) or -1; sgs_failed_instances writes up to
 * `capacity` slot ids to `slots` (may be NULL) and returns how many failed.
 * Their error state is cleared.  The other instances of that sgs_step
 * completed every step (their states advanced) and their rows of `energies`
 * are written as on success; a request loop retires the failed slots and
 * carries on. */
int sgs_failed_instance(const sgs_ctx* ctx);
int sgs_failed_instances(const sgs_ctx* ctx, int* slots, int capacity);

/* Autotuning of the factorisation tile shapes.  With enable = 1, sgs_admit
 * (and sgs_add_state) times the candidate panel widths of the blocked
 * Gauss-Jordan inverse (leaf panels of 8, 12, 16, 20, 24, 32, 48, 64 columns, as shared memory allows)
 * and of the blocked complex Pfaffian (8, 12, 16, 24, 32 column pairs) on the new
 * instance's own pairs,
 * with CUDA events, and keeps the fastest.  Choices are cached per (n, rank,
 * precision) for the process, so a shape is timed once; the scratch of tuned
 * instances is sized for the widest candidate.  Widths change results only
 * by rounding.  Default: off (fixed widths). */
sgs_status sgs_set_autotune(sgs_ctx* ctx, int enable);

/* Panel widths an instance uses; from_cache: -1 not tuned, 0 timed at
 * admission, 1 taken from the cache, 2 set by sgs_set_panel_widths.  Any
 * output may be NULL. */
sgs_status sgs_get_tuning(const sgs_ctx* ctx, int instance, int* gj_width, int* pf_width, int* from_cache);

/* Fix the panel widths of a live instance (for reproducible timings and
 * profiles): each must be one of the autotuner's candidates and fit the
 * instance's scratch (an instance admitted with autotuning on has room for
 * the widest).  Waits for the context's stream; drops a captured step graph.
 * SGS_EINVAL otherwise. */
sgs_status sgs_set_panel_widths(sgs_ctx* ctx, int instance, int gj_width, int pf_width);

/* Rank growth (Sec. III C): append to the live instance `slot` the state
 * Q Gamma_src Q^T with Q = exp(K), a special orthogonal matrix.  The paper
 * grows the ansatz one state at a time from the mean-field (rank-1) solution,
 * copying a state of high amplitude through a random Q close to the identity;
 * the caller draws K (host [n][n], row-major, exactly antisymmetric,
 * ||K||_F <= 8; copied) and so fixes ||Q - 1||_F ~ ||K||_F.  src: index of the
 * state to copy, or -1 for the state with the largest |lambda_mu| of the last
 * amplitude solve (the initial amplitudes before the first step).  The rank
 * grows by one, the slot keeps its index, the new state's amplitude is 0 until
 * the next solve, and all device buffers of the instance are re-allocated
 * (checked against the HBM budget).  Errors: SGS_EINVAL (slot not live, src
 * out of range, rank already 64, K not antisymmetric or too large),
 * SGS_ENOMEM, SGS_ECUDA; on error the instance is unchanged. */
sgs_status sgs_add_state(sgs_ctx* ctx, int slot, const double* K, int src);

/* Graph replay (default on): the first sgs_step of a context captures one step
 * of every live instance into a CUDA graph (one branch per instance, so their
 * kernels overlap), later steps replay it; admit/retire re-capture.  Needs a
 * context stream other than the legacy default stream; off while profiling. */
sgs_status sgs_set_graphs(sgs_ctx* ctx, int enable);

/* Advance every instance by n_steps imaginary-time steps (Sec. III C).
 * energies (may be NULL): [n_instances][n_steps], the energy E of the
 * states at the start of each step with optimal amplitudes.
 * Errors: SGS_ESINGULAR, SGS_ENOTCONV, SGS_ETIMEOUT (a device-side failure
 * of some instances, listed by sgs_failed_instances; their rows of
 * `energies` are left untouched, every other row is written), SGS_ECUDA. */
sgs_status sgs_step(sgs_ctx* ctx, int n_steps, double* energies);

/* Energy of the current states with optimal amplitudes (Eq. eigLambda),
 * without changing the states.  energies: [n_instances]. */
sgs_status sgs_energy(sgs_ctx* ctx, double* energies);

typedef enum {
    SGS_CORR_SPIN_SPIN = 0,      /* C(s) = <S(0).S(s)> (Eq. Cr); sites[i] = s, a site index */
    SGS_CORR_TWO_CHANNEL_K = 1,  /* K(r) = sum_alpha <S_imp.S_alpha(r)> (Eq. K2CK); sites[i] = r >= 1 */
    SGS_CORR_RENYI2 = 2          /* S_2 of the impurity plus the first l sites (App. B); sites[i] = l */
} sgs_corr_kind;

/* Pair-sharded step: one problem over several ranks (one GPU each).  The
 * pairs are independent units (Sec. III C), so an instance admitted with
 * shard_world = W > 1 holds the pairs whose index in the order (0, 1),
 * (0, 2), ..., (M - 2, M - 1) is shard_rank modulo W, and adds the own
 * (beta = mu) terms of the states mu with mu modulo W = shard_rank.  Every
 * rank holds all M states.  One step is three calls with two sums over the
 * ranks between them, which the caller makes (e.g. an all-reduce):
 *   1. sgs_shard_pairs(ctx, i, gh): the pair pass (A1-A5) over this rank's
 *      pairs; writes this rank's share of G and h to gh = [G | h], each
 *      [M][M] complex (re, im), zero where another rank holds the pair.
 *      Summed over the ranks, gh is the whole (G, h).
 *   2. sgs_shard_eom(ctx, i, gh, dgamma, energy): takes the summed gh, solves
 *      the amplitudes (the same solve on every rank), writes the energy E of
 *      the states (host double, may be NULL) and this rank's share of
 *      dGamma/ds to dgamma ([M][n][n]): the terms of its pairs and of its own
 *      states (Eq. EOM-Gamma3 is linear in them).  Summed over the ranks,
 *      dgamma is dGamma/ds.
 *   3. sgs_shard_update(ctx, i, dgamma): takes the summed dgamma and applies
 *      the orthogonal update and re-purification to every state (App. A), the
 *      same on every rank, so the states stay equal across ranks without
 *      another exchange.
 * gh and dgamma may be host or device pointers (copies by cudaMemcpyDefault);
 * device buffers on the context's device let the sums run as NCCL
 * collectives.  A sharded instance does not step through sgs_step or
 * sgs_energy (SGS_EINVAL if one is live in the context) and has no
 * observables or rank growth.  Results equal the unsharded step's up to the
 * order of the sums.  Errors as sgs_step. */
sgs_status sgs_shard_pairs(sgs_ctx* ctx, int instance, double* gh);
sgs_status sgs_shard_eom(sgs_ctx* ctx, int instance, const double* gh, double* dgamma, double* energy);
sgs_status sgs_shard_update(sgs_ctx* ctx, int instance, const double* dgamma);

/* Observables of the current SGS state of one instance, evaluated on its
 * current covariance matrices with optimal amplitudes (a pair pass runs
 * first; the states are not changed).  out: [n_sites].  Sites are spinful
 * sites in the library's mode order: site s holds modes 2s, 2s+1 (Majoranas
 * 4s..4s+3), the impurity is site 0.  For a single chain site s is at
 * distance s from the impurity; for two channels interleaved (as
 * sgs_build_anderson lays them out) channel alpha's r-th site is
 * 1 + 2(r - 1) + alpha.  Renyi-2: A = sites 0..l (the leading 4(1 + l)
 * Majoranas, 4(1 + l) <= 2N); up to l = 12 each Pfaffian runs in one CTA's
 * shared memory, beyond that in chunks through the batched blocked Pfaffian.
 * Errors: SGS_EINVAL for sites out of range. */
sgs_status sgs_correlator(sgs_ctx* ctx, int instance, sgs_corr_kind kind, const int* sites, int n_sites,
                          double* out);

/* Hamiltonian variance (Eq. residual, Sec. IV A): delta_H^2 = <psi|H^2|psi>
 * - <psi|H|psi>^2 of the current states of one instance with optimal
 * amplitudes normalised to <psi|psi> = 1 (a pair pass runs first; the states
 * are not changed).  <H^2> comes from Wick's theorem on each pair's
 * transition matrix in O(n^2) per pair (the quadratic part of H must be
 * sparse for that bound; at most 64 distinct quartic monomials).  The paper
 * extrapolates the energy linearly in delta_H^2 -> 0.  energy, variance: host
 * doubles, either may be NULL.  Errors: SGS_EINVAL (also for a model with
 * terms of more than four Majoranas), SGS_ESINGULAR, SGS_ECUDA. */
sgs_status sgs_variance(sgs_ctx* ctx, int instance, double* energy, double* variance);

void sgs_free(sgs_ctx* ctx);
const char* sgs_last_error(const sgs_ctx* ctx);

/* Checkpoint / resume.  gamma: [rank][n][n]; lambda: [rank] complex. */
sgs_status sgs_get_state(const sgs_ctx* ctx, int instance, double* gamma, double* lambda);
sgs_status sgs_set_state(sgs_ctx* ctx, int instance, const double* gamma, const double* lambda);

/* Intermediate results of the last sgs_step / sgs_energy call of one
 * instance: G and h ([rank][rank] complex, Eq. eigLambda) and, after
 * sgs_step, dGamma/ds of the last step ([rank][n][n], Eq. EOM-Gamma3). */
sgs_status sgs_get_pair_matrices(const sgs_ctx* ctx, int instance, double* G, double* h);
sgs_status sgs_get_derivative(const sgs_ctx* ctx, int instance, double* dgamma);

/* Device memory hook: if set before sgs_init, every device allocation of
 * the library goes through alloc/release (e.g. a framework's caching
 * allocator); otherwise cudaMalloc/cudaFree. */
typedef void* (*sgs_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*sgs_free_fn)(void* ptr, void* user);
void sgs_set_allocator(sgs_alloc_fn alloc, sgs_free_fn release, void* user);

/* Stage profile.  sgs_set_profiling(ctx, 1) resets the counters and records
 * CUDA events (on the context stream) around each stage of every following
 * sgs_step / sgs_energy; sgs_get_profile returns per stage the summed device
 * time (ms), the algorithmic FP64 flops (useful work: an antisymmetric
 * product counts n^3, a general one 2 n^3, the Gauss-Jordan inverse 2 n^3,
 * the complex Pfaffian 4 n^3 / 3), the algorithmic bytes of memory-bound
 * stages, and the number of kernels the library launched.  gemm_f64 (may be
 * NULL) receives [total ms, algorithmic flops, launches] of the FP64 MMA GEMM
 * kernel over all its launches (timed one by one; the pass-through squaring
 * launches of the exponential are left out). */
typedef enum {
    SGS_STAGE_PAIR_INVERSE = 0,    /* S = G_a + G_b, blocked Gauss-Jordan inverse */
    SGS_STAGE_PAIR_DELTA = 1,      /* Im Delta = (G_a - G_b) S^{-1} */
    SGS_STAGE_PHASE_PFAFFIAN = 2,  /* Pf(G_0 + Delta^{a,b}) */
    SGS_STAGE_AMPLITUDES = 3,      /* G, h, Wick contractions, h lambda = E G lambda */
    SGS_STAGE_EOM_W = 4,           /* W = (S^{-1} F) S^{-1} and Gamma F Gamma (antisymmetric products) */
    SGS_STAGE_EOM_V = 5,           /* V = D W: one batched general product over all pairs */
    SGS_STAGE_EOM_X = 6,           /* X = V D (antisymmetric) */
    SGS_STAGE_EOM_ASSEMBLY = 7,    /* Delta F Delta planes, dGamma/ds */
    SGS_STAGE_UPDATE = 8,          /* exp step, R Gamma R^T, re-purification */
    SGS_N_STAGES = 9
} sgs_stage;
sgs_status sgs_set_profiling(sgs_ctx* ctx, int enable);
sgs_status sgs_get_profile(const sgs_ctx* ctx, double* ms, double* flops, double* bytes, long long* launches,
                           double* gemm_f64);

/* Measured throughput (TFLOP/s) of an FP64 pipe of the current device:
 * kind 0 = the m8n8k4 FP64 MMA (mma.sync .f64), kind 1 = FP64 FMA on the
 * CUDA cores (the pipe of the SGS_FP64_FMA products and of the
 * factorisations' panels), kind 2 = both interleaved in one kernel (their sum
 * shows whether the two share one pipe). */
sgs_status sgs_probe_peak(int kind, double* tflops);

/* Majorana form of the Anderson impurity of Sec. IV (H_0 + H_I) with
 * n_channels open bath chains of n_bath sites, hybridisation V, hopping t,
 * chemical potential mu, interaction U n_up n_dn and level eps_d on the
 * impurity.  Site order: impurity, then chain sites interleaved by channel;
 * mode 2*site + spin.  Writes A ([n][n], n = 4 (1 + n_channels n_bath)), one
 * quartic monomial (idx[4], val[1]) and e_const.  Returns the number of
 * modes N, or -1 on bad arguments. */
int sgs_build_anderson(int n_bath, int n_channels, double U, double eps_d, double V, double t, double mu,
                       double* A, int* quartic_idx, double* quartic_val, double* e_const);

/* Majorana form of the lattice two-channel Kondo model of Sec. V:
 * H = -t sum (hopping along each channel) + H_J + H_BC, H_J = J sum_alpha
 * S_imp . S_alpha(1) with a fermionic impurity (site 0, no quadratic term),
 * channels of L - 1 sites interleaved (channel alpha's r-th site is
 * 1 + 2(r - 1) + alpha) and the boundary site 2L - 1 hopping to the last site
 * of both channels (H_BC): 2L sites, n = 8L.  Writes A ([n][n]), the 24
 * quartic monomials of H_J (idx [24][4], val [24]) and e_const (0).  Returns
 * the number of modes N = 4L, or -1 on bad arguments (L < 2). */
int sgs_build_2ck(int L, double J, double t, double* A, int* quartic_idx, double* quartic_val, double* e_const);

/* Failure path of the library's bounded device waits.  Every wait of its
 * kernels (the tensor-core pipelines' mbarrier waits, 2 s) gives up after a
 * time limit: the kernel sets an error bit, drains its own work in flight and
 * returns, and the call reports SGS_ETIMEOUT with the context still usable.
 * This probe runs that wait on its own on a device flag that nothing sets,
 * with limit_ns (1e3 .. 1e10) in place of 2 s: it returns SGS_ETIMEOUT when
 * the wait ran out as it should, and the device time of the launch in
 * *elapsed_ms (may be NULL).  SGS_EINVAL for a limit out of range. */
sgs_status sgs_probe_wait(unsigned long long limit_ns, double* elapsed_ms);

/* Shared-memory set-up of the current device.  Kernels that keep large tiles in
 * shared memory need their dynamic limit raised once per device, with that
 * device current; the first call that launches them on a device does it, and
 * so does this call.  For kernel i < n_out (0 Gauss-Jordan panel, 1 Pfaffian
 * panel, 2 Renyi Pfaffian, 3-5 tensor-core product tf32 / bf16 / 3xtf32,
 * 6 emulated FP64 product, 7 block slicer, 8 emulated FP64 product of
 * 16-column tiles; n_out <= 9) it writes the limit
 * in force to limit[i] and the device's opt-in maximum less the kernel's
 * static shared memory to expected[i]. */
sgs_status sgs_kernel_smem_limits(int n_out, int* limit, int* expected);

/* Building blocks with host buffers, for tests and external callers.
 * fp64_path (sgs_fp64_path) selects the arithmetic of their FP64 products.
 * sgs_kernel_inverse: batch n x n matrices -> inverses (Gauss-Jordan,
 *   partial pivoting, FP64) and log|det|.  Returns SGS_ESINGULAR on a zero
 *   pivot.
 * sgs_kernel_pfaffian: batch complex antisymmetric n x n matrices (re, im
 *   interleaved) -> Pf = phase * exp(logabs), phase as (re, im).
 * sgs_kernel_gemm: batch C = alpha op(A) op(B) + beta Cin + diag I through the
 *   library's FP64 product, op(A) m x k, op(B) k x n, all row-major and
 *   contiguous per batch entry (A stored k x m if trans_a, B stored n x k if
 *   trans_b); Cin may be NULL.  C is in/out: mode 0 writes every element;
 *   mode 1 (m = n) computes the strictly lower part and writes C and -C^T
 *   with a zero diagonal; mode 2 (m = n, Gauss-Jordan delayed update) leaves
 *   columns gj_k0 .. gj_k0 + gj_b - 1 of C unchanged and does not add Cin on
 *   rows in that range.  mode + 4 (k = n, trans_b = 0) declares B
 *   antisymmetric: the emulated path then slices B's rows (op(B)'s columns
 *   negated) and negates alpha; the FMA path ignores it.
 *   emulation_scratch: cap on the operand-slice scratch of the emulated path
 *   (0: 2 GiB, at least 1 MiB); a batch that does not fit runs in chunks,
 *   with bitwise the same result. */
sgs_status sgs_kernel_inverse(const double* S, int n, int batch, int fp64_path, double* inv, double* logabsdet);
sgs_status sgs_kernel_pfaffian(const double* Y, int n, int batch, int fp64_path, double* phase, double* logabs);
sgs_status sgs_kernel_gemm(const double* A, const double* B, const double* Cin, int m, int n, int k, int trans_a,
                           int trans_b, double alpha, double beta, double diag, int mode, int gj_k0, int gj_b,
                           int batch, int fp64_path, size_t emulation_scratch, double* C);

/* sgs_kernel_gemm_tc: batch C = A B on the tcgen05 tensor cores, A: m x k
 * row-major, Bt: n x k row-major (= B^T, the K-major form the tensor core
 * reads), C: m x n FP64.  kind 0 = TF32, 1 = BF16, 2 = 3xTF32 (split
 * operands, three products, fp32 accumulation).  k must be a multiple of 8.
 * Returns SGS_ETIMEOUT if a bounded on-device wait ran out. */
sgs_status sgs_kernel_gemm_tc(const double* A, const double* Bt, int m, int n, int k, int batch, int kind,
                              double* C);

/* Allocation-free variant of sgs_kernel_inverse.  The paper has no
 * counterpart: this is a convenience for callers that must not allocate
 * device memory during a call, such as a host program whose device memory
 * is entirely owned by another framework's pool, or a latency-critical loop
 * that cannot afford cudaMalloc's implicit device synchronisation.
 *   S, inv: DEVICE pointers to batch row-major n x n FP64 matrices (S is read,
 *   inv receives S^{-1}); logabsdet: DEVICE pointer to batch doubles
 *   (log|det S|); stream: a cudaStream_t or NULL (legacy default stream).
 * The call allocates nothing: its scratch is a file-scope device array of
 * about 5.0 MiB that every GPU loading the library holds until exit.  Its
 * products run on the FP64 FMA pipe (the emulated path needs slice scratch).
 * Limits: 1 <= n <= 1024 and batch * n <= 32768; larger sizes return
 * SGS_EINVAL before any GPU work.  The first call on a device does the
 * set-up: it looks up the array's device address (cudaGetSymbolAddress) and
 * raises the panel kernel's shared-memory limit, with that device current;
 * make that first call before any stream capture.  Under lazy module
 * loading that first call may also load the library's device code, which
 * creates the array then: a caller that needs every call free of device
 * allocation makes one warm-up call per device first (a 1 x 1 inverse will
 * do).  Every call shares the array and it keeps the last call's contents,
 * so calls that overlap on the GPU (other streams, other host threads)
 * race; serialise them.  The call waits for its stream and returns
 * SGS_ESINGULAR on a zero pivot, SGS_ECUDA on a CUDA error. */
sgs_status sgs_kernel_inverse_static(const double* S, double* inv, double* logabsdet, int n, int batch,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SGS_H */
