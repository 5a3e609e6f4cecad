/*
 * smc.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of population-based MCMC and SMC samplers, after Lee, Yau, Giles,
 * Doucet & Holmes (2009), "On the utility of graphics cards to perform
 * massively parallel simulation of advanced Monte Carlo methods".
 *
 * Conventions (every entry point):
 *   - Data pointers are DEVICE pointers owned by the caller, unless the
 *     argument says "host".  The library keeps no pointer after a call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Every compute call is asynchronous on that stream and returns before
 *     the work finishes.
 *   - Argument errors are detected on the host and returned at once
 *     (SMC_ERR_ARG); nothing is launched then.  Errors found by a kernel
 *     (non-finite likelihood, zero total weight, weights outside [0,1],
 *     exhausted wait limit) are latched in a device status word of the
 *     context and reported by smc_ctx_check().
 *   - Scratch memory (reduction partials, scan tile descriptors, queue
 *     counters, the status word, the binned layout of the last data set a
 *     population sweep saw) lives in the context.  smc_reserve() sizes
 *     it up front; a call that needs more grows it, which is refused with
 *     SMC_ERR_ARG while the stream is being captured into a CUDA graph.
 *     Calls on one context share that scratch, so they must run one after
 *     another on the GPU (one stream, or streams ordered by events); work
 *     meant to overlap on several streams takes one context per stream.
 *   - Random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11)
 *     in place of the MRG32k3a / xorshift skip-ahead streams of Section
 *     2.5.  key = (seed mod 2^32, seed div 2^32); counter = (index, block,
 *     step mod 2^32, purpose | (step div 2^32) << 8).  Uniforms are
 *     ((w >> 9) + 1/2) 2^-23 in (0,1); normals are Box-Muller on word pairs.
 *     No RNG state is passed or kept: (seed, step) select the draws.
 *   - Layouts: 1-D mixture particles theta are SoA float[K][M] (theta[k*M+p]
 *     is mu_k of particle p); diagonal d-dimensional mixture particles are
 *     float[M][K][d]; log-likelihoods, log-weights and normalised weights
 *     are double[M]; ancestors are int32[M]; particle-filter states are
 *     float[d][M].
 *   - Index arrays passed in device memory (ancestors, population offsets)
 *     are used as given: their values are not read on the host, so the
 *     library cannot check them.  Ancestors must lie in [0, M); those this
 *     library's resampling calls write always do.  The debug build of the
 *     library (libsmc_debug.so, -DSMC_DEBUG_BOUNDS) checks them in the
 *     kernels and reports SMC_ERR_BOUNDS instead of reading outside.
 */
#ifndef SMC_GB300_H
#define SMC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum smc_status {
    SMC_OK = 0,
    SMC_ERR_ARG = -1,          /* bad argument, or workspace growth during capture */
    SMC_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    SMC_ERR_NONFINITE = -3,    /* NaN log-likelihood / log-weight seen by a kernel */
    SMC_ERR_ZERO_WEIGHT = -4,  /* every weight is zero (all log-weights -inf) */
    SMC_ERR_TIMEOUT = -5,      /* a bounded device wait gave up */
    SMC_ERR_UNSUPPORTED = -6,  /* configuration not built (e.g. K too large) */
    SMC_ERR_BOUNDS = -7        /* debug build only: an index failed its bounds check
                                  (the access was skipped; e.g. an ancestor outside [0, M)) */
} smc_status;

typedef struct smc_ctx smc_ctx;

/* Stream purposes of the Philox counter (the fourth counter word). */
enum { SMC_RNG_MOVE = 1, SMC_RNG_ACCEPT = 2, SMC_RNG_RESAMPLE = 3,
       SMC_RNG_EXCHANGE = 4, SMC_RNG_PFNOISE = 5, SMC_RNG_MULTINOMIAL = 6,
       SMC_RNG_PROPOSAL = 7 };

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device` (made current for the call).
 * Allocates the status word and a small initial workspace.  *out receives
 * the handle; SMC_ERR_CUDA if the device cannot be used. */
smc_status smc_create(smc_ctx** out, int device);

/* Free the context and its workspace (synchronises the device first). */
smc_status smc_destroy(smc_ctx* ctx);

/* Size the workspace for up to `max_particles` particles (or chains) and
 * `max_pops` populations so that no later call grows it (required before
 * graph capture).  May allocate; not to be called while capturing. */
smc_status smc_reserve(smc_ctx* ctx, int64_t max_particles, int32_t max_pops);

/* Synchronise `stream`, read and clear the device status word, and return
 * the first error a kernel latched since the last check (SMC_OK if none). */
smc_status smc_ctx_check(smc_ctx* ctx, void* stream);

/* Static English description of a status code. */
const char* smc_status_string(smc_status s);

/* Launch-shape override used by the autotuner.  `op` is one of SMC_OP_*;
 * `lanes` = threads cooperating on one particle's likelihood (1,2,4,8,16,32;
 * Section 4.1.3 splits one likelihood over threads when N is large),
 * `threads` = threads per block (64..256, multiple of 32).  lanes = 0
 * restores the built-in heuristic. */
enum { SMC_OP_LOGLIK = 0, SMC_OP_MOVE = 1, SMC_OP_POPMCMC = 2, SMC_OP_COUNT = 3 };
smc_status smc_set_launch(smc_ctx* ctx, int32_t op, int32_t lanes, int32_t threads);
smc_status smc_get_launch(smc_ctx* ctx, int32_t op, int64_t M, int64_t N, int32_t K,
                          int32_t* lanes, int32_t* threads);

/* Test hook for the bounded device waits (no counterpart in the paper):
 * the number of polls the first wait on a kernel's bulk copy of the data
 * into shared memory makes before it gives up and latches SMC_ERR_TIMEOUT
 * in the context (reported by smc_ctx_check).  A wait that gives up is
 * followed by a second one with the full bound, so no copy is left in
 * flight and the results stay correct; 0 makes every such wait give up at
 * once.  Applies to the 1-D likelihood, move and population-sweep calls of
 * this context.  Default 4,194,304 (seconds of polling). */
smc_status smc_set_wait_limit(smc_ctx* ctx, uint32_t polls);

/* ------------------------------------------------------------------ models */

enum { SMC_GMM_1D = 0, SMC_GMM_DIAG = 1 };
enum { SMC_PREC_FP32 = 0, SMC_PREC_BF16SPLIT = 1 };

/* Gaussian mixture with known weights and a common known sigma
 * (Section 4.1: p(y_j|mu) = sum_i w_i f(y_j|mu_i, sigma); the density of
 * y is the product over j) and a uniform prior on the box [lo, hi]^(K d). */
typedef struct smc_gmm {
    int32_t kind;          /* SMC_GMM_1D or SMC_GMM_DIAG */
    int32_t K;             /* components: 1..64 (1-D), 1..64 (diag) */
    int32_t d;             /* dimension: 1 for SMC_GMM_1D; 1..64 for diag */
    int32_t precision;     /* SMC_PREC_FP32, or SMC_PREC_BF16SPLIT (diag only) */
    const float* log_w;    /* HOST pointer, [K] log mixture weights, copied per call */
    float sigma;           /* component standard deviation (> 0) */
    float lo, hi;          /* prior box, lo < hi */
} smc_gmm;

/* ------------------------------------------------------------ likelihood */

/* Per-particle mixture log-likelihood (Section 4.1), the sum over the N
 * observations of a log-sum-exp over the K components (Section 2.3: log
 * domain; compensated summation over N):
 *   loglik_out[p] = sum_n log sum_k w_k N(y_n | mu_pk, sigma^2 I_d).
 *   y:     1-D float[N]; diag float[N][d].
 *   theta: 1-D float[K][M]; diag float[M][K][d].
 *   loglik_out: double[M].
 *   grad_out (nullable, 1-D only): float[K][M], d loglik / d mu_k =
 *     sum_n r_nk (y_n - mu_k) / sigma^2 with r the responsibilities.
 * The prior box is not applied here.  Diag with SMC_PREC_BF16SPLIT forms
 * mu.y on the tensor cores from bf16 hi/lo splits of y and mu (products
 * hi.hi + hi.lo + lo.hi, FP32 accumulation; relative error of loglik well
 * below 1e-3) and takes d = 16, 32, 48 or 64 and K <= 32 (other shapes:
 * SMC_ERR_UNSUPPORTED, use SMC_PREC_FP32); it uses context scratch of about
 * N (4 d + 8 bytes) + M K (4 d + 32 bytes).  Errors: SMC_ERR_ARG for
 * M < 0, N < 0, K/d out of range, sigma <= 0, NULL pointers with M, N > 0;
 * M == 0 is a no-op; N == 0 gives loglik 0. */
smc_status smc_loglik_batch(smc_ctx* ctx, const smc_gmm* model, const float* y, int64_t N,
                            const float* theta, int64_t M, double* loglik_out, float* grad_out,
                            void* stream);

/* ------------------------------------------------------------------ weights */

/* Incremental reweighting and normalisation (Section 3: W = w / sum w;
 * Section 4.1.2: incremental weight pi_t(x)/pi_{t-1}(x) = exp(dbeta l(x))
 * under the uniform prior; Section 3.2: effective sample size):
 *   logw[i] += dbeta * loglik[i]   (skipped if loglik == NULL or dbeta == 0)
 *   W_out[i] = exp(logw[i] - max) / S1,  S1 = sum exp(logw - max)
 *   scalars_out (device double[4]) = { log Z increment
 *        = LSE(logw new) - LSE(logw old), ESS = S1^2 / S2, max, LSE(new) }
 *   resample_flag_out (device int32, nullable) = ESS < ess_frac * M.
 * logw is in/out (double[M]); W_out is double[M] (nullable: scalars only).
 * Differences are formed in FP64 and exponentiated in FP32 on the reduced
 * argument; sums are FP64.  A NaN latches SMC_ERR_NONFINITE, an all -inf
 * logw SMC_ERR_ZERO_WEIGHT (then W and the scalars are not written). */
smc_status smc_reweight(smc_ctx* ctx, const double* loglik, double dbeta, double* logw,
                        int64_t M, double* W_out, double* scalars_out,
                        int32_t* resample_flag_out, double ess_frac, void* stream);

/* ESS of unnormalised log-weights, (sum w)^2 / sum w^2 (Section 3.2);
 * ess_out is a device double. */
smc_status smc_ess(smc_ctx* ctx, const double* logw, int64_t M, double* ess_out, void* stream);

/* ---------------------------------------------------------------- resampling */

/* Systematic resampling (Section 3.2: build the empirical CDF of the
 * weights and draw M times from it; the parallel scan of Section 4.2), in
 * exact integer arithmetic so the result does not depend on summation
 * order:  q_j = floor(W_j 2^52), C_j = q_0 + ... + q_j, S = C_{M-1}; slot i
 * takes ancestors_out[i] = min { j : C_j M 2^32 > (i 2^32 + u32) S } with
 * u32 the Philox word (seed, RESAMPLE, step, index 0, block 0, word 0).
 *   W: double[M], each in [0,1] (normalised weights; sum <= 2).
 *   ancestors_out: int32[M], non-decreasing.  counts_out: int32[M] offspring
 *     counts (nullable).
 *   do_flag (device int32, nullable): when it holds 0 nothing is resampled;
 *     ancestors_out becomes the identity and counts 1.
 *   logw_reset (nullable): double[M] set to 0 when resampling happened.
 * Exact integer sums per tile of 2048 weights; one CTA turns them into
 * prefixes and forms the call's constants; then each tile is scanned and
 * its output range expanded.  No CTA waits on another.  A weight outside
 * [0,1] or NaN (or weights summing to 2^9 or more) latches SMC_ERR_ARG,
 * S == 0 SMC_ERR_ZERO_WEIGHT; the outputs are then unspecified. */
smc_status smc_resample_systematic(smc_ctx* ctx, const double* W, int64_t M, uint64_t seed,
                                   uint64_t step, int32_t* ancestors_out, int32_t* counts_out,
                                   const int32_t* do_flag, double* logw_reset, void* stream);

/* smc_reweight followed by smc_resample_systematic on its weights, in one
 * call with one pass fewer: the normalisation pass also forms the exact
 * integer tile sums of the quantised weights, so resampling starts from
 * them instead of reading W back.  Same arguments and the same results,
 * bit for bit, as the two calls
 *   smc_reweight(ctx, loglik, dbeta, logw, M, W_out, scalars_out,
 *                resample_flag_out, ess_frac, stream);
 *   smc_resample_systematic(ctx, W_out, M, seed, step, ancestors_out,
 *                           counts_out, resample_flag_out, logw, stream);
 * (resample_flag_out NULL: resample unconditionally; logw is reset to 0
 * when resampling happened).  W_out and ancestors_out are required. */
smc_status smc_reweight_resample(smc_ctx* ctx, const double* loglik, double dbeta, double* logw,
                                 int64_t M, double* W_out, double* scalars_out,
                                 int32_t* resample_flag_out, double ess_frac, uint64_t seed,
                                 uint64_t step, int32_t* ancestors_out, int32_t* counts_out,
                                 void* stream);

/* Multinomial resampling (Section 3.2's resampling step as M independent
 * draws from the empirical CDF), on the exact-integer CDF of
 * smc_resample_systematic (q_j, C_j, S as there):
 *   ancestors_out[i] = min { j : C_j > floor((2 u_i + 1) S / 2^33) },
 *   u_i = word 0 of (seed, MULTINOMIAL = 6, step, index i),
 * i.e. the particle whose CDF interval contains (u_i + 1/2) / 2^32.  The
 * ancestors are in draw order (not sorted).  W, do_flag, logw_reset and the
 * errors as for smc_resample_systematic; no offspring counts.  Scratch:
 * 8 bytes per particle of context workspace on top of the systematic
 * scheme's (smc_reserve sizes it). */
smc_status smc_resample_multinomial(smc_ctx* ctx, const double* W, int64_t M, uint64_t seed,
                                    uint64_t step, int32_t* ancestors_out,
                                    const int32_t* do_flag, double* logw_reset, void* stream);

/* Residual resampling (the resampling step with each particle's integer
 * share of the M slots kept deterministically), in exact integers on the
 * same q_j, S:
 *   n_j = floor(M q_j / S), r_j = M q_j - n_j S;  particle j fills slots
 *   [N_{j-1}, N_j) (N the inclusive prefix of n), in particle order;
 *   the R = M - sum n slots [M - R, M) are multinomial draws (as
 *   smc_resample_multinomial, uniforms v_k = word 0 of (seed, MULTINOMIAL,
 *   step, index k), k < R) on the remainders rho_j = r_j >> s,
 *   s = max(0, bitlen(S) - 32), whose prefix E and total P replace C and S.
 * Arguments, scratch and errors as smc_resample_multinomial. */
smc_status smc_resample_residual(smc_ctx* ctx, const double* W, int64_t M, uint64_t seed,
                                 uint64_t step, int32_t* ancestors_out, const int32_t* do_flag,
                                 double* logw_reset, void* stream);

/* The same systematic resampling as smc_resample_systematic (identical
 * arguments and results, bit for bit), for callers that cannot allocate
 * device memory: processes whose device memory is owned by a pool or a
 * fixed budget they must not bypass, and latency-critical loops that cannot
 * pay the device synchronisation cudaMalloc / cudaFree imply.  It needs no
 * smc_ctx and allocates nothing: its scratch is a 65 KiB static device
 * array inside libsmc.so, which every GPU that loads the library holds
 * until the process exits.  The paper has no counterpart to this entry
 * point; it exists for how the library is called, not for the method.
 *   M must be <= 16,777,216 (2^24); larger M returns SMC_ERR_ARG.
 *   status_out (device uint32, nullable) receives the error bits a kernel
 *   finds, OR-ed in: 8 = a weight outside [0,1] or NaN (or weights far
 *   from normalised), 2 = all weights zero.
 *   The first call on a device (with that device current) looks up the
 *   array's device address; make that first call before any stream capture.
 *   Every call shares the one array.  Nothing in it needs clearing between
 *   calls (each call's first pass overwrites every tile sum it uses, and
 *   its constants are formed anew), but calls whose work overlaps on the
 *   GPU (different streams, or several host threads on one device) race
 *   and give wrong results: serialise them, e.g. on one stream. */
smc_status smc_resample_systematic_noalloc(const double* W, int64_t M, uint64_t seed,
                                           uint64_t step, int32_t* ancestors_out,
                                           int32_t* counts_out, const int32_t* do_flag,
                                           double* logw_reset, uint32_t* status_out,
                                           void* stream);

/* Gather particles by ancestor: for r < rows_f32, dst_f32[r*M + i] =
 * src_f32[r*M + anc[i]] (SoA float[rows][M]); and dst_f64[i] =
 * src_f64[anc[i]] if both are non-NULL.  anc NULL means identity (copy).
 * Source and destination must not overlap. */
smc_status smc_gather(smc_ctx* ctx, const int32_t* anc, int64_t M, int32_t rows_f32,
                      const float* src_f32, float* dst_f32, const double* src_f64,
                      double* dst_f64, void* stream);

/* ---------------------------------------------------------------------- moves */

enum { SMC_MOVE_RW = 0, SMC_MOVE_MALA = 1 };

/* One Metropolis-Hastings move per particle on the tempered target
 * prior(mu) L(mu)^beta (Sections 4.1.1-4.1.2), 1-D mixture only.
 *   Slot p starts from particle src = anc[p] (anc NULL, or *do_flag == 0
 *   when do_flag is given: src = p) -- the gather after resampling fused
 *   into the move.
 *   RW:   mu' = mu + scale z, z ~ N(0, I_K) (purpose MOVE, index p).
 *   MALA: mu' = mu + (h^2/2) beta grad l(mu) + h z with h = scale, and the
 *         log proposal-density ratio added to log alpha.  grad_in / grad_out
 *         are float[K][M] (the gradient at the state; required for MALA).
 *   A proposal outside the prior box is rejected without evaluating l.
 *   Accept iff log u < log alpha, u from purpose ACCEPT word 0 (FP64 test).
 *   beta: device float, beta[p * beta_stride] (stride 0: one temperature).
 *   theta_in/loglik_in/grad_in and theta_out/loglik_out/grad_out must not
 *   overlap when anc is non-NULL; with anc NULL they may be identical.
 *   accept_count (device uint32, nullable) is incremented by the number of
 *   accepted moves. */
smc_status smc_mh_move(smc_ctx* ctx, const smc_gmm* model, const float* y, int64_t N,
                       const float* theta_in, const double* loglik_in, const float* grad_in,
                       const int32_t* anc, const int32_t* do_flag,
                       float* theta_out, double* loglik_out, float* grad_out, int64_t M,
                       const float* beta, int64_t beta_stride, float scale, int32_t kind,
                       uint64_t seed, uint64_t step, uint32_t* accept_count, void* stream);

/* One sweep of population MCMC over many independent populations in one
 * persistent launch (Section 3.1; Section 4.1.1).  Population q owns chains
 * pop_offsets[q] .. pop_offsets[q+1]-1 of theta (float[K][M_total]) and
 * loglik (double[M_total]), updated in place; beta is float[M_total].
 * Stage 1: a random-walk MH move for every chain (as smc_mh_move with
 *   particle index = chain index, step = sweep).
 * Stage 2: exchange moves between adjacent chains of each population, on
 *   the pair set {0,1},{2,3},... (parity bit 0) or {1,2},{3,4},...,{M_q-1,0}
 *   (parity bit 1, the wrap pair only when M_q is even); the bit is
 *   word 0 bit 0 of (seed, EXCHANGE, sweep, index q); pair j swaps iff
 *   log u_j < (beta_a - beta_b)(l_b - l_a), u_j from word 4 + j.
 * The CTAs take equal chunks of chains (dealt round-robin); a population's
 * exchange runs as soon as its last chain has moved, so populations of any
 * size mix freely.  When the average population holds more than two chains
 * per thread of a CTA (M_total > 2 * n_pops * threads, e.g. the single
 * population of Table 1), stage 2 runs instead as a second, grid-wide
 * launch over all pairs, with the same pairs, draws and result.
 * pop_offsets must be non-decreasing with
 * pop_offsets[0] = 0 and pop_offsets[n_pops] = M_total (device data: the
 * library does not read them on the host, so it cannot check them; other
 * values make the launch access chains outside [0, M_total)).
 * stats (device uint64[3], nullable) accumulates {MH accepts, swaps
 *   accepted, swaps attempted}.  Uses n_pops counters of context scratch
 *   (smc_reserve's max_pops sizes them before graph capture).
 * For 512 <= N <= 4096 and K <= 16 the data are sorted into bins once per
 *   data set (a small extra launch when y, N or sigma differ from the
 *   context's previous call, recorded like any launch while capturing) and
 *   the layout is kept in the context; every sweep compares y with the
 *   layout's copy of the data and sorts them itself when they differ, so y
 *   may be overwritten between calls. */
smc_status smc_popmcmc_sweep(smc_ctx* ctx, const smc_gmm* model, const float* y, int64_t N,
                             float* theta, double* loglik, int64_t M_total, const float* beta,
                             const int32_t* pop_offsets, int32_t n_pops, float scale,
                             uint64_t seed, uint64_t sweep, uint64_t* stats, void* stream);

/* ------------------------------------------------------------ importance sampling */

/* Target and proposal of an importance-sampling estimate (Section 2.1's
 * worked example: target 1/2 N(-1, 0.25) + 1/2 N(1.5, 0.25), proposal
 * N(0, 1), test function x^2, expectation 1.875).  Passed by host pointer. */
typedef struct smc_is_problem {
    int32_t K;             /* target components, 1..8 */
    float mu[8];           /* component means */
    float a[8];            /* component weights, > 0 (normalised target: sum 1) */
    float var;             /* common component variance, > 0 */
    float prop_mean;       /* proposal N(prop_mean, prop_sd^2) */
    float prop_sd;         /* > 0 */
    int32_t power;         /* test function phi(x) = x^power, 0..8 */
} smc_is_problem;

/* Importance-sampling sums over N proposal draws (Section 2.1; Section 3:
 * w = target density / proposal density):
 *   out[0] = sum w_i,  out[1] = sum w_i phi(x_i),  out[2] = sum w_i^2
 *   (out: device double[3]).  The plain estimate is out[1] / N, the
 *   self-normalised one out[1] / out[0], the ESS out[0]^2 / out[2].
 *   x: device float[N] draws from the proposal, or NULL to draw
 *      x_i = prop_mean + prop_sd z_i on the device, z_i = normal 0 of
 *      (seed, PROPOSAL = 7, step, index i).
 * Per draw in FP32 (w = exp2 of the log2 ratio; overflows for draws where
 * the target exceeds the proposal by more than 2^128), groups of 8 draws
 * summed in FP32, group sums in FP64 in a fixed order: the same bits on
 * every run.  N = 0 writes zeros.  Uses the context's reduction scratch. */
smc_status smc_is_moments(smc_ctx* ctx, const smc_is_problem* prob, const float* x, int64_t N,
                          uint64_t seed, uint64_t step, double* out, void* stream);

/* ------------------------------------------------------------ particle filter */

enum { SMC_PF_MSV = 0, SMC_PF_LG = 1, SMC_PF_FSV = 2 };

/* State-space model for pf_step, passed by value through a host pointer. */
typedef struct smc_pf_model {
    int32_t kind;          /* SMC_PF_MSV, SMC_PF_LG or SMC_PF_FSV */
    int32_t d;             /* state dimension: 1..8 (FSV: factors K, 1..4) */
    float phi[8];          /* x_t = phi (.) x_{t-1} + L z */
    float chol[64];        /* row-major lower Cholesky factor L of Sigma (d x d) */
    float beta;            /* observation scale (MSV, LG) */
    /* factor stochastic volatility only (Section 4.2): */
    int32_t m;             /* observed series, 1..8 */
    float B[64];           /* row-major m x d factor loadings */
    float psi[8];          /* idiosyncratic variances, > 0 */
} smc_pf_model;

/* One bootstrap particle-filter step (Section 3.2; the model of Section 4.2
 * with multivariate stochastic volatility):
 *   x_out[:, i] = phi (.) x_in[:, anc[i]] + L z_i, z_i ~ N(0, I_d)
 *                 (purpose PFNOISE, index i, step t); anc NULL = identity.
 *   logg_out[i] = log g(y_t | x_out[:, i]):
 *     MSV: sum_j [ -1/2 log(2 pi beta^2) - x_j/2 - y_j^2 exp(-x_j) / (2 beta^2) ]
 *     LG:  sum_j [ -1/2 log(2 pi beta^2) - (y_j - x_j)^2 / (2 beta^2) ]
 *     FSV: log N(y_t; 0, B diag(exp x) B^T + diag(psi)), evaluated through the
 *          Woodbury identity and the matrix determinant lemma (a d x d
 *          Cholesky factor per particle instead of an m x m one).
 *   y_t: device float[d] (FSV: float[m]);  x_in, x_out: float[d][M] (must not overlap);
 *   logg_out: double[M].  Feed logg_out to smc_reweight (dbeta = 1) and
 *   the weights to smc_resample_systematic for the next step's anc. */
smc_status pf_step(smc_ctx* ctx, const smc_pf_model* model, const float* y_t,
                   const float* x_in, const int32_t* anc, float* x_out, double* logg_out,
                   int64_t M, uint64_t seed, uint64_t t, void* stream);

/* One whole bootstrap-filter step (Section 3.2) in one call: pf_step,
 * smc_reweight with dbeta = 1 on its log g, and systematic resampling of
 * the new weights with the normalisation forming the resampling's tile
 * sums (as smc_reweight_resample) -- the kernels of those calls, launched
 * back to back, so every output equals theirs bit for bit:
 *   x_out, logg_out (double[M], required: log g passes through it): as
 *     pf_step, from x_in gathered through anc;
 *   logw[i] += log g_i; W_out, scalars_out, resample_flag_out, ess_frac:
 *     as smc_reweight (resample_flag_out NULL: resample unconditionally);
 *   anc (in/out, int32[M]): read as this step's ancestors, then overwritten
 *     with the ancestors drawn from W_out (uniform word of (seed, RESAMPLE,
 *     t)), or the identity when the flag says no resampling; logw is reset
 *     to 0 when resampling happened; counts_out (nullable): offspring.
 * Errors as pf_step, smc_reweight and smc_resample_systematic; M at most
 * 2^31 - 1. */
smc_status smc_pf_filter_step(smc_ctx* ctx, const smc_pf_model* model, const float* y_t,
                              const float* x_in, int32_t* anc, float* x_out, double* logg_out,
                              double* logw, int64_t M, double* W_out, double* scalars_out,
                              int32_t* resample_flag_out, double ess_frac, uint64_t seed,
                              uint64_t t, int32_t* counts_out, void* stream);

/* ------------------------------------------------------------------- streams */

/* MRG32k3a (L'Ecuyer 1999), the generator Section 2.5 parallelises: thread
 * t of n_threads computes the contiguous block of per_thread numbers that
 * starts at position offset + t * per_thread (mod 2^64) of the one stream
 * that starts at `seed`, reaching it by skip-ahead in O(log n) matrix-vector
 * products mod m (the context holds A^(2^k), k < 64).
 *   x_n = (1403580 x_{n-2} - 810728 x_{n-3}) mod m1,  m1 = 4294967087
 *   y_n = (527612 y_{n-1} - 1370589 y_{n-3}) mod m2,  m2 = 4294944443
 *   z_n = (x_n - y_n) mod m1, taken in [1, m1] (m1 in place of 0);
 *   out_f64 (nullable): u_n = z_n / (m1 + 1), the generator's output, as
 *     (double) z_n * (1 / (m1 + 1));
 *   out_f32 (nullable): u_n = (2 floor(z_n / 2^9) + 1) / 2^24, the same
 *     number cut to the 24 bits a float holds, strictly inside (0, 1).
 *   At least one of the outputs is given.
 *   seed: host uint32[6] = (x_0, x_1, x_2 | y_0, y_1, y_2), oldest first;
 *     x-part < m1, y-part < m2, neither part all zero (else SMC_ERR_ARG).
 *     Position 0 is the first number after the seed state.
 *   Layout of each output [per_thread][n_threads]:
 *     out[j * n_threads + t] = u_{offset + t * per_thread + j}
 *     (slot-major: consecutive threads write consecutive addresses).
 * The SMC / MCMC kernels themselves draw from Philox; this stream serves
 * callers that want the paper's generator. */
smc_status smc_rng_mrg32k3a(smc_ctx* ctx, const uint32_t seed[6], uint64_t offset,
                            int64_t n_threads, int64_t per_thread, float* out_f32,
                            double* out_f64, void* stream);

/* Raw Philox words: out[(i*n_block + b)*4 + w] = word w of
 * (seed, purpose, step, index i, block b), i < n_index, b < n_block. */
smc_status smc_rng_words(smc_ctx* ctx, uint64_t seed, uint32_t purpose, uint64_t step,
                         uint32_t n_index, uint32_t n_block, uint32_t* out, void* stream);

/* Box-Muller normals as the moves draw them: out[i*n + j] = normal j of
 * (seed, purpose, step, index i), float. */
smc_status smc_rng_normals(smc_ctx* ctx, uint64_t seed, uint32_t purpose, uint64_t step,
                           uint32_t n_index, uint32_t n, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SMC_GB300_H */
