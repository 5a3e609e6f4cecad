/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the SMC / population-MCMC
 * hot path of Lee, Yau, Giles, Doucet & Holmes (2009), "On the utility of
 * graphics cards to perform massively parallel simulation of advanced Monte
 * Carlo methods".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; it is written one
 * particle at a time with straight loops so that every function can be read
 * against the paper by eye.  Nothing here is blocked, fused or reordered
 * beyond what the definition states.
 *
 * Precision: every arithmetic step is IEEE double (compiled without
 * -ffast-math).  State arrays that the method stores in single precision
 * (particle positions theta, particle-filter states x, the data y) are taken
 * as float inputs and, where the method writes such a state, the new value is
 * rounded to float exactly as the storage type demands; all arithmetic on
 * them is FP64.
 *
 * Random numbers: the method's draws come from Philox4x32-10 (Salmon, Moraes,
 * Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), written
 * here from its published definition.  Counter layout (identical on the GPU,
 * implemented there independently):
 *     key     = (seed mod 2^32, seed div 2^32)
 *     counter = (index, block, step mod 2^32, purpose | (step div 2^32) << 8)
 * "index" is the particle / chain / population / output slot, "block" picks
 * which group of four 32-bit words, "purpose" separates the streams.
 *
 * Parity status of each function is recorded in its header comment; every
 * function below is pinned by a CPU test against something other than itself
 * (brute force, closed forms, Kalman filter, an independent Philox,
 * invariants).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_PI 3.14159265358979323846

/* stream purposes (the same numbers on the GPU side) */
enum { ORC_P_MOVE = 1, ORC_P_ACCEPT = 2, ORC_P_RESAMPLE = 3,
       ORC_P_EXCHANGE = 4, ORC_P_PFNOISE = 5, ORC_P_MULTINOMIAL = 6, ORC_P_PROPOSAL = 7 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): ten rounds of the 4x32 S-box          */
/* with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments           */
/* 0x9E3779B9 (golden ratio), 0xBB67AE85 (sqrt(3)-1).                        */
/* Replaces the MRG32k3a / xorshift skip-ahead streams of Section 2.5.       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_draw_words(uint64_t seed, uint32_t purpose, uint64_t step,
                    uint32_t index, uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { index, block, (uint32_t)step,
                        (purpose & 0xFFu) | ((uint32_t)(step >> 32) << 8) };
    orc_philox4x32_10(ctr, key, out);
}

/* word -> uniform on the open interval (0,1): the top 23 bits k give
 * (2k+1) / 2^24, which has at most 24 significant bits and is therefore the
 * same number in float and double. */
double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* word w of the stream (seed, purpose, step, index): block w/4, lane w%4 */
static uint32_t orc_word(uint64_t seed, uint32_t purpose, uint64_t step,
                         uint32_t index, uint32_t w)
{
    uint32_t out[4];
    orc_draw_words(seed, purpose, step, index, w >> 2, out);
    return out[w & 3u];
}

/* n standard normals by Box-Muller on consecutive word pairs
 * (words 2p, 2p+1 -> normals 2p, 2p+1):  r = sqrt(-2 ln u1),
 * z_{2p} = r cos(2 pi u2), z_{2p+1} = r sin(2 pi u2).  Section 2.5 says
 * uniforms are "transformed to match various different output
 * distributions"; Box-Muller is that transform here. */
void orc_normals(uint64_t seed, uint32_t purpose, uint64_t step, uint32_t index,
                 int n, double* z)
{
    for (int p = 0; 2 * p < n; ++p) {
        double u1 = orc_u01(orc_word(seed, purpose, step, index, (uint32_t)(2 * p)));
        double u2 = orc_u01(orc_word(seed, purpose, step, index, (uint32_t)(2 * p + 1)));
        double r = sqrt(-2.0 * log(u1));
        z[2 * p] = r * cos(2.0 * ORC_PI * u2);
        if (2 * p + 1 < n) z[2 * p + 1] = r * sin(2.0 * ORC_PI * u2);
    }
}

/* ------------------------------------------------------------------------ */
/* Univariate Gaussian mixture likelihood, Section 4.1:                      */
/*   p(y_j | mu) = sum_i w_i f(y_j | mu_i, sigma),  density of y = prod_j.    */
/* The log of the product is the sum over data of a log-sum-exp over         */
/* components, shifted by the largest term (Section 2.3: work with log-      */
/* likelihoods because of the limited range of floating point).              */
/* ------------------------------------------------------------------------ */
double orc_gmm1d_loglik_one(const float* y, int64_t N, int K, const double* logw,
                            double sigma, const double* mu)
{
    double c = -0.5 * log(2.0 * ORC_PI * sigma * sigma);
    double total = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        double a[64];
        double m = -INFINITY;
        for (int k = 0; k < K; ++k) {
            double d = (double)y[n] - mu[k];
            a[k] = logw[k] + c - d * d / (2.0 * sigma * sigma);
            if (a[k] > m) m = a[k];
        }
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += exp(a[k] - m);
        total += m + log(s);
    }
    return total;
}

/* the same at FP64 means (finite-difference checks of the gradient) */
double orc_gmm1d_loglik_at(const float* y, int64_t N, int K, const double* logw,
                           double sigma, const double* mu)
{
    return orc_gmm1d_loglik_one(y, N, K, logw, sigma, mu);
}

/* theta is SoA: theta[k*M + p] is mu_k of particle p. */
void orc_gmm1d_loglik(const float* y, int64_t N, int K, const double* logw, double sigma,
                      const float* theta, int64_t M, double* out)
{
    double mu[64];
    for (int64_t p = 0; p < M; ++p) {
        for (int k = 0; k < K; ++k) mu[k] = (double)theta[(int64_t)k * M + p];
        out[p] = orc_gmm1d_loglik_one(y, N, K, logw, sigma, mu);
    }
}

/* Gradient of the same log-likelihood with respect to the means:
 *   d l / d mu_k = sum_n r_nk (y_n - mu_k) / sigma^2,
 *   r_nk = w_k f(y_n|mu_k) / sum_i w_i f(y_n|mu_i)   (responsibilities).
 * Differentiating the mixture density of Section 4.1 term by term. */
static void orc_gmm1d_grad_one(const float* y, int64_t N, int K, const double* logw,
                               double sigma, const double* mu, double* g)
{
    double s2 = sigma * sigma;
    for (int k = 0; k < K; ++k) g[k] = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        double a[64];
        double m = -INFINITY;
        for (int k = 0; k < K; ++k) {
            double d = (double)y[n] - mu[k];
            a[k] = logw[k] - d * d / (2.0 * s2);
            if (a[k] > m) m = a[k];
        }
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += exp(a[k] - m);
        for (int k = 0; k < K; ++k) {
            double r = exp(a[k] - m) / s;
            g[k] += r * ((double)y[n] - mu[k]) / s2;
        }
    }
}

void orc_gmm1d_grad(const float* y, int64_t N, int K, const double* logw, double sigma,
                    const float* theta, int64_t M, double* grad /* [K][M] */)
{
    double mu[64], g[64];
    for (int64_t p = 0; p < M; ++p) {
        for (int k = 0; k < K; ++k) mu[k] = (double)theta[(int64_t)k * M + p];
        orc_gmm1d_grad_one(y, N, K, logw, sigma, mu, g);
        for (int k = 0; k < K; ++k) grad[(int64_t)k * M + p] = g[k];
    }
}

/* gradient at FP64 means (used by the MALA move on the proposed point) */
void orc_gmm1d_grad_at(const float* y, int64_t N, int K, const double* logw, double sigma,
                       const double* mu, double* g)
{
    orc_gmm1d_grad_one(y, N, K, logw, sigma, mu, g);
}

/* ------------------------------------------------------------------------ */
/* Diagonal multivariate Gaussian mixture: the Section 4.1 likelihood with    */
/* N(y_n | mu_k, sigma^2 I_d) components; the squared distance is summed     */
/* over dimensions directly (no expansion of the quadratic form).            */
/* Y is [N][d]; theta is [M][K][d].                                          */
/* ------------------------------------------------------------------------ */
void orc_gmmdiag_loglik(const float* Y, int64_t N, int d, int K, const double* logw,
                        double sigma, const float* theta, int64_t M, double* out)
{
    double c = -0.5 * (double)d * log(2.0 * ORC_PI * sigma * sigma);
    for (int64_t p = 0; p < M; ++p) {
        const float* mu = theta + (int64_t)p * K * d;
        double total = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            const float* yn = Y + n * d;
            double a[64];
            double m = -INFINITY;
            for (int k = 0; k < K; ++k) {
                double q = 0.0;
                for (int j = 0; j < d; ++j) {
                    double e = (double)yn[j] - (double)mu[k * d + j];
                    q += e * e;
                }
                a[k] = logw[k] + c - q / (2.0 * sigma * sigma);
                if (a[k] > m) m = a[k];
            }
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += exp(a[k] - m);
            total += m + log(s);
        }
        out[p] = total;
    }
}

/* ------------------------------------------------------------------------ */
/* Importance weights and their normalisation (Section 3, W = w / sum w),    */
/* the SMC-sampler incremental weight pi_t(x)/pi_{t-1}(x) =                  */
/* exp((beta_t - beta_{t-1}) l(x)) under the uniform prior (Section 4.1.2),  */
/* and the effective sample size (Section 3.2, Liu & Chen).                  */
/*   lw_new = lw_old + dbeta * l           (no increment if loglik == NULL)  */
/*   W_i    = exp(lw_new_i - m) / S1,  S1 = sum exp(lw_new - m),             */
/*   ESS    = S1^2 / S2,               S2 = sum exp(2 (lw_new - m)),          */
/*   log Z increment = LSE(lw_new) - LSE(lw_old).                            */
/* scalars = {log Z increment, ESS, max lw_new, LSE(lw_new)}.                */
/* Returns 0, or -4 if every weight is zero, -3 if a value is NaN.           */
/* ------------------------------------------------------------------------ */
int orc_reweight(const double* loglik, double dbeta, double* lw, int64_t M,
                 double* W, double* scalars)
{
    double m_old = -INFINITY;
    for (int64_t i = 0; i < M; ++i) {
        if (isnan(lw[i])) return -3;
        if (lw[i] > m_old) m_old = lw[i];
    }
    double s_old = 0.0;
    for (int64_t i = 0; i < M; ++i) s_old += exp(lw[i] - m_old);
    double lse_old = m_old + log(s_old);

    for (int64_t i = 0; i < M; ++i) {
        if (loglik != NULL && dbeta != 0.0) {
            if (isnan(loglik[i])) return -3;
            lw[i] = lw[i] + dbeta * loglik[i];
        }
    }
    double m = -INFINITY;
    for (int64_t i = 0; i < M; ++i) {
        if (isnan(lw[i])) return -3;
        if (lw[i] > m) m = lw[i];
    }
    if (m == -INFINITY) return -4;
    double S1 = 0.0, S2 = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        double e = exp(lw[i] - m);
        S1 += e;
        S2 += e * e;
    }
    for (int64_t i = 0; i < M; ++i) W[i] = exp(lw[i] - m) / S1;
    scalars[0] = (m + log(S1)) - lse_old;
    scalars[1] = S1 * S1 / S2;
    scalars[2] = m;
    scalars[3] = m + log(S1);
    return 0;
}

/* ESS of unnormalised log-weights: (sum w)^2 / sum w^2. */
double orc_ess(const double* lw, int64_t M)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < M; ++i) if (lw[i] > m) m = lw[i];
    double S1 = 0.0, S2 = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        double e = exp(lw[i] - m);
        S1 += e;
        S2 += e * e;
    }
    return S1 * S1 / S2;
}

/* ------------------------------------------------------------------------ */
/* Systematic resampling (Section 3.2: build the empirical CDF of the        */
/* weights and sample from it N times), in exact integers so that the        */
/* result is independent of summation order:                                 */
/*   q_i = floor(W_i 2^52),  C_j = q_0 + ... + q_j,  S = C_{M-1},            */
/*   slot i takes a_i = min { j : C_j * M * 2^32 > (i * 2^32 + u32) * S },   */
/* i.e. the j whose CDF interval contains (i + u)/M with u = u32 / 2^32.     */
/* Sequential two-pointer merge over slots and particles.                    */
/* Returns 0, -1 if a weight is outside [0,1] or NaN, -4 if S == 0,          */
/* -1 if S does not fit in 64 bits.                                          */
/* ------------------------------------------------------------------------ */
int orc_resample_systematic(const double* W, int64_t M, uint32_t u32,
                            int32_t* anc, int32_t* counts)
{
    typedef unsigned __int128 u128;
    uint64_t* C = (uint64_t*)malloc((size_t)M * sizeof(uint64_t));
    if (!C) return -2;
    u128 acc = 0;
    for (int64_t j = 0; j < M; ++j) {
        double w = W[j];
        if (!(w >= 0.0 && w <= 1.0)) { free(C); return -1; }
        uint64_t q = (uint64_t)floor(w * 4503599627370496.0); /* 2^52 */
        acc += q;
        if (acc >> 64) { free(C); return -1; }
        C[j] = (uint64_t)acc;
    }
    uint64_t S = (uint64_t)acc;
    if (S == 0) { free(C); return -4; }
    if (counts) for (int64_t j = 0; j < M; ++j) counts[j] = 0;
    int64_t j = 0;
    u128 scaleM = (u128)M << 32;
    for (int64_t i = 0; i < M; ++i) {
        u128 T = ((((u128)(uint64_t)i) << 32) + (u128)u32) * (u128)S;
        while (!((u128)C[j] * scaleM > T)) ++j;
        anc[i] = (int32_t)j;
        if (counts) counts[j] += 1;
    }
    free(C);
    return 0;
}

/* word 0 of block 0 of the streams (seed, purpose, step, index i) for     */
/* i = 0..n-1: the per-slot uniforms of multinomial and residual draws.     */
void orc_word_array(uint64_t seed, uint32_t purpose, uint64_t step, int64_t n, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_word(seed, purpose, step, (uint32_t)i, 0);
}

/* First j in [0, n) with C[j] > T (C non-decreasing; n if none). */
static int64_t orc_first_above(const uint64_t* C, int64_t n, uint64_t T)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (C[mid] > T) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* q_j = floor(W_j 2^52) and C_j = q_0 + ... + q_j (exact); 0, -1 (a weight
 * outside [0,1], NaN, or a total beyond 64 bits) or -4 (all zero). */
static int orc_quantised_cdf(const double* W, int64_t M, uint64_t* q, uint64_t* C,
                             uint64_t* S_out)
{
    unsigned __int128 acc = 0;
    for (int64_t j = 0; j < M; ++j) {
        double w = W[j];
        if (!(w >= 0.0 && w <= 1.0)) return -1;
        q[j] = (uint64_t)floor(w * 4503599627370496.0); /* 2^52 */
        acc += q[j];
        if (acc >> 64) return -1;
        C[j] = (uint64_t)acc;
    }
    if (acc == 0) return -4;
    *S_out = (uint64_t)acc;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Multinomial resampling (Section 3.2: M independent draws from the         */
/* empirical CDF of the weights), on the same exact-integer CDF as the       */
/* systematic scheme: slot i takes                                           */
/*   a_i = min { j : C_j > floor((2 u_i + 1) S / 2^33) },                   */
/* the j whose CDF interval (C_{j-1}/S, C_j/S] contains (u_i + 1/2) / 2^32.  */
/* u[i] is the slot's 32-bit uniform (the GPU draws word 0 of (seed,         */
/* MULTINOMIAL, step, index i)).  Returns as orc_resample_systematic.        */
/* ------------------------------------------------------------------------ */
int orc_resample_multinomial(const double* W, int64_t M, const uint32_t* u, int32_t* anc)
{
    uint64_t* q = (uint64_t*)malloc((size_t)M * sizeof(uint64_t));
    uint64_t* C = (uint64_t*)malloc((size_t)M * sizeof(uint64_t));
    uint64_t S = 0;
    int rc = (q && C) ? orc_quantised_cdf(W, M, q, C, &S) : -2;
    if (rc == 0) {
        for (int64_t i = 0; i < M; ++i) {
            unsigned __int128 x = (unsigned __int128)(2ull * u[i] + 1ull) * S;
            anc[i] = (int32_t)orc_first_above(C, M, (uint64_t)(x >> 33));
        }
    }
    free(q);
    free(C);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Residual resampling (a variant of the Section 3.2 resampling step): each  */
/* particle first receives its integer share of the M slots, the rest are    */
/* multinomial draws on the remainders, all in exact integers:               */
/*   n_j = floor(M q_j / S),  r_j = M q_j - n_j S  (0 <= r_j < S),           */
/*   slots [N_{j-1}, N_j) take j (N the prefix of n), in particle order;     */
/*   R = M - sum n residual slots [M - R, M) are multinomial draws on the    */
/*   remainders shifted to 32 bits: rho_j = r_j >> s with                    */
/*   s = max(0, bitlen(S) - 32), E_j = rho_0 + ... + rho_j, P = E_{M-1};     */
/*   residual slot k takes min { j : E_j > floor((2 v_k + 1) P / 2^33) }.    */
/* v[k] (k < R) as u in the multinomial scheme.  R_out (nullable) = R.       */
/* ------------------------------------------------------------------------ */
int orc_resample_residual(const double* W, int64_t M, const uint32_t* v, int32_t* anc,
                          int64_t* R_out)
{
    uint64_t* q = (uint64_t*)malloc((size_t)M * sizeof(uint64_t));
    uint64_t* C = (uint64_t*)malloc((size_t)M * sizeof(uint64_t));
    uint64_t S = 0;
    int rc = (q && C) ? orc_quantised_cdf(W, M, q, C, &S) : -2;
    if (rc == 0) {
        int bits = 64 - __builtin_clzll(S);
        int sh = bits > 32 ? bits - 32 : 0;
        int64_t pos = 0;
        uint64_t P = 0;
        for (int64_t j = 0; j < M; ++j) {
            unsigned __int128 mq = (unsigned __int128)M * q[j];
            uint64_t n = (uint64_t)(mq / S);
            uint64_t r = (uint64_t)(mq - (unsigned __int128)n * S);
            for (uint64_t k = 0; k < n; ++k) anc[pos++] = (int32_t)j;
            P += r >> sh;
            C[j] = P; /* reused: E_j */
        }
        int64_t R = M - pos;
        for (int64_t k = 0; k < R; ++k) {
            unsigned __int128 x = (unsigned __int128)(2ull * v[k] + 1ull) * P;
            anc[pos + k] = (int32_t)orc_first_above(C, M, (uint64_t)(x >> 33));
        }
        if (R_out) *R_out = R;
    }
    free(q);
    free(C);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* MRG32k3a (L'Ecuyer 1999), the generator Section 2.5 parallelises by       */
/* skip-ahead.  Two components of order 3:                                   */
/*   x_n = (1403580 x_{n-2} - 810728 x_{n-3}) mod (2^32 - 209)               */
/*   y_n = (527612 y_{n-1} - 1370589 y_{n-3}) mod (2^32 - 22853)             */
/*   u_n = z_n / (m1 + 1), z_n = (x_n - y_n) mod m1 (m1 in place of 0).      */
/* Writes n numbers starting at position `start` (position 0 = the first     */
/* number after the seed state): out64 = z / (m1 + 1) as (double) z times   */
/* 1 / (m1 + 1); out32 = (2 floor(z / 2^9) + 1) / 2^24 (24 bits, inside     */
/* (0, 1)); either may be NULL.  The state                                   */
/* reaches `start` by multiplying with the one-step matrices raised to the   */
/* power start, by repeated squaring (O(log start) products).                */
/* ------------------------------------------------------------------------ */
static void orc_mat3_mul(const uint64_t* A, const uint64_t* B, uint64_t m, uint64_t* C)
{
    uint64_t r[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            unsigned __int128 acc = 0;
            for (int l = 0; l < 3; ++l) acc += (unsigned __int128)A[3 * i + l] * B[3 * l + j];
            r[3 * i + j] = (uint64_t)(acc % m);
        }
    memcpy(C, r, sizeof(r));
}

void orc_mrg32k3a(const uint32_t seed[6], uint64_t start, int64_t n, float* out32,
                  double* out64)
{
    const uint64_t m1 = 4294967087ull, m2 = 4294944443ull;
    uint64_t A1[9] = {0, 1, 0, 0, 0, 1, m1 - 810728ull, 1403580ull, 0};
    uint64_t A2[9] = {0, 1, 0, 0, 0, 1, m2 - 1370589ull, 0, 527612ull};
    uint64_t P1[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, P2[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (uint64_t e = start; e; e >>= 1) {   /* P = A^start */
        if (e & 1ull) {
            orc_mat3_mul(P1, A1, m1, P1);
            orc_mat3_mul(P2, A2, m2, P2);
        }
        orc_mat3_mul(A1, A1, m1, A1);
        orc_mat3_mul(A2, A2, m2, A2);
    }
    int64_t x[3], y[3];
    for (int i = 0; i < 3; ++i) {
        unsigned __int128 ax = 0, ay = 0;
        for (int k = 0; k < 3; ++k) {
            ax += (unsigned __int128)P1[3 * i + k] * seed[k];
            ay += (unsigned __int128)P2[3 * i + k] * seed[3 + k];
        }
        x[i] = (int64_t)(ax % m1);
        y[i] = (int64_t)(ay % m2);
    }
    for (int64_t j = 0; j < n; ++j) {
        int64_t p1 = (1403580LL * x[1] - 810728LL * x[0]) % (int64_t)m1;
        if (p1 < 0) p1 += (int64_t)m1;
        x[0] = x[1]; x[1] = x[2]; x[2] = p1;
        int64_t p2 = (527612LL * y[2] - 1370589LL * y[0]) % (int64_t)m2;
        if (p2 < 0) p2 += (int64_t)m2;
        y[0] = y[1]; y[1] = y[2]; y[2] = p2;
        int64_t z = (p1 - p2) % (int64_t)m1;
        if (z <= 0) z += (int64_t)m1;
        if (out32) out32[j] = (float)((2.0 * (double)(z >> 9) + 1.0) / 16777216.0);
        if (out64) out64[j] = (double)z * 2.328306549295727688e-10;
    }
}

/* ------------------------------------------------------------------------ */
/* Importance sampling (Section 2.1 and its worked example; Section 3:       */
/* weights are target over proposal).  Target: sum_k a_k N(mu_k, var);      */
/* proposal: N(pm, ps^2); test function phi(x) = x^power.  For each draw     */
/*   w_i = p(x_i) / q(x_i)                                                   */
/* and out = { sum w_i, sum w_i phi(x_i), sum w_i^2 }.  x == NULL draws      */
/* x_i = float(pm + ps z_i), z_i = normal 0 of (seed, PROPOSAL, step, i).    */
/* ------------------------------------------------------------------------ */
void orc_is_moments(int K, const double* mu, const double* a, double var, double pm, double ps,
                    int power, const float* x, int64_t N, uint64_t seed, uint64_t step,
                    double* out)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double xi;
        if (x) {
            xi = (double)x[i];
        } else {
            double z;
            orc_normals(seed, ORC_P_PROPOSAL, step, (uint32_t)i, 1, &z);
            xi = (double)(float)(pm + ps * z);
        }
        double p = 0.0;
        for (int k = 0; k < K; ++k) {
            double d = xi - mu[k];
            p += a[k] * exp(-d * d / (2.0 * var)) / sqrt(2.0 * ORC_PI * var);
        }
        double dq = (xi - pm) / ps;
        double q = exp(-0.5 * dq * dq) / (ps * sqrt(2.0 * ORC_PI));
        double w = p / q;
        double phi = 1.0;
        for (int e = 0; e < power; ++e) phi *= xi;
        s0 += w;
        s1 += w * phi;
        s2 += w * w;
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
}

/* ------------------------------------------------------------------------ */
/* Random-walk Metropolis-Hastings move on the tempered target              */
/* pi_beta(mu) ~ prior(mu) L(mu)^beta, uniform prior on [lo,hi]^K            */
/* (Sections 4.1.1-4.1.2: N(0, I_k) random walk, here scaled by s).          */
/*   mu' = mu + s z,  z ~ N(0, I_K) (purpose MOVE, index p, step)            */
/*   reject if mu' leaves the box; otherwise accept iff                      */
/*   log u < beta (l(mu') - l(mu)),  u from purpose ACCEPT word 0.           */
/* The proposal is stored as float (the state's storage type) and the        */
/* likelihood is evaluated at that stored value.                             */
/* beta[p * beta_stride]; anc (nullable) gathers the input particle first.   */
/* Outputs: theta_out, loglik_out, accepted[p] in {0,1}.                     */
/* ------------------------------------------------------------------------ */
static int orc_in_box(const double* v, int K, double lo, double hi)
{
    for (int k = 0; k < K; ++k) if (!(v[k] >= lo && v[k] <= hi)) return 0;
    return 1;
}

void orc_rwmh_move_slots(const float* y, int64_t N, int K, const double* logw, double sigma,
                         double lo, double hi,
                         const float* theta_in, const double* loglik_in, const int32_t* anc,
                         float* theta_out, double* loglik_out, int64_t M,
                         const float* beta, int64_t beta_stride, float scale,
                         uint64_t seed, uint64_t step, int32_t* accepted,
                         const int32_t* slots, int64_t n_out, double* log_alpha_out)
{
    /* slots (nullable): compute only output slots slots[0..n_out); results
     * are stored compactly at position s (theta_out is [K][n_out]).
     * log_alpha_out (nullable): log acceptance ratio, -inf outside the box. */
    double mu[64], prop[64], z[64];
    for (int64_t s = 0; s < n_out; ++s) {
        int64_t p = slots ? (int64_t)slots[s] : s;
        int64_t src = anc ? (int64_t)anc[p] : p;
        for (int k = 0; k < K; ++k) mu[k] = (double)theta_in[(int64_t)k * M + src];
        double l = loglik_in[src];
        double b = (double)beta[p * beta_stride];
        orc_normals(seed, ORC_P_MOVE, step, (uint32_t)p, K, z);
        for (int k = 0; k < K; ++k) prop[k] = (double)(float)(mu[k] + (double)scale * z[k]);
        int acc = 0;
        double lp = 0.0, la = -INFINITY;
        if (orc_in_box(prop, K, lo, hi)) {
            lp = orc_gmm1d_loglik_one(y, N, K, logw, sigma, prop);
            double u = orc_u01(orc_word(seed, ORC_P_ACCEPT, step, (uint32_t)p, 0));
            la = b * (lp - l);
            if (log(u) < la) acc = 1;
        }
        if (log_alpha_out) log_alpha_out[s] = la;
        for (int k = 0; k < K; ++k)
            theta_out[(int64_t)k * n_out + s] = (float)(acc ? prop[k] : mu[k]);
        loglik_out[s] = acc ? lp : l;
        accepted[s] = acc;
    }
}

void orc_rwmh_move(const float* y, int64_t N, int K, const double* logw, double sigma,
                   double lo, double hi,
                   const float* theta_in, const double* loglik_in, const int32_t* anc,
                   float* theta_out, double* loglik_out, int64_t M,
                   const float* beta, int64_t beta_stride, float scale,
                   uint64_t seed, uint64_t step, int32_t* accepted)
{
    orc_rwmh_move_slots(y, N, K, logw, sigma, lo, hi, theta_in, loglik_in, anc, theta_out,
                        loglik_out, M, beta, beta_stride, scale, seed, step, accepted, NULL, M,
                        NULL);
}

/* ------------------------------------------------------------------------ */
/* MALA move (gradient-informed Langevin proposal) on the same tempered      */
/* target.  The gradient of the tempered log-target is beta * grad l.        */
/*   m(v)  = v + (h^2/2) beta grad l(v)                                      */
/*   mu'   = m(mu) + h z                                                     */
/*   log alpha = beta (l' - l) + log q(mu | mu') - log q(mu' | mu),          */
/*   log q(a | b) = -|a - m(b)|^2 / (2 h^2)                                  */
/* Draws as for the RW move.  grad_in / grad_out are [K][M].                 */
/* ------------------------------------------------------------------------ */
void orc_mala_move_slots(const float* y, int64_t N, int K, const double* logw, double sigma,
                         double lo, double hi,
                         const float* theta_in, const double* loglik_in, const float* grad_in,
                         const int32_t* anc,
                         float* theta_out, double* loglik_out, float* grad_out, int64_t M,
                         const float* beta, int64_t beta_stride, float h,
                         uint64_t seed, uint64_t step, int32_t* accepted,
                         const int32_t* slots, int64_t n_out, double* log_alpha_out)
{
    double mu[64], g[64], prop[64], gp[64], z[64], mf[64], mb[64];
    double hh = (double)h;
    for (int64_t s = 0; s < n_out; ++s) {
        int64_t p = slots ? (int64_t)slots[s] : s;
        int64_t src = anc ? (int64_t)anc[p] : p;
        for (int k = 0; k < K; ++k) {
            mu[k] = (double)theta_in[(int64_t)k * M + src];
            g[k] = (double)grad_in[(int64_t)k * M + src];
        }
        double l = loglik_in[src];
        double b = (double)beta[p * beta_stride];
        orc_normals(seed, ORC_P_MOVE, step, (uint32_t)p, K, z);
        for (int k = 0; k < K; ++k) {
            mf[k] = mu[k] + 0.5 * hh * hh * b * g[k];
            prop[k] = (double)(float)(mf[k] + hh * z[k]);
        }
        int acc = 0;
        double lp = 0.0, la = -INFINITY;
        if (orc_in_box(prop, K, lo, hi)) {
            lp = orc_gmm1d_loglik_one(y, N, K, logw, sigma, prop);
            orc_gmm1d_grad_one(y, N, K, logw, sigma, prop, gp);
            double fwd = 0.0, bwd = 0.0;
            for (int k = 0; k < K; ++k) {
                mb[k] = prop[k] + 0.5 * hh * hh * b * gp[k];
                double df = prop[k] - mf[k];
                double db = mu[k] - mb[k];
                fwd += df * df;
                bwd += db * db;
            }
            double log_alpha = b * (lp - l) + (-bwd / (2.0 * hh * hh)) - (-fwd / (2.0 * hh * hh));
            double u = orc_u01(orc_word(seed, ORC_P_ACCEPT, step, (uint32_t)p, 0));
            la = log_alpha;
            if (log(u) < log_alpha) acc = 1;
        }
        if (log_alpha_out) log_alpha_out[s] = la;
        for (int k = 0; k < K; ++k) {
            theta_out[(int64_t)k * n_out + s] = (float)(acc ? prop[k] : mu[k]);
            grad_out[(int64_t)k * n_out + s] = (float)(acc ? gp[k] : g[k]);
        }
        loglik_out[s] = acc ? lp : l;
        accepted[s] = acc;
    }
}

void orc_mala_move(const float* y, int64_t N, int K, const double* logw, double sigma,
                   double lo, double hi,
                   const float* theta_in, const double* loglik_in, const float* grad_in,
                   const int32_t* anc,
                   float* theta_out, double* loglik_out, float* grad_out, int64_t M,
                   const float* beta, int64_t beta_stride, float h,
                   uint64_t seed, uint64_t step, int32_t* accepted)
{
    orc_mala_move_slots(y, N, K, logw, sigma, lo, hi, theta_in, loglik_in, grad_in, anc,
                        theta_out, loglik_out, grad_out, M, beta, beta_stride, h, seed, step,
                        accepted, NULL, M, NULL);
}

/* ------------------------------------------------------------------------ */
/* One sweep of population MCMC over many independent populations           */
/* (Section 3.1 and Section 4.1.1).  Population q holds the chains           */
/* offsets[q] .. offsets[q+1]-1; chain c of a population has its own beta.   */
/* Stage 1: a random-walk MH move for every chain (as orc_rwmh_move, with    */
/* particle index = global chain index, step = sweep).                       */
/* Stage 2: the basic exchange move between adjacent chains with disjoint    */
/* pairs, chosen by one parity bit b per population and sweep (purpose       */
/* EXCHANGE, index q, block 0, word 0, bit 0):                               */
/*   b = 0: pairs (0,1), (2,3), ...           (last chain idle if M_q odd)   */
/*   b = 1: pairs (1,2), (3,4), ... and (M_q-1, 0) when M_q is even          */
/*          (chain 0 idle if M_q is odd)                                     */
/* Pair j swaps with probability min{1, alpha}, where                        */
/*   log alpha = (beta_a - beta_b)(l_b - l_a)                                */
/* (the ratio pi_a(x_b) pi_b(x_a) / (pi_a(x_a) pi_b(x_b)) for tempered       */
/* targets), u from purpose EXCHANGE, index q, word 4 + j.                   */
/* Chain values theta and l move; the temperatures stay with the slots.      */
/* stats[0] += MH accepts, stats[1] += swaps accepted, stats[2] += swaps     */
/* attempted.                                                                */
/* ------------------------------------------------------------------------ */
/* Stage 2 alone, for populations q0 .. q1-1 (the sweep calls it for all).  */
/* Test hooks (NULL in the sweep): la_out[p] receives log alpha - log u of   */
/* the p-th pair attempted (populations in order, then pairs in order,       */
/* counted from population q0); flip[p] != 0 takes the opposite decision     */
/* for that pair, so a test can replay the stage with chosen decisions.      */
void orc_popmcmc_exchange(int K, float* theta, double* loglik, int64_t Mtot,
                          const float* beta, const int32_t* offsets, int32_t q0, int32_t q1,
                          uint64_t seed, uint64_t sweep, int64_t* stats, double* la_out,
                          const int8_t* flip)
{
    int64_t p = 0;
    for (int32_t q = q0; q < q1; ++q) {
        int64_t base = offsets[q];
        int64_t Mq = (int64_t)offsets[q + 1] - base;
        if (Mq < 2) continue;
        uint32_t b = orc_word(seed, ORC_P_EXCHANGE, sweep, (uint32_t)q, 0) & 1u;
        int64_t npairs;
        if (b == 0) npairs = Mq / 2;
        else npairs = (Mq - 1) / 2 + ((Mq % 2 == 0) ? 1 : 0);
        for (int64_t j = 0; j < npairs; ++j, ++p) {
            int64_t ia, ib;
            if (b == 0) { ia = 2 * j; ib = 2 * j + 1; }
            else if (j < (Mq - 1) / 2) { ia = 2 * j + 1; ib = 2 * j + 2; }
            else { ia = Mq - 1; ib = 0; }
            int64_t ga = base + ia, gb = base + ib;
            double la = loglik[ga], lb = loglik[gb];
            double log_alpha = ((double)beta[ga] - (double)beta[gb]) * (lb - la);
            double u = orc_u01(orc_word(seed, ORC_P_EXCHANGE, sweep, (uint32_t)q, (uint32_t)(4 + j)));
            if (la_out) la_out[p] = log_alpha - log(u);
            int swap = log(u) < log_alpha;
            if (flip && flip[p]) swap = !swap;
            stats[2] += 1;
            if (swap) {
                stats[1] += 1;
                for (int k = 0; k < K; ++k) {
                    float t = theta[(int64_t)k * Mtot + ga];
                    theta[(int64_t)k * Mtot + ga] = theta[(int64_t)k * Mtot + gb];
                    theta[(int64_t)k * Mtot + gb] = t;
                }
                loglik[ga] = lb;
                loglik[gb] = la;
            }
        }
    }
}

void orc_popmcmc_sweep(const float* y, int64_t N, int K, const double* logw, double sigma,
                       double lo, double hi,
                       float* theta, double* loglik, int64_t Mtot,
                       const float* beta, const int32_t* offsets, int32_t n_pops,
                       float scale, uint64_t seed, uint64_t sweep, int64_t* stats)
{
    float* th_new = (float*)malloc((size_t)Mtot * K * sizeof(float));
    double* l_new = (double*)malloc((size_t)Mtot * sizeof(double));
    int32_t* acc = (int32_t*)malloc((size_t)Mtot * sizeof(int32_t));
    orc_rwmh_move(y, N, K, logw, sigma, lo, hi, theta, loglik, NULL, th_new, l_new, Mtot,
                  beta, 1, scale, seed, sweep, acc);
    for (int64_t i = 0; i < Mtot; ++i) stats[0] += acc[i];
    memcpy(theta, th_new, (size_t)Mtot * K * sizeof(float));
    memcpy(loglik, l_new, (size_t)Mtot * sizeof(double));
    orc_popmcmc_exchange(K, theta, loglik, Mtot, beta, offsets, 0, n_pops, seed, sweep, stats,
                         NULL, NULL);
    free(th_new); free(l_new); free(acc);
}

/* ------------------------------------------------------------------------ */
/* Particle filter (Section 3.2, bootstrap proposal) for a d-dimensional     */
/* stochastic-volatility state (the multivariate SV model mentioned in       */
/* Section 4.2) and a linear-Gaussian variant:                               */
/*   x_t = phi (.) x_{t-1} + L z,   z ~ N(0, I_d)  (purpose PFNOISE, index i) */
/*   MSV: log g = sum_j [ -1/2 log(2 pi b^2) - x_j / 2                        */
/*                        - y_j^2 exp(-x_j) / (2 b^2) ]                       */
/*   LG : log g = sum_j [ -1/2 log(2 pi b^2) - (y_j - x_j)^2 / (2 b^2) ]      */
/* x is SoA [d][M]; slot i starts from x_in[anc[i]] (identity if NULL).      */
/* chol is the row-major lower Cholesky factor L of Sigma (d x d).           */
/* The new state is stored as float; log g is evaluated at the stored value.*/
/* ------------------------------------------------------------------------ */
void orc_pf_step(int kind, int d, const double* phi, const double* chol, double bscale,
                 const float* yt, const float* x_in, const int32_t* anc, float* x_out,
                 double* logg_out, int64_t M, uint64_t seed, uint64_t t)
{
    double z[16], xn[16];
    double b2 = bscale * bscale;
    for (int64_t i = 0; i < M; ++i) {
        int64_t src = anc ? (int64_t)anc[i] : i;
        orc_normals(seed, ORC_P_PFNOISE, t, (uint32_t)i, d, z);
        for (int r = 0; r < d; ++r) {
            double v = phi[r] * (double)x_in[(int64_t)r * M + src];
            for (int c = 0; c <= r; ++c) v += chol[r * d + c] * z[c];
            xn[r] = (double)(float)v;
        }
        double lg = 0.0;
        for (int j = 0; j < d; ++j) {
            double yj = (double)yt[j];
            if (kind == 0)
                lg += -0.5 * log(2.0 * ORC_PI * b2) - 0.5 * xn[j] - yj * yj * exp(-xn[j]) / (2.0 * b2);
            else
                lg += -0.5 * log(2.0 * ORC_PI * b2) - (yj - xn[j]) * (yj - xn[j]) / (2.0 * b2);
        }
        for (int j = 0; j < d; ++j) x_out[(int64_t)j * M + i] = (float)xn[j];
        logg_out[i] = lg;
    }
}

/* ------------------------------------------------------------------------ */
/* Whole-run drivers (used for statistical pins and the CPU baseline).       */
/* ------------------------------------------------------------------------ */

/* Bootstrap particle filter with systematic resampling after every step.   */
/* log Z = sum_t [ LSE_i(log g_i) - log M ]; filter means are taken before   */
/* resampling (sum_i W_i x_i).  y is [T][d]; means_out is [T][d] (nullable). */
/* Returns 0 or an error code from reweight / resample.                      */
int orc_pf_run(int kind, int d, const double* phi, const double* chol, double bscale,
               const float* y, int64_t T, int64_t M, uint64_t seed,
               double* logZ_out, double* means_out)
{
    float* xa = (float*)calloc((size_t)d * M, sizeof(float));
    float* xb = (float*)calloc((size_t)d * M, sizeof(float));
    double* lg = (double*)malloc((size_t)M * sizeof(double));
    double* lw = (double*)malloc((size_t)M * sizeof(double));
    double* W = (double*)malloc((size_t)M * sizeof(double));
    int32_t* anc = (int32_t*)malloc((size_t)M * sizeof(int32_t));
    double sc[4];
    double logZ = 0.0;
    int rc = 0;
    for (int64_t i = 0; i < M; ++i) anc[i] = (int32_t)i;
    for (int64_t t = 1; t <= T; ++t) {
        orc_pf_step(kind, d, phi, chol, bscale, y + (t - 1) * d, xa, anc, xb, lg, M, seed, (uint64_t)t);
        for (int64_t i = 0; i < M; ++i) lw[i] = 0.0;
        rc = orc_reweight(lg, 1.0, lw, M, W, sc);
        if (rc) break;
        logZ += sc[0];
        if (means_out) {
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int64_t i = 0; i < M; ++i) s += W[i] * (double)xb[(int64_t)j * M + i];
                means_out[(t - 1) * d + j] = s;
            }
        }
        uint32_t u32 = orc_word(seed, ORC_P_RESAMPLE, (uint64_t)t, 0, 0);
        rc = orc_resample_systematic(W, M, u32, anc, NULL);
        if (rc) break;
        float* tmp = xa; xa = xb; xb = tmp;
    }
    *logZ_out = logZ;
    free(xa); free(xb); free(lg); free(lw); free(W); free(anc);
    return rc;
}

/* Exact log-likelihood of the linear-Gaussian variant by the Kalman filter:
 *   x_t = Phi x_{t-1} + eta, eta ~ N(0, Sigma);  y_t = x_t + eps,
 *   eps ~ N(0, b^2 I);  x_0 = 0 known (m_0 = 0, P_0 = 0).
 * Textbook predict / update recursion with log N(y_t; m_pred, P_pred + R).
 * Sigma is row-major d x d; d <= 8.  means_out [T][d] holds filter means. */
static int orc_chol(const double* A, int d, double* L)
{
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = A[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
        if (!(s > 0.0)) return -1;
        L[j * d + j] = sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double v = A[i * d + j];
            for (int k = 0; k < j; ++k) v -= L[i * d + k] * L[j * d + k];
            L[i * d + j] = v / L[j * d + j];
        }
    }
    return 0;
}

double orc_kalman_lg(int d, const double* phi, const double* Sigma, double bscale,
                     const float* y, int64_t T, double* means_out)
{
    double m[8] = {0}, P[64] = {0}, mp[8], Pp[64], S[64], Ls[64], Kg[64], v[8], w[8];
    double ll = 0.0;
    double R = bscale * bscale;
    for (int64_t t = 0; t < T; ++t) {
        for (int i = 0; i < d; ++i) mp[i] = phi[i] * m[i];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                Pp[i * d + j] = phi[i] * P[i * d + j] * phi[j] + Sigma[i * d + j];
        for (int i = 0; i < d * d; ++i) S[i] = Pp[i];
        for (int i = 0; i < d; ++i) S[i * d + i] += R;
        if (orc_chol(S, d, Ls)) return NAN;
        for (int i = 0; i < d; ++i) v[i] = (double)y[t * d + i] - mp[i];
        /* w = L^{-1} v ; quadratic form = |w|^2 ; log det S = 2 sum log L_ii */
        double logdet = 0.0, quad = 0.0;
        for (int i = 0; i < d; ++i) {
            double s = v[i];
            for (int k = 0; k < i; ++k) s -= Ls[i * d + k] * w[k];
            w[i] = s / Ls[i * d + i];
            quad += w[i] * w[i];
            logdet += 2.0 * log(Ls[i * d + i]);
        }
        ll += -0.5 * ((double)d * log(2.0 * ORC_PI) + logdet + quad);
        /* gain K = Pp S^{-1}: solve S K^T = Pp^T column by column */
        for (int c = 0; c < d; ++c) {
            double rhs[8], tmp[8], sol[8];
            for (int i = 0; i < d; ++i) rhs[i] = Pp[c * d + i]; /* row c of Pp (symmetric) */
            for (int i = 0; i < d; ++i) {
                double s = rhs[i];
                for (int k = 0; k < i; ++k) s -= Ls[i * d + k] * tmp[k];
                tmp[i] = s / Ls[i * d + i];
            }
            for (int i = d - 1; i >= 0; --i) {
                double s = tmp[i];
                for (int k = i + 1; k < d; ++k) s -= Ls[k * d + i] * sol[k];
                sol[i] = s / Ls[i * d + i];
            }
            for (int i = 0; i < d; ++i) Kg[c * d + i] = sol[i];
        }
        for (int i = 0; i < d; ++i) {
            double s = mp[i];
            for (int k = 0; k < d; ++k) s += Kg[i * d + k] * v[k];
            m[i] = s;
        }
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double s = Pp[i * d + j];
                for (int k = 0; k < d; ++k) s -= Kg[i * d + k] * Pp[k * d + j];
                P[i * d + j] = s;
            }
        if (means_out) for (int i = 0; i < d; ++i) means_out[t * d + i] = m[i];
    }
    return ll;
}

/* Factor stochastic volatility (Section 4.2): latent x_t in R^K,
 * observation y_t in R^m (m <= 8, K <= 8):
 *   x_t = Phi x_{t-1} + L_U z,  z ~ N(0, I_K),
 *   y_t | x_t ~ N(0, Sigma_t),  Sigma_t = B diag(exp x_t) B^T + diag(psi).
 * log g(y_t | x_t) by the plain definition: the m x m covariance, its
 * Cholesky factor, the log-determinant and one triangular solve, in FP64.
 * B is row-major m x K; x is [K][M]; yt holds m floats.                    */
static double orc_fsv_logg(int K, int m, const double* B, const double* psi,
                           const double* x, const float* yt)
{
    double S[64], L[64], w[8];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double v = (i == j) ? psi[i] : 0.0;
            for (int k = 0; k < K; ++k) v += B[i * K + k] * exp(x[k]) * B[j * K + k];
            S[i * m + j] = v;
        }
    if (orc_chol(S, m, L)) return NAN;
    double logdet = 0.0, quad = 0.0;
    for (int i = 0; i < m; ++i) {
        double s = (double)yt[i];
        for (int k = 0; k < i; ++k) s -= L[i * m + k] * w[k];
        w[i] = s / L[i * m + i];
        quad += w[i] * w[i];
        logdet += 2.0 * log(L[i * m + i]);
    }
    return -0.5 * ((double)m * log(2.0 * ORC_PI) + logdet + quad);
}

void orc_fsv_step(int K, int m, const double* phi, const double* cholU, const double* B,
                  const double* psi, const float* yt, const float* x_in, const int32_t* anc,
                  float* x_out, double* logg_out, int64_t M, uint64_t seed, uint64_t t)
{
    double z[16], xn[8];
    for (int64_t i = 0; i < M; ++i) {
        int64_t src = anc ? (int64_t)anc[i] : i;
        orc_normals(seed, ORC_P_PFNOISE, t, (uint32_t)i, K, z);
        for (int r = 0; r < K; ++r) {
            double v = phi[r] * (double)x_in[(int64_t)r * M + src];
            for (int c = 0; c <= r; ++c) v += cholU[r * K + c] * z[c];
            xn[r] = (double)(float)v;  /* the state is stored in FP32 */
        }
        for (int r = 0; r < K; ++r) x_out[(int64_t)r * M + i] = (float)xn[r];
        logg_out[i] = orc_fsv_logg(K, m, B, psi, xn, yt);
    }
}

/* Bootstrap filter on the factor SV model, resampling every step as in
 * orc_pf_run; y is [T][m]; means_out [T][K] (nullable). */
int orc_fsv_run(int K, int m, const double* phi, const double* cholU, const double* B,
                const double* psi, const float* y, int64_t T, int64_t M, uint64_t seed,
                double* logZ_out, double* means_out)
{
    float* xa = (float*)calloc((size_t)K * M, sizeof(float));
    float* xb = (float*)calloc((size_t)K * M, sizeof(float));
    double* lg = (double*)malloc((size_t)M * sizeof(double));
    double* lw = (double*)malloc((size_t)M * sizeof(double));
    double* W = (double*)malloc((size_t)M * sizeof(double));
    int32_t* anc = (int32_t*)malloc((size_t)M * sizeof(int32_t));
    double sc[4];
    double logZ = 0.0;
    int rc = 0;
    for (int64_t i = 0; i < M; ++i) anc[i] = (int32_t)i;
    for (int64_t t = 1; t <= T; ++t) {
        orc_fsv_step(K, m, phi, cholU, B, psi, y + (t - 1) * m, xa, anc, xb, lg, M, seed,
                     (uint64_t)t);
        for (int64_t i = 0; i < M; ++i) lw[i] = 0.0;
        rc = orc_reweight(lg, 1.0, lw, M, W, sc);
        if (rc) break;
        logZ += sc[0];
        if (means_out) {
            for (int j = 0; j < K; ++j) {
                double s = 0.0;
                for (int64_t i = 0; i < M; ++i) s += W[i] * (double)xb[(int64_t)j * M + i];
                means_out[(t - 1) * K + j] = s;
            }
        }
        uint32_t u32 = orc_word(seed, ORC_P_RESAMPLE, (uint64_t)t, 0, 0);
        rc = orc_resample_systematic(W, M, u32, anc, NULL);
        if (rc) break;
        float* tmp = xa; xa = xb; xb = tmp;
    }
    *logZ_out = logZ;
    free(xa); free(xb); free(lg); free(lw); free(W); free(anc);
    return rc;
}

/* SMC sampler with tempering (Section 3.3 and Section 4.1.2): particles
 * start from the uniform prior (theta0, supplied), beta_0 = 0; for
 * t = 1..T: reweight by (beta_t - beta_{t-1}) l, resample (systematic) iff
 * ESS < ess_frac * M, then n_moves random-walk MH moves (kind 0) or MALA
 * moves (kind 1) targeting pi_{beta_t} (Section 4.1.2 uses 10 per
 * temperature).  Move r of step t draws with step counter t + r 2^32 (so
 * a single move uses step t); only move 0 starts from the ancestors.
 * log Z = sum_t log Z increment.
 * theta is [K][M] in/out; ess_out [T] (nullable) records the ESS before
 * resampling, resampled_out [T] (nullable) the decisions. */
int orc_smc_run(const float* y, int64_t N, int K, const double* logw, double sigma,
                double lo, double hi, float* theta, int64_t M,
                const double* betas /* [T+1], betas[0] = 0 */, int64_t T,
                int kind, float scale, int n_moves, double ess_frac, uint64_t seed,
                double* logZ_out, double* ess_out, int32_t* resampled_out)
{
    float* th2 = (float*)malloc((size_t)K * M * sizeof(float));
    float* g = (float*)malloc((size_t)K * M * sizeof(float));
    float* g2 = (float*)malloc((size_t)K * M * sizeof(float));
    double* l = (double*)malloc((size_t)M * sizeof(double));
    double* l2 = (double*)malloc((size_t)M * sizeof(double));
    double* lw = (double*)calloc((size_t)M, sizeof(double));
    double* W = (double*)malloc((size_t)M * sizeof(double));
    double* gd = (double*)malloc((size_t)K * M * sizeof(double));
    int32_t* anc = (int32_t*)malloc((size_t)M * sizeof(int32_t));
    int32_t* acc = (int32_t*)malloc((size_t)M * sizeof(int32_t));
    double sc[4];
    double logZ = 0.0;
    int rc = 0;
    orc_gmm1d_loglik(y, N, K, logw, sigma, theta, M, l);
    if (kind == 1) {
        orc_gmm1d_grad(y, N, K, logw, sigma, theta, M, gd);
        for (int64_t i = 0; i < (int64_t)K * M; ++i) g[i] = (float)gd[i];
    }
    for (int64_t t = 1; t <= T; ++t) {
        rc = orc_reweight(l, betas[t] - betas[t - 1], lw, M, W, sc);
        if (rc) break;
        logZ += sc[0];
        if (ess_out) ess_out[t - 1] = sc[1];
        int do_rs = sc[1] < ess_frac * (double)M;
        if (resampled_out) resampled_out[t - 1] = do_rs;
        if (do_rs) {
            uint32_t u32 = orc_word(seed, ORC_P_RESAMPLE, (uint64_t)t, 0, 0);
            rc = orc_resample_systematic(W, M, u32, anc, NULL);
            if (rc) break;
            for (int64_t i = 0; i < M; ++i) lw[i] = 0.0;
        } else {
            for (int64_t i = 0; i < M; ++i) anc[i] = (int32_t)i;
        }
        float bt = (float)betas[t];
        for (int r = 0; r < n_moves; ++r) {
            const int32_t* a = r == 0 ? anc : NULL;
            uint64_t st = (uint64_t)t + ((uint64_t)r << 32);
            if (kind == 0) {
                orc_rwmh_move(y, N, K, logw, sigma, lo, hi, theta, l, a, th2, l2, M,
                              &bt, 0, scale, seed, st, acc);
            } else {
                orc_mala_move(y, N, K, logw, sigma, lo, hi, theta, l, g, a, th2, l2, g2, M,
                              &bt, 0, scale, seed, st, acc);
                memcpy(g, g2, (size_t)K * M * sizeof(float));
            }
            memcpy(theta, th2, (size_t)K * M * sizeof(float));
            memcpy(l, l2, (size_t)M * sizeof(double));
        }
    }
    *logZ_out = logZ;
    free(th2); free(g); free(g2); free(l); free(l2); free(lw); free(W); free(gd);
    free(anc); free(acc);
    return rc;
}
