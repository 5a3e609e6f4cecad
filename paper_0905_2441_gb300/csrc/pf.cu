// pf.cu -- pf_step: one bootstrap particle-filter step (Section 3.2) for
// the multivariate stochastic-volatility state of Section 4.2, a
// linear-Gaussian variant and the factor stochastic-volatility model of
// Section 4.2 (Table 3): gather by ancestor, propagate, weight, fused in one
// pass (one thread per particle; SoA states, coalesced except for the
// ancestor gather, which reads mostly increasing addresses).
#include <cmath>

#include "ctx.hpp"
#include "device.cuh"
#include "bounds.cuh"
#include "reweight.cuh"

using namespace smc_host;

namespace smc {

struct PfArgs {
    float phi[8];
    float chol[64];
    float cst;        // -1/2 log(2 pi beta^2) per dimension
    float inv2b2;     // 1 / (2 beta^2)
};

template <int D, bool MSV>
__global__ void __launch_bounds__(256) k_pf_step(PfArgs A, const float* __restrict__ yt,
                                                 const float* __restrict__ x_in,
                                                 const int32_t* __restrict__ anc,
                                                 float* __restrict__ x_out,
                                                 double* __restrict__ logg, int64_t M,
                                                 uint64_t seed, uint64_t t, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    float y[D];
#pragma unroll
    for (int j = 0; j < D; ++j) y[j] = yt[j];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        int64_t src = anc ? (int64_t)anc[i] : i;
        if (!SMC_IN_BOUNDS(src >= 0 && src < M, status)) src = i;
        float z[D], xn[D];
        normals<D>(seed, RNG_PFNOISE, t, (uint32_t)i, D, z);
        float lg = 0.0f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float v = A.phi[r] * x_in[(int64_t)r * M + src];
#pragma unroll
            for (int c = 0; c <= r; ++c) v = fmaf(A.chol[r * D + c], z[c], v);
            xn[r] = v;
            x_out[(int64_t)r * M + i] = v;
            if (MSV) {
                // y^2 exp(-x) / (2 b^2) with exp(-x) = 2^(-x log2 e)
                float e = ex2(-v * 1.4426950408889634f);
                lg += A.cst - 0.5f * v - y[r] * y[r] * e * A.inv2b2;
            } else {
                float d = y[r] - v;
                lg += A.cst - d * d * A.inv2b2;
            }
        }
        if (lg != lg) raise_status(status, ST_NONFINITE);
        logg[i] = f2d_bits(lg);  // normal floats only (log g is finite, |log g| >= 2^-126 or 0)
    }
}

// Factor stochastic volatility (Section 4.2): x_t in R^D (factor
// log-variances), y_t in R^m with y_t | x_t ~ N(0, Sigma), Sigma = Psi +
// B H B^T, H = diag(exp x).  With the Woodbury identity and the matrix
// determinant lemma, for A = H^-1 + C, C = B^T Psi^-1 B:
//   y^T Sigma^-1 y = q - |L_A^-1 v|^2,   v = B^T Psi^-1 y,  q = y^T Psi^-1 y
//   log det Sigma  = log det Psi + sum_k x_k + log det A
// so one particle needs a D x D Cholesky factor of A (D = 3 for the paper's
// model) instead of the m x m one of Sigma.
struct FsvArgs {
    float phi[4];
    float chol[16];    // L_U, row-major D x D
    float C[16];       // B^T Psi^-1 B
    float BtPi[32];    // B^T Psi^-1, row-major D x m
    float inv_psi[8];
    float cst;         // -(m/2) log 2 pi - 1/2 log det Psi
    int m;
};

template <int D>
__global__ void __launch_bounds__(256) k_pf_fsv(FsvArgs A, const float* __restrict__ yt,
                                                const float* __restrict__ x_in,
                                                const int32_t* __restrict__ anc,
                                                float* __restrict__ x_out,
                                                double* __restrict__ logg, int64_t M,
                                                uint64_t seed, uint64_t t, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    // the observation's projections, the same for every particle
    float v[D], q = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = 0.0f;
    for (int j = 0; j < A.m; ++j) {
        const float yj = yt[j];
        q = fmaf(A.inv_psi[j] * yj, yj, q);
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = fmaf(A.BtPi[k * 8 + j], yj, v[k]);
    }
    constexpr float kLog2e = 1.4426950408889634f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        int64_t src = anc ? (int64_t)anc[i] : i;
        if (!SMC_IN_BOUNDS(src >= 0 && src < M, status)) src = i;
        float z[D], x[D];
        normals<D>(seed, RNG_PFNOISE, t, (uint32_t)i, D, z);
        float sx = 0.0f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float val = A.phi[r] * x_in[(int64_t)r * M + src];
#pragma unroll
            for (int c = 0; c <= r; ++c) val = fmaf(A.chol[r * D + c], z[c], val);
            x[r] = val;
            x_out[(int64_t)r * M + i] = val;
            sx += val;
        }
        // A = C + diag(exp(-x)); L L^T = A by Cholesky (rsqrt pivots); w = L^-1 v
        float L[D][D], inv[D], w[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
#pragma unroll
            for (int c = 0; c <= r; ++c) {
                float a = A.C[r * D + c];
                if (c == r) a += ex2(-x[r] * kLog2e);
#pragma unroll
                for (int k = 0; k < c; ++k) a = fmaf(-L[r][k], L[c][k], a);
                if (c == r) {
                    inv[r] = rsqrtf(a);
                    L[r][r] = a * inv[r];
                } else {
                    L[r][c] = a * inv[c];
                }
            }
            float s = v[r];
#pragma unroll
            for (int k = 0; k < r; ++k) s = fmaf(-L[r][k], w[k], s);
            w[r] = s * inv[r];
        }
        float prod = 1.0f, ww = 0.0f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            prod *= L[r][r];
            ww = fmaf(w[r], w[r], ww);
        }
        // log det A = 2 ln(prod L_rr)
        const float lg = A.cst - 0.5f * (sx + 2.0f * 0.69314718055994531f * lg2(prod)) -
                         0.5f * (q - ww);
        if (lg != lg) raise_status(status, ST_NONFINITE);
        logg[i] = f2d_bits(lg);
    }
}

}  // namespace smc

static smc_status pf_fsv(smc_ctx* ctx, const smc_pf_model* model, const float* y_t,
                         const float* x_in, const int32_t* anc, float* x_out, double* logg_out,
                         int64_t M, uint64_t seed, uint64_t t, cudaStream_t s) {
    const int d = model->d, m = model->m;
    if (d < 1 || d > 4 || m < 1 || m > 8) return SMC_ERR_ARG;
    for (int j = 0; j < m; ++j)
        if (!(model->psi[j] > 0.0f) || !std::isfinite(model->psi[j])) return SMC_ERR_ARG;
    smc::FsvArgs A = {};
    A.m = m;
    double logdet_psi = 0.0;
    for (int j = 0; j < m; ++j) {
        A.inv_psi[j] = (float)(1.0 / (double)model->psi[j]);
        logdet_psi += std::log((double)model->psi[j]);
    }
    for (int r = 0; r < d; ++r) {
        A.phi[r] = model->phi[r];
        for (int c = 0; c <= r; ++c) A.chol[r * d + c] = model->chol[r * d + c];
        for (int j = 0; j < m; ++j)
            A.BtPi[r * 8 + j] = (float)((double)model->B[j * d + r] / (double)model->psi[j]);
        for (int c = 0; c < d; ++c) {
            double v = 0.0;
            for (int j = 0; j < m; ++j)
                v += (double)model->B[j * d + r] * (double)model->B[j * d + c] /
                     (double)model->psi[j];
            A.C[r * d + c] = (float)v;
        }
    }
    A.cst = (float)(-0.5 * (double)m * std::log(2.0 * M_PI) - 0.5 * logdet_psi);
    int64_t blocks = (M + 255) / 256;
    if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
#define SMC_FSV(DD)                                                                       \
    return launch_pdl(smc::k_pf_fsv<DD>, dim3((unsigned)blocks), dim3(256), 0, s, A, y_t, x_in, \
                      anc, x_out, logg_out, M, seed, t, ctx->d_status)
    switch (d) {
        case 1: SMC_FSV(1);
        case 2: SMC_FSV(2);
        case 3: SMC_FSV(3);
        case 4: SMC_FSV(4);
    }
#undef SMC_FSV
    return SMC_ERR_ARG;
}

extern "C" smc_status pf_step(smc_ctx* ctx, const smc_pf_model* model, const float* y_t,
                              const float* x_in, const int32_t* anc, float* x_out,
                              double* logg_out, int64_t M, uint64_t seed, uint64_t t,
                              void* stream) {
    if (!ctx || !model || M < 0) return SMC_ERR_ARG;
    if (model->kind != SMC_PF_MSV && model->kind != SMC_PF_LG && model->kind != SMC_PF_FSV)
        return SMC_ERR_ARG;
    if (model->kind != SMC_PF_FSV && (model->d < 1 || model->d > 8 || !(model->beta > 0.0f)))
        return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    if (!y_t || !x_in || !x_out || !logg_out || x_in == x_out) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    if (model->kind == SMC_PF_FSV)
        return pf_fsv(ctx, model, y_t, x_in, anc, x_out, logg_out, M, seed, t, as_stream(stream));
    smc::PfArgs A;
    const int d = model->d;
    for (int i = 0; i < 8; ++i) A.phi[i] = i < d ? model->phi[i] : 0.0f;
    for (int i = 0; i < 64; ++i) A.chol[i] = 0.0f;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c <= r; ++c) A.chol[r * d + c] = model->chol[r * d + c];
    double b2 = (double)model->beta * (double)model->beta;
    A.cst = (float)(-0.5 * std::log(2.0 * M_PI * b2));
    A.inv2b2 = (float)(1.0 / (2.0 * b2));
    int64_t blocks = (M + 255) / 256;
    if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
    cudaStream_t s = as_stream(stream);
    bool msv = model->kind == SMC_PF_MSV;
#define SMC_PF(DD)                                                                        \
    return msv ? launch_pdl(smc::k_pf_step<DD, true>, dim3((unsigned)blocks), dim3(256), 0, s, \
                            A, y_t, x_in, anc, x_out, logg_out, M, seed, t, ctx->d_status)   \
               : launch_pdl(smc::k_pf_step<DD, false>, dim3((unsigned)blocks), dim3(256), 0, \
                            s, A, y_t, x_in, anc, x_out, logg_out, M, seed, t, ctx->d_status)
    switch (d) {
        case 1: SMC_PF(1);
        case 2: SMC_PF(2);
        case 3: SMC_PF(3);
        case 4: SMC_PF(4);
        case 5: SMC_PF(5);
        case 6: SMC_PF(6);
        case 7: SMC_PF(7);
        case 8: SMC_PF(8);
    }
#undef SMC_PF
    return SMC_ERR_ARG;
}

// the reweighting reduction of smc_reweight and the normalisation and
// resampling half of smc_reweight_resample (weights.cu)
smc_status reweight_reduce_launch(smc_ctx* ctx, const double* loglik, double dbeta, double* logw,
                                  int64_t M, double* scalars_out, int32_t* resample_flag,
                                  double ess_frac, cudaStream_t s, smc::RwArgs* defer_to);
smc_status normalize_resample_launch(smc_ctx* ctx, const smc::RwArgs& rw, double* logw,
                                     int64_t M, double* W_out, int32_t* resample_flag,
                                     uint64_t seed, uint64_t step, int32_t* ancestors_out,
                                     int32_t* counts_out, cudaStream_t s);

extern "C" smc_status smc_pf_filter_step(smc_ctx* ctx, const smc_pf_model* model,
                                         const float* y_t, const float* x_in, int32_t* anc,
                                         float* x_out, double* logg_out, double* logw, int64_t M,
                                         double* W_out, double* scalars_out,
                                         int32_t* resample_flag_out, double ess_frac,
                                         uint64_t seed, uint64_t t, int32_t* counts_out,
                                         void* stream) {
    if (!ctx || M <= 0 || M > 0x7FFFFFFF || !anc || !logw || !W_out || !logg_out ||
        std::isnan(ess_frac))
        return SMC_ERR_ARG;
    smc_status st = pf_step(ctx, model, y_t, x_in, anc, x_out, logg_out, M, seed, t, stream);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    smc::RwArgs rw;
    st = reweight_reduce_launch(ctx, logg_out, 1.0, logw, M, scalars_out, resample_flag_out,
                                ess_frac, s, &rw);
    if (st != SMC_OK) return st;
    return normalize_resample_launch(ctx, rw, logw, M, W_out, resample_flag_out, seed, t, anc,
                                     counts_out, s);
}
