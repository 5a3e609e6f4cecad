// pf.cu -- pf_step: one bootstrap particle-filter step (Section 3.2) for
// the multivariate stochastic-volatility state of Section 4.2 and a
// linear-Gaussian variant: gather by ancestor, propagate, weight, fused in
// one pass (one thread per particle; SoA states, coalesced except for the
// ancestor gather, which reads mostly increasing addresses).
#include <cmath>

#include "ctx.hpp"
#include "device.cuh"

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
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    float y[D];
#pragma unroll
    for (int j = 0; j < D; ++j) y[j] = yt[j];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        const int64_t src = anc ? (int64_t)anc[i] : i;
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

}  // namespace smc

extern "C" smc_status pf_step(smc_ctx* ctx, const smc_pf_model* model, const float* y_t,
                              const float* x_in, const int32_t* anc, float* x_out,
                              double* logg_out, int64_t M, uint64_t seed, uint64_t t,
                              void* stream) {
    if (!ctx || !model || M < 0) return SMC_ERR_ARG;
    if (model->kind != SMC_PF_MSV && model->kind != SMC_PF_LG) return SMC_ERR_ARG;
    if (model->d < 1 || model->d > 8 || !(model->beta > 0.0f)) return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    if (!y_t || !x_in || !x_out || !logg_out || x_in == x_out) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
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
#define SMC_PF(DD)                                                                          \
    do {                                                                                    \
        if (msv)                                                                            \
            smc::k_pf_step<DD, true><<<(unsigned)blocks, 256, 0, s>>>(                      \
                A, y_t, x_in, anc, x_out, logg_out, M, seed, t, ctx->d_status);             \
        else                                                                                \
            smc::k_pf_step<DD, false><<<(unsigned)blocks, 256, 0, s>>>(                     \
                A, y_t, x_in, anc, x_out, logg_out, M, seed, t, ctx->d_status);             \
    } while (0)
    switch (d) {
        case 1: SMC_PF(1); break;
        case 2: SMC_PF(2); break;
        case 3: SMC_PF(3); break;
        case 4: SMC_PF(4); break;
        case 5: SMC_PF(5); break;
        case 6: SMC_PF(6); break;
        case 7: SMC_PF(7); break;
        case 8: SMC_PF(8); break;
    }
#undef SMC_PF
    return cuda_ok(cudaGetLastError());
}
