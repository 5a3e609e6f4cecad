// loglik.cu -- smc_loglik_batch: per-particle mixture log-likelihoods
// (Section 4.1) for the univariate model (CUDA cores, MUFU-bound) and the
// diagonal d-dimensional model (CUDA-core FP32 path here; the tensor-core
// BF16-split path lives in diag_tc.cu).
#include <cmath>
#include <vector>

#include "ctx.hpp"
#include "gmm1d.cuh"

using namespace smc_host;

namespace smc {

// One block = (blockDim / L) particles, L lanes each; y streamed through
// shared memory in chunks (bulk asynchronous copies).
template <int K, bool GRAD, bool EQW>
__global__ void __launch_bounds__(256) k_loglik_gmm1d(const float* __restrict__ y, int64_t N,
                                                      const float* __restrict__ theta, int64_t M,
                                                      double* __restrict__ loglik_out,
                                                      float* __restrict__ grad_out,
                                                      Gmm1dArgs P, int L, int Kreal, int ychunk,
                                                      uint32_t* status) {
    extern __shared__ __align__(16) float ys[];
    init_mbar(ychunk_mbar(ys, ychunk));
    const int lane = threadIdx.x % L;
    const int ppb = blockDim.x / L;
    const int64_t p = (int64_t)blockIdx.x * ppb + threadIdx.x / L;
    const bool active = p < M;
    float nu[K], lw2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float mu = (active && k < Kreal) ? theta[(int64_t)k * M + p] : 0.0f;
        nu[k] = -mu * P.r;
        lw2[k] = P.lw2[k];
    }
    uint32_t phase = 0;
    float g[K];
    double ll;
    if constexpr (EQW) {
        SliceAccEqW<K, GRAD> acc;
        slice_over_data_eq(acc, ys, ychunk, y, N, active, lane, L, nu, P.r, phase, status,
                           P.wait_limit);
        ll = acc.finish(L, P, g);
    } else {
        SliceAcc<K, GRAD, EQW> acc;
        slice_over_data(acc, ys, ychunk, y, N, active, lane, L, nu, lw2, P.r, phase, status,
                        P.wait_limit);
        ll = acc.finish(L, P, g);
    }
    if (active && lane == 0) {
        if (ll != ll) raise_status(status, ST_NONFINITE);
        loglik_out[p] = ll;
        if constexpr (GRAD) {
            if (grad_out) {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (k < Kreal) grad_out[(int64_t)k * M + p] = g[k];
            }
        }
    }
}

// Diagonal d-dimensional mixture on CUDA cores, FP32 arithmetic with the
// squared distance summed directly over dimensions: PPB particles per block,
// their means in shared memory, one datum per thread and step.
constexpr int kDiagPPB = 4;

struct DiagLw2 {
    float v[64];  // log2 w_k
};

__global__ void __launch_bounds__(256) k_loglik_diag_fp32(const float* __restrict__ Y, int64_t N,
                                                          int d, int K,
                                                          const float* __restrict__ theta,
                                                          int64_t M, double* __restrict__ out,
                                                          float c2,  // log2(e) / (2 sigma^2)
                                                          DiagLw2 lw2g, double cst,
                                                          uint32_t* status) {
    extern __shared__ __align__(16) float sm[];
    float* mu = sm;                               // [PPB][K][d]
    float* lw2 = sm + kDiagPPB * K * d;           // [K]
    __shared__ double red[kDiagPPB][8];
    const int64_t p0 = (int64_t)blockIdx.x * kDiagPPB;
    for (int i = threadIdx.x; i < kDiagPPB * K * d; i += blockDim.x) {
        int64_t p = p0 + i / (K * d);
        mu[i] = p < M ? theta[p0 * K * d + i] : 0.0f;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) lw2[k] = lw2g.v[k];
    __syncthreads();
    Kahan acc[kDiagPPB];
    float yv[64];
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        const float* yn = Y + n * d;
        for (int j = 0; j < d; ++j) yv[j] = yn[j];
        for (int q = 0; q < kDiagPPB; ++q) {
            const float* mq = mu + q * K * d;
            float m = -INFINITY;
            float a[64];
            for (int k = 0; k < K; ++k) {
                float s = 0.0f;
                for (int j = 0; j < d; ++j) {
                    float e = yv[j] - mq[k * d + j];
                    s = fmaf(e, e, s);
                }
                a[k] = fmaf(-c2, s, lw2[k]);
                m = fmaxf(m, a[k]);
            }
            float s = 0.0f;
            for (int k = 0; k < K; ++k) s += ex2(a[k] - m);
            acc[q].add(m + lg2(s));
        }
    }
    for (int q = 0; q < kDiagPPB; ++q) {
        double v = (double)acc[q].s - (double)acc[q].c;
        v = warp_sum_d(v);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagPPB) {
        int q = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[q][w];
        int64_t p = p0 + q;
        if (p < M) {
            double ll = t * kLn2 + cst;
            if (ll != ll) raise_status(status, ST_NONFINITE);
            out[p] = ll;
        }
    }
}

}  // namespace smc

// -------------------------------------------------------------- host side

namespace smc_host {

// Shared argument preparation for every 1-D mixture entry point.
smc_status gmm1d_prepare(const smc_gmm* model, int64_t N, smc::Gmm1dArgs* P, int* Kpad,
                         bool* eqw) {
    if (!model || model->kind != SMC_GMM_1D || model->d != 1) return SMC_ERR_ARG;
    int K = model->K;
    if (K < 1 || !model->log_w || !(model->sigma > 0.0f) || !(model->lo < model->hi))
        return SMC_ERR_ARG;
    if (K > smc::kMaxK1d) return SMC_ERR_UNSUPPORTED;
    int kp = 1;
    while (kp < K) kp *= 2;
    double s = (double)model->sigma;
    P->r = (float)std::sqrt(smc::kLog2e / (2.0 * s * s));
    P->cf = (float)(smc::kLog2e / (2.0 * s * s));
    // w = 2^floor(log2(4 / sqrt(cf))), so that cf (w/2)^2 <= 4
    P->binw = (float)std::ldexp(1.0, (int)std::floor(std::log2(4.0 / std::sqrt((double)P->cf))));
    P->binw_inv = 1.0f / P->binw;
    P->wait_limit = smc::kSpinLimit;
    P->gscale = (float)(1.0 / (s * s * (double)P->r));
    P->lo = model->lo;
    P->hi = model->hi;
    bool equal = (kp == K);
    for (int k = 0; k < K; ++k) {
        if (std::isnan(model->log_w[k])) return SMC_ERR_ARG;
        if (model->log_w[k] != model->log_w[0]) equal = false;
    }
    double per = -0.5 * std::log(2.0 * M_PI * s * s);
    for (int k = 0; k < smc::kMaxK1d; ++k)
        P->lw2[k] = k < K ? (float)((double)model->log_w[k] * smc::kLog2e) : -INFINITY;
    if (equal) {
        per += (double)model->log_w[0];
        for (int k = 0; k < smc::kMaxK1d; ++k) P->lw2[k] = k < K ? 0.0f : -INFINITY;
    }
    P->cst = (double)N * per;
    *Kpad = kp;
    *eqw = equal;
    return SMC_OK;
}

template <int K, bool GRAD, bool EQW>
static void launch_1d(int blocks, int threads, cudaStream_t s, const float* y, int64_t N,
                      const float* theta, int64_t M, double* out, float* grad,
                      const smc::Gmm1dArgs& P, int L, int Kreal, uint32_t* st) {
    const int yc = smc::ychunk_for(N);
    smc::k_loglik_gmm1d<K, GRAD, EQW><<<blocks, threads, smc::ysmem_bytes(yc), s>>>(
        y, N, theta, M, out, grad, P, L, Kreal, yc, st);
}

template <int K>
static void dispatch_1d(bool grad, bool eqw, int blocks, int threads, cudaStream_t s,
                        const float* y, int64_t N, const float* theta, int64_t M, double* out,
                        float* g, const smc::Gmm1dArgs& P, int L, int Kreal, uint32_t* st) {
    if (grad) {
        if (eqw) launch_1d<K, true, true>(blocks, threads, s, y, N, theta, M, out, g, P, L, Kreal, st);
        else launch_1d<K, true, false>(blocks, threads, s, y, N, theta, M, out, g, P, L, Kreal, st);
    } else {
        if (eqw) launch_1d<K, false, true>(blocks, threads, s, y, N, theta, M, out, g, P, L, Kreal, st);
        else launch_1d<K, false, false>(blocks, threads, s, y, N, theta, M, out, g, P, L, Kreal, st);
    }
}

}  // namespace smc_host

// defined in diag_tc.cu
smc_status smc_diag_tc_loglik(smc_ctx* ctx, const smc_gmm* model, const float* Y, int64_t N,
                              const float* theta, int64_t M, double* out, cudaStream_t s);

extern "C" smc_status smc_loglik_batch(smc_ctx* ctx, const smc_gmm* model, const float* y,
                                       int64_t N, const float* theta, int64_t M,
                                       double* loglik_out, float* grad_out, void* stream) {
    if (!ctx || !model || M < 0 || N < 0) return SMC_ERR_ARG;
    if (M > 0 && (!theta || !loglik_out || (N > 0 && !y))) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    if (model->kind == SMC_GMM_DIAG) {
        int K = model->K, d = model->d;
        if (K < 1 || K > 64 || d < 1 || d > 64 || !model->log_w || !(model->sigma > 0.0f) ||
            grad_out)
            return SMC_ERR_ARG;
        if (M == 0) return SMC_OK;
        if (model->precision == SMC_PREC_BF16SPLIT)
            return smc_diag_tc_loglik(ctx, model, y, N, theta, M, loglik_out, s);
        if (model->precision != SMC_PREC_FP32) return SMC_ERR_ARG;
        double sg = (double)model->sigma;
        double cst = (double)N * (-0.5 * d * std::log(2.0 * M_PI * sg * sg));
        smc::DiagLw2 lw2;
        for (int k = 0; k < 64; ++k)
            lw2.v[k] = k < K ? (float)((double)model->log_w[k] * smc::kLog2e) : 0.0f;
        size_t smem = (size_t)smc::kDiagPPB * K * d * sizeof(float) + K * sizeof(float);
        if (smem > 200 * 1024) return SMC_ERR_UNSUPPORTED;
        cudaFuncSetAttribute(smc::k_loglik_diag_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int64_t blocks = (M + smc::kDiagPPB - 1) / smc::kDiagPPB;
        float c2 = (float)(smc::kLog2e / (2.0 * sg * sg));
        smc::k_loglik_diag_fp32<<<(unsigned)blocks, 256, smem, s>>>(y, N, d, K, theta, M,
                                                                   loglik_out, c2, lw2, cst,
                                                                   ctx->d_status);
        return cuda_ok(cudaGetLastError());
    }
    smc::Gmm1dArgs P;
    int Kp;
    bool eqw;
    st = gmm1d_prepare(model, N, &P, &Kp, &eqw);
    if (st != SMC_OK) return st;
    P.wait_limit = ctx->wait_limit;
    if (M == 0) return SMC_OK;
    int L, threads;
    launch_shape(ctx, SMC_OP_LOGLIK, M, N, model->K, &L, &threads);
    int ppb = threads / L;
    int64_t blocks = (M + ppb - 1) / ppb;
    if (blocks > 0x7FFFFFFF) return SMC_ERR_ARG;
    bool g = grad_out != nullptr;
    const int Kr = model->K;
    uint32_t* sw = ctx->d_status;
    switch (Kp) {
        case 1: smc_host::dispatch_1d<1>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        case 2: smc_host::dispatch_1d<2>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        case 4: smc_host::dispatch_1d<4>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        case 8: smc_host::dispatch_1d<8>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        case 16: smc_host::dispatch_1d<16>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        case 32: smc_host::dispatch_1d<32>(g, eqw, (int)blocks, threads, s, y, N, theta, M, loglik_out, grad_out, P, L, Kr, sw); break;
        default: return SMC_ERR_UNSUPPORTED;
    }
    return cuda_ok(cudaGetLastError());
}
