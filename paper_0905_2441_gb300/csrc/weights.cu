// weights.cu -- smc_reweight and smc_ess: incremental weights, FP64
// normalisation, log-evidence increment and effective sample size
// (Section 3: W = w / sum w; Section 4.1.2: incremental weight
// exp(dbeta l(x)); Section 3.2: ESS).
//
// One grid-stride pass reads l and logw, writes the new logw and reduces
// (max, sum e, sum e^2) of the new log-weights and (max, sum e) of the old
// ones online; the last block to finish combines the per-block partials
// and writes the scalars.  A second pass writes W = e / S1.  Per element the
// only FP64 instructions are the logw update and one subtraction; the
// exponential runs in FP32 on the exactly split difference.
#include <cmath>

#include "ctx.hpp"
#include "device.cuh"

using namespace smc_host;

namespace smc {

// exp(x) for an FP64 x <= 0, FP32 accuracy, as float
__device__ __forceinline__ float expd(double x) {
    float hi, lo;
    split_double(x, hi, lo);
    return exp_hilo(hi, lo);
}

// thread-level online accumulator: m is the running max, s1 = sum e^(x-m),
// s2 = sum e^(2(x-m))
struct OnlineLse {
    double m = -INFINITY;
    float s1 = 0.0f, s2 = 0.0f;
    __device__ __forceinline__ void add(double x) {
        if (dkey(x) > dkey(m)) {
            float f = (m == -INFINITY) ? 0.0f : expd(m - x);
            s1 = fmaf(s1, f, 1.0f);
            s2 = fmaf(s2, f * f, 1.0f);
            m = x;
        } else if (x != -INFINITY) {
            float e = expd(x - m);
            s1 += e;
            s2 = fmaf(e, e, s2);
        }
    }
};

// block / grid level: FP64 sums
struct Lse {
    double m, s1, s2;
};

__device__ __forceinline__ Lse lse_merge(Lse a, Lse b) {
    if (b.m == -INFINITY) return a;
    if (a.m == -INFINITY) return b;
    if (dkey(b.m) > dkey(a.m)) { Lse t = a; a = b; b = t; }
    double f = (double)expd(b.m - a.m);
    a.s1 += b.s1 * f;
    a.s2 += b.s2 * f * f;
    return a;
}

__device__ __forceinline__ Lse warp_merge(Lse v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Lse w;
        w.m = __shfl_xor_sync(0xFFFFFFFFu, v.m, o);
        w.s1 = __shfl_xor_sync(0xFFFFFFFFu, v.s1, o);
        w.s2 = __shfl_xor_sync(0xFFFFFFFFu, v.s2, o);
        v = lse_merge(v, w);
    }
    return v;
}

// merge a value across the block; result valid in every thread
__device__ __forceinline__ Lse block_merge(Lse v, Lse* sh /* [32] */) {
    v = warp_merge(v);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        Lse t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : Lse{-INFINITY, 0.0, 0.0};
        t = warp_merge(t);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    Lse r = sh[0];
    __syncthreads();
    return r;
}

// partial slot layout (doubles): [b*8 + 0..4] = {m, s1, s2, m_old, s_old}
// final slot at kMaxPartialBlocks-1: {m, S1, S2, valid, lse, ...}
__global__ void __launch_bounds__(256) k_reweight_reduce(const double* __restrict__ ll,
                                                         double dbeta, double* __restrict__ lw,
                                                         int64_t M, int has_inc,
                                                         double* __restrict__ partials,
                                                         unsigned long long* ticket,
                                                         double* __restrict__ scalars,
                                                         int32_t* __restrict__ flag,
                                                         double ess_frac, int final_slot,
                                                         uint32_t* status) {
    __shared__ Lse sh[32];
    __shared__ bool last;
    OnlineLse cur, old;
    bool nan_seen = false;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        double x = lw[i];
        if (has_inc) {
            double v = ll[i];
            nan_seen |= disnan(x) | disnan(v);
            old.add(x);
            x = fma(dbeta, v, x);
            lw[i] = x;
        }
        nan_seen |= disnan(x);
        cur.add(x);
    }
    if (nan_seen) raise_status(status, ST_NONFINITE);
    Lse c = block_merge(Lse{cur.m, (double)cur.s1, (double)cur.s2}, sh);
    Lse o = has_inc ? block_merge(Lse{old.m, (double)old.s1, 0.0}, sh) : Lse{-INFINITY, 0.0, 0.0};
    if (threadIdx.x == 0) {
        double* P = partials + (size_t)blockIdx.x * 8;
        P[0] = c.m; P[1] = c.s1; P[2] = c.s2; P[3] = o.m; P[4] = o.s1;
        __threadfence();
        unsigned long long t = atomicAdd(ticket, 1ull);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last block: combine every partial
    Lse tc{-INFINITY, 0.0, 0.0}, to{-INFINITY, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        volatile double* P = partials + (size_t)b * 8;
        tc = lse_merge(tc, Lse{P[0], P[1], P[2]});
        to = lse_merge(to, Lse{P[3], P[4], 0.0});
    }
    tc = block_merge(tc, sh);
    to = block_merge(to, sh);
    if (threadIdx.x == 0) {
        *ticket = 0ull;
        double* F = partials + (size_t)final_slot * 8;
        bool valid = tc.m != -INFINITY && !disnan(tc.m);
        if (!valid) {
            if (!disnan(tc.m)) raise_status(status, ST_ZERO_WEIGHT);
            F[3] = 0.0;
            if (flag) *flag = 0;
            return;
        }
        double lse = tc.m + log(tc.s1);
        double ess = tc.s1 * tc.s1 / tc.s2;
        F[0] = tc.m; F[1] = tc.s1; F[2] = tc.s2; F[3] = 1.0; F[4] = lse;
        if (scalars) {
            double inc = 0.0;
            if (has_inc) inc = lse - (to.m + log(to.s1));
            scalars[0] = inc;
            scalars[1] = ess;
            scalars[2] = tc.m;
            scalars[3] = lse;
        }
        if (flag) *flag = (ess < ess_frac * (double)M) ? 1 : 0;
    }
}

// W_i = exp(lw_i - m) / S1, computed in FP32 on the exact FP64 difference;
// values below 2^-126 are written as 0.
__global__ void __launch_bounds__(256) k_reweight_normalize(const double* __restrict__ lw,
                                                            int64_t M,
                                                            const double* __restrict__ fin,
                                                            double* __restrict__ W) {
    if (fin[3] == 0.0) return;
    const double m = fin[0];
    const float inv = (float)(1.0 / fin[1]);
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        float e = expd(lw[i] - m);
        W[i] = f2d_bits(e * inv);
    }
}

__global__ void __launch_bounds__(256) k_ess_reduce(const double* __restrict__ lw, int64_t M,
                                                    double* __restrict__ partials,
                                                    unsigned long long* ticket,
                                                    double* __restrict__ ess_out,
                                                    uint32_t* status) {
    __shared__ Lse sh[32];
    __shared__ bool last;
    OnlineLse cur;
    bool nan_seen = false;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        double x = lw[i];
        nan_seen |= disnan(x);
        cur.add(x);
    }
    if (nan_seen) raise_status(status, ST_NONFINITE);
    Lse c = block_merge(Lse{cur.m, (double)cur.s1, (double)cur.s2}, sh);
    if (threadIdx.x == 0) {
        double* P = partials + (size_t)blockIdx.x * 8;
        P[0] = c.m; P[1] = c.s1; P[2] = c.s2;
        __threadfence();
        unsigned long long t = atomicAdd(ticket, 1ull);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Lse tc{-INFINITY, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        volatile double* P = partials + (size_t)b * 8;
        tc = lse_merge(tc, Lse{P[0], P[1], P[2]});
    }
    tc = block_merge(tc, sh);
    if (threadIdx.x == 0) {
        *ticket = 0ull;
        if (tc.m == -INFINITY) {
            raise_status(status, ST_ZERO_WEIGHT);
            return;
        }
        *ess_out = tc.s1 * tc.s1 / tc.s2;
    }
}

}  // namespace smc

namespace smc_host {

static int reduce_blocks(const smc_ctx* ctx, int64_t M) {
    int64_t b = (M + 256 * 8 - 1) / (256 * 8);
    int64_t cap = (int64_t)ctx->num_sms * 8;
    if (cap > kMaxPartialBlocks - 2) cap = kMaxPartialBlocks - 2;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace smc_host

extern "C" smc_status smc_reweight(smc_ctx* ctx, const double* loglik, double dbeta,
                                   double* logw, int64_t M, double* W_out, double* scalars_out,
                                   int32_t* resample_flag_out, double ess_frac, void* stream) {
    if (!ctx || M <= 0 || !logw || std::isnan(dbeta) || std::isnan(ess_frac)) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    int has_inc = (loglik != nullptr && dbeta != 0.0) ? 1 : 0;
    int blocks = reduce_blocks(ctx, M);
    const int final_slot = kMaxPartialBlocks - 1;
    smc::k_reweight_reduce<<<blocks, 256, 0, s>>>(loglik, dbeta, logw, M, has_inc, ctx->d_partials,
                                                  ctx->d_counters + CNT_REWEIGHT_TICKET, scalars_out,
                                                  resample_flag_out, ess_frac, final_slot,
                                                  ctx->d_status);
    SMC_CUDA(cudaGetLastError());
    if (W_out) {
        int nb = (int)((M + 255) / 256);
        int cap = ctx->num_sms * 16;
        if (nb > cap) nb = cap;
        smc::k_reweight_normalize<<<nb, 256, 0, s>>>(logw, M,
                                                     ctx->d_partials + (size_t)final_slot * 8, W_out);
        SMC_CUDA(cudaGetLastError());
    }
    return SMC_OK;
}

extern "C" smc_status smc_ess(smc_ctx* ctx, const double* logw, int64_t M, double* ess_out,
                              void* stream) {
    if (!ctx || M <= 0 || !logw || !ess_out) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    int blocks = reduce_blocks(ctx, M);
    smc::k_ess_reduce<<<blocks, 256, 0, s>>>(logw, M, ctx->d_partials,
                                             ctx->d_counters + CNT_ESS_TICKET, ess_out,
                                             ctx->d_status);
    return cuda_ok(cudaGetLastError());
}
