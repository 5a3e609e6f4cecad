// is.cu -- smc_is_moments: importance-sampling sums for a one-dimensional
// Gaussian-mixture target and a Gaussian proposal (Section 2.1's worked
// example; Section 3: w = target / proposal).
//
// One pass over the draws (read from device memory, or drawn on the device
// from Philox), everything per draw in FP32: log p by a shifted
// log-sum-exp over the components, log q, w = exp(log p - log q),
// phi = x^power.  Groups of eight draws are summed in FP32 and the group
// sums in FP64; blocks combine in a fixed order and the last block to
// finish adds the block partials in a fixed order, so the result has the
// same bits on every run (for a given grid).
#include "ctx.hpp"
#include "device.cuh"

using namespace smc_host;

namespace smc {

struct IsArgs {
    int K;
    float mu[8];
    float la2[8];    // log2 a_k - log2 sqrt(2 pi var)
    float c2;        // log2(e) / (2 var)
    float pm, rps;   // proposal mean, 1 / sd
    float lq2;       // -log2(sd sqrt(2 pi))
    int power;
};

constexpr int kIsGroup = 8;

__device__ __forceinline__ float is_x(const float* __restrict__ x, int64_t i, const IsArgs& A,
                                      uint64_t seed, uint64_t step, float ps) {
    if (x) return x[i];
    const uint4 w = draw(seed, RNG_PROPOSAL, step, (uint32_t)i, 0u);
    float z0, z1;
    box_muller(w.x, w.y, z0, z1);
    return fmaf(ps, z0, A.pm);
}

// w and w phi of one draw (KP components: the real ones, then padding with
// weight zero, whose terms ex2 flushes to zero)
template <int KP>
__device__ __forceinline__ void is_term(float xi, const IsArgs& A, float& w, float& wphi) {
    float t[KP], m = -INFINITY;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const float d = xi - A.mu[k];
        t[k] = fmaf(-A.c2, d * d, A.la2[k]);
        m = fmaxf(m, t[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KP; ++k) s += ex2(t[k] - m);
    const float dq = (xi - A.pm) * A.rps;
    const float lq = fmaf(-0.72134752044448170368f, dq * dq, A.lq2);  // -log2(e)/2 dq^2 + lq2
    w = ex2(m + lg2(s) - lq);
    float phi = 1.0f;
    for (int e = 0; e < A.power; ++e) phi *= xi;
    wphi = w * phi;
}

template <int KP>
__global__ void __launch_bounds__(256, 4) k_is_moments(IsArgs A, const float* __restrict__ x,
                                                    int64_t N, uint64_t seed, uint64_t step,
                                                    float ps, double* __restrict__ partials,
                                                    unsigned long long* ticket,
                                                    double* __restrict__ out) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    __shared__ double s_p[3][8];
    __shared__ bool last;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t ngroups = (N + kIsGroup - 1) / kIsGroup;
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        // draws in memory, 16-byte aligned: the whole groups are software
        // pipelined (the next group's two 16-byte loads are issued before
        // this group's arithmetic, so a load is always in flight)
        const int64_t nfull = N / kIsGroup;
        const float4* xv = reinterpret_cast<const float4*>(x);
        float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
        if (g < nfull) {
            n0 = __ldcs(xv + 2 * g);
            n1 = __ldcs(xv + 2 * g + 1);
        }
        for (; g < nfull; g += G) {
            const float4 v0 = n0, v1 = n1;
            if (g + G < nfull) {
                n0 = __ldcs(xv + 2 * (g + G));
                n1 = __ldcs(xv + 2 * (g + G) + 1);
            }
            const float xs[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
#pragma unroll
            for (int j = 0; j < kIsGroup; ++j) {
                float w, wp;
                is_term<KP>(xs[j], A, w, wp);
                f0 += w;
                f1 += wp;
                f2 = fmaf(w, w, f2);
            }
            a0 += (double)f0;
            a1 += (double)f1;
            a2 += (double)f2;
        }
        // g is now this thread's first group at or past nfull: the partial
        // last group (N not a multiple of 8) goes to the generic loop below
    }
    for (; g < ngroups; g += G) {
        float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
        const int64_t i0 = g * kIsGroup;
        for (int j = 0; j < kIsGroup && i0 + j < N; ++j) {
            float w, wp;
            is_term<KP>(is_x(x, i0 + j, A, seed, step, ps), A, w, wp);
            f0 += w;
            f1 += wp;
            f2 = fmaf(w, w, f2);
        }
        a0 += (double)f0;
        a1 += (double)f1;
        a2 += (double)f2;
    }
    // fixed-order block combine: warp trees, then warps in index order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, o);
        a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
        a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_p[0][wid] = a0;
        s_p[1][wid] = a1;
        s_p[2][wid] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b0 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            b0 += s_p[0][w];
            b1 += s_p[1][w];
            b2 += s_p[2][w];
        }
        double* P = partials + (size_t)blockIdx.x * 8;
        P[0] = b0;
        P[1] = b1;
        P[2] = b2;
        __threadfence();
        last = atomicAdd(ticket, 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block adds the partials: thread t takes blocks t, t + 256, ...
    // in order, then the same fixed-order combine as above
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        t0 += __ldcg(partials + (size_t)b * 8 + 0);
        t1 += __ldcg(partials + (size_t)b * 8 + 1);
        t2 += __ldcg(partials + (size_t)b * 8 + 2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xFFFFFFFFu, t0, o);
        t1 += __shfl_xor_sync(0xFFFFFFFFu, t1, o);
        t2 += __shfl_xor_sync(0xFFFFFFFFu, t2, o);
    }
    __syncthreads();  // s_p reused
    if ((threadIdx.x & 31) == 0) {
        s_p[0][wid] = t0;
        s_p[1][wid] = t1;
        s_p[2][wid] = t2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b0 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            b0 += s_p[0][w];
            b1 += s_p[1][w];
            b2 += s_p[2][w];
        }
        out[0] = b0;
        out[1] = b1;
        out[2] = b2;
        *ticket = 0ull;
    }
}

}  // namespace smc

extern "C" smc_status smc_is_moments(smc_ctx* ctx, const smc_is_problem* prob, const float* x,
                                     int64_t N, uint64_t seed, uint64_t step, double* out,
                                     void* stream) {
    if (!ctx || !prob || N < 0 || !out) return SMC_ERR_ARG;
    if (prob->K < 1 || prob->K > 8 || !(prob->var > 0.0f) || !(prob->prop_sd > 0.0f) ||
        prob->power < 0 || prob->power > 8)
        return SMC_ERR_ARG;
    for (int k = 0; k < prob->K; ++k)
        if (!(prob->a[k] > 0.0f)) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    smc::IsArgs A;
    const double l2e = 1.4426950408889634;
    const double v = (double)prob->var, ps = (double)prob->prop_sd;
    A.K = prob->K;
    for (int k = 0; k < 8; ++k) {  // padding components: weight 0 (log2 = -inf)
        A.mu[k] = k < A.K ? prob->mu[k] : 0.0f;
        A.la2[k] = k < A.K ? (float)(std::log2((double)prob->a[k]) -
                                     0.5 * std::log2(2.0 * M_PI * v))
                           : -INFINITY;
    }
    A.c2 = (float)(l2e / (2.0 * v));
    A.pm = prob->prop_mean;
    A.rps = (float)(1.0 / ps);
    A.lq2 = (float)(-std::log2(ps * std::sqrt(2.0 * M_PI)));
    A.power = prob->power;
    cudaStream_t s = as_stream(stream);
    int64_t blocks = (N + 256 * smc::kIsGroup - 1) / (256 * smc::kIsGroup);
    int64_t cap = (int64_t)ctx->num_sms * 4;  // one resident wave
    if (cap > kMaxPartialBlocks) cap = kMaxPartialBlocks;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    auto kern = A.K <= 1 ? smc::k_is_moments<1>
                : A.K <= 2 ? smc::k_is_moments<2>
                : A.K <= 4 ? smc::k_is_moments<4> : smc::k_is_moments<8>;
    return launch_pdl(kern, dim3((unsigned)blocks), dim3(256), 0, s, A, x, N, seed, step,
                      prob->prop_sd, ctx->d_partials, ctx->d_counters + CNT_IS_TICKET, out);
}
