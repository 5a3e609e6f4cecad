// diag_tc.cu -- diagonal d-dimensional mixture log-likelihood (Section 4.1's
// mixture with components N(mu_k, sigma^2 I_d)) with the mu . y contraction
// on the tensor cores.
//
// In log2 units, with alpha = log2(e) / sigma^2,
//   a_{n,pk} = log2 w_k - (alpha/2) (|y_n|^2 - 2 y_n . mu_pk + |mu_pk|^2)
//            = alpha S_{n,pk} + beta_pk - gamma_n,
//   S = y . mu,  beta_pk = log2 w_k - (alpha/2)|mu_pk|^2,  gamma_n = (alpha/2)|y_n|^2,
// so  log2 sum_k 2^a = LSE2_k(alpha S + beta) - gamma_n  and the gamma_n sum
// over the data is one constant for every particle.  alpha S + beta is a
// GEMM [N x (d+16)] . [(d+16) x M K] that is never stored: tcgen05.mma
// forms 128 data x 128 particle-components per instruction group in tensor
// memory from bf16 hi/lo splits of y and alpha mu (hi.hi + hi.lo + lo.hi,
// FP32 accumulation) plus one product of a constant ones column with beta
// split three ways in bf16 (24 bits), and the epilogue warps read the
// exponents back (tcgen05.ld) for the per-datum log-sum-exp over the K
// components of each particle and the sum over n.
//
// Kernels: k_dtc_prep_y / k_dtc_prep_mu convert y and mu to bf16 hi/lo in
// the tensor cores' no-swizzle K-major layout (8-row x 16-byte core
// matrices) and compute beta and the gamma sum; k_dtc_main is persistent,
// one CTA per SM, warp-specialised: warp 0 moves tiles with bulk async
// copies (cp.async.bulk, mbarrier completion), warp 1 issues the MMAs from
// one thread, warps 2..17 are the epilogue; k_dtc_combine adds the units
// of each particle in a fixed order.  Every wait is bounded; a timeout
// sets ST_TIMEOUT, drains what is in flight and ends the CTA.
#include <cmath>
#include <cstdint>

#include <cuda_bf16.h>

#include "ctx.hpp"
#include "device.cuh"

using namespace smc_host;

namespace smc {
namespace dtc {

constexpr int kRows = 128;     // data per tile = MMA M = TMEM lanes
constexpr int kHalf = 128;     // particle-components per MMA (N) and per TMEM buffer
constexpr int kBlockCols = 2 * kHalf;  // particle-components per particle block
constexpr int kStages = 4;     // ring of data tiles (at most; fewer at large d)
constexpr int kEpiWarps = 16;  // four warpgroups: (tile parity, half) each
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 512; // 4 buffers of 128 FP32 columns

// byte offset of element (r, j) of a rows x d bf16 block in the no-swizzle
// K-major layout: 8-row x 8-element core matrices of 128 contiguous bytes,
// K-adjacent core matrices 128 B apart, 8-row groups d * 16 B apart
__host__ __device__ inline uint32_t cm_off(int r, int j, int d) {
    return (uint32_t)((r >> 3) * (d * 16) + (j >> 3) * 128 + (r & 7) * 16 + (j & 7) * 2);
}

struct Lw2 {
    float v[32];  // log2 w_k, k < K (padding components: -inf)
};

// shared-memory plan (bytes from a 1024-aligned base)
constexpr uint32_t kOnesBytes = kRows * 16 * 2;       // ones operand: 128 rows x 16 bf16
constexpr uint32_t kBetaPart = kBlockCols * 16 * 2;   // beta operand: 256 rows x 16 bf16

struct Plan {
    uint32_t ypart;   // one bf16 part (hi or lo) of a data tile: 128 * d * 2
    uint32_t bpart;   // one part of a particle block: 256 * d * 2
    uint32_t bblock;  // a particle block in memory: hi, lo, beta parts
    uint32_t y0, b0, ones0, acc0, bar0, tmemslot, total;
    int ny, nb;       // data-tile stages (2..4) and particle-block buffers (1..2)
};

__host__ __device__ inline Plan plan(int d, int ppw, int ny, int nb) {
    Plan p;
    p.ny = ny;
    p.nb = nb;
    p.ypart = (uint32_t)(kRows * d * 2);
    p.bpart = (uint32_t)(kBlockCols * d * 2);
    p.bblock = 2 * p.bpart + kBetaPart;
    p.y0 = 0;
    p.b0 = p.y0 + (uint32_t)ny * 2 * p.ypart;
    p.ones0 = p.b0 + (uint32_t)nb * p.bblock;
    p.acc0 = p.ones0 + kOnesBytes;
    p.bar0 = p.acc0 + (uint32_t)(32 * kEpiWarps * ppw * 4);  // a float per thread and particle
    p.tmemslot = p.bar0 + 24 * 8;
    p.total = p.tmemslot + 16;
    return p;
}

// barrier slots
enum { B_FULL = 0, B_EMPTY = kStages, B_BFULL = 2 * kStages, B_BFREE = B_BFULL + 2,
       B_TFULL = B_BFREE + 2, B_TEMPTY = B_TFULL + 2, B_DRAIN = B_TEMPTY + 2, B_COUNT };
static_assert(B_COUNT <= 24, "barrier slots");

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(a), "r"(phase) : "memory");
    return done != 0;
}
// bounded wait for the phase with parity `phase` to complete; false on
// timeout, or early once another role has aborted (abort != nullptr)
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t phase, const volatile int* abort) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        if (mbar_test(a, phase)) return true;
        if (it > 256) {
            if (abort && *abort) return false;
            __nanosleep(128);
        }
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// shared-memory matrix descriptor, no swizzle, K-major: LBO = 128 B between
// K-adjacent core matrices, SBO = d * 16 B between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: bf16 A and B, FP32 D, both K-major,
// M = 128 data, N = 256 particle-components (one instruction per split
// product and K step covers the whole particle block)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kBlockCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(dtm), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}
// 16 columns of this warp's 32 lanes, without waiting: the registers are
// valid after tmem_wait()
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// waits for every tcgen05.ld of the thread; r (the last load's registers)
// is passed through so no use of them is scheduled before the wait
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ prep
// y -> bf16 hi/lo tiles (tile t: hi part then lo part, rows >= N zero) and
// per-block partial sums of |y_n|^2 (FP64).  One thread per row.
__global__ void __launch_bounds__(256) k_dtc_prep_y(const float* __restrict__ Y, int64_t N, int d,
                                                    int64_t ntiles, uint8_t* __restrict__ yt,
                                                    double* __restrict__ gpart) {
    __shared__ double red[8];
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (row < ntiles * kRows) {
        const int64_t t = row / kRows;
        const int r = (int)(row % kRows);
        uint8_t* hi = yt + (size_t)t * 2 * (kRows * d * 2);
        uint8_t* lo = hi + kRows * d * 2;
        for (int j0 = 0; j0 < d; j0 += 8) {
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float v0 = 0.0f, v1 = 0.0f;
                if (row < N) {
                    v0 = Y[row * d + j0 + e];
                    v1 = Y[row * d + j0 + e + 1];
                    sq += (double)v0 * v0 + (double)v1 * v1;
                }
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
                wh[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) |
                            ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                wl[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) |
                            ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            const uint32_t off = cm_off(r, j0, d);
            *reinterpret_cast<uint4*>(hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4*>(lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
    }
    sq = warp_sum_d(sq);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        gpart[blockIdx.x] = s;
    }
}

// alpha mu -> bf16 hi/lo particle blocks (block b: rows rho = p_local * KP
// + k; hi part, lo part, then the beta part: row rho holds beta_rho split
// into three bf16 (columns 0..2, rest 0)), beta = log2 w_k - (alpha/2)|mu|^2
// from the FP32 mu.  Padding components and particles beyond M: mu = 0 and
// beta = -1e30 (finite, so the splits stay finite; 2^(-1e30 - m) = 0).
__global__ void __launch_bounds__(256) k_dtc_prep_mu(const float* __restrict__ theta, int64_t M,
                                                     int K, int KP, int d, int64_t nblocks,
                                                     float alpha, Lw2 lw2,
                                                     uint8_t* __restrict__ bt) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nblocks * kBlockCols) return;
    const int64_t b = row / kBlockCols;
    const int rho = (int)(row % kBlockCols);
    const int64_t p = b * (kBlockCols / KP) + rho / KP;
    const int k = rho % KP;
    const bool real = p < M && k < K;
    const float* mu = theta + ((size_t)p * K + k) * d;
    const uint32_t bpart = kBlockCols * d * 2;
    uint8_t* hi = bt + (size_t)b * (2 * bpart + kBetaPart);
    uint8_t* lo = hi + bpart;
    uint8_t* bb = lo + bpart;
    float sq = 0.0f;
    for (int j0 = 0; j0 < d; j0 += 8) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float v0 = 0.0f, v1 = 0.0f;
            if (real) {
                v0 = mu[j0 + e];
                v1 = mu[j0 + e + 1];
            }
            sq = fmaf(v0, v0, sq);
            sq = fmaf(v1, v1, sq);
            v0 *= alpha;
            v1 *= alpha;
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
            wh[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            wl[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        const uint32_t off = cm_off(rho, j0, d);
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
    const float beta = real ? fmaf(-0.5f * alpha, sq, lw2.v[k]) : -1e30f;
    const __nv_bfloat16 b0 = __float2bfloat16_rn(beta);
    const float r1 = beta - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
    const uint32_t w0 = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
    const uint32_t w1 = (uint32_t)__bfloat16_as_ushort(b2);
    *reinterpret_cast<uint4*>(bb + cm_off(rho, 0, 16)) = make_uint4(w0, w1, 0u, 0u);
    *reinterpret_cast<uint4*>(bb + cm_off(rho, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------------ main
// Work unit u: particle block u / nsplit (256 particle-components), data
// tiles [split * T / nsplit, (split + 1) * T / nsplit), split = u % nsplit.
// partial[u][e][i] = sum over the unit's data seen by epilogue warp e (its
// lane quarter of every tile) of LSE2_k(alpha S + beta) for particle i of
// the warp's column quarter of the block.
template <int KP>
__global__ void __launch_bounds__(kThreads, 1) k_dtc_main(
    const uint8_t* __restrict__ yt, const uint8_t* __restrict__ bt, int64_t N, int d,
    int64_t ntiles, int nsplit, int64_t units, double* __restrict__ partial, uint32_t* status,
    int ny, int nbuf) {
    constexpr int PPW = 64 / KP;          // particles per epilogue warp
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                             ~(uintptr_t)1023);
    const Plan pl = plan(d, PPW, ny, nbuf);
    const int NY = pl.ny, NB = pl.nb;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar = smem_u32(sm + pl.bar0);
    auto B = [&](int i) { return bar + 8u * (uint32_t)i; };
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + pl.tmemslot);

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NY; ++s) {
            mbar_init(B(B_FULL + s), 1);
            mbar_init(B(B_EMPTY + s), 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(B(B_BFULL + j), 1);
            mbar_init(B(B_BFREE + j), 1);
            mbar_init(B(B_TFULL + j), 1);
            mbar_init(B(B_TEMPTY + j), kEpiWarps);
        }
        mbar_init(B(B_DRAIN), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the constant ones operand (columns 0..2 = 1, the rest 0) of the beta product
    for (int r = threadIdx.x; r < kRows; r += blockDim.x) {
        const uint32_t one2 = 0x3F803F80u;  // two bf16 ones
        *reinterpret_cast<uint4*>(sm + pl.ones0 + cm_off(r, 0, 16)) =
            make_uint4(one2, 0x3F80u, 0u, 0u);
        *reinterpret_cast<uint4*>(sm + pl.ones0 + cm_off(r, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
    }
    // written through the generic proxy, read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {  // tensor memory: 4 accumulator buffers of 128 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    volatile int* abort = &s_abort;
    auto fail = [&]() {
        raise_status(status, ST_TIMEOUT);
        *abort = 1;
    };

    const uint32_t tile_bytes = 2 * pl.ypart;
    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            // ring positions kept incrementally (no division in the loops):
            // stage s of fill round k for the data tiles, buffer bb of round
            // kb for the particle blocks
            int64_t it = 0;
            int ui = 0, s = 0, bb = 0;
            uint32_t k = 0, kb = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x, ++ui) {
                const int64_t pb = u / nsplit, sp = u % nsplit;
                if (kb > 0 && !mbar_wait(B(B_BFREE + bb), (kb - 1) & 1, abort)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(B(B_BFULL + bb), pl.bblock);
                bulk_g2s(smem_u32(sm + pl.b0 + bb * pl.bblock), bt + (size_t)pb * pl.bblock,
                         pl.bblock, B(B_BFULL + bb));
                if (++bb == NB) { bb = 0; ++kb; }
                const int64_t t0 = sp * ntiles / nsplit, t1 = (sp + 1) * ntiles / nsplit;
                for (int64_t t = t0; t < t1; ++t, ++it) {
                    if (k > 0 && !mbar_wait(B(B_EMPTY + s), (k - 1) & 1, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(B(B_FULL + s), tile_bytes);
                    bulk_g2s(smem_u32(sm + pl.y0 + s * tile_bytes), yt + (size_t)t * tile_bytes,
                             tile_bytes, B(B_FULL + s));
                    if (++s == NY) { s = 0; ++k; }
                }
            }
            if (!ok) fail();
            // drain: every copy issued has landed before the CTA ends (fill
            // number k of a stage or buffer completes phase k)
            for (int s = 0; s < NY; ++s)
                if (it > s) mbar_wait(B(B_FULL + s), (uint32_t)(((it - 1 - s) / NY) & 1), nullptr);
            for (int b2 = 0; b2 < NB; ++b2)
                if (ui > b2) mbar_wait(B(B_BFULL + b2), (uint32_t)(((ui - 1 - b2) / NB) & 1), nullptr);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int64_t it = 0;
            int ui = 0, s = 0, bb = 0;
            uint32_t k = 0, kb = 0;  // as the producer's
            bool ok = true;
            const uint32_t sbo = (uint32_t)d * 16u;
            const int ksteps = d / 16;
            for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x, ++ui) {
                const int64_t sp = u % nsplit;
                if (!mbar_wait(B(B_BFULL + bb), kb & 1, abort)) {
                    ok = false;
                    break;
                }
                const uint32_t bhi = smem_u32(sm + pl.b0 + bb * pl.bblock);
                const uint64_t dbhi = smem_desc(bhi, sbo);
                const uint64_t dblo = smem_desc(bhi + pl.bpart, sbo);
                const uint64_t dbeta = smem_desc(bhi + 2 * pl.bpart, 256u);
                const uint64_t dones = smem_desc(smem_u32(sm + pl.ones0), 256u);
                const int64_t t0 = sp * ntiles / nsplit, t1 = (sp + 1) * ntiles / nsplit;
                for (int64_t t = t0; t < t1; ++t, ++it) {
                    const int j = (int)(it & 1);
                    if (it >= 2 &&
                        !mbar_wait(B(B_TEMPTY + j), (uint32_t)(((it >> 1) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(B(B_FULL + s), k & 1, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors advance along K by 256 B = 16 address units
                    const uint64_t ahi = smem_desc(smem_u32(sm + pl.y0 + s * tile_bytes), sbo);
                    const uint64_t alo = ahi + (pl.ypart >> 4);
                    const uint32_t dtm = tbase + (uint32_t)(j * kBlockCols);
                    uint32_t acc = 0;
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t ko = (uint64_t)ks * 16u;
                        mma_bf16(dtm, ahi + ko, dbhi + ko, acc);
                        acc = 1;
                        mma_bf16(dtm, ahi + ko, dblo + ko, 1);
                        mma_bf16(dtm, alo + ko, dbhi + ko, 1);
                    }
                    // + beta: ones column times the three bf16 parts of beta
                    mma_bf16(dtm, dones, dbeta, 1);
                    mma_commit(B(B_EMPTY + s));
                    mma_commit(B(B_TFULL + j));
                    if (++s == NY) { s = 0; ++k; }
                }
                mma_commit(B(B_BFREE + bb));
                if (++bb == NB) { bb = 0; ++kb; }
            }
            if (!ok) fail();
            // every MMA issued has completed before tensor memory is freed
            mma_commit(B(B_DRAIN));
            mbar_wait(B(B_DRAIN), 0, nullptr);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // warp e reads lanes 32 q.. (q = its tensor-memory lane quarter) and
        // columns 64 cq.. (cq = e / 4) of every tile: PPW particles.  It copies
        // them to registers, releases the buffer at once (so the next MMA
        // group can start), then reduces.
        const int e = warp - 2;
        const int q = warp & 3;
        const int cq = e >> 2;
        int64_t it = 0;
        bool ok = true;
        float* sacc = reinterpret_cast<float*>(sm + pl.acc0) + (threadIdx.x - 64);
        for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const int64_t sp = u % nsplit;
            // per-thread sums of this unit in shared memory (registers are the
            // epilogue's limit), sacc[i * 512 + epilogue thread]: a few
            // flushes of 16 tiles each, so FP32 holds them to ~1e-7
#pragma unroll
            for (int i = 0; i < PPW; ++i) sacc[i * 32 * kEpiWarps] = 0.0f;
            // per particle: product of the per-datum sums (each in [1, KP])
            // and sum of the shifts over up to 16 tiles, then one lg2
            float pr[PPW], ms[PPW];
#pragma unroll
            for (int i = 0; i < PPW; ++i) { pr[i] = 1.0f; ms[i] = 0.0f; }
            int ngroup = 0;
            const int64_t t0 = sp * ntiles / nsplit, t1 = (sp + 1) * ntiles / nsplit;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                const int j = (int)(it & 1);
                if (!mbar_wait(B(B_TFULL + j), (uint32_t)((it >> 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tcol = tbase + ((uint32_t)(q * 32) << 16) +
                                      (uint32_t)(j * kBlockCols + cq * 64);
                uint32_t r[4][16];
#pragma unroll
                for (int c = 0; c < 4; ++c) tmem_ld16_async(tcol + (uint32_t)(c * 16), r[c]);
#pragma unroll
                for (int c = 0; c < 4; ++c) tmem_wait(r[c]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(B(B_TEMPTY + j));
                const bool valid = t * kRows + q * 32 + lane < N;
#pragma unroll
                for (int ip = 0; ip < PPW; ++ip) {
                    float a[KP];  // exponents alpha S + beta of one particle
#pragma unroll
                    for (int k = 0; k < KP; ++k)
                        a[k] = __uint_as_float(r[(ip * KP + k) >> 4][(ip * KP + k) & 15]);
                    float m = max3(a[0], a[1], a[2]);
#pragma unroll
                    for (int k = 3; k + 1 < KP; k += 2) m = max3(m, a[k], a[k + 1]);
                    if constexpr ((KP - 3) % 2 == 1) m = fmaxf(m, a[KP - 1]);
                    const float2 NM = make_float2(-m, -m);
                    float2 E[KP / 2];
#pragma unroll
                    for (int k = 0; k < KP / 2; ++k) {
                        const float2 x = __fadd2_rn(make_float2(a[2 * k], a[2 * k + 1]), NM);
                        E[k] = make_float2(ex2(x.x), ex2(x.y));
                    }
#pragma unroll
                    for (int w2 = 1; w2 < KP / 2; w2 <<= 1)
#pragma unroll
                        for (int k = 0; k + w2 < KP / 2; k += 2 * w2)
                            E[k] = __fadd2_rn(E[k], E[k + w2]);
                    if (valid) {
                        pr[ip] *= E[0].x + E[0].y;
                        ms[ip] += m;
                    }
                }
                if (++ngroup == 16) {  // 16 sums of at most KP <= 32 each: below 2^80
#pragma unroll
                    for (int i = 0; i < PPW; ++i) {
                        sacc[i * 32 * kEpiWarps] += ms[i] + lg2(pr[i]);
                        pr[i] = 1.0f;
                        ms[i] = 0.0f;
                    }
                    ngroup = 0;
                }
            }
            if (!ok) break;
#pragma unroll
            for (int i = 0; i < PPW; ++i) sacc[i * 32 * kEpiWarps] += ms[i] + lg2(pr[i]);
            // per-particle sums over the warp's lanes; the 4 warps of each
            // column quarter are added by k_dtc_combine in a fixed order
            double* dst = partial + ((size_t)u * kEpiWarps + e) * PPW;
#pragma unroll
            for (int i = 0; i < PPW; ++i) {
                const double vsum = warp_sum_d((double)sacc[i * 32 * kEpiWarps]);
                if (lane == 0) dst[i] = vsum;
            }
        }
        if (!ok) fail();
    }
    // ---------------------------------------------------------- teardown
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tbase), "r"(kTmemCols) : "memory");
}

// l_p = ln2 (sum over the units and warps of p - sum_n gamma_n) + N c0,
// added in a fixed order (splits, then the 4 warps of p's column quarter)
__global__ void __launch_bounds__(256) k_dtc_combine(const double* __restrict__ partial,
                                                     int nsplit, int kp, int64_t M,
                                                     const double* __restrict__ gpart, int ngpart,
                                                     double half_alpha, double ncst,
                                                     double* __restrict__ out, uint32_t* status) {
    __shared__ double red[256];
    double g = 0.0;
    for (int i = threadIdx.x; i < ngpart; i += blockDim.x) g += gpart[i];
    red[threadIdx.x] = g;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double gamma = half_alpha * red[0];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int ppb = kBlockCols / kp, ppw = 64 / kp;
    const int64_t pb = p / ppb;
    const int ib = (int)(p % ppb);
    const int cq = ib / ppw, i = ib % ppw;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) {
        const double* base = partial + ((size_t)(pb * nsplit + sp) * kEpiWarps) * ppw;
        for (int w = 0; w < 4; ++w) s += base[(size_t)(4 * cq + w) * ppw + i];
    }
    const double ll = (s - gamma) * kLn2 + ncst;
    if (ll != ll) raise_status(status, ST_NONFINITE);
    out[p] = ll;
}

}  // namespace dtc
}  // namespace smc

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// components padded to 4, 8, 16 or 32
int comp_pad(int K) { return K <= 4 ? 4 : (K <= 8 ? 8 : (K <= 16 ? 16 : 32)); }

// the deepest pipeline whose shared-memory plan fits one CTA (with 1 KiB of
// alignment slack): data-tile stages 4..2 with two particle-block buffers,
// then 4..2 with one
bool pick_plan(const smc_ctx* ctx, int d, int ppw, int* ny, int* nb) {
    const size_t cap = ctx->smem_optin > 0 ? (size_t)ctx->smem_optin : (size_t)227 * 1024;
    for (int b = 2; b >= 1; --b)
        for (int y = smc::dtc::kStages; y >= 2; --y)
            if (smc::dtc::plan(d, ppw, y, b).total + 1024 + 1088 <= cap) {  // + static shared memory
                *ny = y;
                *nb = b;
                return true;
            }
    return false;
}

template <int KP>
smc_status launch_main(const smc_ctx* ctx, int64_t grid, size_t smem, const uint8_t* yt,
                       const uint8_t* bt, int64_t N, int d, int64_t ntiles, int nsplit,
                       int64_t units, double* partial, cudaStream_t s, int ny, int nb) {
    auto kern = smc::dtc::k_dtc_main<KP>;
    cudaFuncAttributes fa;
    SMC_CUDA(cudaFuncGetAttributes(&fa, kern));
    if (fa.maxThreadsPerBlock < smc::dtc::kThreads) return SMC_ERR_UNSUPPORTED;
    SMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, smc::dtc::kThreads, smem, s>>>(yt, bt, N, d, ntiles, nsplit, units,
                                                         partial, ctx->d_status, ny, nb);
    return cuda_ok(cudaGetLastError());
}

}  // namespace

// Workspace bytes of one call (data tiles, particle blocks, beta, partials).
size_t smc_diag_tc_ws_bytes(int64_t N, int64_t M, int K, int d, int sms) {
    using namespace smc::dtc;
    const int KP = comp_pad(K);
    const int64_t ntiles = (N + kRows - 1) / kRows;
    const int64_t nblocks = (M + kBlockCols / KP - 1) / (kBlockCols / KP);
    int nsplit = 1;
    while (nblocks * nsplit < 4 * (int64_t)sms && ntiles / (2 * nsplit) >= 8) nsplit *= 2;
    const int64_t units = nblocks * nsplit;
    const int64_t gblocks = (ntiles * kRows + 255) / 256;
    size_t b = 0;
    b += align_up((size_t)ntiles * 2 * kRows * d * 2, 1024);
    b += align_up((size_t)nblocks * (2 * kBlockCols * d * 2 + kBetaPart), 1024);
    b += align_up((size_t)gblocks * 8, 1024);
    b += align_up((size_t)units * kEpiWarps * (64 / KP) * 8, 1024);
    return b;
}

smc_status smc_diag_tc_loglik(smc_ctx* ctx, const smc_gmm* model, const float* Y, int64_t N,
                              const float* theta, int64_t M, double* out, cudaStream_t s) {
    using namespace smc::dtc;
    const int K = model->K, d = model->d;
    // tensor-core path: K <= 32 components, d a multiple of 16 up to 64
    if (K < 1 || K > 32 || d < 16 || d > 64 || d % 16 != 0) return SMC_ERR_UNSUPPORTED;
    // the shared-memory plan: as many data-tile stages and particle-block
    // buffers as fit (4 and 2 up to d = 32; fewer at d = 48, 64)
    const int KP = comp_pad(K);
    int ny = 0, nb = 0;
    if (!pick_plan(ctx, d, 64 / KP, &ny, &nb)) return SMC_ERR_UNSUPPORTED;
    if (N == 0) return cuda_ok(cudaMemsetAsync(out, 0, (size_t)M * sizeof(double), s));
    const int64_t ntiles = (N + kRows - 1) / kRows;
    const int64_t nblocks = (M + kBlockCols / KP - 1) / (kBlockCols / KP);
    int nsplit = 1;
    while (nblocks * nsplit < 4 * (int64_t)ctx->num_sms && ntiles / (2 * nsplit) >= 8) nsplit *= 2;
    const int64_t units = nblocks * nsplit;
    const int64_t gblocks = (ntiles * kRows + 255) / 256;
    if (units > 0x7FFFFFFF || gblocks > 0x7FFFFFFF) return SMC_ERR_ARG;
    smc_status st = ensure_ws(ctx, smc_diag_tc_ws_bytes(N, M, K, d, ctx->num_sms), s);
    if (st != SMC_OK) return st;
    uint8_t* w = static_cast<uint8_t*>(ctx->ws);
    uint8_t* yt = w;
    w += align_up((size_t)ntiles * 2 * kRows * d * 2, 1024);
    uint8_t* bt = w;
    w += align_up((size_t)nblocks * (2 * kBlockCols * d * 2 + kBetaPart), 1024);
    double* gpart = reinterpret_cast<double*>(w);
    w += align_up((size_t)gblocks * 8, 1024);
    double* partial = reinterpret_cast<double*>(w);

    const double sg = (double)model->sigma;
    const double alpha = smc::kLog2e / (sg * sg);
    Lw2 lw2;
    for (int k = 0; k < 32; ++k)
        lw2.v[k] = k < K ? (float)((double)model->log_w[k] * smc::kLog2e) : -INFINITY;
    k_dtc_prep_y<<<(unsigned)gblocks, 256, 0, s>>>(Y, N, d, ntiles, yt, gpart);
    SMC_CUDA(cudaGetLastError());
    k_dtc_prep_mu<<<(unsigned)((nblocks * kBlockCols + 255) / 256), 256, 0, s>>>(
        theta, M, K, KP, d, nblocks, (float)alpha, lw2, bt);
    SMC_CUDA(cudaGetLastError());
    const Plan pl = plan(d, 64 / KP, ny, nb);
    // + alignment slack; at least half an SM's shared memory so that one CTA
    // (and one 512-column tensor-memory allocation) runs per SM
    size_t smem = pl.total + 1024;
    if (ctx->smem_per_sm > 0 && smem < (size_t)ctx->smem_per_sm / 2 + 1024)
        smem = (size_t)ctx->smem_per_sm / 2 + 1024;
    int64_t grid = units < ctx->num_sms ? units : ctx->num_sms;
    switch (KP) {
        case 4: st = launch_main<4>(ctx, grid, smem, yt, bt, N, d, ntiles, nsplit, units, partial, s, ny, nb); break;
        case 8: st = launch_main<8>(ctx, grid, smem, yt, bt, N, d, ntiles, nsplit, units, partial, s, ny, nb); break;
        case 16: st = launch_main<16>(ctx, grid, smem, yt, bt, N, d, ntiles, nsplit, units, partial, s, ny, nb); break;
        default: st = launch_main<32>(ctx, grid, smem, yt, bt, N, d, ntiles, nsplit, units, partial, s, ny, nb); break;
    }
    if (st != SMC_OK) return st;
    const double ncst = (double)N * (-0.5 * d * std::log(2.0 * M_PI * sg * sg));
    k_dtc_combine<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(partial, nsplit, KP, M,
                                                              gpart, (int)gblocks, 0.5 * alpha,
                                                              ncst, out, ctx->d_status);
    return cuda_ok(cudaGetLastError());
}
