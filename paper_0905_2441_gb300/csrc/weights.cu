// weights.cu -- smc_reweight and smc_ess: incremental weights, FP64
// normalisation, log-evidence increment and effective sample size
// (Section 3: W = w / sum w; Section 4.1.2: incremental weight
// exp(dbeta l(x)); Section 3.2: ESS).
//
// One grid-stride pass reads l and logw, writes the new logw and reduces
// (sum e, sum e^2) of the new log-weights and (sum e) of the old ones
// against slack references, plus the exact maximum (integer keys), into
// per-block partials.  A second pass writes W = e / S1 (smc_reweight_resample:
// the same pass also forms the exact tile sums of pass 1 of systematic
// resampling from the W it writes); every block of that pass combines the
// partials itself while its first tiles load, and its block 0 writes the
// scalars.  Without a second pass the reduction's last block combines them.
// Per element the only FP64 instruction is the log-weight update (GB300
// issues FP64 at ~1/64 of FP32); differences and exponentials run in FP32
// on hi/lo splits.
#include <climits>
#include <cmath>

#include "ctx.hpp"
#include "device.cuh"
#include "resample.cuh"
#include "reweight.cuh"
#include "bulk.cuh"

using namespace smc_host;

namespace smc {

// partial slot layout (doubles): [b*8 + 0..5] = {ref, s1, s2, ref_old, s_old, max}
// final slot: {max, S1, S2, valid, lse, (float) 1/S1 in the low word of [5]},
// S1 and S2 relative to the true maximum
__global__ void __launch_bounds__(256, 2) k_reweight_reduce(const double* __restrict__ ll,
                                                         double dbeta, double* __restrict__ lw,
                                                         int64_t M, int has_inc,
                                                         double* __restrict__ partials,
                                                         unsigned long long* ticket, int defer,
                                                         double* __restrict__ scalars,
                                                         int32_t* __restrict__ flag,
                                                         double ess_frac, int final_slot,
                                                         uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    RefSums cur, old;
    bool nan_seen = false;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // chunks of 8 only when every thread gets one (large M); otherwise one
    // element per thread keeps each thread's dependent chain short
    const bool vec = aligned16(lw) && (!has_inc || aligned16(ll)) && M >= G * kChunk;
    const int64_t nchunk = vec ? M / kChunk : 0;
    // the new log-weights stay in L2 in preference to the data read once
    // (the normalisation reads them back, last written first)
    const uint64_t keep = l2_evict_last_policy();
    // the next chunk's loads are issued before this chunk's arithmetic
    double xn[kChunk], vn[kChunk];
    if (t0 < nchunk) {
        load8_cs(lw + t0 * kChunk, xn);
        if (has_inc) load8_cs(ll + t0 * kChunk, vn);
    }
    for (int64_t ch = t0; ch < nchunk; ch += G) {
        double x[kChunk], v[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            x[j] = xn[j];
            v[j] = vn[j];
        }
        if (ch + G < nchunk) {
            load8_cs(lw + (ch + G) * kChunk, xn);
            if (has_inc) load8_cs(ll + (ch + G) * kChunk, vn);
        }
        if (has_inc) {
            double n[kChunk];
#pragma unroll
            for (int j = 0; j < kChunk; ++j) {
                n[j] = fma(dbeta, v[j], x[j]);
                nan_seen |= disnan(n[j]);  // a NaN in x or v makes n NaN
            }
            store8_keep(lw + ch * kChunk, n, keep);
            add8(old, x, false);
            add8(cur, n, true);
        } else {
#pragma unroll
            for (int j = 0; j < kChunk; ++j) nan_seen |= disnan(x[j]);
            add8(cur, x, true);
        }
    }
    for (int64_t i = nchunk * kChunk + t0; i < M; i += G) {  // tail / unaligned
        const double x = lw[i];
        nan_seen |= disnan(x);
        if (has_inc) {
            const double v = ll[i];
            const double n = fma(dbeta, v, x);
            nan_seen |= disnan(v) | disnan(n);
            lw[i] = n;
            old.add(x);
            cur.add(n);
        } else {
            cur.add(x);
        }
    }
    if (nan_seen) raise_status(status, ST_NONFINITE);
    reweight_finish(cur, old, has_inc, M, partials, ticket, defer, scalars, flag, ess_frac,
                    final_slot, status);
}

// W_i = exp(lw_i - m) / S1 with the difference taken on float hi/lo splits
// as in RefSums (no FP64 instruction per element); values below 2^-126 are
// written as 0.
__global__ void __launch_bounds__(256) k_reweight_normalize(const double* __restrict__ lw,
                                                            int64_t M, RwArgs rw,
                                                            double* __restrict__ W,
                                                            uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const RwFinal fin = rw_final(rw, status);
    if (!fin.valid) return;
    float mh, ml;
    split_double(fin.m, mh, ml);
    const float inv = fin.inv;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nchunk = (aligned16(lw) && aligned16(W)) ? M / kChunk : 0;
    // descending: the reduction wrote the log-weights ascending, so the most
    // recently written ones (still in L2) come first
    for (int64_t k = t0; k < nchunk; k += G) {
        const int64_t ch = nchunk - 1 - k;
        double x[kChunk], w[kChunk];
        load8_cs(lw + ch * kChunk, x);
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            float xh, xl;
            split_double(x[j], xh, xl);
            w[j] = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
        }
        store8(W + ch * kChunk, w);
    }
    for (int64_t i = nchunk * kChunk + t0; i < M; i += G) {
        float xh, xl;
        split_double(lw[i], xh, xl);
        W[i] = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
    }
}

// k_reweight_normalize with the tiles moved by bulk copies: whole tiles of
// kNrmTile log-weights are loaded into a ring of kNrmStages shared-memory
// buffers (one cp.async.bulk each, completion on an mbarrier), turned into
// weights in shared memory and stored back by one bulk copy per tile, so a
// tile costs two memory instructions instead of 2 x 4 per thread per 8
// elements (the per-thread form is throttled by the load/store queues).
// Tiles are taken in descending order (the reduction wrote the log-weights
// ascending: the most recent, still in L2, come first); the elements past
// the last whole tile take the per-thread form.  Same values as
// k_reweight_normalize.
constexpr int kNrmThreads = 256;
constexpr int kNrmTile = 2048;  // doubles: 16 KB
constexpr int kNrmStages = 3;
constexpr size_t kNrmSmem = (size_t)(kNrmStages + 2) * kNrmTile * sizeof(double) + 64;
__global__ void __launch_bounds__(kNrmThreads) k_reweight_normalize_bulk(
    const double* __restrict__ lw, int64_t M, RwArgs rw, double* __restrict__ W,
    uint32_t* status, uint32_t limit) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    extern __shared__ __align__(128) double nsm[];
    double* in = nsm;                               // [kNrmStages][kNrmTile]
    double* out = nsm + kNrmStages * kNrmTile;      // [2][kNrmTile]
    uint64_t* full = reinterpret_cast<uint64_t*>(out + 2 * kNrmTile);
    const int tid = threadIdx.x;
    const int64_t ntiles = M / kNrmTile;
    const int64_t nmine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t k) { return ntiles - 1 - (blockIdx.x + k * gridDim.x); };
    constexpr uint32_t kBytes = kNrmTile * sizeof(double);
    const uint64_t drop = l2_evict_first_policy();  // the log-weights' last read
    if (tid == 0) {
        for (int st = 0; st < kNrmStages; ++st) mb_init(&full[st], 1);
        mb_init_fence();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < kNrmStages && k < nmine; ++k) {
            mb_expect_tx(&full[k], kBytes);
            bulk_load_hint(in + k * kNrmTile, lw + tile_of(k) * kNrmTile, kBytes, &full[k], drop);
        }
    // the normalisation constants, while the first tiles load
    const RwFinal fin = rw_final(rw, status);
    if (!fin.valid) {  // no weights to write: let the loads in flight land first
        for (int k = 0; k < kNrmStages && k < nmine; ++k) mb_wait(&full[k], 0, status, limit);
        return;
    }
    float mh, ml;
    split_double(fin.m, mh, ml);
    const float inv = fin.inv;
    int st = 0;
    uint32_t round = 0;
    for (int64_t k = 0; k < nmine; ++k) {
        const int ob = (int)(k & 1);
        mb_wait(&full[st], round & 1, status, limit);
        if (tid == 0 && k >= 2) bulk_wait_read<1>();  // out[ob]'s last store has read it
        __syncthreads();
        const double2* src = reinterpret_cast<const double2*>(in + st * kNrmTile);
        double2* dst = reinterpret_cast<double2*>(out + ob * kNrmTile);
#pragma unroll
        for (int j = 0; j < kNrmTile / 2 / kNrmThreads; ++j) {
            const double2 x = src[tid + j * kNrmThreads];
            float h0, l0, h1, l1;
            split_double(x.x, h0, l0);
            split_double(x.y, h1, l1);
            dst[tid + j * kNrmThreads] = make_double2(f2d_bits(exp_hl(h0 - mh, l0 - ml) * inv),
                                                      f2d_bits(exp_hl(h1 - mh, l1 - ml) * inv));
        }
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            bulk_store_hint(W + tile_of(k) * kNrmTile, out + ob * kNrmTile, kBytes, drop);
            bulk_commit();
            if (k + kNrmStages < nmine) {  // the ring slot just read takes tile k + stages
                fence_async_shared();
                mb_expect_tx(&full[st], kBytes);
                bulk_load_hint(in + st * kNrmTile, lw + tile_of(k + kNrmStages) * kNrmTile,
                               kBytes, &full[st], drop);
            }
        }
        if (++st == kNrmStages) { st = 0; ++round; }
    }
    if (tid == 0) bulk_wait_all();
    // the elements past the last whole tile
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = ntiles * kNrmTile + (int64_t)blockIdx.x * blockDim.x + tid; i < M; i += G) {
        float xh, xl;
        split_double(lw[i], xh, xl);
        W[i] = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
    }
}

__global__ void __launch_bounds__(256) k_ess_reduce(const double* __restrict__ lw, int64_t M,
                                                    double* __restrict__ partials,
                                                    unsigned long long* ticket,
                                                    double* __restrict__ ess_out,
                                                    uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    __shared__ long long s_key[48];
    __shared__ float s_a[32], s_b[32];
    __shared__ bool last;
    RefSums cur;
    bool nan_seen = false;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nchunk = aligned16(lw) ? M / kChunk : 0;
    for (int64_t ch = t0; ch < nchunk; ch += G) {
        double x[kChunk];
        load8(lw + ch * kChunk, x);
#pragma unroll
        for (int j = 0; j < kChunk; ++j) { nan_seen |= disnan(x[j]); cur.add(x[j]); }
    }
    for (int64_t i = nchunk * kChunk + t0; i < M; i += G) {
        const double x = lw[i];
        nan_seen |= disnan(x);
        cur.add(x);
    }
    if (nan_seen) raise_status(status, ST_NONFINITE);
    double bmax;
    const Lse c = block_combine(cur, s_key, s_a, s_b, &bmax);
    if (threadIdx.x == 0) {
        double* P = partials + (size_t)blockIdx.x * 8;
        P[0] = c.m; P[1] = c.s1; P[2] = c.s2;
        __threadfence();
        const unsigned long long t = atomicAdd(ticket, 1ull);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const Lse tc = combine_partials(partials, gridDim.x, 0, s_key);
    if (threadIdx.x == 0) {
        *ticket = 0ull;
        if (is_neg_inf(tc.m)) {
            raise_status(status, ST_ZERO_WEIGHT);
            return;
        }
        const float s1f = (float)tc.s1;
        *ess_out = f2d_bits(s1f * (s1f / (float)tc.s2));
    }
}

// Normalisation fused with pass 1 of systematic resampling: every tile of
// 2048 weights is written as k_reweight_normalize writes it, and the exact
// integer sum of q = floor(W 2^52) of those same values is stored for the
// tile (what k_resample_total would form by reading W back).  Invalid
// weights (the reduction found none positive) leave zero tile sums, so the
// resampling that follows reports SMC_ERR_ZERO_WEIGHT and writes nothing.
__global__ void __launch_bounds__(kRsThreads) k_normalize_tiles(const double* __restrict__ lw,
                                                                int64_t M, RwArgs rw,
                                                                double* __restrict__ W,
                                                                RsScratch sc, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    __shared__ unsigned long long sh[kRsThreads / 32];
    const RwFinal fin = rw_final(rw, status);
    const bool valid = fin.valid;
    float mh = 0.0f, ml = 0.0f, inv = 0.0f;
    if (valid) {
        split_double(fin.m, mh, ml);
        inv = fin.inv;
    }
    const int64_t ntiles = rs_tiles(M);
    // descending: the reduction wrote the log-weights ascending (the most
    // recent, still in L2, first); the resampling scan then runs ascending
    for (int64_t k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const int64_t t = ntiles - 1 - k;
        unsigned long long acc = 0;
        if (valid) {
            double x[kRsIpt], w[kRsIpt];
            load_tile_raw_cs(lw, M, t, x);
            const int64_t g0 = t * kRsTile + (int64_t)threadIdx.x * kRsIpt;
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j) {
                float xh, xl;
                split_double(x[j], xh, xl);
                w[j] = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
                acc += g0 + j < M ? q_fast(w[j]) : 0ull;  // w in [0, 1]
            }
            if (g0 + kRsIpt <= M && aligned16(W + g0)) {
                store8(W + g0, w);
            } else {
#pragma unroll
                for (int j = 0; j < kRsIpt; ++j)
                    if (g0 + j < M) W[g0 + j] = w[j];
            }
        }
        const unsigned long long ts = block_sum_u64(acc, sh);
        if (threadIdx.x == 0) sc.tile_sum[t] = ts;
    }
}

// k_normalize_tiles with the whole tiles moved by bulk copies (a ring of
// kNtStages 16 KB slots for the log-weights, two for the weights; thread t
// takes elements t + 256 j), tiles descending as there; the partial last
// tile, if any, goes to block 0 in the per-thread form first.  Same weights
// and tile sums.
constexpr int kNtStages = 3;
constexpr size_t kNtSmem = (size_t)(kNtStages + 2) * kRsTile * sizeof(double) + 64;
__global__ void __launch_bounds__(kRsThreads) k_normalize_tiles_bulk(
    const double* __restrict__ lw, int64_t M, RwArgs rw, double* __restrict__ W, RsScratch sc,
    uint32_t* status, uint32_t limit) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    extern __shared__ __align__(128) double ntm[];
    double* in = ntm;                            // [kNtStages][kRsTile]
    double* out = ntm + kNtStages * kRsTile;     // [2][kRsTile]
    uint64_t* full = reinterpret_cast<uint64_t*>(out + 2 * kRsTile);
    __shared__ unsigned long long sh[2][kRsThreads / 32];
    const int tid = threadIdx.x, wid = tid >> 5;
    const int64_t nfull = M / kRsTile;
    const int64_t nmine = nfull > blockIdx.x ? (nfull - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t k) { return nfull - 1 - (blockIdx.x + k * gridDim.x); };
    constexpr uint32_t kBytes = kRsTile * sizeof(double);
    if (tid == 0) {
        for (int st = 0; st < kNtStages; ++st) mb_init(&full[st], 1);
        mb_init_fence();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < kNtStages && k < nmine; ++k) {
            mb_expect_tx(&full[k], kBytes);
            bulk_load(in + k * kRsTile, lw + tile_of(k) * kRsTile, kBytes, &full[k]);
        }
    // the normalisation constants, while the first tiles load
    const RwFinal fin = rw_final(rw, status);
    if (!fin.valid) {  // no valid weights: zero tile sums, W untouched
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + tid; t < rs_tiles(M);
             t += (int64_t)gridDim.x * blockDim.x)
            sc.tile_sum[t] = 0ull;
        for (int k = 0; k < kNtStages && k < nmine; ++k) mb_wait(&full[k], 0, status, limit);
        return;
    }
    float mh, ml;
    split_double(fin.m, mh, ml);
    const float inv = fin.inv;
    int buf = 0;
    auto tile_total = [&](unsigned long long acc) {  // valid in thread 0 after the barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((tid & 31) == 0) sh[buf][wid] = acc;
        __syncthreads();
        unsigned long long ts = 0;
        if (tid == 0)
#pragma unroll
            for (int w = 0; w < kRsThreads / 32; ++w) ts += sh[buf][w];
        buf ^= 1;
        return ts;
    };
    if (blockIdx.x == 0 && nfull * kRsTile < M) {  // the partial last tile
        double x[kRsIpt];
        load_tile_raw_cs(lw, M, nfull, x);
        const int64_t g0 = nfull * kRsTile + (int64_t)tid * kRsIpt;
        unsigned long long acc = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            if (g0 + j < M) {
                float xh, xl;
                split_double(x[j], xh, xl);
                const double w = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
                W[g0 + j] = w;
                acc += q_fast(w);
            }
        }
        const unsigned long long ts = tile_total(acc);
        if (tid == 0) sc.tile_sum[nfull] = ts;
    }
    int st = 0;
    uint32_t round = 0;
    for (int64_t k = 0; k < nmine; ++k) {
        const int ob = (int)(k & 1);
        mb_wait(&full[st], round & 1, status, limit);
        if (tid == 0 && k >= 2) bulk_wait_read<1>();  // out[ob]'s last store has read it
        __syncthreads();
        const double* src = in + st * kRsTile;
        double* dst = out + ob * kRsTile;
        unsigned long long acc = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            float xh, xl;
            split_double(src[tid + kRsThreads * j], xh, xl);
            const double w = f2d_bits(exp_hl(xh - mh, xl - ml) * inv);
            dst[tid + kRsThreads * j] = w;
            acc += q_fast(w);  // w in [0, 1]
        }
        fence_async_shared();
        const unsigned long long ts = tile_total(acc);  // its barrier: slot st read, out[ob] written
        if (tid == 0) {
            const int64_t t = tile_of(k);
            sc.tile_sum[t] = ts;
            bulk_store(W + t * kRsTile, dst, kBytes);
            bulk_commit();
            if (k + kNtStages < nmine) {
                fence_async_shared();
                mb_expect_tx(&full[st], kBytes);
                bulk_load(in + st * kRsTile, lw + tile_of(k + kNtStages) * kRsTile, kBytes,
                          &full[st]);
            }
        }
        if (++st == kNtStages) { st = 0; ++round; }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace smc

namespace smc_host {

smc::RsScratch resample_scratch(unsigned long long* base, int64_t M, bool heavy);
smc_status resample_launch(int num_sms, const double* W, int64_t M, uint64_t seed, uint64_t step,
                           int32_t* anc, int32_t* counts, const int32_t* do_flag, double* lwreset,
                           const smc::RsScratch& sc, uint32_t* status, cudaStream_t s,
                           bool tiles_ready);

// Up to cap * 256 elements: one element per thread (short dependent chains:
// the reduction is latency-bound there); beyond, chunks of 8 per thread,
// with at most as many blocks as are resident at once (two per SM).
static bool aligned16h(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static int reduce_blocks(const smc_ctx* ctx, int64_t M) {
    int64_t cap = (int64_t)ctx->num_sms * 2;
    if (cap > smc::kRwMaxParts) cap = smc::kRwMaxParts;  // what one combination reads
    int64_t b = (M + 255) / 256;
    if (b > cap) b = (M + 256 * 8 - 1) / (256 * 8);
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace smc_host

smc_status reweight_reduce_launch(smc_ctx* ctx, const double* loglik, double dbeta, double* logw,
                                  int64_t M, double* scalars_out, int32_t* resample_flag,
                                  double ess_frac, cudaStream_t s, smc::RwArgs* defer_to);

extern "C" smc_status smc_reweight(smc_ctx* ctx, const double* loglik, double dbeta,
                                   double* logw, int64_t M, double* W_out, double* scalars_out,
                                   int32_t* resample_flag_out, double ess_frac, void* stream) {
    if (!ctx || M <= 0 || !logw || std::isnan(dbeta) || std::isnan(ess_frac)) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    smc::RwArgs rw;
    st = reweight_reduce_launch(ctx, loglik, dbeta, logw, M, scalars_out, resample_flag_out,
                                ess_frac, s, W_out ? &rw : nullptr);
    if (st != SMC_OK) return st;
    if (W_out) {
        if (aligned16h(logw) && aligned16h(W_out) && M >= (int64_t)smc::kNrmTile * ctx->num_sms) {
            // bulk tiles: two 80 KB blocks per SM
            static bool attr_set[64] = {};
            const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
            if (!attr_set[dev]) {
                SMC_CUDA(cudaFuncSetAttribute(smc::k_reweight_normalize_bulk,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smc::kNrmSmem));
                attr_set[dev] = true;
            }
            st = launch_pdl(smc::k_reweight_normalize_bulk, dim3((unsigned)ctx->num_sms * 2),
                            dim3(smc::kNrmThreads), smc::kNrmSmem, s, (const double*)logw, M, rw,
                            W_out, ctx->d_status, ctx->wait_limit);
        } else {
            int nb = (int)((M + 256 * 8 - 1) / (256 * 8));
            int cap = ctx->num_sms * 8;
            if (nb > cap) nb = cap;
            st = launch_pdl(smc::k_reweight_normalize, dim3(nb), dim3(256), 0, s,
                            (const double*)logw, M, rw, W_out, ctx->d_status);
        }
        if (st != SMC_OK) return st;
    }
    return SMC_OK;
}

size_t smc_resample_ws_bytes(int64_t M);

// After a deferred reweighting reduction (rw: its partials and outputs): W
// and the exact tile sums in one pass that also combines the partials, then
// systematic resampling from those tile sums (the ancestors, the log-weight
// reset).
smc_status normalize_resample_launch(smc_ctx* ctx, const smc::RwArgs& rw, double* logw,
                                     int64_t M, double* W_out, int32_t* resample_flag,
                                     uint64_t seed, uint64_t step, int32_t* ancestors_out,
                                     int32_t* counts_out, cudaStream_t s) {
    smc_status st = ensure_ws(ctx, smc_resample_ws_bytes(M), s);
    if (st != SMC_OK) return st;
    const smc::RsScratch sc =
        resample_scratch(reinterpret_cast<unsigned long long*>(ctx->ws), M, true);
    if (aligned16h(logw) && aligned16h(W_out) &&
        M >= (int64_t)smc::kRsTile * ctx->num_sms * 2) {
        // whole tiles by bulk copies: two 80 KB blocks per SM
        static bool attr_set[64] = {};
        const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
        if (!attr_set[dev]) {
            SMC_CUDA(cudaFuncSetAttribute(smc::k_normalize_tiles_bulk,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smc::kNtSmem));
            attr_set[dev] = true;
        }
        st = launch_pdl(smc::k_normalize_tiles_bulk, dim3((unsigned)ctx->num_sms * 2),
                        dim3(smc::kRsThreads), smc::kNtSmem, s, (const double*)logw, M, rw,
                        W_out, sc, ctx->d_status, ctx->wait_limit);
    } else {
        int64_t nb = smc::rs_tiles(M);
        if (nb > (int64_t)ctx->num_sms * 8) nb = (int64_t)ctx->num_sms * 8;
        st = launch_pdl(smc::k_normalize_tiles, dim3((unsigned)nb), dim3(smc::kRsThreads), 0, s,
                        (const double*)logw, M, rw, W_out, sc, ctx->d_status);
    }
    if (st != SMC_OK) return st;
    return resample_launch(ctx->num_sms, W_out, M, seed, step, ancestors_out, counts_out,
                           resample_flag, logw, sc, ctx->d_status, s, true);
}

// The reweighting reduction (logw += dbeta loglik, the per-block partials).
// With defer_to null its last block also writes the final slot, the scalars
// and the flag; otherwise *defer_to receives what the kernel that consumes
// the weights (launched next on the same stream) needs to do that itself.
smc_status reweight_reduce_launch(smc_ctx* ctx, const double* loglik, double dbeta, double* logw,
                                  int64_t M, double* scalars_out, int32_t* resample_flag,
                                  double ess_frac, cudaStream_t s, smc::RwArgs* defer_to) {
    const int has_inc = (loglik != nullptr && dbeta != 0.0) ? 1 : 0;
    const int blocks = reduce_blocks(ctx, M);
    const int final_slot = kMaxPartialBlocks - 1;
    if (defer_to)
        *defer_to = smc::RwArgs{ctx->d_partials, blocks,        has_inc,   M,
                                scalars_out,     resample_flag, ess_frac, final_slot};
    return launch_pdl(smc::k_reweight_reduce, dim3(blocks), dim3(256), 0, s, loglik, dbeta, logw,
                      M, has_inc, ctx->d_partials, ctx->d_counters + CNT_REWEIGHT_TICKET,
                      defer_to ? 1 : 0, scalars_out, resample_flag, ess_frac, final_slot,
                      ctx->d_status);
}

extern "C" smc_status smc_reweight_resample(smc_ctx* ctx, const double* loglik, double dbeta,
                                            double* logw, int64_t M, double* W_out,
                                            double* scalars_out, int32_t* resample_flag_out,
                                            double ess_frac, uint64_t seed, uint64_t step,
                                            int32_t* ancestors_out, int32_t* counts_out,
                                            void* stream) {
    if (!ctx || M <= 0 || M > 0x7FFFFFFF || !logw || !W_out || !ancestors_out ||
        std::isnan(dbeta) || std::isnan(ess_frac))
        return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    smc::RwArgs rw;
    st = reweight_reduce_launch(ctx, loglik, dbeta, logw, M, scalars_out, resample_flag_out,
                                ess_frac, s, &rw);
    if (st != SMC_OK) return st;
    return normalize_resample_launch(ctx, rw, logw, M, W_out, resample_flag_out, seed, step,
                                     ancestors_out, counts_out, s);
}

extern "C" smc_status smc_ess(smc_ctx* ctx, const double* logw, int64_t M, double* ess_out,
                              void* stream) {
    if (!ctx || M <= 0 || !logw || !ess_out) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    int blocks = reduce_blocks(ctx, M);
    return launch_pdl(smc::k_ess_reduce, dim3(blocks), dim3(256), 0, s, logw, M, ctx->d_partials,
                      ctx->d_counters + CNT_ESS_TICKET, ess_out, ctx->d_status);
}
