// resample_var.cu -- smc_resample_multinomial and smc_resample_residual.
//
// Two further resampling schemes (Section 3.2's resampling step: draws from
// the empirical CDF of the weights) on the exact-integer CDF of the
// systematic scheme, q_j = floor(W_j 2^52), C_j = q_0 + ... + q_j, S = C_{M-1}:
//
//   multinomial: slot i takes min { j : C_j > floor((2 u_i + 1) S / 2^33) },
//     u_i = word 0 of (seed, MULTINOMIAL, step, index i);
//   residual: n_j = floor(M q_j / S) copies of particle j fill slots
//     [N_{j-1}, N_j) in particle order; the R = M - sum n remaining slots
//     [M - R, M) are multinomial draws on the remainders
//     rho_j = (M q_j - n_j S) >> s, s = max(0, bitlen(S) - 32), with the
//     uniforms v_k = word 0 of (seed, MULTINOMIAL, step, index k).
//
// Pass 1 and the one-CTA finalize of the systematic scheme give the tile
// prefixes and S.  Multinomial: one pass writes the inclusive CDF, then one
// thread per slot bisects first the tile prefixes, then its tile's 2048
// entries.  Residual: one pass sums n and rho per tile, one CTA turns those
// sums into prefixes (and R, P = sum rho), one pass expands the
// deterministic copies (staged through shared memory, balanced over the
// block) and writes the inclusive rho prefix, and the multinomial search
// fills the last R slots.
#include "ctx.hpp"
#include "device.cuh"
#include "resample.cuh"

using namespace smc_host;

namespace smc {

// constants of one residual call, formed by k_rd_finalize
struct RdConst {
    unsigned long long R;  // residual slots
    unsigned long long P;  // total of the shifted remainders
    uint32_t ok;
};

struct VarScratch {
    RsScratch rs;               // tile sums / prefixes and the call constants (S)
    unsigned long long* cum;    // [M] inclusive CDF: C_j (multinomial) or E_j (residual)
    unsigned long long* tn;     // [ntiles] residual: sums of n per tile, then prefixes
    unsigned long long* tr;     // [ntiles] residual: sums of rho per tile, then prefixes
    RdConst* rd;
};

constexpr int kRdStage = 2 * kRsTile;  // deterministic slots of a tile staged in shared memory

// exclusive block scan of one 64-bit value per thread; *total = block sum
__device__ __forceinline__ unsigned long long block_excl_u64(unsigned long long v,
                                                             unsigned long long* s_warp,
                                                             unsigned long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();  // s_warp free
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    unsigned long long off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) {
        if (w < wid) off += s_warp[w];
        tot += s_warp[w];
    }
    *total = tot;
    return off + incl - v;
}

// this item's share n = floor(M q / S) and shifted remainder rho
__device__ __forceinline__ void residual_split(unsigned long long q, unsigned long long MM,
                                               const RsConst& k, int sh, unsigned long long& n,
                                               unsigned long long& rho) {
    unsigned long long r;
    divmod_cm(q, MM, k, n, r);
    rho = r >> sh;
}

__device__ __forceinline__ int remainder_shift(unsigned long long S) {
    const int bits = 64 - __clzll((long long)S);
    return bits > 32 ? bits - 32 : 0;
}

// Multinomial: the inclusive CDF C_j of every item (persistent over tiles).
__global__ void __launch_bounds__(kRsThreads) k_mn_prefix(const double* __restrict__ W,
                                                          int64_t M, const int32_t* do_flag,
                                                          VarScratch vs,
                                                          double* __restrict__ lwreset) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    if (!vs.rs.cst->ok) return;
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    const int64_t ntiles = rs_tiles(M);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        double v[kRsIpt];
        load_tile_raw(W, M, tile, v);
        unsigned long long q[kRsIpt], tsum = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            quantise(v[j], q[j]);  // pass 1 reported bad weights
            tsum += q[j];
        }
        unsigned long long tot;
        unsigned long long c = __ldcg(vs.rs.tile_sum + tile) + block_excl_u64(tsum, s_warp, &tot);
        const int64_t g0 = tile * kRsTile + (int64_t)threadIdx.x * kRsIpt;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            c += q[j];
            if (g0 + j < M) vs.cum[g0 + j] = c;
        }
        if (lwreset)
            for (int j = threadIdx.x; j < kRsTile; j += kRsThreads)
                if (tile * kRsTile + j < M) lwreset[tile * kRsTile + j] = 0.0;
    }
}

// Residual: per tile, the sums of n and rho.
__global__ void __launch_bounds__(kRsThreads) k_rd_tiles(const double* __restrict__ W, int64_t M,
                                                         const int32_t* do_flag, VarScratch vs) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    const RsConst cst = *vs.rs.cst;
    if (!cst.ok) return;
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    const int sh = remainder_shift(cst.S);
    const unsigned long long MM = (unsigned long long)M;
    const int64_t ntiles = rs_tiles(M);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        double v[kRsIpt];
        load_tile_raw(W, M, tile, v);
        unsigned long long sn = 0, sr = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            unsigned long long q, n, rho;
            quantise(v[j], q);
            residual_split(q, MM, cst, sh, n, rho);
            sn += n;
            sr += rho;
        }
        unsigned long long tn, tr;
        block_excl_u64(sn, s_warp, &tn);
        block_excl_u64(sr, s_warp, &tr);
        if (threadIdx.x == 0) {
            vs.tn[tile] = tn;
            vs.tr[tile] = tr;
        }
    }
}

// exclusive prefix of a[0..n) in place by one CTA; returns the total
__device__ unsigned long long cta_prefix_inplace(unsigned long long* a, int64_t n,
                                                 unsigned long long* s_w) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (n + kRsFinThreads - 1) / kRsFinThreads;
    const int64_t t0 = (int64_t)tid * per;
    const int64_t t1 = t0 + per < n ? t0 + per : n;
    unsigned long long own = 0;
    for (int64_t t = t0; t < t1; ++t) own += __ldcg(a + t);
    unsigned long long incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    __syncthreads();
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    unsigned long long off = 0, total = 0;
    for (int w = 0; w < kRsFinThreads / 32; ++w) {
        if (w < wid) off += s_w[w];
        total += s_w[w];
    }
    unsigned long long run = off + incl - own;
    for (int64_t t = t0; t < t1; ++t) {
        const unsigned long long v = __ldcg(a + t);
        a[t] = run;
        run += v;
    }
    return total;
}

// Residual, one CTA: prefixes of the per-tile sums, R and P.
__global__ void __launch_bounds__(kRsFinThreads) k_rd_finalize(int64_t M, const int32_t* do_flag,
                                                               VarScratch vs, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long s_w[kRsFinThreads / 32];
    const bool ok = vs.rs.cst->ok != 0;
    const int64_t ntiles = rs_tiles(M);
    const unsigned long long nsum = ok ? cta_prefix_inplace(vs.tn, ntiles, s_w) : 0ull;
    __syncthreads();
    const unsigned long long P = ok ? cta_prefix_inplace(vs.tr, ntiles, s_w) : 0ull;
    if (threadIdx.x == 0) {
        RdConst c;
        c.ok = 0;
        c.R = 0;
        c.P = P;
        if (ok) {
            // sum n <= M by construction, and P > 0 whenever R > 0
            if (nsum > (unsigned long long)M || (nsum < (unsigned long long)M && P == 0))
                raise_status(status, ST_BADARG);
            else {
                c.R = (unsigned long long)M - nsum;
                c.ok = 1;
            }
        }
        *vs.rd = c;
    }
}

// Residual: the deterministic copies and the inclusive remainder prefix E.
__global__ void __launch_bounds__(kRsThreads) k_rd_expand(const double* __restrict__ W, int64_t M,
                                                          const int32_t* do_flag, VarScratch vs,
                                                          int32_t* __restrict__ anc,
                                                          double* __restrict__ lwreset,
                                                          uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) {  // no resampling this step: identity
        for (int64_t g = (int64_t)blockIdx.x * kRsThreads + threadIdx.x; g < M;
             g += (int64_t)gridDim.x * kRsThreads)
            anc[g] = (int32_t)g;
        return;
    }
    const RsConst cst = *vs.rs.cst;
    if (!cst.ok || !vs.rd->ok) return;
    __shared__ uint32_t s_hi[kRsTile];  // inclusive N of each item of the tile
    __shared__ int32_t s_anc[kRdStage];
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    const int sh = remainder_shift(cst.S);
    const unsigned long long MM = (unsigned long long)M;
    const int64_t ntiles = rs_tiles(M);
    const int tid = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kRsTile;
        double v[kRsIpt];
        load_tile_raw(W, M, tile, v);
        unsigned long long n[kRsIpt], rho[kRsIpt], sn = 0, sr = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            unsigned long long q;
            quantise(v[j], q);
            residual_split(q, MM, cst, sh, n[j], rho[j]);
            sn += n[j];
            sr += rho[j];
        }
        unsigned long long tot_n, tot_r;
        const unsigned long long on = block_excl_u64(sn, s_warp, &tot_n);
        const unsigned long long orr = block_excl_u64(sr, s_warp, &tot_r);
        const unsigned long long nbase = __ldcg(vs.tn + tile);
        unsigned long long e = __ldcg(vs.tr + tile) + orr;
        const int64_t g0 = base + (int64_t)tid * kRsIpt;
        unsigned long long f = nbase + on;  // first slot of this thread's item 0
        const uint32_t F0 = (uint32_t)f;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            e += rho[j];
            if (g0 + j < M) vs.cum[g0 + j] = e;
            f += n[j];
            s_hi[tid * kRsIpt + j] = (uint32_t)f;
        }
        if (lwreset)
            for (int j = tid; j < kRsTile; j += kRsThreads)
                if (base + j < M) lwreset[base + j] = 0.0;
        __syncthreads();
        const uint32_t lo = (uint32_t)nbase, hi = s_hi[kRsTile - 1];
        if (hi < lo || (unsigned long long)hi > MM) {  // cannot happen with consistent sums
            if (tid == 0) raise_status(status, ST_BADARG);
            __syncthreads();
            continue;
        }
        const uint32_t range = hi - lo;
        if (range <= (uint32_t)kRdStage) {  // stage the tile's slots, store slot-major
            uint32_t s0 = F0;
            for (int j = 0; j < kRsIpt; ++j) {
                const uint32_t s1 = s_hi[tid * kRsIpt + j];
                for (uint32_t sl = s0; sl < s1; ++sl)
                    if (SMC_IN_BOUNDS(sl - lo < (uint32_t)kRdStage, status))
                        s_anc[sl - lo] = (int32_t)(g0 + j);
                s0 = s1;
            }
            __syncthreads();
            for (uint32_t k = tid; k < range; k += kRsThreads) anc[lo + k] = s_anc[k];
        } else {  // heavy tile: contiguous runs of slots per thread
            const uint32_t per = (range + kRsThreads - 1) / kRsThreads;
            const uint32_t s0 = lo + (uint32_t)tid * per;
            const uint32_t s1 = s0 + per < hi ? s0 + per : hi;
            if (s0 < s1) {
                int a = 0, b = kRsTile - 1;  // first item whose inclusive N exceeds s0
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if (s_hi[mid] > s0) b = mid;
                    else a = mid + 1;
                }
                int item = a;
                for (uint32_t sl = s0; sl < s1; ++sl) {
                    while (SMC_IN_BOUNDS(item < kRsTile, status) && s_hi[item] <= sl) ++item;
                    if (SMC_IN_BOUNDS(sl < (uint32_t)M && item < kRsTile, status))
                        anc[sl] = (int32_t)(base + item);
                }
            }
        }
        __syncthreads();  // shared memory reused by the next tile
    }
}

// One thread per drawn slot: the first item whose inclusive CDF exceeds
// floor((2 u + 1) total / 2^33), by bisection of the tile prefixes and then
// of the tile.  Multinomial: all M slots; residual: the last R slots.
template <bool RESIDUAL>
__global__ void __launch_bounds__(256) k_mn_draw(int64_t M, uint64_t seed, uint64_t step,
                                                 const int32_t* do_flag, VarScratch vs,
                                                 int32_t* __restrict__ anc, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (do_flag && *do_flag == 0) {
        if (!RESIDUAL)  // identity (the residual expand kernel wrote it already)
            for (int64_t g = i0; g < M; g += G) anc[g] = (int32_t)g;
        return;
    }
    if (!vs.rs.cst->ok) return;
    unsigned long long total, nslots;
    const unsigned long long* tpre;
    if (RESIDUAL) {
        const RdConst rd = *vs.rd;
        if (!rd.ok) return;
        total = rd.P;
        nslots = rd.R;
        tpre = vs.tr;
    } else {
        total = vs.rs.cst->S;
        nslots = (unsigned long long)M;
        tpre = vs.rs.tile_sum;
    }
    const int64_t slot0 = M - (int64_t)nslots;
    const int64_t ntiles = rs_tiles(M);
    bool bad = false;
    for (int64_t k = i0; k < (int64_t)nslots; k += G) {
        const uint32_t u = draw(seed, RNG_MULTINOMIAL, step, (uint32_t)k, 0u).x;
        const unsigned long long T = __umul64hi((2ull * u + 1ull) << 31, total);
        int64_t a = 0, b = ntiles;  // last tile whose exclusive prefix is <= T
        while (b - a > 1) {
            const int64_t mid = (a + b) >> 1;
            if (__ldg(tpre + mid) <= T) a = mid;
            else b = mid;
        }
        int64_t lo = a * kRsTile, hi = lo + kRsTile < M ? lo + kRsTile : M;
        while (lo < hi) {  // first item of the tile with cum > T
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(vs.cum + mid) > T) hi = mid;
            else lo = mid + 1;
        }
        if (lo >= M) {  // cannot happen with consistent sums
            bad = true;
            lo = M - 1;
        }
        anc[slot0 + k] = (int32_t)lo;
    }
    if (bad) raise_status(status, ST_BADARG);
}

}  // namespace smc

namespace smc_host {

smc::RsScratch resample_scratch(unsigned long long* base, int64_t M, bool heavy);
smc_status resample_finalize_launch(int64_t M, uint64_t seed, uint64_t step,
                                    const int32_t* do_flag, const smc::RsScratch& sc,
                                    uint32_t* status, cudaStream_t s);

}  // namespace smc_host

// scratch of the multinomial / residual entry points, in words: the
// systematic scheme's tile sums and constants, the inclusive CDF, the two
// residual tile tables and the residual constants
static int64_t var_words(int64_t M) {
    return smc::rs_words(M) + M + 2 * smc::rs_tiles(M) + 4;
}

size_t smc_resample_var_ws_bytes(int64_t M) {
    return (size_t)var_words(M) * sizeof(unsigned long long) + 512;
}

static smc_status resample_var(smc_ctx* ctx, bool residual, const double* W, int64_t M,
                               uint64_t seed, uint64_t step, int32_t* anc, const int32_t* do_flag,
                               double* lwreset, void* stream) {
    if (!ctx || M < 0 || M > 0x7FFFFFFF) return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    if (!W || !anc) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    st = ensure_ws(ctx, smc_resample_var_ws_bytes(M), s);
    if (st != SMC_OK) return st;
    unsigned long long* base = reinterpret_cast<unsigned long long*>(ctx->ws);
    const int64_t tiles = smc::rs_tiles(M);
    smc::VarScratch vs;
    vs.rs = resample_scratch(base, M, false);
    vs.cum = base + smc::rs_words(M);
    vs.tn = vs.cum + M;
    vs.tr = vs.tn + tiles;
    vs.rd = reinterpret_cast<smc::RdConst*>(vs.tr + tiles);
    // pass 1 and the finalize of the systematic scheme: tile prefixes and S
    int64_t b1 = tiles < (int64_t)ctx->num_sms * 4 ? tiles : (int64_t)ctx->num_sms * 4;
    st = launch_pdl(smc::k_resample_total, dim3((unsigned)b1), dim3(smc::kRsThreads), 0, s, W, M,
                    do_flag, vs.rs, ctx->d_status);
    if (st != SMC_OK) return st;
    st = resample_finalize_launch(M, seed, step, do_flag, vs.rs, ctx->d_status, s);
    if (st != SMC_OK) return st;
    int64_t gt = tiles < (int64_t)ctx->num_sms * 4 ? tiles : (int64_t)ctx->num_sms * 4;
    int64_t gd = (M + 255) / 256;
    if (gd > (int64_t)ctx->num_sms * 16) gd = (int64_t)ctx->num_sms * 16;
    if (!residual) {
        st = launch_pdl(smc::k_mn_prefix, dim3((unsigned)gt), dim3(smc::kRsThreads), 0, s, W, M,
                        do_flag, vs, lwreset);
        if (st != SMC_OK) return st;
        return launch_pdl(smc::k_mn_draw<false>, dim3((unsigned)gd), dim3(256), 0, s, M, seed,
                          step, do_flag, vs, anc, ctx->d_status);
    }
    st = launch_pdl(smc::k_rd_tiles, dim3((unsigned)gt), dim3(smc::kRsThreads), 0, s, W, M,
                    do_flag, vs);
    if (st != SMC_OK) return st;
    st = launch_pdl(smc::k_rd_finalize, dim3(1), dim3(smc::kRsFinThreads), 0, s, M, do_flag, vs,
                    ctx->d_status);
    if (st != SMC_OK) return st;
    st = launch_pdl(smc::k_rd_expand, dim3((unsigned)gt), dim3(smc::kRsThreads), 0, s, W, M,
                    do_flag, vs, anc, lwreset, ctx->d_status);
    if (st != SMC_OK) return st;
    return launch_pdl(smc::k_mn_draw<true>, dim3((unsigned)gd), dim3(256), 0, s, M, seed, step,
                      do_flag, vs, anc, ctx->d_status);
}

extern "C" smc_status smc_resample_multinomial(smc_ctx* ctx, const double* W, int64_t M,
                                               uint64_t seed, uint64_t step,
                                               int32_t* ancestors_out, const int32_t* do_flag,
                                               double* logw_reset, void* stream) {
    return resample_var(ctx, false, W, M, seed, step, ancestors_out, do_flag, logw_reset, stream);
}

extern "C" smc_status smc_resample_residual(smc_ctx* ctx, const double* W, int64_t M,
                                            uint64_t seed, uint64_t step, int32_t* ancestors_out,
                                            const int32_t* do_flag, double* logw_reset,
                                            void* stream) {
    return resample_var(ctx, true, W, M, seed, step, ancestors_out, do_flag, logw_reset, stream);
}
