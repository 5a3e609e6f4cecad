// resample.cuh -- kernels of the exact-integer systematic resampler
// (included by resample.cu only).  The scratch words they use are passed
// in explicitly, so any owner of suitable device memory can run them.
//
// Pass 1 (k_resample_total): every tile of kRsTile weights is quantised
// (q = floor(W 2^52) from the FP64 bits) and reduced exactly; the tile's
// integer sum is stored.
// Between the passes (k_resample_finalize, one CTA): the tile sums become
// exclusive prefixes and the call's constants (S, the uniform, fixed-point
// reciprocals) are formed once.
// Pass 2 (k_resample_scan, persistent over tiles): each tile reads its
// prefix (no waiting on other CTAs), is scanned in shared memory, F is
// evaluated at every prefix and the tile's contiguous output range is
// expanded; ranges too long for one CTA go to k_resample_heavy.
#pragma once
#include "device.cuh"

namespace smc {

constexpr int kRsThreads = 256;
constexpr int kRsIpt = 8;                      // weights per thread
constexpr int kRsTile = kRsThreads * kRsIpt;   // weights per tile
constexpr unsigned long long kMaxTotal = 1ull << 61;   // S must stay below this
constexpr int kRsStage = 2 * kRsTile;          // output slots of a tile staged in shared memory

// constants of one resampling call, formed once by k_resample_finalize
struct RsConst {
    unsigned long long S;       // exact total of the quantised weights
    unsigned long long Rth;     // floor(u32 S / 2^32)
    unsigned long long qheavy;  // items with q above this are divided afresh
    unsigned long long mfx;     // floor(M 2^64 / S) when M < S, else 0 (use FP64)
    unsigned long long ifx;     // floor(2^64 / S) when S > 1, else 0
    double m_over_s;            // M / S (FP64 estimates, only when M >= S)
    uint32_t ok;                // 0: nothing to resample (status already raised)
};
constexpr int kRsConstWords = 8;

struct RsScratch {
    unsigned long long* tile_sum;   // [ntiles]: tile sums, then their exclusive prefixes
    RsConst* cst;                   // after the tile sums
    // grid-wide expansion of tiles with many output slots (optional: when
    // null, such a tile is expanded by its own CTA)
    unsigned long long* heavy_count;  // chunk records written, zero before pass 2
    uint4* heavy_list;                // {tile, tile's first slot, chunk begin, chunk end}
    uint32_t* fpos;                   // [M] inclusive F of the items of heavy tiles
};

__host__ __device__ inline int64_t rs_tiles(int64_t M) { return (M + kRsTile - 1) / kRsTile; }
// words of scratch for M weights: tile sums, constants
__host__ __device__ inline int64_t rs_words(int64_t M) { return rs_tiles(M) + kRsConstWords; }
// output slots of one heavy-expansion chunk, and the most chunk records M
// weights can produce (a tile's range is split into chunks; ranges add to M)
constexpr int kRsChunk = 4096;
__host__ __device__ inline int64_t rs_heavy_records(int64_t M) {
    return rs_tiles(M) + M / kRsChunk + 1;
}

// floor(w 2^52) from the bits of w in [0,1]; false if w is outside [0,1] or NaN
__device__ __forceinline__ bool quantise(double w, unsigned long long& q) {
    unsigned long long b = (unsigned long long)__double_as_longlong(w);
    if (b >> 63) {                       // negative (or -0)
        q = 0;
        return b == 0x8000000000000000ull;
    }
    uint32_t e = (uint32_t)(b >> 52);
    unsigned long long man = b & 0xFFFFFFFFFFFFFull;
    if (e > 1023 || (e == 1023 && man != 0)) { q = 0; return false; }  // > 1, inf, NaN
    uint32_t sh = 1023u - e;
    q = sh > 52 ? 0ull : (((1ull << 52) | man) >> sh);
    if (e == 0) q = 0;                   // zero / subnormal
    return true;
}

// this thread's kRsIpt weights of tile `tile`, quantised (0 past M)
__device__ __forceinline__ bool load_tile_items(const double* __restrict__ W, int64_t M,
                                                int64_t tile, unsigned long long (&q)[kRsIpt]) {
    const int64_t g0 = tile * kRsTile + (int64_t)threadIdx.x * kRsIpt;
    bool bad = false;
    if (g0 + kRsIpt <= M && ((reinterpret_cast<uintptr_t>(W + g0) & 15u) == 0)) {
        const double2* p = reinterpret_cast<const double2*>(W + g0);
        double2 v[kRsIpt / 2];
#pragma unroll
        for (int j = 0; j < kRsIpt / 2; ++j) v[j] = p[j];
#pragma unroll
        for (int j = 0; j < kRsIpt / 2; ++j) {
            bad |= !quantise(v[j].x, q[2 * j]);
            bad |= !quantise(v[j].y, q[2 * j + 1]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            q[j] = 0;
            if (g0 + j < M) bad |= !quantise(W[g0 + j], q[j]);
        }
    }
    return bad;
}

// this thread's kRsIpt raw weights of tile `tile` (0 past M), for loading
// one tile ahead of its use
__device__ __forceinline__ void load_tile_raw(const double* __restrict__ W, int64_t M,
                                              int64_t tile, double (&v)[kRsIpt]) {
    const int64_t g0 = tile * kRsTile + (int64_t)threadIdx.x * kRsIpt;
    if (g0 + kRsIpt <= M && ((reinterpret_cast<uintptr_t>(W + g0) & 15u) == 0)) {
        const double2* p = reinterpret_cast<const double2*>(W + g0);
#pragma unroll
        for (int j = 0; j < kRsIpt / 2; ++j) {
            const double2 d = p[j];
            v[2 * j] = d.x;
            v[2 * j + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) v[j] = g0 + j < M ? W[g0 + j] : 0.0;
    }
}

// block-wide sum of 64-bit values; result valid in thread 0
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Pass 1: the exact integer sum of every tile (each CTA a contiguous range
// of tiles, the next tile's weights loading while one is reduced).
static __global__ void __launch_bounds__(kRsThreads) k_resample_total(const double* __restrict__ W,
                                                               int64_t M, const int32_t* do_flag,
                                                               RsScratch sc, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long sh[kRsThreads / 32];
    const int64_t ntiles = rs_tiles(M);
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
    bool bad = false;
    double vn[kRsIpt];
    if (t0 < t1) load_tile_raw(W, M, t0, vn);
    for (int64_t t = t0; t < t1; ++t) {
        unsigned long long q[kRsIpt];
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) bad |= !quantise(vn[j], q[j]);
        if (t + 1 < t1) load_tile_raw(W, M, t + 1, vn);  // next tile in flight
        unsigned long long acc = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) acc += q[j];  // <= 8 * 2^52: no wrap
        const unsigned long long ts = block_sum_u64(acc, sh);  // <= 2^63: no wrap
        if (threadIdx.x == 0) {
            sc.tile_sum[t] = ts;
            if (ts >= kMaxTotal) bad = true;  // far from normalised
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, ST_BADARG);
}

// 128-bit unsigned arithmetic for the exact quotient fix-up
struct U128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ U128 mul64(unsigned long long a, unsigned long long b) {
    return U128{a * b, __umul64hi(a, b)};
}
__device__ __forceinline__ U128 sub128(U128 a, U128 b) {
    U128 r;
    r.lo = a.lo - b.lo;
    r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
    return r;
}
__device__ __forceinline__ bool lt128(U128 a, U128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Slot i lies strictly below the CDF value c iff (i + u) S < c M, with
// u = u32 / 2^32.  Writing c M = Q S + R (0 <= R < S):
//   F(c) = #{i >= 0 : (i + u) S < c M} = Q + [R 2^32 > u32 S] = Q + [R > Rth],
//   Rth = floor(u32 S / 2^32)
// (R integer: R 2^32 > X  <=>  R > floor(X / 2^32)).  Advancing c by an item's
// q adds q M to R and carries whole S into Q.

// c M = Q S + R exactly (c <= S < 2^61, M < 2^31).  The estimate of Q is
// c times the fixed-point reciprocal mfx = floor(M 2^64 / S) (integer
// multiply-high: off by at most one below), fixed up exactly; without it
// (M >= S, degenerate totals) an FP64 estimate, fixed up the same way.
static __device__ __noinline__ void divmod_cm(unsigned long long c, unsigned long long M,
                                       const RsConst& k, unsigned long long& Q,
                                       unsigned long long& R) {
    const unsigned long long S = k.S;
    unsigned long long q;
    if (k.mfx) {
        q = __umul64hi(c, k.mfx);
    } else {
        const double qe = floor((double)c * k.m_over_s);
        q = qe > 0.0 ? (unsigned long long)qe : 0ull;
    }
    const U128 P = mul64(c, M);
    U128 QS = mul64(q, S);
    for (int it = 0; it < 64 && lt128(P, QS); ++it) {  // estimate too high
        --q;
        QS = sub128(QS, U128{S, 0ull});
    }
    U128 r = sub128(P, QS);
    for (int it = 0; it < 64 && (r.hi != 0 || r.lo >= S); ++it) {  // too low
        ++q;
        r = sub128(r, U128{S, 0ull});
    }
    Q = q;
    R = r.lo;
}

// floor(hi 2^64 / d) for hi < d < 2^63 (once per call): an FP64 estimate
// (53 bits), the exact 128-bit remainder, a second FP64 estimate of the
// correction from it, then unit steps until 0 <= remainder < d.
static __device__ unsigned long long div_shift64(unsigned long long hi, unsigned long long d) {
    const double two64 = 18446744073709551616.0;
    double e = (double)hi / (double)d * two64;  // < 2^64 (hi < d), relative error ~2^-52
    unsigned long long q = e >= two64 ? ~0ull : (unsigned long long)e;
    const U128 N{0ull, hi};  // hi 2^64
    for (int pass = 0; pass < 2; ++pass) {
        const U128 qd = mul64(q, d);
        if (lt128(N, qd)) {  // q too large by ceil((qd - N) / d)
            const U128 r = sub128(qd, N);
            const double c = ((double)r.hi * two64 + (double)r.lo) / (double)d;
            q -= (unsigned long long)c + 1ull;
        } else {
            const U128 r = sub128(N, qd);
            if (r.hi == 0 && r.lo < d) return q;
            const double c = ((double)r.hi * two64 + (double)r.lo) / (double)d;
            q += c >= 1.0 ? (unsigned long long)c - 1ull : 0ull;
        }
    }
    // within a few units now: exact steps
    U128 qd = mul64(q, d);
    for (int it = 0; it < 64 && lt128(N, qd); ++it) {
        --q;
        qd = sub128(qd, U128{d, 0ull});
    }
    U128 r = sub128(N, qd);
    for (int it = 0; it < 64 && (r.hi != 0 || r.lo >= d); ++it) {
        ++q;
        r = sub128(r, U128{d, 0ull});
    }
    return q;
}

// Between the passes, one CTA: the exact total S from the tile sums, the
// call's uniform and constants, and every tile's exclusive prefix (the tile
// sums are replaced in place), so that no tile of pass 2 repeats this work.
constexpr int kRsFinThreads = 1024;
static __global__ void __launch_bounds__(kRsFinThreads) k_resample_finalize(
    int64_t M, uint64_t seed, uint64_t step, const int32_t* do_flag, RsScratch sc,
    uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long s_w[kRsFinThreads / 32];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = rs_tiles(M);
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // each thread scans a contiguous run of tile sums (up to 8 loads in
    // flight at a time)
    const int64_t per = (ntiles + kRsFinThreads - 1) / kRsFinThreads;
    const int64_t t0 = (int64_t)tid * per;
    const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
    // up to 8 tiles per thread (M <= 2^24): the run stays in registers
    // between the sum and the prefix writes
    const bool in_regs = per <= 8;
    unsigned long long v0[8];
    unsigned long long own = 0;
    bool ovf = false;
    for (int64_t t = t0; t < t1; t += 8) {
        unsigned long long v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = t + k < t1 ? __ldcg(sc.tile_sum + t + k) : 0ull;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v0[k] = v[k];
            const unsigned long long n = own + v[k];
            ovf |= n < own;
            own = n;
        }
    }
    // block exclusive scan of the runs
    unsigned long long incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) {
            ovf |= incl + v < incl;
            incl += v;
        }
    }
    if (lane == 31) s_w[wid] = incl;
    if (ovf) s_bad = 1;
    __syncthreads();
    unsigned long long off = 0, S = 0;
    bool ovf2 = s_bad != 0;
    for (int w = 0; w < kRsFinThreads / 32; ++w) {
        if (w < wid) off += s_w[w];
        const unsigned long long n = S + s_w[w];
        ovf2 |= n < S;
        S = n;
    }
    unsigned long long run = off + incl - own;
    if (in_regs) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (t0 + k < t1) sc.tile_sum[t0 + k] = run;
            run += t0 + k < t1 ? v0[k] : 0ull;
        }
    } else {
        for (int64_t t = t0; t < t1; t += 8) {
            unsigned long long v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = t + k < t1 ? __ldcg(sc.tile_sum + t + k) : 0ull;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (t + k < t1) sc.tile_sum[t + k] = run;
                run += v[k];
            }
        }
    }
    if (tid == 0 && sc.heavy_count) *sc.heavy_count = 0ull;  // the scan appends from zero
    if (tid == 0) {
        RsConst c;
        c.ok = 0;
        if (S == 0 || S >= kMaxTotal || ovf2) {
            raise_status(status, S == 0 && !ovf2 ? ST_ZERO_WEIGHT : ST_BADARG);
        } else {
            const uint32_t u32 = draw(seed, RNG_RESAMPLE, step, 0u, 0u).x;
            const unsigned long long MM = (unsigned long long)M;
            c.S = S;
            c.Rth = __umul64hi((unsigned long long)u32 << 32, S);  // floor(u32 S / 2^32)
            c.m_over_s = (double)MM / (double)S;
            c.mfx = MM < S ? div_shift64(MM, S) : 0ull;
            c.ifx = S > 1 ? div_shift64(1ull, S) : 0ull;
            // R + q M < 8 S + S < 2^64 while S < 2^60 (else every item is divided)
            c.qheavy = S < (1ull << 60) && c.ifx ? (7ull * S) / MM : 0ull;
            c.ok = 1;
        }
        *sc.cst = c;
    }
}

// Minimum resident blocks per SM asked of the register allocator for the
// scan (compile-time tuning knob).
#ifndef SMC_RS_MINB
#define SMC_RS_MINB 3
#endif

// Pass 2: one CTA per tile.
static __global__ void __launch_bounds__(kRsThreads, SMC_RS_MINB) k_resample_scan(
    const double* __restrict__ W, int64_t M, uint64_t seed, uint64_t step,
    const int32_t* do_flag, RsScratch sc, int32_t* __restrict__ anc,
    int32_t* __restrict__ counts, double* __restrict__ lwreset, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    __shared__ uint32_t s_hi[kRsTile];            // F at each item's inclusive prefix
    __shared__ int32_t s_anc[kRsStage];           // the tile's ancestors, staged for coalesced stores
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    __shared__ uint32_t s_lo;
    __shared__ unsigned long long s_qr[2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = rs_tiles(M);
    (void)seed;
    (void)step;

    if (do_flag && *do_flag == 0) {  // no resampling this step: identity
        for (int64_t g = (int64_t)blockIdx.x * kRsThreads + tid; g < M;
             g += (int64_t)gridDim.x * kRsThreads) {
            anc[g] = (int32_t)g;
            if (counts) counts[g] = 1;
        }
        return;
    }
    // ---- the call's constants (finalize)
    const RsConst cst = *sc.cst;
    if (!cst.ok) return;
    const unsigned long long S = cst.S;
    const unsigned long long MM = (unsigned long long)M;
    const unsigned long long Rth = cst.Rth;
    const unsigned long long qheavy = cst.qheavy;
    const unsigned long long ifx = cst.ifx;
    // persistent over tiles; the next tile's weights and prefix load while
    // the current one is processed
    int64_t tile = blockIdx.x;
    double vn[kRsIpt];
    unsigned long long pn = 0;
    if (tile < ntiles) {
        load_tile_raw(W, M, tile, vn);
        pn = __ldcg(sc.tile_sum + tile);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kRsTile;
        unsigned long long q[kRsIpt];
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) quantise(vn[j], q[j]);  // pass 1 reported bad weights
        const unsigned long long tpre = pn;  // the tile's exclusive prefix (finalize)
        if (tile + gridDim.x < ntiles) {
            load_tile_raw(W, M, tile + gridDim.x, vn);
            pn = __ldcg(sc.tile_sum + tile + gridDim.x);
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) tsum += q[j];
        // ---- block exclusive scan of the thread sums
        unsigned long long incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        __syncthreads();  // the previous tile is done with shared memory
        if (lane == 31) s_warp[wid] = incl;
        if (tid == 0) {  // the tile's own c M = Q S + R, divided once
            unsigned long long Qt, Rt;
            divmod_cm(tpre, MM, cst, Qt, Rt);
            s_qr[0] = Qt;
            s_qr[1] = Rt;
        }
        __syncthreads();
        unsigned long long woff = 0;
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w)
            if (w < wid) woff += s_warp[w];
        const unsigned long long off = woff + (incl - tsum);  // this thread's offset in the tile
        unsigned long long c = tpre + off;                    // C before this thread's item 0
        unsigned long long Q = s_qr[0], R = s_qr[1];
        if (off <= qheavy) {  // carry the tile's Q, R by off M (< 8 S)
            const unsigned long long R2 = R + off * MM;
            unsigned long long n = __umul64hi(R2, ifx);
            unsigned long long r = R2 - n * S;
            const bool hi1 = r >= S;
            Q += n + (hi1 ? 1ull : 0ull);
            R = r - (hi1 ? S : 0ull);
        } else {
            divmod_cm(c, MM, cst, Q, R);
        }
        const uint32_t F0 = (uint32_t)(Q + (R > Rth ? 1ull : 0ull));
        if (tid == 0) s_lo = F0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            c += q[j];
            if (q[j] > qheavy) {  // rare: a heavy item, divided afresh
                divmod_cm(c, MM, cst, Q, R);
            } else {
                // carry R + q M (< 9 S < 2^64) into Q without a data-dependent
                // loop: n = floor((R + q M) / S) in [0, 8] from the
                // fixed-point reciprocal ifx = floor(2^64 / S) (integer
                // multiply-high, off by at most one below) and one correction
                const unsigned long long R2 = R + q[j] * MM;
                unsigned long long n = __umul64hi(R2, ifx);
                unsigned long long r = R2 - n * S;
                const bool hi1 = r >= S;
                n += hi1 ? 1ull : 0ull;
                r -= hi1 ? S : 0ull;
                Q += n;
                R = r;
            }
            uint32_t Fn = (uint32_t)(Q + (R > Rth ? 1ull : 0ull));
            if (Fn > (uint32_t)M) Fn = (uint32_t)M;
            s_hi[tid * kRsIpt + j] = Fn;
        }
        __syncthreads();
        // ---- offspring counts and the log-weight reset, item-major (coalesced)
        const uint32_t lo = s_lo, hi = s_hi[kRsTile - 1];
        if (counts)
            for (int j = tid; j < kRsTile; j += kRsThreads)
                if (base + j < M) counts[base + j] = (int32_t)(s_hi[j] - (j ? s_hi[j - 1] : lo));
        if (lwreset) {
            if (base + kRsTile <= M && ((reinterpret_cast<uintptr_t>(lwreset + base) & 15u) == 0)) {
                double2* d2 = reinterpret_cast<double2*>(lwreset + base);
                for (int j = tid; j < kRsTile / 2; j += kRsThreads) d2[j] = make_double2(0.0, 0.0);
            } else {
                for (int j = tid; j < kRsTile; j += kRsThreads)
                    if (base + j < M) lwreset[base + j] = 0.0;
            }
        }
        // ---- expand the tile's output range [lo, hi).  Usual case (the range
        // fits in shared memory): each thread writes its own items' slots there,
        // then the block stores them slot-major.  A larger range (heavy weights)
        // is split into chunks for k_resample_heavy, which all CTAs share;
        // without that scratch the CTA expands it itself (contiguous blocks of
        // slots per thread, stored directly).
        if (hi < lo || hi > (uint32_t)M) {  // cannot happen with consistent sums
            if (tid == 0) raise_status(status, ST_BADARG);
            continue;
        }
        const uint32_t range = hi - lo;
        if (range <= (uint32_t)kRsStage) {  // uniform over the block
            // each item writes its first 4 slots with predicated stores; the
            // rare items with more slots finish in a loop
            uint32_t f = F0;
            const int32_t i0 = (int32_t)(base + (int64_t)tid * kRsIpt);
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j) {
                const uint32_t e = s_hi[tid * kRsIpt + j];
#pragma unroll
                for (uint32_t k = 0; k < 4; ++k)
                    if (f + k < e) s_anc[f + k - lo] = i0 + j;
                for (uint32_t sl = f + 4; sl < e; ++sl) s_anc[sl - lo] = i0 + j;
                f = e;
            }
            __syncthreads();
            for (uint32_t k = tid; k < range; k += kRsThreads) anc[lo + k] = s_anc[k];
            continue;
        }
        if (sc.heavy_list) {
            for (int j = tid; j < kRsTile; j += kRsThreads)
                if (base + j < M) sc.fpos[base + j] = s_hi[j];
            if (tid == 0) {
                const uint32_t nch = (range + kRsChunk - 1) / kRsChunk;
                const unsigned long long r0 = atomicAdd(sc.heavy_count, (unsigned long long)nch);
                for (uint32_t k = 0; k < nch; ++k) {
                    const uint32_t b = lo + k * kRsChunk;
                    const uint32_t e = b + kRsChunk < hi ? b + kRsChunk : hi;
                    sc.heavy_list[r0 + k] = make_uint4((uint32_t)tile, lo, b, e);
                }
            }
            continue;
        }
        const uint32_t per = (range + kRsThreads - 1) / kRsThreads;
        const uint32_t s0 = lo + (uint32_t)tid * per;
        const uint32_t s1 = s0 + per < hi ? s0 + per : hi;
        if (s0 < s1) {
            int a = 0, b = kRsTile - 1;  // first item whose inclusive F exceeds s0
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (s_hi[mid] > s0) b = mid;
                else a = mid + 1;
            }
            int item = a;
            for (uint32_t sl = s0; sl < s1; ++sl) {
                while (s_hi[item] <= sl) ++item;
                anc[sl] = (int32_t)(base + item);
            }
        }
    }
}

// Pass 3: the chunks of heavy tiles, shared by all CTAs (grid-stride).  A
// chunk's first item is found by bisection on the tile's inclusive F
// values; its slots are staged in shared memory and stored slot-major.
static __global__ void __launch_bounds__(kRsThreads) k_resample_heavy(
    const int32_t* do_flag, RsScratch sc, int64_t M, int32_t* __restrict__ anc) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ int32_t s_anc[kRsChunk];
    const unsigned long long n = __ldcg(sc.heavy_count);
    for (unsigned long long r = blockIdx.x; r < n; r += gridDim.x) {
        const uint4 rec = sc.heavy_list[r];
        const int64_t base = (int64_t)rec.x * kRsTile;
        const int nit = (int)(M - base < kRsTile ? M - base : kRsTile);
        const uint32_t* f = sc.fpos + base;
        const uint32_t b = rec.z, e = rec.w;
        const uint32_t per = (e - b + kRsThreads - 1) / kRsThreads;
        const uint32_t s0 = b + (uint32_t)threadIdx.x * per;
        const uint32_t s1 = s0 + per < e ? s0 + per : e;
        if (s0 < s1) {
            int a = 0, hi = nit - 1;  // first item whose inclusive F exceeds s0
            while (a < hi) {
                const int mid = (a + hi) >> 1;
                if (f[mid] > s0) hi = mid;
                else a = mid + 1;
            }
            int item = a;
            for (uint32_t sl = s0; sl < s1; ++sl) {
                while (f[item] <= sl) ++item;
                s_anc[sl - b] = (int32_t)(base + item);
            }
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < e - b; k += kRsThreads) anc[b + k] = s_anc[k];
        __syncthreads();
    }
}

}  // namespace smc
