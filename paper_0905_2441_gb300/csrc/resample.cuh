// resample.cuh -- kernels of the exact-integer systematic resampler
// (included by resample.cu only).  The scratch words they use are passed
// in explicitly, so any owner of suitable device memory can run them.
//
// Pass 1 (k_resample_total): every tile of kRsTile weights is quantised
// (q = floor(W 2^52) from the FP64 bits) and reduced exactly; the tile's
// integer sum is stored, and added atomically to its group of 64 tiles and
// to the grand total S (integer addition: order-free and exact).
// Pass 2 (k_resample_scan): one CTA per tile obtains its exclusive prefix
// from the group sums before it and the tile sums before it in its group
// (one parallel read, no waiting on other CTAs), scans the tile in shared
// memory, evaluates F at every prefix and expands the tile's contiguous
// output range.
#pragma once
#include "device.cuh"

namespace smc {

constexpr int kRsThreads = 256;
constexpr int kRsIpt = 8;                      // weights per thread
constexpr int kRsTile = kRsThreads * kRsIpt;   // weights per tile
constexpr int kRsGroup = 64;                   // tiles per group sum
constexpr unsigned long long kMaxTotal = 1ull << 61;   // S must stay below this

struct RsScratch {
    unsigned long long* tile_sum;   // [ntiles]
    unsigned long long* group_sum;  // [ceil(ntiles / kRsGroup)], zero before pass 1
};

__host__ __device__ inline int64_t rs_tiles(int64_t M) { return (M + kRsTile - 1) / kRsTile; }
__host__ __device__ inline int64_t rs_groups(int64_t M) {
    return (rs_tiles(M) + kRsGroup - 1) / kRsGroup;
}
// words of scratch for M weights: tile sums, group sums
__host__ __device__ inline int64_t rs_words(int64_t M) { return rs_tiles(M) + rs_groups(M); }

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

// Pass 1: tile sums and group sums.  Each CTA takes a contiguous range of
// tiles and adds to a group sum once per group it touches (integer atomics
// on distinct words), so no word receives more than a few atomics; the
// grand total is formed from the group sums in pass 2.
__global__ void __launch_bounds__(kRsThreads) k_resample_total(const double* __restrict__ W,
                                                               int64_t M, const int32_t* do_flag,
                                                               RsScratch sc, uint32_t* status) {
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long sh[kRsThreads / 32];
    const int64_t ntiles = rs_tiles(M);
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
    bool bad = false;
    unsigned long long gacc = 0;
    int64_t gcur = t0 / kRsGroup;
    for (int64_t t = t0; t < t1; ++t) {
        unsigned long long q[kRsIpt];
        bad |= load_tile_items(W, M, t, q);
        unsigned long long acc = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) acc += q[j];  // <= 8 * 2^52: no wrap
        const unsigned long long ts = block_sum_u64(acc, sh);  // <= 2^63: no wrap
        if (threadIdx.x == 0) {
            sc.tile_sum[t] = ts;
            const int64_t g = t / kRsGroup;
            if (g != gcur) {
                const unsigned long long old = atomicAdd(sc.group_sum + gcur, gacc);
                if (old + gacc < old) bad = true;
                gacc = 0;
                gcur = g;
            }
            const unsigned long long n = gacc + ts;
            if (n < gacc || ts >= kMaxTotal) bad = true;  // far from normalised
            gacc = n;
        }
    }
    if (threadIdx.x == 0 && t0 < t1) {
        const unsigned long long old = atomicAdd(sc.group_sum + gcur, gacc);
        if (old + gacc < old) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, ST_BADARG);
}

// 128-bit unsigned arithmetic for the exact slot test
struct U128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ U128 mul64(unsigned long long a, unsigned long long b) {
    return U128{a * b, __umul64hi(a, b)};
}
__device__ __forceinline__ U128 add128(U128 a, U128 b) {
    U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
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

// Slot i lies strictly below the CDF value c iff
//   A_i = (i 2^32 + u32) S  <  X = c M 2^32.
// A walker keeps A_i for its current i, so a step to i +- 1 is one 128-bit
// addition of S 2^32, and F(c) = the first i with A_i >= X (or M).
struct SlotWalker {
    U128 step;          // S 2^32
    uint32_t M;
    uint32_t i;         // current slot
    U128 A;             // (i 2^32 + u32) S
    __device__ __forceinline__ void init(unsigned long long S, uint32_t u32, uint32_t Mv,
                                         uint32_t i0) {
        step = U128{S << 32, S >> 32};
        M = Mv;
        i = i0;
        A = mul64(((unsigned long long)i0 << 32) | u32, S);
    }
    // move to slot j (a 32 x 128-bit multiply-add)
    __device__ __forceinline__ void jump(uint32_t j) {
        if (j >= i) {
            const U128 d = mul64((unsigned long long)(j - i) << 32, S_of());
            A = add128(A, d);
        } else {
            const U128 d = mul64((unsigned long long)(i - j) << 32, S_of());
            A = sub128(A, d);
        }
        i = j;
    }
    __device__ __forceinline__ unsigned long long S_of() const {
        return (step.lo >> 32) | (step.hi << 32);
    }
    // F(X) for X at or above the X of the current slot's F: only steps up
    // (the merge walk of slots against a non-decreasing CDF)
    __device__ __forceinline__ uint32_t walk_up(U128 X) {
        while (i < M && lt128(A, X)) {
            A = add128(A, step);
            ++i;
        }
        return i;
    }
    // F(X): first slot whose A is not below X, starting near the current slot
    __device__ __forceinline__ uint32_t first_not_below(U128 X) {
        if (i < M && lt128(A, X)) {                       // walk up
            for (int it = 0; it < 64; ++it) {
                A = add128(A, step);
                ++i;
                if (i == M || !lt128(A, X)) return i;
            }
        } else {                                          // walk down
            for (int it = 0; it < 64; ++it) {
                if (i == 0) return 0;
                const U128 Ap = sub128(A, step);
                if (lt128(Ap, X)) return i;
                A = Ap;
                --i;
            }
        }
        // far from the estimate: bisection on the exact test
        uint32_t lo = 0, hi = M;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            jump(mid);
            if (lt128(A, X)) lo = mid + 1;
            else hi = mid;
        }
        jump(lo);
        return lo;
    }
};

// float -> int by its bits, truncated toward zero, 0 below 1, at most
// 2^30 (estimates only)
__device__ __forceinline__ int est_int(float v) {
    if (!(v >= 1.0f)) return 0;
    const uint32_t b = __float_as_uint(v);
    int e = (int)(b >> 23) - 127;
    if (e > 30) return 1 << 30;
    const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
    return (int)(e >= 23 ? (m << (e - 23)) : (m >> (23 - e)));
}

// uint64 -> float from 16-bit pieces (exact pieces, a few roundings;
// estimates only)
__device__ __forceinline__ float u32_to_f(uint32_t x) {
    return fmaf(u23_to_f(x >> 16), 65536.0f, u23_to_f(x & 0xFFFFu));
}
__device__ __forceinline__ float u64_to_f(unsigned long long v) {
    return fmaf(u32_to_f((uint32_t)(v >> 32)), 4294967296.0f, u32_to_f((uint32_t)v));
}

// Pass 2: one CTA per tile.
__global__ void __launch_bounds__(kRsThreads) k_resample_scan(
    const double* __restrict__ W, int64_t M, uint64_t seed, uint64_t step,
    const int32_t* do_flag, RsScratch sc, int32_t* __restrict__ anc,
    int32_t* __restrict__ counts, double* __restrict__ lwreset, uint32_t* status) {
    __shared__ uint32_t s_hi[kRsTile];            // F at each item's inclusive prefix
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    __shared__ unsigned long long s_pre[kRsThreads / 32];
    __shared__ unsigned long long s_tot[kRsThreads / 32];
    __shared__ uint32_t s_lo;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kRsTile;

    if (do_flag && *do_flag == 0) {  // no resampling this step: identity
        for (int j = tid; j < kRsTile; j += kRsThreads) {
            const int64_t g = base + j;
            if (g < M) {
                anc[g] = (int32_t)g;
                if (counts) counts[g] = 1;
            }
        }
        return;
    }
    // ---- total S and this tile's exclusive prefix from the group / tile sums
    const int64_t ngroups = rs_groups(M);
    const int64_t grp = tile / kRsGroup;
    unsigned long long tot = 0, pre = 0;
    bool ovf = false;
    for (int64_t i = tid; i < ngroups; i += kRsThreads) {
        const unsigned long long v = __ldcg(sc.group_sum + i);
        const unsigned long long n = tot + v;
        ovf |= n < tot;
        tot = n;
        if (i < grp) pre += v;
    }
    for (int64_t i = grp * kRsGroup + tid; i < tile; i += kRsThreads) pre += __ldcg(sc.tile_sum + i);
    // ---- this thread's items
    unsigned long long q[kRsIpt];
    load_tile_items(W, M, tile, q);  // pass 1 already reported bad weights
    unsigned long long tsum = 0;
#pragma unroll
    for (int j = 0; j < kRsIpt; ++j) tsum += q[j];
    // ---- block scan of the thread sums; block sums of the prefix and total
    unsigned long long incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
        const unsigned long long t2 = __shfl_xor_sync(0xFFFFFFFFu, tot, o);
        const unsigned long long n = tot + t2;
        ovf |= n < tot;
        tot = n;
    }
    if (lane == 31) s_warp[wid] = incl;
    if (lane == 0) { s_pre[wid] = pre; s_tot[wid] = tot; }
    const bool any_ovf = __syncthreads_or(ovf);
    unsigned long long woff = 0, excl = 0, S = 0;
    bool ovf2 = any_ovf;
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) {
        if (w < wid) woff += s_warp[w];
        excl += s_pre[w];
        const unsigned long long n = S + s_tot[w];
        ovf2 |= n < S;
        S = n;
    }
    if (S == 0 || S >= kMaxTotal || ovf2) {
        if (tid == 0 && tile == 0) raise_status(status, S == 0 && !ovf2 ? ST_ZERO_WEIGHT : ST_BADARG);
        return;
    }
    // ---- F at every prefix of this thread's items (exact, 128-bit walker)
    const uint32_t u32 = draw(seed, RNG_RESAMPLE, step, 0u, 0u).x;
    const unsigned long long MM = (unsigned long long)M << 32;
    unsigned long long c = excl + woff + (incl - tsum);  // C before this thread's item 0
    // M / S in FP32 (S < 2^61): estimate of the slots below c, fixed up exactly
    const float ms = u64_to_f((unsigned long long)M) / u64_to_f(S);
    const float u = u32_to_f(u32) * 2.3283064365386963e-10f;
    U128 X = mul64(c, MM);
    SlotWalker wk;
    int e0 = est_int(u64_to_f(c) * ms - u) + 1;
    if (e0 > (int)M) e0 = (int)M;
    wk.init(S, u32, (uint32_t)M, (uint32_t)e0);
    uint32_t F = wk.first_not_below(X);
    if (tid == 0) s_lo = F;
    // items expected to own more than 16 slots jump by an estimate; the
    // others advance the walker one slot at a time (128-bit add + compare)
    const float qthr_f = 16.0f / ms;
#pragma unroll
    for (int j = 0; j < kRsIpt; ++j) {
        const int64_t g = base + (int64_t)tid * kRsIpt + j;
        uint32_t Fn = F;
        if (q[j]) {
            X = add128(X, mul64(q[j], MM));
            const float qf = u64_to_f(q[j]);
            if (qf > qthr_f) {
                long long e = (long long)F + est_int(qf * ms);
                if (e > (long long)M) e = M;
                if ((uint32_t)e != wk.i) wk.jump((uint32_t)e);
                Fn = wk.first_not_below(X);
            } else {
                Fn = wk.walk_up(X);
            }
        }
        s_hi[tid * kRsIpt + j] = Fn;
        if (g < M) {
            if (counts) counts[g] = (int32_t)(Fn - F);
            if (lwreset) lwreset[g] = 0.0;
        }
        F = Fn;
    }
    __syncthreads();
    // ---- expand the tile's output range [s_lo, s_hi[last]) (blocked per thread)
    const uint32_t lo = s_lo, hi = s_hi[kRsTile - 1];
    const uint32_t range = hi - lo;
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

}  // namespace smc
