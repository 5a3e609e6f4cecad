// resample.cuh -- kernels of the exact-integer systematic resampler
// (included by resample.cu only).  The scratch words they use are passed
// in explicitly, so any owner of suitable device memory can run them.
#pragma once
#include "device.cuh"

namespace smc {

constexpr int kRsThreads = 256;
constexpr int kRsIpt = 8;                      // weights per thread
constexpr int kRsTile = kRsThreads * kRsIpt;   // weights per tile
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kFlagErr = 3ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr unsigned long long kMaxTotal = 1ull << 61;   // S must stay below this

struct RsScratch {
    unsigned long long* tiles;   // [ntiles] tile descriptors: flag << 62 | value
    unsigned long long* ticket;  // dynamic tile index (reset by the last tile)
    unsigned long long* sum;     // exact total S (reset by the last tile)
    unsigned long long* done;    // finished tiles (reset by the last tile)
};

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

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Pass 1: exact total of the quantised weights; clears the tile descriptors.
__global__ void __launch_bounds__(256) k_resample_total(const double* __restrict__ W, int64_t M,
                                                        const int32_t* do_flag, RsScratch sc,
                                                        int64_t ntiles, uint32_t* status) {
    if (do_flag && *do_flag == 0) return;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < ntiles; i += G) sc.tiles[i] = 0ull;
    unsigned long long acc = 0;
    bool bad = false;
    for (int64_t i = t0; i < M; i += G) {
        unsigned long long q;
        bad |= !quantise(W[i], q);
        unsigned long long n = acc + q;
        bad |= n >= (1ull << 55);  // far from normalised; keeps block sums below 2^63
        acc = n;
    }
    __shared__ unsigned long long sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, ST_BADARG);
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        bool ovf = false;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            unsigned long long n = t + sh[w];
            ovf |= n < t;
            t = n;
        }
        unsigned long long old = atomicAdd(sc.sum, t);
        if (ovf || old + t < old || old + t >= kMaxTotal) raise_status(status, ST_BADARG);
    }
}

struct SlotGeom {
    unsigned long long S;    // total
    unsigned long long MM;   // M << 32
    uint32_t u32;
    uint32_t M;
};

// slot i lies strictly below CDF value c:  (i 2^32 + u32) S < c M 2^32
__device__ __forceinline__ bool slot_below(uint32_t i, unsigned long long c, const SlotGeom& g) {
    unsigned long long L = ((unsigned long long)i << 32) | g.u32;
    unsigned long long lh = __umul64hi(L, g.S), lo = L * g.S;
    unsigned long long rh = __umul64hi(c, g.MM), rl = c * g.MM;
    return lh < rh || (lh == rh && lo < rl);
}

// F(c) = number of slots below c, starting from an estimate: a short
// two-sided walk, then bisection if the estimate was far off.
__device__ __forceinline__ uint32_t slots_below(unsigned long long c, long long est,
                                                const SlotGeom& g) {
    uint32_t i = est < 0 ? 0u : (est > (long long)g.M ? g.M : (uint32_t)est);
    int it = 0;
    while (i > 0 && !slot_below(i - 1, c, g) && it < 4) { --i; ++it; }
    while (i < g.M && slot_below(i, c, g) && it < 8) { ++i; ++it; }
    bool ok = (i == 0 || slot_below(i - 1, c, g)) && (i == g.M || !slot_below(i, c, g));
    if (ok) return i;
    uint32_t lo = 0, hi = g.M;  // first i with !below
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (slot_below(mid, c, g)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Pass 2: one tile of kRsTile weights per block, tiles taken in ticket order.
__global__ void __launch_bounds__(kRsThreads) k_resample_scan(
    const double* __restrict__ W, int64_t M, uint64_t seed, uint64_t step,
    const int32_t* do_flag, RsScratch sc, uint32_t ntiles, int32_t* __restrict__ anc,
    int32_t* __restrict__ counts, double* __restrict__ lwreset, uint32_t* status) {
    __shared__ uint32_t s_hi[kRsTile];            // F at each item's inclusive prefix
    __shared__ unsigned long long s_warp[kRsThreads / 32];
    __shared__ unsigned long long s_excl, s_total;
    __shared__ uint32_t s_tile, s_u32, s_lo;
    __shared__ int s_state;                       // 0 ok, 1 identity, 2 abort
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    if (tid == 0) {
        s_tile = (uint32_t)atomicAdd(sc.ticket, 1ull);
        int state = 0;
        if (do_flag && *do_flag == 0) state = 1;
        s_state = state;
        s_u32 = draw(seed, RNG_RESAMPLE, step, 0u, 0u).x;
        s_total = *(volatile unsigned long long*)sc.sum;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kRsTile;

    if (s_state == 1) {  // no resampling this step: identity
        for (int j = tid; j < kRsTile; j += kRsThreads) {
            int64_t g = base + j;
            if (g < M) {
                anc[g] = (int32_t)g;
                if (counts) counts[g] = 1;
            }
        }
    } else {
        const unsigned long long S = s_total;
        if (S == 0 || S >= kMaxTotal) {
            if (tid == 0 && S == 0) raise_status(status, ST_ZERO_WEIGHT);
            if (tid == 0) st_release(sc.tiles + tile, kFlagErr);
        } else {
            // ---- load and quantise this thread's items (blocked)
            unsigned long long q[kRsIpt];
            unsigned long long tsum = 0;
            bool bad = false;
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j) {
                int64_t g = base + (int64_t)tid * kRsIpt + j;
                q[j] = 0;
                if (g < M) bad |= !quantise(W[g], q[j]);
                tsum += q[j];
            }
            if (bad) raise_status(status, ST_BADARG);
            // ---- block exclusive scan of the thread sums
            unsigned long long incl = tsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) s_warp[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                unsigned long long v = lane < kRsThreads / 32 ? s_warp[lane] : 0ull;
                unsigned long long vi = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, vi, o);
                    if (lane >= o) vi += u;
                }
                if (lane < kRsThreads / 32) s_warp[lane] = vi - v;  // exclusive warp offsets
                const unsigned long long agg = __shfl_sync(0xFFFFFFFFu, vi, kRsThreads / 32 - 1);
                // ---- decoupled look-back (warp 0)
                unsigned long long excl = 0;
                int state = 0;
                if (tile == 0) {
                    if (lane == 0) st_release(sc.tiles, kFlagInc | agg);
                } else {
                    if (lane == 0) st_release(sc.tiles + tile, kFlagAgg | agg);
                    long long j = (long long)tile - 1;
                    uint32_t spins = 0;
                    while (true) {
                        long long idx = j - lane;
                        unsigned long long v2 = idx >= 0 ? ld_acquire(sc.tiles + idx) : kFlagInc;
                        unsigned long long f = v2 & ~kValMask;
                        unsigned inc_mask = __ballot_sync(0xFFFFFFFFu, f == kFlagInc);
                        int first = inc_mask ? __ffs(inc_mask) - 1 : 32;
                        // only the predecessors up to the nearest inclusive prefix matter
                        unsigned need = first == 32 ? 0xFFFFFFFFu : ((2u << first) - 1u);
                        if (__ballot_sync(0xFFFFFFFFu, f == kFlagErr) & need) { state = 2; break; }
                        if (__ballot_sync(0xFFFFFFFFu, f == 0ull) & need) {
                            if (++spins > kSpinLimit) { state = 3; break; }
                            __nanosleep(spins < 64 ? 32 : 256);
                            continue;
                        }
                        unsigned long long mine = (lane <= first) ? (v2 & kValMask) : 0ull;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
                        excl += mine;
                        if (first < 32) break;
                        j -= 32;
                    }
                    if (lane == 0) {
                        if (state == 0 && excl + agg >= kMaxTotal) state = 2;
                        if (state == 3) raise_status(status, ST_TIMEOUT);
                        if (state == 2) raise_status(status, ST_BADARG);
                        st_release(sc.tiles + tile, state ? kFlagErr : (kFlagInc | (excl + agg)));
                    }
                }
                if (lane == 0) {
                    s_excl = excl;
                    s_state = state ? 2 : 0;
                }
            }
            __syncthreads();
            if (s_state == 0) {
                // ---- F at every prefix of this thread's items
                SlotGeom geo;
                geo.S = S;
                geo.M = (uint32_t)M;
                geo.MM = (unsigned long long)M << 32;
                geo.u32 = s_u32;
                unsigned long long c = s_excl + s_warp[wid] + (incl - tsum);  // C before item 0
                // first estimate in FP64 (once per thread): ceil(c M / S - u)
                const double ms = (double)M / (double)S;
                double x = (double)c * ms - (double)geo.u32 * 2.3283064365386963e-10;
                uint32_t F = slots_below(c, (long long)ceil(x), geo);
                if (tid == 0) s_lo = F;
                const float msf = (float)ms;
#pragma unroll
                for (int j = 0; j < kRsIpt; ++j) {
                    int64_t g = base + (int64_t)tid * kRsIpt + j;
                    uint32_t Fn = F;
                    if (q[j]) {
                        c += q[j];
                        float cnt = __ull2float_rn(q[j]) * msf;
                        Fn = slots_below(c, (long long)F + (long long)cnt, geo);
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
                uint32_t s0 = lo + (uint32_t)tid * per;
                uint32_t s1 = s0 + per < hi ? s0 + per : hi;
                if (s0 < s1) {
                    // first item whose inclusive F exceeds s0
                    int a = 0, b = kRsTile - 1;
                    while (a < b) {
                        int mid = (a + b) >> 1;
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
    }
    // ---- the last tile to finish resets the shared counters
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned long long d = atomicAdd(sc.done, 1ull);
        if (d == (unsigned long long)ntiles - 1) {
            *sc.ticket = 0ull;
            *sc.sum = 0ull;
            __threadfence();
            *sc.done = 0ull;
        }
    }
}

}  // namespace smc
