// resample.cuh -- kernels of the exact-integer systematic resampler
// (included by resample.cu and resample_var.cu).  The scratch words they
// use are passed in explicitly, so any owner of suitable device memory can
// run them.
//
// Pass 1 (k_resample_total): every tile of kRsTile weights is quantised
// (q = floor(W 2^52) from the FP64 bits) and reduced exactly; the tile's
// integer sum is stored.
// Between the passes (k_resample_finalize, one CTA): the tile sums become
// exclusive prefixes c_t and the call's constants (S, the uniform,
// fixed-point reciprocals) are formed once.
// Pass 2 (k_resample_scan, persistent over tiles): each tile reads its
// prefix (no waiting on other CTAs), each warp scans its 256 items, each
// thread divides its own starting c M = Q S + R by the fixed-point
// reciprocal (one correction) and carries F item by item, and each warp
// expands its own contiguous output range through shared memory; ranges
// too long for a warp go to k_resample_heavy.
//
// Pass 1 (and the normalisation of smc_reweight_resample, which forms the
// tile sums itself) runs over the tiles in descending order and pass 2 in
// ascending order, so the second read of the weights finds the most
// recently touched ones still in L2; loads and stores that are a datum's
// last use carry the streaming (evict-first) hint.
#pragma once
#include "device.cuh"
#include "bounds.cuh"

namespace smc {

constexpr int kRsThreads = 256;
constexpr int kRsIpt = 8;                      // weights per thread
constexpr int kRsTile = kRsThreads * kRsIpt;   // weights per tile
constexpr unsigned long long kMaxTotal = 1ull << 61;   // S must stay below this

// constants of one resampling call, formed once by k_resample_finalize
struct RsConst {
    unsigned long long S;       // exact total of the quantised weights
    unsigned long long Rth;     // floor(u32 S / 2^32)
    unsigned long long qheavy;  // items (and offsets) with q above this are divided afresh
    unsigned long long mfx;     // floor(M 2^64 / S) when M < S, else 0 (use FP64)
    unsigned long long ifx;     // floor(2^64 / S) when S > 1, else 0
    double m_over_s;            // M / S (FP64 estimates, only when M >= S)
    unsigned long long qlight;  // a thread run with total q up to this keeps every R' + d M < 2^64 - S
    uint32_t ok;                // 0: nothing to resample (status already raised)
};
constexpr int kRsConstWords = 8;

struct RsScratch {
    unsigned long long* tile_sum;   // [ntiles]: tile sums, then their exclusive prefixes
    RsConst* cst;                   // after the tile sums
    // grid-wide expansion of tiles with many output slots (optional: when
    // null, such a tile is expanded by its own CTA)
    unsigned long long* heavy_count;  // chunk records written, zero before pass 2
    uint4* heavy_list;                // {first item, items, chunk begin, chunk end}
    uint32_t* fpos;                   // [M] inclusive F of the items of heavy warp segments
};

__host__ __device__ constexpr int64_t rs_tiles(int64_t M) { return (M + kRsTile - 1) / kRsTile; }
// words of scratch for M weights: tile sums, constants
__host__ __device__ constexpr int64_t rs_words(int64_t M) {
    return rs_tiles(M) + kRsConstWords;
}
// items of one warp's segment of a tile in pass 2; a warp's staging row in
// shared memory (16 positions a lane) and the longest output range it
// expands there (the range start may sit up to 3 positions into the row)
constexpr int kRsSeg = 32 * kRsIpt;
constexpr int kRsWarpRow = 32 * 16;
constexpr int kRsWarpFill = kRsWarpRow - 4;
// output slots of one heavy-expansion chunk, and the most chunk records M
// weights can produce (a segment's range is split into chunks; ranges add to M)
constexpr int kRsChunk = 4096;
__host__ __device__ inline int64_t rs_heavy_records(int64_t M) {
    return rs_tiles(M) * (kRsTile / kRsSeg) + M / kRsChunk + 1;
}

// floor(w 2^52) from the bits of w in [0,1]; false if w is outside [0,1] or
// NaN.  On the 32-bit halves of w (an integer test on the whole word may be
// compiled to an FP64 comparison, and the FP64 pipe is narrow on this part).
__device__ __forceinline__ bool quantise(double w, unsigned long long& q) {
    const uint32_t hw = (uint32_t)__double2hiint(w), lw = (uint32_t)__double2loint(w);
    const uint32_t e = (hw >> 20) & 0x7FFu;
    const uint32_t mh = hw & 0xFFFFFu;
    const bool neg = (hw >> 31) != 0;
    const bool above = e > 1023u || (e == 1023u && (mh | lw) != 0u);  // > 1, inf, NaN
    const uint32_t sh = 1023u - e;                                     // w < 2^-sh ... 2^(1-sh)
    const unsigned long long man = ((unsigned long long)(mh | 0x100000u) << 32) | lw;
    const unsigned long long v = sh > 52u ? 0ull : (man >> (sh & 63u));
    q = (neg || above || e == 0u) ? 0ull : v;  // zero / subnormal / negative / invalid: 0
    return neg ? (hw == 0x80000000u && lw == 0u) : !above;  // -0 is a valid zero
}

// floor(w 2^52) for w in [0, 1] (what quantise gives there), without the
// validity test: q_fast's result for an invalid w is unspecified, and
// w_invalid tells whether w lies outside [0, 1] (or is NaN), -0 counting as
// a valid zero.  Branch-free, on the 32-bit halves.
__device__ __forceinline__ unsigned long long q_fast(double w) {
    // (2^52 + mantissa) >> sh with sh = 1023 - e, as 32-bit funnel shifts
    // (clamped: a shift of 32 or more leaves the high word, or 0)
    const uint32_t hw = (uint32_t)__double2hiint(w), lw = (uint32_t)__double2loint(w);
    const uint32_t e = (hw >> 20) & 0x7FFu;
    const uint32_t sh = 1023u - e;  // wraps for e > 1023 (invalid); 1023 for e = 0
    const uint32_t m21 = (hw & 0xFFFFFu) | 0x100000u;
    const uint32_t lo_a = __funnelshift_rc(lw, m21, sh);         // sh < 32
    const uint32_t lo_b = __funnelshift_rc(m21, 0u, sh - 32u);   // sh >= 32 (0 from 53 on)
    const uint32_t hi = __funnelshift_rc(m21, 0u, sh);           // 0 for sh >= 32
    const uint32_t lo = sh < 32u ? lo_a : lo_b;
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ bool w_invalid(double w) {
    const uint32_t hw = (uint32_t)__double2hiint(w), lw = (uint32_t)__double2loint(w);
    const bool neg_zero = (hw == 0x80000000u) & (lw == 0u);
    const bool above_one = (hw > 0x3FF00000u) | ((hw == 0x3FF00000u) & (lw != 0u));
    return above_one & !neg_zero;  // sign set, > 1, inf or NaN (all above 1.0's bits)
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

// load_tile_raw with the streaming hint (the weights' last read)
__device__ __forceinline__ void load_tile_raw_cs(const double* __restrict__ W, int64_t M,
                                                 int64_t tile, double (&v)[kRsIpt]) {
    const int64_t g0 = tile * kRsTile + (int64_t)threadIdx.x * kRsIpt;
    if (g0 + kRsIpt <= M && ((reinterpret_cast<uintptr_t>(W + g0) & 15u) == 0)) {
        const double2* p = reinterpret_cast<const double2*>(W + g0);
#pragma unroll
        for (int j = 0; j < kRsIpt / 2; ++j) {
            const double2 d = __ldcs(p + j);
            v[2 * j] = d.x;
            v[2 * j + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) v[j] = g0 + j < M ? __ldcs(W + g0 + j) : 0.0;
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

// Pass 1: the exact integer sum of every tile; tiles dealt round-robin in
// descending order, the next tile's weights loading while one is reduced,
// one barrier per tile (the warp sums alternate between two arrays).
static __global__ void __launch_bounds__(kRsThreads) k_resample_total(const double* __restrict__ W,
                                                               int64_t M, const int32_t* do_flag,
                                                               RsScratch sc, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long sh[2][kRsThreads / 32];
    const int64_t ntiles = rs_tiles(M);
    const int wid = threadIdx.x >> 5;
    bool bad = false;
    double vn[kRsIpt];
    int64_t kk = blockIdx.x;  // the kk-th tile from the top
    if (kk < ntiles) load_tile_raw(W, M, ntiles - 1 - kk, vn);
    for (int buf = 0; kk < ntiles; kk += gridDim.x, buf ^= 1) {
        const int64_t tile = ntiles - 1 - kk;
        unsigned long long acc = 0;  // <= 8 * 2^52: no wrap
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) {
            bad |= w_invalid(vn[j]);
            acc += q_fast(vn[j]);
        }
        if (kk + gridDim.x < ntiles) load_tile_raw(W, M, tile - gridDim.x, vn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0) sh[buf][wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long ts = 0;  // <= 2^63: no wrap
#pragma unroll
            for (int w = 0; w < kRsThreads / 32; ++w) ts += sh[buf][w];
            sc.tile_sum[tile] = ts;
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
struct QR {
    unsigned long long Q, R;
};
// (the constants by value: a call with a reference to the caller's copy
// would move that copy to local memory)
static __device__ __noinline__ QR divmod_cm_v(unsigned long long c, unsigned long long M,
                                              unsigned long long S, unsigned long long mfx,
                                              double m_over_s) {
    unsigned long long q;
    if (mfx) {
        q = __umul64hi(c, mfx);
    } else {
        const double qe = floor((double)c * m_over_s);
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
    return QR{q, r.lo};
}
__device__ __forceinline__ void divmod_cm(unsigned long long c, unsigned long long M,
                                          const RsConst& k, unsigned long long& Q,
                                          unsigned long long& R) {
    const QR t = divmod_cm_v(c, M, k.S, k.mfx, k.m_over_s);
    Q = t.Q;
    R = t.R;
}

// floor(Y / S) for Y = Rp + d M < 2^64 - S, S > 2^32 and a quotient below
// 2^31, from the fixed-point reciprocal f = floor(2^64 / S) < 2^32: the
// estimate n = floor(Y f / 2^64) (a 96-bit multiply-high by 32-bit pieces)
// is the quotient or one below it, and n + 1 is taken when Y >= (n + 1) S.
// Written in PTX so that every 64-bit step is one wide multiply-add.
__device__ __forceinline__ uint32_t quot_fx32(unsigned long long Rp, unsigned long long d,
                                              uint32_t m, uint32_t f, unsigned long long S) {
    uint32_t n;
    asm("{\n\t"
        ".reg .u32 dl, dh, yl, yh, lo, q, q1, tl, th, sl, sh;\n\t"
        ".reg .u64 Y, P, T, L;\n\t"
        ".reg .pred ge;\n\t"
        "mov.b64 {dl, dh}, %2;\n\t"
        "mad.wide.u32 Y, dl, %3, %1;\n\t"
        "mov.b64 {yl, yh}, Y;\n\t"
        "mad.lo.u32 yh, dh, %3, yh;\n\t"
        "mov.b64 Y, {yl, yh};\n\t"
        "mul.hi.u32 lo, yl, %4;\n\t"
        "cvt.u64.u32 L, lo;\n\t"
        "mad.wide.u32 P, yh, %4, L;\n\t"
        "mov.b64 {tl, q}, P;\n\t"
        "add.u32 q1, q, 1;\n\t"
        "mov.b64 {sl, sh}, %5;\n\t"
        "mul.wide.u32 T, q1, sl;\n\t"
        "mov.b64 {tl, th}, T;\n\t"
        "mad.lo.u32 th, q1, sh, th;\n\t"
        "mov.b64 T, {tl, th};\n\t"
        "setp.ge.u64 ge, Y, T;\n\t"
        "selp.u32 %0, q1, q, ge;\n\t"
        "}"
        : "=r"(n)
        : "l"(Rp), "l"(d), "r"(m), "r"(f), "l"(S));
    return n;
}

// c M = Q S + R exactly from the fixed-point reciprocal mfx = floor(M 2^64 /
// S) (M < S, c <= S < 2^61): Q' = floor(c mfx / 2^64) is Q or Q - 1 (the
// reciprocal's error times c is below 2^61 / 2^64), so one correction
// suffices; inline, no loop.
__device__ __forceinline__ void divmod_mfx(unsigned long long c, unsigned long long M,
                                           unsigned long long S, unsigned long long mfx,
                                           unsigned long long& Q, unsigned long long& R) {
    unsigned long long q = __umul64hi(c, mfx);
    const U128 r = sub128(mul64(c, M), mul64(q, S));  // < 2 S < 2^62: hi is 0
    const bool up = r.lo >= S;
    Q = q + (up ? 1ull : 0ull);
    R = r.lo - (up ? S : 0ull);
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

// The call's constants from the exact total S, into c: lane 0 of warps
// 0..5 forms one each (integer divisions side by side, no FP64 loop); the
// caller synchronises the block before reading c.  c.ok is not touched.
static __device__ __noinline__ void rs_form_constants(unsigned long long S, int64_t M, uint64_t seed,
                                                  uint64_t step, RsConst& c) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane != 0) return;
    const unsigned long long MM = (unsigned long long)M;
    if (wid == 0) {
        const uint32_t u32 = draw(seed, RNG_RESAMPLE, step, 0u, 0u).x;
        c.S = S;
        c.Rth = __umul64hi((unsigned long long)u32 << 32, S);  // floor(u32 S / 2^32)
    } else if (wid == 1) {
        c.mfx = MM < S ? (unsigned long long)(((unsigned __int128)MM << 64) / S) : 0ull;
    } else if (wid == 2) {
        c.ifx = S > 1 ? (0ull - S) / S + 1ull : 0ull;  // floor(2^64 / S)
    } else if (wid == 3) {
        // items (and thread runs) with q M <= 2^64 - S keep R + q M < 2^64,
        // where the fixed-point quotient is off by at most one (heavier
        // ones are divided afresh)
        c.qheavy = S > 1 ? (0ull - S) / MM : 0ull;
    } else if (wid == 4) {
        // R' < 2 S: d M <= 2^64 - 3 S keeps R' + d M below 2^64 - S
        c.qlight = S > 1 ? (0ull - 3ull * S) / MM : 0ull;
    } else if (wid == 5) {
        c.m_over_s = (double)MM / (double)S;
    }
}

// Between the passes, one CTA: the exact total S from the tile sums, the
// call's uniform and constants, and every tile's exclusive prefix c_t (the
// tile sums are replaced in place), so that no tile of pass 2 repeats this
// work.  kRsFinTiles tile sums at a time: each thread loads 8 consecutive
// ones (all loads in flight at once) and sums them, a warp scan and one
// scan of the 32 warp totals give every thread its offset, and each thread
// writes its 8 prefixes.  The four fixed-point constants are formed by four
// warps side by side (integer divisions, no FP64 loop).
constexpr int kRsFinThreads = 1024;
constexpr int kRsFinTiles = 8 * kRsFinThreads;
static __global__ void __launch_bounds__(kRsFinThreads) k_resample_finalize(
    int64_t M, uint64_t seed, uint64_t step, const int32_t* do_flag, RsScratch sc,
    uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ unsigned long long s_w[kRsFinThreads / 32];
    __shared__ unsigned long long s_tot;
    __shared__ int s_bad;
    __shared__ RsConst s_c;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = rs_tiles(M);
    if (tid == 0) s_bad = 0;
    unsigned long long run = 0;  // total of the blocks before this one
    bool ovf = false;
    for (int64_t base = 0; base < ntiles; base += kRsFinTiles) {
        const int64_t i0 = base + (int64_t)tid * 8;
        unsigned long long v[8];
        if (i0 + 8 <= ntiles && (reinterpret_cast<uintptr_t>(sc.tile_sum) & 15u) == 0) {
            const ulonglong2* p = reinterpret_cast<const ulonglong2*>(sc.tile_sum + i0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const ulonglong2 t = __ldcg(p + j);
                v[2 * j] = t.x;
                v[2 * j + 1] = t.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = i0 + j < ntiles ? __ldcg(sc.tile_sum + i0 + j) : 0ull;
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            tsum += v[j];
            ovf |= tsum < v[j];
        }
        unsigned long long incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) {
                incl += u;
                ovf |= incl < u;
            }
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {  // exclusive scan of the warp totals, in place
            const unsigned long long t = s_w[lane];
            unsigned long long x = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) {
                    x += u;
                    ovf |= x < u;
                }
            }
            s_w[lane] = x - t;
            if (lane == 31) s_tot = x;
        }
        __syncthreads();
        unsigned long long c = run + s_w[wid] + (incl - tsum);  // before this thread's first tile
        ovf |= c < run;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned long long x = v[j];
            v[j] = c;
            c += x;
        }
        if (i0 + 8 <= ntiles && (reinterpret_cast<uintptr_t>(sc.tile_sum) & 15u) == 0) {
            ulonglong2* p = reinterpret_cast<ulonglong2*>(sc.tile_sum + i0);
#pragma unroll
            for (int j = 0; j < 4; ++j) p[j] = make_ulonglong2(v[2 * j], v[2 * j + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (i0 + j < ntiles) sc.tile_sum[i0 + j] = v[j];
        }
        const unsigned long long nrun = run + s_tot;
        ovf |= nrun < run;
        run = nrun;
        __syncthreads();  // s_w and s_tot are rewritten by the next block
    }
    if (ovf) s_bad = 1;
    __syncthreads();
    const unsigned long long S = run;
    const bool good = !(S == 0 || S >= kMaxTotal || s_bad);
    if (good) rs_form_constants(S, M, seed, step, s_c);
    __syncthreads();
    if (tid == 0) {
        if (sc.heavy_count) *sc.heavy_count = 0ull;  // the scan appends from zero
        RsConst c = s_c;
        c.ok = good ? 1u : 0u;
        if (!good) raise_status(status, S == 0 && !s_bad ? ST_ZERO_WEIGHT : ST_BADARG);
        *sc.cst = c;
    }
}

// Minimum resident blocks per SM asked of the register allocator for the
// scan (compile-time tuning knob).
#ifndef SMC_RS_MINB
#define SMC_RS_MINB 3
#endif

// Pass 2, persistent over tiles in ascending order (each CTA's tiles too).
// Per tile: each thread quantises its 8 weights and each warp scans its 256
// items with shuffles; one barrier exchanges the warp totals; each thread
// divides c M = Q S + R at its own offset c and forms F at each inclusive
// prefix of its run from (Q, R); each warp writes its items' offspring
// counts and log-weight reset, and expands its own output range [lo, hi):
// by a fill-forward through shared memory when it holds at most kRsWarpFill
// slots, else as chunks for k_resample_heavy (or, without that scratch, by
// the warp itself).
static __global__ void __launch_bounds__(kRsThreads, SMC_RS_MINB) k_resample_scan(
    const double* __restrict__ W, int64_t M, const int32_t* do_flag, RsScratch sc,
    int32_t* __restrict__ anc, int32_t* __restrict__ counts, double* __restrict__ lwreset,
    uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    __shared__ uint32_t s_hi[kRsTile];                          // inclusive F of each item
    // a warp's staged slots, from its range start rounded down to 4 slots
    __shared__ __align__(16) int32_t s_anc[kRsThreads / 32][kRsWarpRow];
    __shared__ unsigned long long s_warp[2][kRsThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = rs_tiles(M);

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
    const bool ifx32 = ifx != 0 && (ifx >> 32) == 0;  // S > 2^32
    const bool anc16 = (reinterpret_cast<uintptr_t>(anc) & 15u) == 0;
    // carry R + a M (< 2^64 for a <= qheavy) into Q: n = floor((R + a M) / S)
    // from the fixed-point reciprocal ifx = floor(2^64 / S) (integer
    // multiply-high, off by at most one below) and one correction
    auto carry = [&](unsigned long long& Q, unsigned long long& R, unsigned long long a) {
        const unsigned long long R2 = R + a * MM;
        unsigned long long n = __umul64hi(R2, ifx);
        unsigned long long r = R2 - n * S;
        const bool hi1 = r >= S;
        Q += n + (hi1 ? 1ull : 0ull);
        R = r - (hi1 ? S : 0ull);
    };
    // persistent over tiles; the next tile's weights, prefix, Q and R load
    // while the current one is processed
    int64_t k = blockIdx.x;
    {  // the staging rows start below every mark
        int4* mine = reinterpret_cast<int4*>(s_anc[wid] + 16 * lane);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mine[kk] = make_int4(-1, -1, -1, -1);
        __syncwarp();
    }
    double vn[kRsIpt];
    unsigned long long pn = 0;
    if (k < ntiles) {
        const int64_t t = k;
        load_tile_raw_cs(W, M, t, vn);
        pn = __ldcg(sc.tile_sum + t);
    }
    for (int buf = 0; k < ntiles; k += gridDim.x, buf ^= 1) {
        const int64_t tile = k;
        const int64_t base = tile * kRsTile;
        unsigned long long q[kRsIpt];
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) q[j] = q_fast(vn[j]);  // pass 1 reported bad weights
        const unsigned long long tpre = pn;
        if (k + gridDim.x < ntiles) {
            const int64_t t = k + gridDim.x;
            load_tile_raw_cs(W, M, t, vn);
            pn = __ldcg(sc.tile_sum + t);
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) tsum += q[j];
        // ---- warp inclusive scan, then the warp totals across the block
        unsigned long long incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[buf][wid] = incl;
        __syncthreads();
        unsigned long long woff = 0;
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w)
            if (w < wid) woff += s_warp[buf][w];
        const unsigned long long off = woff + (incl - tsum);  // this thread's offset in the tile
        unsigned long long c = tpre + off;                    // C before this thread's item 0
        unsigned long long Q, R;
        uint32_t Fv[kRsIpt];
        uint32_t F0;
        // the usual case, taken per warp: the starting quotient from the
        // fixed-point reciprocal, and the thread's whole run light enough
        // that R' + d M < 2^64 for every prefix d of its run.  With
        // R' = R + S - 1 - Rth (< 2 S), floor((R' + d M) / S) counts the
        // slots below the prefix beyond Q: writing R + d M = n S + r,
        // R' + d M = n S + r + S - 1 - Rth, whose quotient is n + [r > Rth].
        // So each item's F = Q + floor((R' + d_j M) / S) comes from the
        // thread's (Q, R') independently of the other items, and the eight
        // divisions overlap instead of forming a chain.
        const bool light = cst.mfx != 0 && tsum <= cst.qlight;
        if (__all_sync(0xFFFFFFFFu, light)) {
            divmod_mfx(c, MM, S, cst.mfx, Q, R);
            const unsigned long long Rp = R + (S - 1ull - Rth);
            F0 = (uint32_t)Q + (Rp >= S ? 1u : 0u);
            unsigned long long d = 0;
            if (ifx32) {
                // S > 2^32 (normalised weights give S ~ 2^52): the
                // reciprocal and every quotient fit 32 bits
                const uint32_t f32 = (uint32_t)ifx, m32 = (uint32_t)MM;
#pragma unroll
                for (int j = 0; j < kRsIpt; ++j) {
                    d += q[j];
                    const uint32_t Fn = (uint32_t)Q + quot_fx32(Rp, d, m32, f32, S);
                    Fv[j] = Fn < (uint32_t)M ? Fn : (uint32_t)M;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kRsIpt; ++j) {
                    d += q[j];
                    const unsigned long long Y = Rp + d * MM;
                    const unsigned long long n = __umul64hi(Y, ifx);
                    const bool up = Y - n * S >= S;
                    const unsigned long long Fn = Q + n + (up ? 1ull : 0ull);
                    Fv[j] = Fn < MM ? (uint32_t)Fn : (uint32_t)M;
                }
            }
        } else {
            divmod_cm(c, MM, cst, Q, R);
            F0 = (uint32_t)(Q + (R > Rth ? 1ull : 0ull));
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j) {
                c += q[j];
                if (q[j] > qheavy) divmod_cm(c, MM, cst, Q, R);  // a heavy item, divided afresh
                else carry(Q, R, q[j]);
                const uint32_t Fn = (uint32_t)(Q + (R > Rth ? 1ull : 0ull));
                Fv[j] = Fn < (uint32_t)M ? Fn : (uint32_t)M;
            }
        }
        // ---- offspring counts and log-weight reset: 8 consecutive per thread
        const int64_t g0 = base + (int64_t)tid * kRsIpt;
        const bool full = g0 + kRsIpt <= M;
        if (counts) {
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j)
                if (g0 + j < M) __stcs(counts + g0 + j, (int32_t)(Fv[j] - (j ? Fv[j - 1] : F0)));
        }
        if (lwreset) {
            if (full && ((reinterpret_cast<uintptr_t>(lwreset + g0) & 15u) == 0)) {
                double2* d2 = reinterpret_cast<double2*>(lwreset + g0);
#pragma unroll
                for (int j = 0; j < kRsIpt / 2; ++j) __stcs(d2 + j, make_double2(0.0, 0.0));
            } else {
#pragma unroll
                for (int j = 0; j < kRsIpt; ++j)
                    if (g0 + j < M) __stcs(lwreset + g0 + j, 0.0);
            }
        }
        // ---- this warp's output range [lo, hi)
        const uint32_t lo = __shfl_sync(0xFFFFFFFFu, F0, 0);
        const uint32_t hi = __shfl_sync(0xFFFFFFFFu, Fv[kRsIpt - 1], 31);
        if (hi < lo || hi > (uint32_t)M) {  // cannot happen with consistent sums
            if (lane == 0) raise_status(status, ST_BADARG);
            continue;
        }
        const uint32_t range = hi - lo;
        const int32_t i0 = (int32_t)g0;  // this thread's first item
        if (range <= (uint32_t)kRsWarpFill) {  // uniform over the warp
            // Fill-forward through shared memory: each item with offspring
            // marks its first slot with its index, and each slot's ancestor
            // is the largest mark at or before it (items increase with
            // their slots).  The rows are never cleared: a CTA's tiles
            // ascend, so marks left by earlier tiles are smaller than this
            // tile's, and the slot at lo always holds one of this tile's.
            // Lane l owns row positions [16 l, 16 l + 16): the maximum of
            // its 16, a warp maximum-scan across the lanes, then a running
            // maximum from the lanes before.  Slot sl sits at sl - lo_al
            // (lo_al = lo rounded down to 4 slots when the ancestors are
            // 16-byte aligned, so 4 positions are one 16-byte store).  No
            // loops and no divergence, whatever the offspring counts.
            const uint32_t lo_al = anc16 ? (lo & ~3u) : lo;
            int32_t* row = s_anc[wid];
            const int4* mine = reinterpret_cast<const int4*>(row + 16 * lane);
            uint32_t f = F0;
#pragma unroll
            for (int j = 0; j < kRsIpt; ++j) {
                const uint32_t e = Fv[j];
                if (e > f) row[f - lo_al] = i0 + j;
                f = e;
            }
            __syncwarp();
            int32_t v[16];
#pragma unroll
            for (int kq = 0; kq < 4; ++kq) {
                const int4 t = mine[kq];
                v[4 * kq] = t.x;
                v[4 * kq + 1] = t.y;
                v[4 * kq + 2] = t.z;
                v[4 * kq + 3] = t.w;
            }
            int32_t run = max(max(max(v[0], v[1]), max(v[2], v[3])),
                              max(max(v[4], v[5]), max(v[6], v[7])));
            run = max(run, max(max(max(v[8], v[9]), max(v[10], v[11])),
                               max(max(v[12], v[13]), max(v[14], v[15]))));
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xFFFFFFFFu, run, o);
                if (lane >= o) run = max(run, u);
            }
            int32_t before = __shfl_up_sync(0xFFFFFFFFu, run, 1);
            v[0] = lane ? max(v[0], before) : v[0];
#pragma unroll
            for (int kq = 1; kq < 16; ++kq) v[kq] = max(v[kq], v[kq - 1]);
            const uint32_t s0 = lo_al + 16u * (uint32_t)lane;  // the slot of v[0]
            if (anc16) {
                // 4 slots a store; a group cut by the range's ends (at most
                // one at each end of the warp's range) slot by slot
#pragma unroll
                for (int kq = 0; kq < 4; ++kq) {
                    const uint32_t sg = s0 + 4u * kq;
                    if (sg >= lo && sg + 4u <= hi) {
                        __stcs(reinterpret_cast<int4*>(anc + sg),
                               make_int4(v[4 * kq], v[4 * kq + 1], v[4 * kq + 2], v[4 * kq + 3]));
                    } else if (sg < hi && sg + 4u > lo) {
#pragma unroll
                        for (int t = 0; t < 4; ++t)
                            if (sg + t >= lo && sg + t < hi) __stcs(anc + sg + t, v[4 * kq + t]);
                    }
                }
            } else if (s0 < hi) {
#pragma unroll
                for (int kq = 0; kq < 16; ++kq)
                    if (s0 + kq < hi) __stcs(anc + s0 + kq, v[kq]);
            }
            __syncwarp();
            continue;
        }
        // a long range (heavy weights): the items' inclusive F for the
        // bisections, then chunks for k_resample_heavy or the warp itself
        const int64_t sbase = base + (int64_t)wid * kRsSeg;  // the warp's first item
        const int nit = (int)(M - sbase < kRsSeg ? M - sbase : kRsSeg);
        uint32_t* fs = s_hi + wid * kRsSeg;
#pragma unroll
        for (int j = 0; j < kRsIpt; ++j) fs[lane * kRsIpt + j] = Fv[j];
        __syncwarp();
        if (sc.heavy_list) {
            for (int j = lane; j < nit; j += 32) sc.fpos[sbase + j] = fs[j];
            if (lane == 0) {
                const uint32_t nch = (range + kRsChunk - 1) / kRsChunk;
                const unsigned long long r0 = atomicAdd(sc.heavy_count, (unsigned long long)nch);
                for (uint32_t kk = 0; kk < nch; ++kk) {
                    const uint32_t b = lo + kk * kRsChunk;
                    const uint32_t e = b + kRsChunk < hi ? b + kRsChunk : hi;
                    sc.heavy_list[r0 + kk] = make_uint4((uint32_t)sbase, (uint32_t)nit, b, e);
                }
            }
            continue;
        }
        const uint32_t per = (range + 31) / 32;
        const uint32_t s0 = lo + (uint32_t)lane * per;
        const uint32_t s1 = s0 + per < hi ? s0 + per : hi;
        if (s0 < s1) {
            int a = 0, b = nit - 1;  // first item whose inclusive F exceeds s0
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (fs[mid] > s0) b = mid;
                else a = mid + 1;
            }
            int item = a;
            for (uint32_t sl = s0; sl < s1; ++sl) {
                while (SMC_IN_BOUNDS(item < nit, status) && fs[item] <= sl) ++item;
                if (SMC_IN_BOUNDS(sl < (uint32_t)M && item < nit, status))
                    anc[sl] = (int32_t)(sbase + item);
            }
        }
    }
}

// Pass 3: the chunks of heavy warp segments, shared by all CTAs
// (grid-stride).  A chunk's first item is found by bisection on the
// segment's inclusive F values; its slots are staged in shared memory and
// stored slot-major.
static __global__ void __launch_bounds__(kRsThreads) k_resample_heavy(
    const int32_t* do_flag, RsScratch sc, int64_t M, int32_t* __restrict__ anc,
    uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    if (do_flag && *do_flag == 0) return;
    __shared__ int32_t s_anc[kRsChunk];
    const unsigned long long n = __ldcg(sc.heavy_count);
    for (unsigned long long r = blockIdx.x; r < n; r += gridDim.x) {
        const uint4 rec = sc.heavy_list[r];
        const int64_t base = (int64_t)rec.x;
        const int nit = (int)rec.y;
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
                while (SMC_IN_BOUNDS(item < nit, status) && f[item] <= sl) ++item;
                if (SMC_IN_BOUNDS(sl - b < (uint32_t)kRsChunk && item < nit, status))
                    s_anc[sl - b] = (int32_t)(base + item);
            }
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < e - b; k += kRsThreads)
            if (SMC_IN_BOUNDS(k < (uint32_t)kRsChunk && (int64_t)b + k < M, status))
                __stcs(anc + b + k, s_anc[k]);
        __syncthreads();
    }
}

}  // namespace smc
