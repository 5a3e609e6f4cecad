// device.cuh -- device primitives shared by the sm_103a kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) written from its
// published definition, the uniform and Box-Muller transforms of the
// library's random streams, MUFU wrappers, warp reductions, the device
// status word and the helpers that keep FP64 instructions out of per-element
// loops (GB300 has very little FP64 throughput).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace smc {

// ---------------------------------------------------------------- status
enum : uint32_t {
    ST_NONFINITE = 1u, ST_ZERO_WEIGHT = 2u, ST_TIMEOUT = 4u, ST_BADARG = 8u
};

__device__ __forceinline__ void raise_status(uint32_t* st, uint32_t bit) {
    if (st) atomicOr(st, bit);
}

// Upper bound on polls of a flag written by another CTA; with the
// nanosleep back-off this is a few seconds, far beyond any legal wait.
constexpr uint32_t kSpinLimit = 4u << 20;

// ---------------------------------------------------------------- Philox
enum : uint32_t {
    RNG_MOVE = 1, RNG_ACCEPT = 2, RNG_RESAMPLE = 3, RNG_EXCHANGE = 4, RNG_PFNOISE = 5,
    RNG_MULTINOMIAL = 6, RNG_PROPOSAL = 7
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// counter = (index, block, step lo, purpose | step hi << 8), key = seed halves
__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t purpose, uint64_t step,
                                      uint32_t index, uint32_t block) {
    uint4 c = make_uint4(index, block, (uint32_t)step,
                         (purpose & 0xFFu) | ((uint32_t)(step >> 32) << 8));
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int i) {
    return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

// Integer <-> float helpers built from float bit patterns.  On sm_103a the
// conversion instructions share the narrow FP64 pipe, so per-element code
// avoids them.
// m in [0, 2^23) -> float, exactly (m is the mantissa of 2^23 + m)
__device__ __forceinline__ float u23_to_f(uint32_t m) {
    return __uint_as_float(0x4B000000u | m) - 8388608.0f;
}
// round to the nearest integer for |x| < 2^22: float value and int value
__device__ __forceinline__ float round_magic(float x, int& ki) {
    const float t = x + 12582912.0f;  // 1.5 * 2^23
    ki = (int)__float_as_uint(t) - 0x4B400000;
    return t - 12582912.0f;
}

// (2k+1) 2^-24 with k the top 23 bits: exact in float, strictly inside (0,1)
// (k 2^-23 is 1.k - 1 read from the bits, then + 2^-24, both exact)
__device__ __forceinline__ float u01(uint32_t w) {
    return (__uint_as_float(0x3F800000u | (w >> 9)) - 1.0f) + 5.9604644775390625e-08f;
}

// Box-Muller on one word pair: r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2)
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    float r = sqrtf(-2.0f * logf(u01(a)));
    float s, c;
    sincospif(2.0f * u01(b), &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// normals j < n of (seed, purpose, step, index): pair p uses words 2p, 2p+1
template <int NMAX>
__device__ __forceinline__ void normals(uint64_t seed, uint32_t purpose, uint64_t step,
                                        uint32_t index, int n, float (&z)[NMAX]) {
#pragma unroll
    for (int b = 0; b < (NMAX + 3) / 4; ++b) {
        if (4 * b < n) {
            uint4 w = draw(seed, purpose, step, index, (uint32_t)b);
            float z0, z1, z2, z3;
            box_muller(w.x, w.y, z0, z1);
            box_muller(w.z, w.w, z2, z3);
            if (4 * b + 0 < NMAX) z[4 * b + 0] = z0;
            if (4 * b + 1 < NMAX) z[4 * b + 1] = z1;
            if (4 * b + 2 < NMAX) z[4 * b + 2] = z2;
            if (4 * b + 3 < NMAX) z[4 * b + 3] = z3;
        }
    }
}

// ---------------------------------------------------------------- MUFU
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr double kLn2 = 0.6931471805599453094;
constexpr double kLog2e = 1.4426950408889634074;

// ---------------------------------------------------------------- FP64-light helpers
// Split of a double into hi + lo floats by integer operations only (no
// FP64 pipe): hi keeps the top 24 significant bits (truncated), lo the next
// 23 (truncated), so hi + lo is within 2^-46 of the double, relatively.  The magnitude
// is first clamped to [2^-74, 2^100) by the exponent field: smaller values
// (zero included) become +-2^-74 and larger ones (infinities too) about
// +-2^100 -- the callers only exponentiate differences of such splits, for
// which both ends are exact enough.  Branch-free.
__device__ __forceinline__ void split_double(double d, float& hi, float& lo) {
    const uint32_t hw = (uint32_t)__double2hiint(d), lw = (uint32_t)__double2loint(d);
    const uint32_t sign = hw & 0x80000000u;
    // |d|'s high word with the exponent clamped to [1023 - 74, 1023 + 99]
    const uint32_t a = min(max(hw & 0x7FFFFFFFu, 0x3B500000u), 0x462FFFFFu);
    // hi: exponent re-biased from 1023 to 127, 20 + 3 mantissa bits
    hi = __uint_as_float(sign | __funnelshift_l(lw, a - 0x38000000u, 3));
    // lo: the next 23 mantissa bits m, worth m 2^(e - 1075 + 6): the float
    // (2^23 + m) 2^(e - 1069 - 23) less 2^(e - 1069), signs alike (exact)
    const uint32_t eb = sign | (((a & 0x7FF00000u) - (919u << 20)) << 3);
    lo = __uint_as_float(eb | ((lw >> 6) & 0x7FFFFFu)) - __uint_as_float(eb);
}

// exp(d) for an FP64 d <= 0 given as hi + lo floats, in FP32: the argument
// is reduced in double-float (Cody-Waite style split of log2 e), 2^f comes
// from ex2.approx and 2^k is assembled in the exponent.  Results below
// 2^-126 flush to 0.  Relative error ~ 2^-22.
__device__ __forceinline__ float exp_hilo(float hi, float lo) {
    const float L2E_HI = 1.44269502162933349609375f;   // log2(e) rounded to float
    const float L2E_LO = 1.925963033500011e-08f;       // log2(e) - L2E_HI
    const float ph = hi * L2E_HI;
    // below 2^-126 (also -inf): 0, selected at the end (no branch)
    const float phc = fmaxf(ph, -127.5f);
    int ki;
    const float k = round_magic(phc, ki);              // |phc| < 2^22 here
    const float pl = fmaf(hi, L2E_HI, -ph);
    const float f = (phc - k) + (pl + fmaf(hi, L2E_LO, lo * L2E_HI));
    const float p2 = __uint_as_float((uint32_t)(ki + 127) << 23);
    return (ph < -127.0f || ki < -126) ? 0.0f : ex2(f) * p2;
}

// Programmatic dependent launch: kernels of consecutive calls on a stream are
// launched with programmatic serialisation; grid_dep_wait() holds the thread
// until the previous grid has finished and its writes are visible, and
// grid_dep_launch() lets the next grid start launching.  Both are no-ops for
// a launch without the programmatic attribute.
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// FP64 -> sortable signed 64-bit key (total order for non-NaN values)
__device__ __forceinline__ long long dkey(double x) {
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
// on the 32-bit halves (an integer test on the whole word may be compiled
// to an FP64 comparison, and the FP64 pipe is narrow on this part)
__device__ __forceinline__ bool disnan(double x) {
    const uint32_t h = (uint32_t)__double2hiint(x) & 0x7FFFFFFFu;
    return (h > 0x7FF00000u) | ((h == 0x7FF00000u) & (__double2loint(x) != 0));
}

// float -> double by integer operations (subnormal floats give 0)
__device__ __forceinline__ double f2d_bits(float f) {
    uint32_t u = __float_as_uint(f);
    uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    if (e == 255) return (double)f;  // inf / NaN
    unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                           ((unsigned long long)(e - 127 + 1023) << 52) |
                           ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum_d(double v, unsigned mask = 0xFFFFFFFFu) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Kahan accumulation in FP32 (the accumulated values share one sign here)
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

}  // namespace smc
