// reweight.cuh -- the reweighting reduction shared by smc_reweight,
// smc_reweight_resample and the fused particle-filter step: per-thread sums
// of exp(logw - r) against slack references on float hi/lo splits (no FP64
// instruction per element), block and grid combination in FP64, and the
// final scalars (log-evidence increment, ESS, maximum, LSE).
#pragma once
#include <climits>
#include <cmath>

#include "ctx.hpp"
#include "device.cuh"

namespace smc {

// exp(dh + dl) for a non-positive difference given as float hi/lo parts,
// per element: one FFMA, one FMUL and ex2.approx (flushes below 2^-126 to
// 0).  The rounding of the base-2 argument t = (dh + dl) log2(e) is about
// 2^-24 |t|, so the relative error is ~2^-22 + 4.1e-8 |t| -- within the
// weights' stated error of 1e-6 + 1e-7 |ln(W / W_max)| at every t, and
// below 2e-7 of a sum for the usual spread of log-weights.
__device__ __forceinline__ float exp_hl(float dh, float dl) {
    const float L2E = 1.44269504088896340736f;
    return ex2(fmaf(dh, L2E, dl * L2E));
}

// exp(x) for an FP64 x <= 64 (FP32 accuracy, float result)
__device__ __forceinline__ float expd(double x) {
    float hi, lo;
    split_double(x, hi, lo);
    return exp_hilo(hi, lo);
}

constexpr double kNegInf = -INFINITY;
__device__ __forceinline__ bool is_neg_inf(double x) {  // on the 32-bit halves
    return (uint32_t)__double2hiint(x) == 0xFFF00000u && __double2loint(x) == 0;
}

// Element loops take chunks of 8 consecutive doubles per thread and
// iteration (four 16-byte loads issued before any use), so each SM keeps
// enough bytes in flight to cover HBM latency; a scalar loop handles the
// tail and unaligned arrays.
constexpr int kChunk = 8;

__device__ __forceinline__ bool aligned16(const void* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

__device__ __forceinline__ void load8(const double* __restrict__ p, double (&v)[kChunk]) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 t[kChunk / 2];
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j) t[j] = q[j];
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j) { v[2 * j] = t[j].x; v[2 * j + 1] = t[j].y; }
}

// load8 with the streaming hint (the data's last read)
__device__ __forceinline__ void load8_cs(const double* __restrict__ p, double (&v)[kChunk]) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 t[kChunk / 2];
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j) t[j] = __ldcs(q + j);
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j) { v[2 * j] = t[j].x; v[2 * j + 1] = t[j].y; }
}

__device__ __forceinline__ void store8(double* __restrict__ p, const double (&v)[kChunk]) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j) q[j] = make_double2(v[2 * j], v[2 * j + 1]);
}

// An L2 eviction policy that keeps lines longer than the default (the
// data's next read follows soon in the same call), and store8 with it.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void store8_keep(double* __restrict__ p, const double (&v)[kChunk],
                                            uint64_t pol) {
#pragma unroll
    for (int j = 0; j < kChunk / 2; ++j)
        asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;"
                     :: "l"(p + 2 * j), "d"(v[2 * j]), "d"(v[2 * j + 1]), "l"(pol) : "memory");
}

// FP32 sum with its rounding error carried (Knuth's two-sum): the running
// error stays below 2^-24 of the sum's magnitude times a few, without the
// long-latency FP64 pipe.
struct F2Sum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float bb = t - s;
        c += (s - (t - bb)) + (x - bb);
        s = t;
    }
    __device__ __forceinline__ void add(const F2Sum& o) {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ void warp_sum() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            F2Sum o;
            o.s = __shfl_xor_sync(0xFFFFFFFFu, s, off);
            o.c = __shfl_xor_sync(0xFFFFFFFFu, c, off);
            add(o);
        }
    }
    __device__ __forceinline__ double value() const { return f2d_bits(s) + f2d_bits(c); }
};

// Thread-level sums against a slack reference r: e = exp(x - r) may exceed
// 1 (up to e^32) so the reference moves only when an element exceeds it by
// more than 32 nats, not at every new maximum.  No FP64 instruction per
// element: x and r are split into float hi + lo parts by integer operations
// and x - r is taken as the pair (xh - rh, xl - rl); the hi difference is
// exact when x and r are within a factor 2 and otherwise rounded once
// (relative error 2^-24 of the difference), which the exponential turns
// into a relative error of at most 2^-24 |x - r| in e.
struct RefSums {
    double r = kNegInf;
    float rh = -1e30f, rl = 0.0f;            // (below every weight until one arrives)
    float s1 = 0.0f, s2 = 0.0f;
    float c1 = 0.0f, c2 = 0.0f;              // rounding errors carried by add8's merges
    bool any = false;
    long long kmax = LLONG_MIN;               // key of the largest element
    __device__ __forceinline__ float sum1() const { return s1 + c1; }
    __device__ __forceinline__ float sum2() const { return s2 + c2; }
    __device__ __forceinline__ void add(double x) {
        if (is_neg_inf(x)) return;            // zero weight
        const long long k = dkey(x);
        kmax = k > kmax ? k : kmax;
        float xh, xl;
        split_double(x, xh, xl);
        if (!any) { r = x; rh = xh; rl = xl; s1 = 1.0f; s2 = 1.0f; any = true; return; }
        const float dh = xh - rh, dl = xl - rl;
        if (dh > 32.0f) {                     // move the reference up to x
            const float f = exp_hl(-dh, -dl);
            s1 = fmaf(s1, f, 1.0f);
            s2 = fmaf(s2, f * f, 1.0f);
            r = x; rh = xh; rl = xl;
        } else {
            const float e = exp_hl(dh, dl);
            s1 += e;
            s2 = fmaf(e, e, s2);
        }
    }
};

// Eight elements at once against the thread's running reference r (no
// exact chunk maximum, no key compares unless the maximum is tracked): e_j
// = exp(x_j - r) on float hi/lo splits as in RefSums::add, tree sums of e
// and e^2, then a two-sum merge into the running sums (the rounding errors
// carried in c1, c2).  The reference moves to a chunk element whose hi part
// exceeds it (the sums are rescaled by one exponential, at most 1), so the
// dominant terms keep small exponents and their FP32 arguments small
// errors; the first chunk holding a weight sets it.  Zero weights (-inf,
// split to -1e30) add nothing.  With track_max the exact maximum (integer
// keys) is kept too.
__device__ __forceinline__ void add8(RefSums& t, const double (&x)[kChunk], bool track_max) {
    float xh[kChunk], xl[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) split_double(x[j], xh[j], xl[j]);
    if (track_max) {
        long long km = dkey(x[0]);
#pragma unroll
        for (int j = 1; j < kChunk; ++j) {
            const long long k = dkey(x[j]);
            km = k > km ? k : km;
        }
        t.kmax = km > t.kmax ? km : t.kmax;
    }
    float mh = xh[0];
#pragma unroll
    for (int j = 1; j < kChunk; ++j) mh = fmaxf(mh, xh[j]);
    if (mh > t.rh) {  // a new reference: the (last) element with the largest hi part
        double rn = x[0];
        float nh = xh[0], nl = xl[0];
#pragma unroll
        for (int j = 1; j < kChunk; ++j) {
            const bool m = xh[j] == mh;
            rn = m ? x[j] : rn;
            nh = m ? xh[j] : nh;
            nl = m ? xl[j] : nl;
        }
        if (t.any) {
            const float f = exp_hl(t.rh - nh, t.rl - nl);
            t.s1 *= f;
            t.c1 *= f;
            t.s2 *= f * f;
            t.c2 *= f * f;
        }
        t.r = rn;
        t.rh = nh;
        t.rl = nl;
        t.any = true;
    }
    if (!t.any) return;  // only zero weights so far
    float e[kChunk], e2[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
        e[j] = exp_hl(xh[j] - t.rh, xl[j] - t.rl);  // ~<= 1
        e2[j] = e[j] * e[j];
    }
#pragma unroll
    for (int w = 1; w < kChunk; w <<= 1)
#pragma unroll
        for (int j = 0; j + w < kChunk; j += 2 * w) {
            e[j] += e[j + w];
            e2[j] += e2[j + w];
        }
    F2Sum a{t.s1, t.c1}, b{t.s2, t.c2};
    a.add(e[0]);
    b.add(e2[0]);
    t.s1 = a.s;
    t.c1 = a.c;
    t.s2 = b.s;
    t.c2 = b.c;
}

// block / grid level: FP64 sums relative to a reference m
struct Lse {
    double m, s1, s2;
};

__device__ __forceinline__ double key_to_double(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

__device__ __forceinline__ long long warp_max_key(long long key) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xFFFFFFFFu, key, o);
        key = k2 > key ? k2 : key;
    }
    return key;
}

// Block combination of thread sums: the block's reference is the largest
// thread reference (integer comparison of FP64 keys), every thread rescales
// its FP32 sums to it with one exponential, then FP32 block sums.  Result
// valid in thread 0.
__device__ __forceinline__ Lse block_combine(const RefSums& t, long long* s_key, float* s_a,
                                             float* s_b, double* max_out) {
    long long key = warp_max_key(t.any ? dkey(t.r) : LLONG_MIN);
    long long kmx = warp_max_key(t.kmax);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_key[w] = key; s_key[16 + w] = kmx; }
    __syncthreads();
    long long bk = LLONG_MIN, bm = LLONG_MIN;
    for (int i = 0; i < nw; ++i) {
        bk = s_key[i] > bk ? s_key[i] : bk;
        bm = s_key[16 + i] > bm ? s_key[16 + i] : bm;
    }
    __syncthreads();
    Lse out{kNegInf, 0.0, 0.0};
    *max_out = bm == LLONG_MIN ? kNegInf : key_to_double(bm);
    if (bk == LLONG_MIN) return out;  // every weight zero in this block
    const double R = key_to_double(bk);
    float a = 0.0f, b = 0.0f;
    if (t.any) {
        const float f = expd(t.r - R);  // <= 1
        a = t.sum1() * f;
        b = t.sum2() * f * f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { s_a[w] = a; s_b[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float A = 0.0f, B = 0.0f;
        for (int i = 0; i < nw; ++i) { A += s_a[i]; B += s_b[i]; }
        out = Lse{R, f2d_bits(A), f2d_bits(B)};
    }
    __syncthreads();
    return out;
}

// Combine the per-block partials in the last block: the common reference is
// the largest block reference (integer keys), each partial is scaled to it
// with one FP32 exponential and the sums are reduced in FP64 as a parallel
// tree -- no long serial chain of FP64 operations (FP64 latency is long on
// this part).  Result valid in thread 0; `off` selects {ref, s1, s2} at 0 or
// {ref_old, s_old} at 3.
__device__ __forceinline__ Lse combine_partials(const double* partials, int nblocks, int off,
                                                long long* s_key) {
    long long k = LLONG_MIN;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double r = __ldcg(partials + (size_t)b * 8 + off);
        if (!is_neg_inf(r)) { const long long kk = dkey(r); k = kk > k ? kk : k; }
    }
    k = warp_max_key(k);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) s_key[w] = k;
    __syncthreads();
    long long bk = LLONG_MIN;
    for (int i = 0; i < nw; ++i) bk = s_key[i] > bk ? s_key[i] : bk;
    __syncthreads();
    Lse out{kNegInf, 0.0, 0.0};
    if (bk == LLONG_MIN) return out;
    float Rh, Rl;
    const double R = key_to_double(bk);
    split_double(R, Rh, Rl);
    // FP64 accumulation, but only short dependent chains: a few partials per
    // thread, then a 5-level shuffle tree and 8 warp totals
    double a = 0.0, bsum = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* P = partials + (size_t)b * 8 + off;
        const double r = __ldcg(P);
        if (is_neg_inf(r)) continue;
        float h, l;
        split_double(r, h, l);
        const float f = exp_hilo(h - Rh, l - Rl);  // <= 1
        a = fma(__ldcg(P + 1), f2d_bits(f), a);
        if (off == 0) bsum = fma(__ldcg(P + 2), f2d_bits(f * f), bsum);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        bsum += __shfl_xor_sync(0xFFFFFFFFu, bsum, o);
    }
    __shared__ double s_da[32], s_db[32];
    if ((threadIdx.x & 31) == 0) { s_da[w] = a; s_db[w] = bsum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int i = 0; i < nw; ++i) { A += s_da[i]; B += s_db[i]; }
        out = Lse{R, A, B};
    }
    __syncthreads();
    return out;
}

__device__ __forceinline__ double ln_sum(double s) {
    return (double)(lg2((float)s) * 0.69314718055994531f);
}

// Both block combinations of the reweight reduction in one pass (the new
// log-weights' sums with their maximum, and the old ones' sums): the same
// references, scalings and summation orders as two calls of block_combine,
// with two barriers instead of eight.  Results valid in thread 0.
__device__ __forceinline__ void block_combine2(const RefSums& c, const RefSums& o, bool has_old,
                                               long long* s_key, float* s_f, Lse* outc,
                                               Lse* outo, double* max_out) {
    const long long kc = warp_max_key(c.any ? dkey(c.r) : LLONG_MIN);
    const long long km = warp_max_key(c.kmax);
    const long long ko = has_old ? warp_max_key(o.any ? dkey(o.r) : LLONG_MIN) : LLONG_MIN;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_key[w] = kc; s_key[16 + w] = km; s_key[32 + w] = ko; }
    __syncthreads();
    long long bc = LLONG_MIN, bm = LLONG_MIN, bo = LLONG_MIN;
    for (int i = 0; i < nw; ++i) {
        bc = s_key[i] > bc ? s_key[i] : bc;
        bm = s_key[16 + i] > bm ? s_key[16 + i] : bm;
        bo = s_key[32 + i] > bo ? s_key[32 + i] : bo;
    }
    *max_out = bm == LLONG_MIN ? kNegInf : key_to_double(bm);
    float a = 0.0f, b = 0.0f, ao = 0.0f;
    if (bc != LLONG_MIN && c.any) {
        const float f = expd(c.r - key_to_double(bc));  // <= 1
        a = c.sum1() * f;
        b = c.sum2() * f * f;
    }
    if (has_old && bo != LLONG_MIN && o.any) ao = o.sum1() * expd(o.r - key_to_double(bo));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, off);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, off);
        ao += __shfl_xor_sync(0xFFFFFFFFu, ao, off);
    }
    if ((threadIdx.x & 31) == 0) { s_f[w] = a; s_f[32 + w] = b; s_f[64 + w] = ao; }
    __syncthreads();
    *outc = Lse{kNegInf, 0.0, 0.0};
    *outo = Lse{kNegInf, 0.0, 0.0};
    if (threadIdx.x == 0) {
        float A = 0.0f, B = 0.0f, AO = 0.0f;
        for (int i = 0; i < nw; ++i) { A += s_f[i]; B += s_f[32 + i]; AO += s_f[64 + i]; }
        if (bc != LLONG_MIN) *outc = Lse{key_to_double(bc), f2d_bits(A), f2d_bits(B)};
        if (bo != LLONG_MIN) *outo = Lse{key_to_double(bo), f2d_bits(AO), 0.0};
    }
}

// A double that holds a normal float (or zero) exactly, back to that
// float by integer operations (no conversion on the FP64 pipe).
__device__ __forceinline__ float d2f_exact(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t f = (hi & 0x80000000u) | ((e - 1023u + 127u) << 23) | ((hi & 0xFFFFFu) << 3) |
                       (lo >> 29);
    return e == 0u ? 0.0f : __uint_as_float(f);
}

// The final combination of a reweighting reduction: the per-block partials
// {ref, s1, s2, ref_old, s_old, max} of at most kRwMaxParts blocks are read
// once into registers (two per thread at 256 threads), the common
// references and the maximum are found by integer keys, every partial's sums
// are scaled to its reference by one FP32 exponential and added as FP32
// two-sums (the block sums are FP32 values: only the final addition of each
// total runs on the FP64 pipe), then the sums are expressed relative to the
// true maximum.  Every thread of the calling block calls it and gets the
// normalisation constants; with `write` (one block) the final slot {max, S1,
// S2, valid, LSE, 1/S1 (float)}, the scalars {log Z increment, ESS, max,
// LSE} and the resampling flag are written too.  It runs either in the
// reduction's last block or, redundantly, in every block of the kernel that
// consumes the weights, whose first tile loads are then already in flight.
constexpr int kRwMaxParts = 512;

struct RwFinal {
    double m;     // maximum log-weight
    float inv;    // 1 / sum exp(logw - m), FP32
    bool valid;   // some weight positive, no NaN
};

__device__ __forceinline__ RwFinal reweight_combine(double* partials,
                                                    int nblocks, int has_inc, int64_t M,
                                                    bool write, double* __restrict__ scalars,
                                                    int32_t* __restrict__ flag, double ess_frac,
                                                    int final_slot, uint32_t* status) {
    __shared__ long long s_key[96];
    __shared__ float s_f[192];
    __shared__ double s_m;
    __shared__ float s_inv;
    __shared__ int s_valid;
    const bool has_old = has_inc != 0;
    const int tid = threadIdx.x, w = tid >> 5, nw = blockDim.x >> 5;
    double rc[2], s1[2], s2[2], ro[2], so[2];
    long long kc = LLONG_MIN, ko = LLONG_MIN, km = LLONG_MIN;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int b = tid + p * (int)blockDim.x;
        rc[p] = kNegInf; ro[p] = kNegInf;
        s1[p] = 0.0; s2[p] = 0.0; so[p] = 0.0;
        if (b < nblocks) {
            const double2* P = reinterpret_cast<const double2*>(partials + (size_t)b * 8);
            const double2 u = __ldcg(P), v = __ldcg(P + 1), x = __ldcg(P + 2);
            rc[p] = u.x; s1[p] = u.y; s2[p] = v.x; ro[p] = v.y; so[p] = x.x;
            if (!is_neg_inf(u.x)) { const long long k = dkey(u.x); kc = k > kc ? k : kc; }
            if (has_old && !is_neg_inf(v.y)) { const long long k = dkey(v.y); ko = k > ko ? k : ko; }
            if (!is_neg_inf(x.y)) { const long long k = dkey(x.y); km = k > km ? k : km; }
        }
    }
    kc = warp_max_key(kc);
    ko = warp_max_key(ko);
    km = warp_max_key(km);
    if ((tid & 31) == 0) { s_key[w] = kc; s_key[32 + w] = ko; s_key[64 + w] = km; }
    __syncthreads();
    long long bc = LLONG_MIN, bo = LLONG_MIN, bm = LLONG_MIN;
    for (int i = 0; i < nw; ++i) {
        bc = s_key[i] > bc ? s_key[i] : bc;
        bo = s_key[32 + i] > bo ? s_key[32 + i] : bo;
        bm = s_key[64 + i] > bm ? s_key[64 + i] : bm;
    }
    float Rch = 0.0f, Rcl = 0.0f, Roh = 0.0f, Rol = 0.0f;
    if (bc != LLONG_MIN) split_double(key_to_double(bc), Rch, Rcl);
    if (bo != LLONG_MIN) split_double(key_to_double(bo), Roh, Rol);
    F2Sum a, bs, ao;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        if (bc != LLONG_MIN && !is_neg_inf(rc[p])) {
            float h, l;
            split_double(rc[p], h, l);
            const float f = exp_hilo(h - Rch, l - Rcl);  // <= 1
            a.add(d2f_exact(s1[p]) * f);
            bs.add(d2f_exact(s2[p]) * (f * f));
        }
        if (has_old && bo != LLONG_MIN && !is_neg_inf(ro[p])) {
            float h, l;
            split_double(ro[p], h, l);
            ao.add(d2f_exact(so[p]) * exp_hilo(h - Roh, l - Rol));
        }
    }
    a.warp_sum();
    bs.warp_sum();
    ao.warp_sum();
    if ((tid & 31) == 0) {
        s_f[2 * w] = a.s; s_f[2 * w + 1] = a.c;
        s_f[64 + 2 * w] = bs.s; s_f[64 + 2 * w + 1] = bs.c;
        s_f[128 + 2 * w] = ao.s; s_f[128 + 2 * w + 1] = ao.c;
    }
    __syncthreads();
    if (tid == 0) {
        F2Sum A, B, AO;
        for (int i = 0; i < nw; ++i) {
            A.add(F2Sum{s_f[2 * i], s_f[2 * i + 1]});
            B.add(F2Sum{s_f[64 + 2 * i], s_f[64 + 2 * i + 1]});
            AO.add(F2Sum{s_f[128 + 2 * i], s_f[128 + 2 * i + 1]});
        }
        Lse tc{kNegInf, 0.0, 0.0}, to{kNegInf, 0.0, 0.0};
        if (bc != LLONG_MIN) tc = Lse{key_to_double(bc), A.value(), B.value()};
        if (bo != LLONG_MIN) to = Lse{key_to_double(bo), AO.value(), 0.0};
        const double mx = bm == LLONG_MIN ? kNegInf : key_to_double(bm);
        double* F = partials + (size_t)final_slot * 8;
        const bool valid = !is_neg_inf(tc.m) && !disnan(tc.m);
        float inv = 0.0f;
        if (valid) {  // express the sums relative to the true maximum
            const double f = f2d_bits(expd(tc.m - mx));
            tc = Lse{mx, tc.s1 * f, tc.s2 * f * f};
            const double lse = tc.m + ln_sum(tc.s1);
            const float s1f = (float)tc.s1;
            inv = 1.0f / s1f;
            if (write) {
                const double ess = f2d_bits(s1f * (s1f / (float)tc.s2));  // FP32 division
                F[0] = tc.m; F[1] = tc.s1; F[2] = tc.s2; F[3] = 1.0; F[4] = lse;
                reinterpret_cast<float*>(F + 5)[0] = inv;
                if (scalars) {
                    double inc = 0.0;
                    if (has_inc) inc = lse - (to.m + ln_sum(to.s1));
                    scalars[0] = inc;
                    scalars[1] = ess;
                    scalars[2] = tc.m;
                    scalars[3] = lse;
                }
                if (flag) *flag = (ess < ess_frac * (double)M) ? 1 : 0;
            }
        } else if (write) {
            if (!disnan(tc.m)) raise_status(status, ST_ZERO_WEIGHT);
            F[3] = 0.0;
            if (flag) *flag = 0;
        }
        s_m = tc.m;
        s_inv = inv;
        s_valid = valid ? 1 : 0;
    }
    __syncthreads();
    return RwFinal{s_m, s_inv, s_valid != 0};
}

// What a kernel that consumes a deferred reduction's weights needs to
// combine its partials (reweight_combine); block 0 writes the results.
struct RwArgs {
    double* partials;
    int nparts;          // blocks of the reduction
    int has_inc;
    int64_t M;
    double* scalars;     // may be null
    int32_t* flag;       // may be null
    double ess_frac;
    int final_slot;
};

__device__ __forceinline__ RwFinal rw_final(const RwArgs& a, uint32_t* status) {
    return reweight_combine(a.partials, a.nparts, a.has_inc, a.M, blockIdx.x == 0, a.scalars,
                            a.flag, a.ess_frac, a.final_slot, status);
}

// The end of a reweighting reduction's block: its sums (thread sums cur of
// the new log-weights and old of the old ones) go to the block's partial
// slot.  Unless `defer` (the kernel that consumes the weights combines the
// partials itself), the last block to finish runs reweight_combine and
// writes the final slot, the scalars and the flag.  Every thread of the
// block calls it once, after its element loop.
__device__ __forceinline__ void reweight_finish(const RefSums& cur, const RefSums& old,
                                                int has_inc, int64_t M, double* __restrict__ partials,
                                                unsigned long long* ticket, int defer,
                                                double* __restrict__ scalars, int32_t* __restrict__ flag,
                                                double ess_frac, int final_slot, uint32_t* status) {
    __shared__ long long s_key[48];
    __shared__ float s_f[96];
    __shared__ bool last;
    double bmax;
    Lse c, o;
    block_combine2(cur, old, has_inc != 0, s_key, s_f, &c, &o, &bmax);
    if (threadIdx.x == 0) {
        double* P = partials + (size_t)blockIdx.x * 8;
        P[0] = c.m; P[1] = c.s1; P[2] = c.s2; P[3] = o.m; P[4] = o.s1; P[5] = bmax;
        if (!defer) {
            __threadfence();
            const unsigned long long t = atomicAdd(ticket, 1ull);
            last = (t == gridDim.x - 1);
        }
    }
    if (defer) return;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0ull;
    reweight_combine(partials, gridDim.x, has_inc, M, true, scalars, flag, ess_frac, final_slot,
                     status);
}

}  // namespace smc
