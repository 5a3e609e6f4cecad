// binned.cuh -- the univariate mixture log-likelihood over data sorted into
// bins of width w, evaluated with one packed FMA per datum pair and
// component (Section 4.1 product-sum, Section 2.3 log domain).
//
// In base-2 units with c = log2(e) / (2 sigma^2), a datum y of the bin with
// centre y0 = j w has the exact offset delta = y - y0 (|delta| <= w/2), and
// with e_k = y0 - mu_k
//   log2 w_k - c (y - mu_k)^2 = delta A_k + B_k - c delta^2,
//   A_k = -2 c e_k,   B_k = log2 w_k - c e_k^2.
// The term -c delta^2 is the same for every particle: its sum over the data
// is one constant per data set.  Per bin, m_b = max over the bin's data range
// of max_k (delta A_k + B_k) is taken out (both ends of the range bound the
// linear arguments), so the per-datum sum
//   S = sum_k 2^(delta A_k + B_k - m_b)
// lies in (0, K] and each of its terms costs one FFMA2 half and one ex2.
// w is the largest power of two with c (w/2)^2 <= 4: every delta is exact
// (y and j w lie within a factor two of each other) and the rounding of
// A_k, B_k and the FMA stays a few units of 2^-24 of quantities of size
// c delta^2 <= 4 for the dominant components.  Data whose bin index lies
// outside [-15, 15] (or that are not finite) form a last class evaluated
// by the max-shifted direct form.
#pragma once
#include <climits>
#include <cstddef>

#include "device.cuh"

namespace smc {

constexpr int kBinHalf = 15;                    // bins j = -15 .. 15
constexpr int kClasses = 2 * kBinHalf + 2;      // 31 bins + the data outside them
constexpr int kOutlier = kClasses - 1;
constexpr int kBinnedMaxN = 4096;               // data held in shared memory
// below this many data the per-sweep binning and the round structure cost
// more than they save (measured: K = 8, 34,591 chains: break-even near 500)
constexpr int kBinnedMinN = 512;
constexpr int kBinnedMaxWarps = 16;

struct __align__(16) BinTable {
    // (start .. dconst form the table's core: what the sweep reads after the
    // partition; the cached layout holds exactly these bytes)
    int start[kClasses + 1];  // first slot of each class in the sorted list (even);
                              // start[kClasses] = padded length of the list
    int count[kClasses];
    float y0[kClasses];       // bin centre j w
    int dlo[kClasses];        // order keys of the smallest / largest delta of the bin
    int dhi[kClasses];
    double dconst;            // -c sum over the binned data of delta^2 (log2 units)
    int cnt[kBinnedMaxWarps][kClasses];  // partition scratch: per-warp counts, then bases
    float2 csum[kClasses];    // per bin: compensated sum of delta^2 (s, c)
};

// order-preserving integer key of a float (total order for non-NaN values)
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b ^ ((b >> 31) & 0x7FFFFFFF);
}
__device__ __forceinline__ float fkey_inv(int k) {
    return __int_as_float(k ^ ((k >> 31) & 0x7FFFFFFF));
}

// class of a datum and its exact offset from the bin centre (integer and
// FP32 operations only: conversions would take the narrow FP64 pipe)
__device__ __forceinline__ int bin_class(float v, float binw, float binw_inv, float& dl) {
    const float x = v * binw_inv;  // exact (binw_inv is a power of two)
    if (!(fabsf(x) < (float)kBinHalf + 0.5f)) {  // outside the bins, or NaN
        dl = v;
        return kOutlier;
    }
    int q;
    const float qf = round_magic(x, q);  // rint(x), |q| <= 15
    dl = v - qf * binw;  // exact: v and q w lie within a factor two (or q = 0)
    return q + kBinHalf;
}

// x 2^32 rounded to the nearest integer (ties away from zero), for |x| < 2^31,
// by integer operations: a deterministic fixed-point image of a float
__device__ __forceinline__ long long fixed32(float x) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e == 0) return 0;                               // zero (and subnormals)
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 127 - 23 + 32;                   // x 2^32 = m 2^sh
    long long v;
    if (sh >= 0) v = m << sh;
    else if (sh > -25) v = (m + (1LL << (-sh - 1))) >> (-sh);
    else v = 0;
    return (b >> 31) ? -v : v;
}

// Sort the staged data ys[0, N) by class into yb (each class starting at an
// even slot; an odd class is followed by one unused slot): bin data as their
// offsets delta, the last class as raw values.  Stable (data order within a
// class is kept), so every CTA builds the same list and sums in the same
// order.  rk is scratch for N ranks.  Then, per bin, the range of its
// offsets, and the sum of delta^2 over the binned data.  The whole block
// calls this (barriers); blockDim.x is a multiple of 32, at most 512.
__device__ void bin_partition(const float* ys, int N, float* yb, uint16_t* rk, BinTable& bt,
                              float binw, float binw_inv, float cf) {
    const int nw = (int)(blockDim.x >> 5), w = (int)(threadIdx.x >> 5), l = threadIdx.x & 31;
    const unsigned lt = (1u << l) - 1u;
    for (int i = threadIdx.x; i < kBinnedMaxWarps * kClasses; i += blockDim.x)
        (&bt.cnt[0][0])[i] = 0;
    __syncthreads();
    // each warp ranks a contiguous range of data, 32 at a time
    const int per = (((N + nw - 1) / nw) + 31) & ~31;
    const int w0 = w * per;
    for (int r = 0; r < per; r += 32) {
        const int i = w0 + r + l;
        int cls = -1;
        float dl = 0.0f;
        if (i < N) cls = bin_class(ys[i], binw, binw_inv, dl);
        const unsigned m = __match_any_sync(0xFFFFFFFFu, cls);
        const int before = cls >= 0 ? bt.cnt[w][cls] : 0;
        __syncwarp();
        if (cls >= 0) {
            rk[i] = (uint16_t)(before + __popc(m & lt));
            if ((m & lt) == 0u) bt.cnt[w][cls] = before + __popc(m);
        }
        __syncwarp();
    }
    __syncthreads();
    // per (class, warp): exclusive prefix over warps and the class total
    int pre = 0;
    const int t = threadIdx.x;
    const int tc = t / nw, tw = t % nw;
    const bool owner = t < nw * kClasses;
    if (owner) {
        int tot = 0;
        for (int v = 0; v < nw; ++v) {
            const int c = bt.cnt[v][tc];
            if (v < tw) pre += c;
            tot += c;
        }
        if (tw == 0) bt.count[tc] = tot;
    }
    __syncthreads();
    if (w == 0) {  // class starts: exclusive scan of the even-padded counts
        const int c = bt.count[l];
        const int tp = c + (c & 1);
        int inc = tp;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (l >= o) inc += v;
        }
        bt.start[l] = inc - tp;
        bt.y0[l] = l < kOutlier ? (float)(l - kBinHalf) * binw : 0.0f;
        if (l == kClasses - 1) bt.start[kClasses] = inc;
    }
    __syncthreads();
    if (owner) bt.cnt[tw][tc] = bt.start[tc] + pre;
    __syncthreads();
    for (int r = 0; r < per; r += 32) {
        const int i = w0 + r + l;
        if (i < N) {
            float dl;
            const int cls = bin_class(ys[i], binw, binw_inv, dl);
            yb[bt.cnt[w][cls] + rk[i]] = dl;
        }
    }
    if (t < kClasses && (bt.count[t] & 1)) yb[bt.start[t] + bt.count[t]] = 0.0f;
    __syncthreads();
    // per bin (one warp each, in turn): smallest and largest offset and the
    // compensated sum of delta^2; then the data set's sum, bins in order
    for (int c = w; c < kOutlier; c += nw) {
        const int a = bt.start[c], n = bt.count[c];
        float lo = INFINITY, hi = -INFINITY;
        Kahan q;
        for (int i = l; i < n; i += 32) {
            const float d = yb[a + i];
            lo = fminf(lo, d);
            hi = fmaxf(hi, d);
            q.add(d * d);
        }
        float s2 = q.s, c2 = q.c;
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
            const float so = __shfl_xor_sync(0xFFFFFFFFu, s2, o);
            const float co = __shfl_xor_sync(0xFFFFFFFFu, c2, o);
            const float tt = s2 + so;  // two-sum
            const float bp = tt - s2;
            const float err = (s2 - (tt - bp)) + (so - bp);
            s2 = tt;
            c2 = (c2 + co) - err;
        }
        if (l == 0) {
            bt.dlo[c] = fkey(lo);
            bt.dhi[c] = fkey(hi);
            bt.csum[c] = make_float2(s2, c2);
        }
    }
    __syncthreads();
    if (w == 0) {  // sum over the bins, lane c holding bin c, compensated
        float s2 = 0.0f, c2 = 0.0f;
        if (l < kOutlier) {
            s2 = bt.csum[l].x;
            c2 = bt.csum[l].y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float so = __shfl_xor_sync(0xFFFFFFFFu, s2, o);
            const float co = __shfl_xor_sync(0xFFFFFFFFu, c2, o);
            const float tt = s2 + so;
            const float bp = tt - s2;
            const float err = (s2 - (tt - bp)) + (so - bp);
            s2 = tt;
            c2 = (c2 + co) - err;
        }
        if (l == 0) bt.dconst = -(double)cf * (f2d_bits(s2) - f2d_bits(c2));
    }
    __syncthreads();
}

// Pieces of the sorted list: each class's slots cut into runs of at most
// kPieceSlots (even), listed largest first; the same for every chain.
constexpr int kPieceSlots = 128;
constexpr int kMaxPieces = kClasses + kBinnedMaxN / kPieceSlots + 1;

// Warp 0 builds the piece list (a, b, class) after bin_partition: every
// class's full-size pieces first (classes in order), then the remainders
// (classes in order), a fixed order shared by every CTA that hands out the
// larger pieces first.  Returns the count in *np (a shared variable); the
// caller synchronises after it.
__device__ void bin_pieces(const BinTable& bt, int3* pieces, int* np) {
    if (threadIdx.x >= 32) return;
    const int l = threadIdx.x;  // class l
    const int a = bt.start[l], n = bt.count[l];
    const int nf = n / kPieceSlots, nr = (n % kPieceSlots) ? 1 : 0;
    int incf = nf, incr = nr;
    for (int o = 1; o < 32; o <<= 1) {
        const int vf = __shfl_up_sync(0xFFFFFFFFu, incf, o);
        const int vr = __shfl_up_sync(0xFFFFFFFFu, incr, o);
        if (l >= o) {
            incf += vf;
            incr += vr;
        }
    }
    const int totf = __shfl_sync(0xFFFFFFFFu, incf, 31);
    for (int j = 0; j < nf; ++j)
        pieces[incf - nf + j] = make_int3(a + j * kPieceSlots, a + (j + 1) * kPieceSlots, l);
    if (nr) pieces[totf + incr - 1] = make_int3(a + nf * kPieceSlots, a + n, l);
    if (l == 31) *np = totf + incr;
    __syncwarp();
}

// The binned layout of one data set, kept in global memory between sweeps
// (it depends only on the data, the bin width and c): a 16-byte header
// {N, piece count, bin width bits, c bits}, a copy of the data (to check
// that the data are still those), the sorted list, the table's core and the
// pieces -- each section a multiple of 16 bytes, so that a sweep moves each
// by one bulk copy into the place its own partition would have filled.
constexpr size_t kBinCoreBytes = (offsetof(BinTable, cnt) + 15) / 16 * 16;
constexpr size_t kPiecesBytes = (kMaxPieces * sizeof(int3) + 15) / 16 * 16;
static_assert(offsetof(BinTable, dconst) + sizeof(double) <= kBinCoreBytes, "core ends at dconst");
static_assert(kBinCoreBytes <= offsetof(BinTable, cnt), "the core does not reach the scratch");
__host__ __device__ inline size_t bcache_ycopy_bytes(int64_t N) { return (size_t)((N + 3) & ~3LL) * 4; }
__host__ __device__ inline size_t bcache_yb_off(int64_t N) { return 16 + bcache_ycopy_bytes(N); }
__host__ __device__ inline size_t bcache_core_off(int64_t N, int yb_len) {
    return bcache_yb_off(N) + (size_t)yb_len * 4;
}
__host__ __device__ inline size_t bcache_pieces_off(int64_t N, int yb_len) {
    return bcache_core_off(N, yb_len) + kBinCoreBytes;
}
__host__ __device__ inline size_t bcache_bytes(int64_t N, int yb_len) {
    return bcache_pieces_off(N, yb_len) + kPiecesBytes;
}

// log2 of sum_k w_k 2^(-c (y - mu_k)^2), max-shifted (the class outside the bins)
template <int K>
__device__ __forceinline__ float direct_log2(float v, const float (&mu)[K], const float (&lw2)[K],
                                             float r) {
    float a[K];
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float t = (v - mu[k]) * r;
        a[k] = fmaf(-t, t, lw2[k]);
        m = fmaxf(m, a[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) s += ex2(a[k] - m);
    return m + lg2(s);
}

// Threshold below which a datum's bin-shifted sum is re-formed with its own
// shift: above it, the terms ex2 flushes to zero (< 2^-126) are below 2^-64
// of the sum, and the product of two sums stays a normal float.
constexpr float kBinFloor = 0x1p-62f;

// Accumulates log2 terms of one particle over a range of the sorted list.
template <int K>
struct BinnedAcc {
    Kahan ll;                                     // shifts, exponents, single data
    float2 pr = {1.0f, 1.0f};                     // mantissa of the product of sums
    int ex = 0;                                   // biased exponents split off pr
    int nsp = 0;                                  // number of splits

    __device__ __forceinline__ void fold(float2 S) {
        pr = __fmul2_rn(pr, S);
        const uint32_t bx = __float_as_uint(pr.x), by = __float_as_uint(pr.y);
        ex += (int)(bx >> 23) + (int)(by >> 23);
        ++nsp;
        pr = make_float2(__uint_as_float((bx & 0x7FFFFFu) | 0x3F800000u),
                         __uint_as_float((by & 0x7FFFFFu) | 0x3F800000u));
    }

    // one datum with its own shift: returns S in [1, K], adds the shift
    __device__ __forceinline__ float own_shift(float d, const float2 (&A2)[K],
                                               const float2 (&B2)[K]) {
        float a[K];
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a[k] = fmaf(d, A2[k].x, B2[k].x);
            m = fmaxf(m, a[k]);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) s += ex2(a[k] - m);
        ll.add(m);
        return s;
    }

    __device__ __forceinline__ float2 pair_sum(float2 D, const float2 (&A2)[K],
                                               const float2 (&B2)[K]) {
        float2 e[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 T = __ffma2_rn(D, A2[k], B2[k]);
            e[k] = make_float2(ex2(T.x), ex2(T.y));
        }
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) e[k] = __fadd2_rn(e[k], e[k + s]);
        return e[0];
    }

    // the sorted list's slots [ia, ib) of one bin (ia even); the proposal's
    // means are read from mu[k * stride]
    __device__ __forceinline__ void bin_range(const float* yb, int ia, int ib, float y0, float dlo,
                                              float dhi, const float* mu, int stride,
                                              const float* lw2, float cf) {
        float2 A2[K], B2[K];
        float mb = -INFINITY;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float e = y0 - mu[k * stride];
            const float c = cf * e;
            const float A = -2.0f * c;
            const float B = fmaf(-c, e, lw2[k]);
            mb = fmaxf(mb, fmaxf(fmaf(dlo, A, B), fmaf(dhi, A, B)));
            A2[k] = make_float2(A, A);
            B2[k] = make_float2(B, B);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            B2[k].x -= mb;
            B2[k].y = B2[k].x;
        }
        // the shift, once per datum: n m_b with its rounding error
        const float nf = u23_to_f((uint32_t)(ib - ia));
        const float p = nf * mb;
        ll.add(p);
        ll.add(fmaf(nf, mb, -p));
        // two pairs per step; a datum whose sum fell below the floor (rare)
        // is re-formed with its own shift, the test taken once per warp
        const float2* y2 = reinterpret_cast<const float2*>(yb + ia);
        const float2* const y2e = y2 + ((ib - ia) >> 2) * 2;
#pragma unroll 1
        for (; y2 != y2e; y2 += 2) {
            const float2 D0 = y2[0], D1 = y2[1];
            float2 S0 = pair_sum(D0, A2, B2);
            float2 S1 = pair_sum(D1, A2, B2);
            const float mn = fminf(fminf(S0.x, S0.y), fminf(S1.x, S1.y));
            if (__any_sync(0xFFFFFFFFu, mn < kBinFloor)) {
                if (S0.x < kBinFloor) S0.x = own_shift(D0.x, A2, B2);
                if (S0.y < kBinFloor) S0.y = own_shift(D0.y, A2, B2);
                if (S1.x < kBinFloor) S1.x = own_shift(D1.x, A2, B2);
                if (S1.y < kBinFloor) S1.y = own_shift(D1.y, A2, B2);
            }
            fold(__fmul2_rn(S0, S1));
        }
        int i = ia + (((ib - ia) >> 2) << 2);
        if (i + 2 <= ib) {
            const float2 D0 = *reinterpret_cast<const float2*>(yb + i);
            float2 S0 = pair_sum(D0, A2, B2);
            if (S0.x < kBinFloor) S0.x = own_shift(D0.x, A2, B2);
            if (S0.y < kBinFloor) S0.y = own_shift(D0.y, A2, B2);
            fold(S0);
            i += 2;
        }
        if (i < ib) ll.add(lg2(own_shift(yb[i], A2, B2)));
    }

    // slots [a, b) of class cls of the sorted list (a even)
    __device__ __forceinline__ void piece(const float* yb, const BinTable& bt, int a, int b, int cls,
                                          const float* mu, int stride, const float* lw2, float cf,
                                          float r) {
        if (cls == kOutlier) {
            float m[K], w[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                m[k] = mu[k * stride];
                w[k] = lw2[k];
            }
#pragma unroll 1
            for (int i = a; i < b; ++i) ll.add(direct_log2(yb[i], m, w, r));
        } else {
            bin_range(yb, a, b, bt.y0[cls], fkey_inv(bt.dlo[cls]), fkey_inv(bt.dhi[cls]), mu,
                      stride, lw2, cf);
        }
    }

    // the partial sum in log2 units as an unevaluated pair (s - c)
    __device__ __forceinline__ float2 partial() {
        ll.add((float)(ex - 254 * nsp));
        ll.add(lg2(pr.x) + lg2(pr.y));
        return make_float2(ll.s, ll.c);
    }
};

}  // namespace smc
