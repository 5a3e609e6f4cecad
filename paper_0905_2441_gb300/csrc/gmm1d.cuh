// gmm1d.cuh -- the univariate mixture log-likelihood of one particle,
// evaluated by a slice of L cooperating lanes over data staged in shared
// memory (Section 4.1 product-sum; Section 4.1.3: one likelihood split over
// several threads when the data are many).
//
// Arithmetic, per datum n and component k, in base-2 log units:
//   t_k   = (y_n - mu_k) r            r = sqrt(log2(e) / (2 sigma^2))
//         = fma(y_n, r, nu_k)         nu_k = -mu_k r
//   a_k   = log2 w_k - t_k^2
//   m_n   = max_k a_k,  s_n = sum_k 2^(a_k - m_n) in [1, K]
//   log2 p(y_n | mu) = m_n + log2 s_n + const
// The products of 16 consecutive s_n are formed before one lg2 (each
// s_n <= K <= 32, so the product stays below 2^80), the m_n of the same 16
// data are summed in FP32 and each group total enters a Kahan accumulator.
// The lane partials meet in FP32 (two-sum), the FP64 total forms once.  Gradient: d l / d mu_k =
// sum_n r_nk (y_n - mu_k) / sigma^2 = (1/(sigma^2 r)) sum_n (e_k / s_n) t_k.
#pragma once
#include "device.cuh"

namespace smc {

constexpr int kMaxK1d = 32;

// Reduce Kahan pairs (s, c) (true sum s - c) over the L lanes of a slice in
// FP32 with error-free additions, then form the FP64 total once.
__device__ __forceinline__ double slice_total(float s, float c, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s, o);
        const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
        const float t = s + s2;                 // two-sum: t + err == s + s2 exactly
        const float bp = t - s;
        const float err = (s - (t - bp)) + (s2 - bp);
        s = t;
        c = (c + c2) - err;
    }
    return f2d_bits(s) - f2d_bits(c);  // conversions by integer ops (no FP64-pipe convert)
}


struct Gmm1dArgs {
    float r;            // sqrt(log2(e) / (2 sigma^2))
    float gscale;       // 1 / (sigma^2 r)
    float lo, hi;       // prior box
    float cf;           // log2(e) / (2 sigma^2)
    float binw;         // bin width of the binned form: largest power of 2 with cf (w/2)^2 <= 4
    float binw_inv;     // 1 / binw (a power of two)
    double cst;         // N (-1/2 ln(2 pi sigma^2)) [+ N ln w when weights are equal]
    float lw2[kMaxK1d]; // log2 w_k (padding components: -inf)
    uint32_t wait_limit;  // polls of the first wait on a bulk data copy (the context's)
};

// Stage y[n0, n0+cnt) into shared memory.  A bulk asynchronous copy moves
// the 16-byte aligned body (completion on an mbarrier); the unaligned head
// and tail use plain loads.  stage_y_issue starts the copy (every thread of
// the block calls it; returns whether the bulk copy was used), other work
// may follow, and stage_y_wait completes it.  stage_y does both.
__device__ __forceinline__ bool stage_y_issue(float* ys, const float* __restrict__ y, int64_t n0,
                                              int cnt, uint64_t* mbar) {
    const float* src = y + n0;
    uintptr_t a = reinterpret_cast<uintptr_t>(src);
    int head = (int)(((16u - (uint32_t)(a & 15u)) & 15u) / 4u);
    if ((a & 3u) != 0) head = cnt;  // not even float-aligned: plain loads only
    if (head > cnt) head = cnt;
    int body = ((cnt - head) / 4) * 4;
    // the shared destination must share the source's 16-byte phase
    bool bulk = body >= 64 && ((reinterpret_cast<uintptr_t>(ys + head) & 15u) == 0);
    if (!bulk) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) ys[i] = src[i];
        return false;
    }
    uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        // order earlier generic-proxy reads of this buffer before the async write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        uint32_t bytes = (uint32_t)body * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(mb), "r"(bytes) : "memory");
        uint32_t dst = (uint32_t)__cvta_generic_to_shared(ys + head);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            :: "r"(dst), "l"(src + head), "r"(bytes), "r"(mb) : "memory");
    }
    for (int i = threadIdx.x; i < head; i += blockDim.x) ys[i] = src[i];
    for (int i = head + body + threadIdx.x; i < cnt; i += blockDim.x) ys[i] = src[i];
    return true;
}

// Completes stage_y_issue: every thread of the block calls it.  The wait on
// the bulk copy is bounded (`limit` polls, the context's setting); on timeout
// the status word gets ST_TIMEOUT and a second wait, with the full bound,
// lets the copy finish, so none is left in flight and the data are complete.
__device__ __forceinline__ void stage_y_wait(bool bulk, uint64_t* mbar, uint32_t& phase,
                                             uint32_t* status, uint32_t limit = kSpinLimit) {
    if (!bulk) {
        __syncthreads();
        return;
    }
    uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mb), "r"(phase) : "memory");
        if (!done && it > 64) __nanosleep(64);
    }
    if (!done) {
        raise_status(status, ST_TIMEOUT);
        // wait once more, again bounded, so no copy is left in flight
        for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done) : "r"(mb), "r"(phase) : "memory");
            __nanosleep(256);
        }
    }
    phase ^= 1u;
    __syncthreads();
}

__device__ __forceinline__ void stage_y(float* ys, const float* __restrict__ y, int64_t n0,
                                        int cnt, uint64_t* mbar, uint32_t& phase,
                                        uint32_t* status, uint32_t limit = kSpinLimit) {
    stage_y_wait(stage_y_issue(ys, y, n0, cnt, mbar), mbar, phase, status, limit);
}

__device__ __forceinline__ void init_mbar(uint64_t* mbar) {
    if (threadIdx.x == 0) {
        uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Per-lane partial over the data this lane owns in a staged chunk
// ys[0, cnt): n = lane, lane + L, ...  The state carries across chunks.
template <int K, bool GRAD, bool EQW>
struct SliceAcc {
    static constexpr int KG = GRAD ? K : 1;
    Kahan ll;          // sum over groups of (sum m_n + log2 prod s_n)
    float msum = 0.0f; // current group's sum of m_n
    float prod = 1.0f; // current group's product of s_n
    int cnt = 0;
    float gch[KG];
    Kahan gacc[KG];

    __device__ __forceinline__ SliceAcc() {
#pragma unroll
        for (int k = 0; k < KG; ++k) gch[k] = 0.0f;
    }

    __device__ __forceinline__ void flush() {
        ll.add(msum + lg2(prod));
        msum = 0.0f;
        prod = 1.0f;
        cnt = 0;
        if constexpr (GRAD) {
#pragma unroll
            for (int k = 0; k < KG; ++k) {
                gacc[k].add(gch[k]);
                gch[k] = 0.0f;
            }
        }
    }

    __device__ __forceinline__ void run(const float* ys, int cnt_total, int lane, int L,
                                        const float (&nu)[K], const float (&lw2)[K], float r) {
#pragma unroll 2
        for (int n = lane; n < cnt_total; n += L) {
            float yv = ys[n];
            float t[K], a[K];
            float m = -INFINITY;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                t[k] = fmaf(yv, r, nu[k]);
                if constexpr (EQW) a[k] = -t[k] * t[k];
                else a[k] = fmaf(-t[k], t[k], lw2[k]);
                m = fmaxf(m, a[k]);
            }
            float s = 0.0f;
            float e[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                e[k] = ex2(a[k] - m);
                s += e[k];
            }
            msum += m;
            prod *= s;
            if constexpr (GRAD) {
                float rs = rcp(s);
#pragma unroll
                for (int k = 0; k < KG; ++k) gch[k] = fmaf(e[k] * rs, t[k], gch[k]);
            }
            if (++cnt == 16) flush();
        }
    }

    // Reduce over the slice; every lane of the warp must call this.
    // Returns the particle's log-likelihood; g receives the gradient.
    __device__ __forceinline__ double finish(int L, const Gmm1dArgs& P, float (&g)[K]) {
        if (cnt) flush();
        const double part = slice_total(ll.s, ll.c, L);
        if constexpr (GRAD) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float v = gacc[k].s - gacc[k].c;
                for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                g[k] = v * P.gscale;
            }
        }
        return part * kLn2 + P.cst;
    }
};

// Equal component weights, no gradient: the common case, written for the
// issue rate of sm_103a.  Two data are evaluated at once in packed f32x2
// registers (one FFMA2 / FMUL2 / FADD2 instruction per pair):
//   t_k = y r + nu_k,   s = sum_k 2^(-t_k^2)   (log2 units: a_k = c0 - t_k^2)
// Unlike the max-shifted form, no shift is computed: s is taken as is
// whenever s >= 2^-100, where every term ex2 flushes to zero (< 2^-126) is
// below 2^-23 s, i.e. under the FP32 rounding of s itself.  Only data far
// from every component (s < 2^-100) take the shifted path, with
// c = -min_k t_k^2 added to the total exactly as in the scalar path.  Per
// datum and component this leaves half a packed FFMA (t), half a packed
// FMUL (t^2), one MUFU ex2 and half a packed FADD (the sum).  The product
// of the s_n is kept as mantissa in [1, 2) times an integer power of two
// (exponent bits split off after every pair), so one lg2 per slice lane
// closes the whole sum instead of one per datum.
__device__ __forceinline__ float ex2_neg(float p) {
    float y;
    asm("{\n\t.reg .f32 t;\n\tneg.f32 t, %1;\n\tex2.approx.ftz.f32 %0, t;\n\t}" : "=f"(y) : "f"(p));
    return y;
}

// Pairs of data evaluated per block of the packed path (compile-time tuning
// knob: more pairs give more independent work per warp, and more registers
// per thread).
#ifndef SMC_EQW_UNROLL
#define SMC_EQW_UNROLL 2
#endif
constexpr int kEqwUnroll = SMC_EQW_UNROLL;

template <int K, bool GRAD = false>
struct SliceAccEqW {
    Kahan ll;                              // log2 terms: exponents, shifts, scalar data
    float2 pr[2] = {{1.0f, 1.0f}, {1.0f, 1.0f}};  // mantissa products of s (even / odd
                                                 // pairs of a block), in [1, 2)
    // gradient (GRAD): per component, sum over the data of r_nk t_nk with the
    // responsibilities r_nk = e_nk / s_n (shift-free, so the unshifted sums
    // serve), one half per datum of a pair
    float2 G[GRAD ? K : 1];

    __device__ __forceinline__ SliceAccEqW() {
#pragma unroll
        for (int k = 0; k < (GRAD ? K : 1); ++k) G[k] = make_float2(0.0f, 0.0f);
    }

    // one datum on the shifted scalar path; returns s and adds the shift to
    // the sum, and (GRAD) its responsibilities times t_k to G[k].x or .y
    __device__ __forceinline__ float one_shifted(float yv, const float (&nu)[K], float r,
                                                 bool upper_half) {
        float t[K];
        float tm = INFINITY;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            t[k] = fmaf(yv, r, nu[k]);
            tm = fminf(tm, fabsf(t[k]));
        }
        const float c = -tm * tm;
        float e[K];
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            e[k] = ex2_neg(fmaf(t[k], t[k], c));
            s += e[k];
        }
        ll.add(c);
        if constexpr (GRAD) {
            const float inv = rcp(s);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float v = e[k] * t[k] * inv;
                if (upper_half) G[k].y += v;
                else G[k].x += v;
            }
        }
        return s;
    }

    // one datum on the scalar path (odd tail of a chunk)
    __device__ __forceinline__ void one(float yv, const float (&nu)[K], float r) {
        const float s = one_shifted(yv, nu, r, false);
        ll.add(lg2(s));
    }

    // U pairs p, p + L, ..., p + (U-1) L: their sums are computed
    // independently (straight-line code the scheduler can interleave), with
    // one test for the rare rescue (data whose unshifted sum fell below
    // 2^-100 take the shifted path), then folded into the products
    template <int U>
    __device__ __forceinline__ void pairs(const float2* ys2, int p, int L, float2 R2,
                                          const float2 (&NU)[K], const float (&nu)[K], float r,
                                          int& ex) {
        float2 Y[U], S[U];
        float2 E[GRAD ? U : 1][K];  // the terms, kept for the gradient
#pragma unroll
        for (int u = 0; u < U; ++u) Y[u] = ys2[p + u * L];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float2 e[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float2 T = __ffma2_rn(Y[u], R2, NU[k]);
                const float2 Q = __fmul2_rn(T, T);
                e[k] = make_float2(ex2_neg(Q.x), ex2_neg(Q.y));
                if constexpr (GRAD) E[u][k] = e[k];
            }
            // balanced tree keeps the dependency chain short (log2 K)
#pragma unroll
            for (int w = 1; w < K; w <<= 1)
#pragma unroll
                for (int k = 0; k + w < K; k += 2 * w) e[k] = __fadd2_rn(e[k], e[k + w]);
            S[u] = e[0];
        }
        bool resc[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) { resc[u][0] = false; resc[u][1] = false; }
        float mn = fminf(S[0].x, S[0].y);
#pragma unroll
        for (int u = 1; u < U; ++u) mn = fminf(mn, fminf(S[u].x, S[u].y));
        if (mn < 0x1p-100f) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (S[u].x < 0x1p-100f) {
                    resc[u][0] = true;
                    S[u].x = one_shifted(Y[u].x, nu, r, false);
                }
                if (S[u].y < 0x1p-100f) {
                    resc[u][1] = true;
                    S[u].y = one_shifted(Y[u].y, nu, r, true);
                }
            }
        }
        if constexpr (GRAD) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // rescued halves added their own (shifted) contribution
                const float2 INV = make_float2(resc[u][0] ? 0.0f : rcp(S[u].x),
                                               resc[u][1] ? 0.0f : rcp(S[u].y));
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float2 T = __ffma2_rn(Y[u], R2, NU[k]);
                    G[k] = __ffma2_rn(__fmul2_rn(E[u][k], T), INV, G[k]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float2& acc = pr[u & 1];
            acc = __fmul2_rn(acc, S[u]);  // in [2^-100, 2^4): normal
            const uint32_t bx = __float_as_uint(acc.x), by = __float_as_uint(acc.y);
            ex += (int)(bx >> 23) + (int)(by >> 23);
            acc = make_float2(__uint_as_float((bx & 0x7FFFFFu) | 0x3F800000u),
                              __uint_as_float((by & 0x7FFFFFu) | 0x3F800000u));
        }
    }

    // data ys[0, cnt_total): pairs p = lane, lane + L, ...; the odd last
    // datum (if any) goes to lane 0
    __device__ __forceinline__ void run(const float* ys, int cnt_total, int lane, int L,
                                        const float (&nu)[K], float r) {
        const float2* ys2 = reinterpret_cast<const float2*>(ys);
        const int np = cnt_total >> 1;
        const float2 R2 = make_float2(r, r);
        float2 NU[K];
#pragma unroll
        for (int k = 0; k < K; ++k) NU[k] = make_float2(nu[k], nu[k]);
        int ex = 0;  // biased exponents split off pr in this chunk (< 2^21 in all)
        int p = lane;
#pragma unroll 1
        for (; p + (kEqwUnroll - 1) * L < np; p += kEqwUnroll * L)
            pairs<kEqwUnroll>(ys2, p, L, R2, NU, nu, r, ex);
#pragma unroll 1
        for (; p < np; p += L) pairs<1>(ys2, p, L, R2, NU, nu, r, ex);
        // remove the bias 2 x 127 of each pair; the result, at most
        // 4096 x 200 in size, is exact in FP32
        const int npairs = lane < np ? (np - 1 - lane) / L + 1 : 0;
        ll.add((float)(ex - 254 * npairs));
        if ((cnt_total & 1) && lane == 0) one(ys[cnt_total - 1], nu, r);
    }

    __device__ __forceinline__ double finish(int L, const Gmm1dArgs& P) {
        ll.add((lg2(pr[0].x) + lg2(pr[0].y)) + (lg2(pr[1].x) + lg2(pr[1].y)));
        const double part = slice_total(ll.s, ll.c, L);
        return part * kLn2 + P.cst;
    }
    // with the gradient d l / d mu_k = sum_n r_nk (y_n - mu_k) / sigma^2
    // = gscale sum_n r_nk t_nk, reduced over the slice's lanes
    __device__ __forceinline__ double finish(int L, const Gmm1dArgs& P, float (&g)[K]) {
        if constexpr (GRAD) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float v = G[k].x + G[k].y;
                for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                g[k] = v * P.gscale;
            }
        }
        return finish(L, P);
    }
};

// The random draws of one chain's move, computed once per slice of L lanes
// instead of redundantly on every lane.  The slice has P + 1 tasks (P =
// ceil(K/2) Box-Muller pairs; pair p uses Philox block p/2 of the MOVE
// stream, words 2p, 2p+1; task P is the ACCEPT block), dealt to its lanes
// in ceil((P+1)/L) rounds; shuffles hand the K normals and the accept word
// to every lane of the slice.  Every lane of the warp must call this.
template <int K>
__device__ __forceinline__ void slice_draws(uint64_t seed, uint64_t step, uint32_t index,
                                            int lane, int L, int Kreal, float (&z)[K],
                                            uint32_t& accept_word) {
    constexpr int PMAX = (K + 1) / 2;
    const int P = (Kreal + 1) / 2;
    const int base = (int)(threadIdx.x & 31) - lane;  // warp lane of this slice's lane 0
    const int R = (P + L) / L;                        // rounds = ceil((P + 1) / L)
    float z0[PMAX + 1], z1[PMAX + 1];
    uint32_t wx[PMAX + 1];
#pragma unroll
    for (int r = 0; r <= PMAX; ++r) {
        z0[r] = 0.0f; z1[r] = 0.0f; wx[r] = 0u;
        if (r < R) {
            const int t = r * L + lane;              // this lane's task in round r
            const bool acc = t == P;
            const int p = t < P ? t : 0;
            const uint4 w = draw(seed, acc ? RNG_ACCEPT : RNG_MOVE, step, index,
                                 acc ? 0u : (uint32_t)(p >> 1));
            if (p & 1) box_muller(w.z, w.w, z0[r], z1[r]);
            else box_muller(w.x, w.y, z0[r], z1[r]);
            wx[r] = w.x;
        }
    }
    // task t sits in round t / L on slice lane t % L (warp-uniform for fixed t)
    {
        const int r = P / L;
        uint32_t v = wx[0];
#pragma unroll
        for (int rr = 1; rr <= PMAX; ++rr) v = rr == r ? wx[rr] : v;
        accept_word = __shfl_sync(0xFFFFFFFFu, v, base + P % L);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int t = k >> 1, r = t / L;
        float a = z0[0], b = z1[0];
#pragma unroll
        for (int rr = 1; rr <= PMAX; ++rr) {
            a = rr == r ? z0[rr] : a;
            b = rr == r ? z1[rr] : b;
        }
        a = __shfl_sync(0xFFFFFFFFu, a, base + t % L);
        b = __shfl_sync(0xFFFFFFFFu, b, base + t % L);
        z[k] = k < Kreal ? ((k & 1) ? b : a) : 0.0f;
    }
}

// Largest chunk of staged data (floats).  A launch sizes its buffer to
// ychunk = min(kYChunk, N rounded up to 4) floats, followed by the mbarrier,
// so small data sets leave shared memory for more resident CTAs.
constexpr int kYChunk = 8192;

__host__ __device__ inline int ychunk_for(int64_t N) {
    int64_t c = N < 4 ? 4 : ((N + 3) / 4) * 4;
    return (int)(c < kYChunk ? c : kYChunk);
}
__host__ __device__ inline size_t ysmem_bytes(int ychunk) {
    return (size_t)ychunk * sizeof(float) + 16;
}

__device__ __forceinline__ uint64_t* ychunk_mbar(float* ys, int ychunk) {
    return reinterpret_cast<uint64_t*>(ys + ychunk);
}

// Run one slice accumulator over all N data, staging chunk by chunk.  The
// whole block calls this (it contains barriers); `active` slices compute.
template <int K, bool GRAD, bool EQW>
__device__ __forceinline__ void slice_over_data(SliceAcc<K, GRAD, EQW>& acc, float* ys, int ychunk,
                                                const float* __restrict__ y, int64_t N,
                                                bool active, int lane, int L,
                                                const float (&nu)[K], const float (&lw2)[K],
                                                float r, uint32_t& phase, uint32_t* status,
                                                uint32_t limit = kSpinLimit) {
    uint64_t* mbar = ychunk_mbar(ys, ychunk);
    for (int64_t c0 = 0; c0 < N; c0 += ychunk) {
        int cnt = (int)((N - c0) < ychunk ? (N - c0) : ychunk);
        stage_y(ys, y, c0, cnt, mbar, phase, status, limit);
        if (active) acc.run(ys, cnt, lane, L, nu, lw2, r);
        __syncthreads();
    }
}

// The same chunked streaming for the packed equal-weight accumulator.
template <int K, bool GRAD>
__device__ __forceinline__ void slice_over_data_eq(SliceAccEqW<K, GRAD>& acc, float* ys, int ychunk,
                                                   const float* __restrict__ y, int64_t N,
                                                   bool active, int lane, int L,
                                                   const float (&nu)[K], float r,
                                                   uint32_t& phase, uint32_t* status,
                                                   uint32_t limit = kSpinLimit) {
    uint64_t* mbar = ychunk_mbar(ys, ychunk);
    for (int64_t c0 = 0; c0 < N; c0 += ychunk) {
        int cnt = (int)((N - c0) < ychunk ? (N - c0) : ychunk);
        stage_y(ys, y, c0, cnt, mbar, phase, status, limit);
        if (active) acc.run(ys, cnt, lane, L, nu, r);
        __syncthreads();
    }
}

}  // namespace smc
