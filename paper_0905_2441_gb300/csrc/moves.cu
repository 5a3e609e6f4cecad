// moves.cu -- smc_mh_move (random-walk MH and MALA with the gather after
// resampling fused in) and smc_popmcmc_sweep (many independent populations
// of tempered chains in one persistent launch, chains dealt in equal items).
// Sections 3.1, 4.1.1, 4.1.2 of Lee, Yau, Giles, Doucet & Holmes (2009).
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "binned.cuh"
#include "bulk.cuh"
#include "gmm1d.cuh"
#include "bounds.cuh"

using namespace smc_host;

namespace smc {

// accept test: log u < log alpha, compared in FP32 (log alpha arrives as a
// float hi/lo pair from an FP64 difference; the FP32 likelihoods already
// set a decision band far wider than this rounding)
__device__ __forceinline__ bool accept(uint32_t w, float log_alpha) {
    return logf(u01(w)) < log_alpha;
}

// beta (l' - l) with one FP64 subtraction; the product in FP32.  A NaN
// difference gives -inf, so the move is rejected.
__device__ __forceinline__ float tempered_diff(float beta, double lp, double l) {
    const double d = lp - l;
    if (disnan(d)) return -INFINITY;
    float hi, lo;
    split_double(d, hi, lo);
    return beta * (hi + lo);
}

// Block-wide count of accepted moves, one global atomic per block.
__device__ __forceinline__ void count_accepts(bool a, uint32_t* accept_count, uint32_t* s_cnt) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, a);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(s_cnt, (uint32_t)__popc(m));
    __syncthreads();
    if (threadIdx.x == 0 && accept_count && *s_cnt) atomicAdd(accept_count, *s_cnt);
}

// Minimum resident 256-thread blocks per SM asked of the register
// allocator for the move kernel with K <= 8 (the state of the move is
// stashed in shared memory across the likelihood loop, so two blocks fit
// without spilling).
#ifndef SMC_MOVE_MINB
#define SMC_MOVE_MINB 2
#endif

template <int K, bool MALA, bool EQW>
__global__ void __launch_bounds__(256, (K <= 8 ? SMC_MOVE_MINB : 1)) k_mh_move(
    const float* __restrict__ y, int64_t N, const float* theta_in, const double* ll_in,
    const float* grad_in, const int32_t* __restrict__ anc, const int32_t* __restrict__ do_flag,
    float* theta_out, double* ll_out, float* grad_out, int64_t M, const float* __restrict__ beta,
    int64_t beta_stride, float scale, uint64_t seed, uint64_t step, uint32_t* accept_count,
    Gmm1dArgs P, int L, int Kreal, int ychunk, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    extern __shared__ __align__(16) float ys[];
    __shared__ uint32_t s_cnt;
    // K <= 8: the particle's current state, gradient and proposal wait out
    // the likelihood loop here (written and read back by the particle's
    // lane 0 only), not in registers
    constexpr bool STASH = K <= 8;
    __shared__ float s_st[STASH ? 3 * K * 256 : 1];
    if (threadIdx.x == 0) s_cnt = 0;
    init_mbar(ychunk_mbar(ys, ychunk));
    const int lane = threadIdx.x % L;
    const int ppb = blockDim.x / L;
    const int pi = threadIdx.x / L;
    const int64_t p = (int64_t)blockIdx.x * ppb + pi;
    const bool active = p < M;

    int64_t src = p;
    if (active && anc && (!do_flag || *do_flag != 0)) src = anc[p];
    if (active && !SMC_IN_BOUNDS(src >= 0 && src < M, status)) src = p;
    float mu[K], g[K], z[K], prop[K];
    double l = 0.0;
    float b = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) { mu[k] = 0.0f; g[k] = 0.0f; }
    uint32_t aw;
    slice_draws<K>(seed, step, (uint32_t)(active ? p : 0), lane, L, Kreal, z, aw);
    if (active) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k < Kreal) {
                mu[k] = theta_in[(int64_t)k * M + src];
                if (MALA) g[k] = grad_in[(int64_t)k * M + src];
            }
        }
        l = ll_in[src];
        b = beta[p * beta_stride];
    }
    const float hh2 = 0.5f * scale * scale;
    bool in_box = active;
    float mf[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        mf[k] = MALA ? fmaf(hh2 * b, g[k], mu[k]) : mu[k];
        prop[k] = k < Kreal ? fmaf(scale, z[k], mf[k]) : 0.0f;
        if (k < Kreal) in_box &= (prop[k] >= P.lo) & (prop[k] <= P.hi);
    }
    float nu[K], lw2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        nu[k] = -prop[k] * P.r;
        lw2[k] = P.lw2[k];
    }
    if constexpr (STASH) {
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                s_st[k * 256 + pi] = mu[k];
                if (MALA) s_st[(K + k) * 256 + pi] = g[k];
                s_st[(2 * K + k) * 256 + pi] = prop[k];
            }
        }
    }
    uint32_t phase = 0;
    float gp[K];
    double lp;
    if constexpr (EQW) {
        SliceAccEqW<K, MALA> acc;
        slice_over_data_eq(acc, ys, ychunk, y, N, in_box, lane, L, nu, P.r, phase, status,
                           P.wait_limit);
        lp = acc.finish(L, P, gp);
    } else {
        SliceAcc<K, MALA, EQW> acc;
        slice_over_data(acc, ys, ychunk, y, N, in_box, lane, L, nu, lw2, P.r, phase, status,
                        P.wait_limit);
        lp = acc.finish(L, P, gp);
    }

    if constexpr (STASH) {  // back from shared memory (lane 0 is the only reader)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            mu[k] = lane == 0 ? s_st[k * 256 + pi] : 0.0f;
            g[k] = (MALA && lane == 0) ? s_st[(K + k) * 256 + pi] : 0.0f;
            prop[k] = lane == 0 ? s_st[(2 * K + k) * 256 + pi] : 0.0f;
            mf[k] = MALA ? fmaf(hh2 * b, g[k], mu[k]) : mu[k];
        }
    }
    bool acc_ok = false;
    if (in_box && lane == 0) {
        float log_alpha = tempered_diff(b, lp, l);
        if (MALA) {
            float fwd = 0.0f, bwd = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k < Kreal) {
                    float df = prop[k] - mf[k];
                    float db = mu[k] - fmaf(hh2 * b, gp[k], prop[k]);
                    fwd = fmaf(df, df, fwd);
                    bwd = fmaf(db, db, bwd);
                }
            }
            log_alpha += (fwd - bwd) / (2.0f * scale * scale);
        }
        if (lp != lp) raise_status(status, ST_NONFINITE);
        acc_ok = accept(aw, log_alpha);
    }
    if (active && lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k < Kreal) {
                theta_out[(int64_t)k * M + p] = acc_ok ? prop[k] : mu[k];
                if (MALA) grad_out[(int64_t)k * M + p] = acc_ok ? gp[k] : g[k];
            }
        }
        ll_out[p] = acc_ok ? lp : l;
    }
    count_accepts(acc_ok, accept_count, &s_cnt);
}

// ------------------------------------------------------------------ population MCMC
// Work items are chunks of (blockDim / L) consecutive chains of the flat
// chain array, dealt round-robin to the CTAs, so every item costs the same
// whatever the population sizes.  After an item's moves, one lane adds the
// item's chain count to each population it touches (one acquire-release
// atomic per population); the CTA that completes a population runs that
// population's exchange moves at once, its pairs dealt over all the CTA's
// threads, so no CTA ever waits on another.  The counters are left at zero
// for the next sweep.
__device__ __forceinline__ int pop_of(const int32_t* __restrict__ offsets, int n_pops, int64_t c) {
    int lo = 0, hi = n_pops;  // largest q with offsets[q] <= c
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(offsets + mid) <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}


// Pairs of one exchange move (Section 3.3: adjacent temperatures, disjoint
// pairs chosen by a parity bit): parity 0 pairs (2j, 2j+1); parity 1 pairs
// (2j+1, 2j+2) and, for an even population, the wrap-around pair (Mq-1, 0).
__device__ __forceinline__ int exchange_npairs(int Mq, uint32_t par) {
    return par == 0 ? Mq / 2 : (Mq - 1) / 2 + ((Mq % 2 == 0) ? 1 : 0);
}

// Exchange move of pair j of population q (chains base..base+Mq-1): the
// chains' states and log-likelihoods are loaded together (one round trip),
// then swapped if accepted with log alpha = (beta_a - beta_b)(l_b - l_a).
template <int K>
__device__ __forceinline__ bool exchange_pair(float* theta, double* ll, int64_t Mtot,
                                              const float* __restrict__ beta, int64_t base,
                                              int Mq, uint32_t par, int q, int j, int Kreal,
                                              uint64_t seed, uint64_t sweep, uint32_t* status) {
    int ia, ib;
    if (par == 0) { ia = 2 * j; ib = 2 * j + 1; }
    else if (j < (Mq - 1) / 2) { ia = 2 * j + 1; ib = 2 * j + 2; }
    else { ia = Mq - 1; ib = 0; }
    const int64_t ga = base + ia, gb = base + ib;
    // (chain indices come from the caller's population offsets)
    if (!SMC_IN_BOUNDS(base >= 0 && ga < Mtot && gb < Mtot, status)) return false;
    const double la = __ldcg(ll + ga), lb = __ldcg(ll + gb);
    float ta[K], tb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ta[k] = k < Kreal ? __ldcg(theta + (int64_t)k * Mtot + ga) : 0.0f;
        tb[k] = k < Kreal ? __ldcg(theta + (int64_t)k * Mtot + gb) : 0.0f;
    }
    const uint4 w = draw(seed, RNG_EXCHANGE, sweep, (uint32_t)q, 1u + (uint32_t)(j >> 2));
    const float log_alpha = tempered_diff(beta[ga] - beta[gb], lb, la);
    if (!accept(word_of(w, j & 3), log_alpha)) return false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (k < Kreal) {
            __stcg(theta + (int64_t)k * Mtot + ga, tb[k]);
            __stcg(theta + (int64_t)k * Mtot + gb, ta[k]);
        }
    }
    __stcg(ll + ga, lb);
    __stcg(ll + gb, la);
    return true;
}

// Minimum resident 256-thread blocks per SM asked of the register
// allocator for the sweep (compile-time tuning knob; 1 leaves it free).
#ifndef SMC_POP_MINB
#define SMC_POP_MINB 2
#endif

// add with acquire-release ordering at GPU scope: publishes the writes the
// calling CTA made before its last barrier, and sees those of every CTA that
// added before it
__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Warp 0 of a CTA finds the first population overlapping chain c0 (a 32-way
// parallel search of the CSR offsets) and the bounds [qa, qb) of population
// qlo + lane; the whole warp calls this.
__device__ __forceinline__ void pop_search(const int32_t* __restrict__ offsets, int n_pops,
                                           int64_t c0, int l32, int& qlo, int64_t& qa,
                                           int64_t& qb) {
    int qhi = n_pops;  // offsets[qlo] <= c0 < offsets[qhi]
    while (qhi - qlo > 1) {
        // 32 probes split [qlo, qhi) into 33 parts
        const int span = qhi - qlo;
        const int probe = qlo + (int)(((int64_t)span * (l32 + 1)) / 33);
        const bool inside = probe > qlo && probe < qhi;
        const int64_t op = inside ? (int64_t)offsets[probe] : 0;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, inside && op <= c0);
        const unsigned gt = __ballot_sync(0xFFFFFFFFu, inside && op > c0);
        int nlo = qlo, nhi = qhi;
        if (m) nlo = __shfl_sync(0xFFFFFFFFu, probe, 31 - __clz(m));
        if (gt) nhi = __shfl_sync(0xFFFFFFFFu, probe, __ffs(gt) - 1);
        if (nlo == qlo && nhi == qhi) {  // fewer than 33 candidates left: scan
            const int cand = qlo + 1 + l32;
            const bool le2 = cand < qhi && (int64_t)offsets[cand] <= c0;
            const unsigned m2 = __ballot_sync(0xFFFFFFFFu, le2);
            if (m2) nlo = qlo + 1 + (31 - __clz(m2));
            nhi = nlo + 1;
        }
        qlo = nlo;
        qhi = nhi;
    }
    const int q = qlo + l32;
    if (q < n_pops) {
        qa = offsets[q];
        qb = offsets[q + 1];
    }
}

// After a CTA's moves of chains [c0, c1): count them per population (one
// lane of warp 0 per touched population adds its count with release
// semantics, publishing the moves); the lane whose add completes a
// population acquires every other CTA's moves of it and lists it; then the
// CTA runs the exchange moves of the populations it completed, their pairs
// dealt over all its threads, and clears their counters for the next sweep.
// The whole block calls this; (qlo, qa, qb) come from pop_search in warp 0.
template <int K>
__device__ __forceinline__ void pop_exchange(float* theta, double* ll, int64_t Mtot,
                                             const float* __restrict__ beta,
                                             const int32_t* __restrict__ offsets, int n_pops,
                                             uint64_t seed, uint64_t sweep, uint32_t* pop_done,
                                             int64_t c0, int64_t c1, int qlo, int64_t qa,
                                             int64_t qb, int4* exb, int* s_nex, uint32_t* s_sw,
                                             uint32_t* s_try, int Kreal, uint32_t* status) {
    const int warp = threadIdx.x >> 5, l32 = threadIdx.x & 31;
    if (threadIdx.x == 0) *s_nex = 0;
    __syncthreads();  // the moves are done (and ordered before warp 0's release)
    if (warp == 0) {
        for (int q = qlo + l32;; q += 32) {
            if (q >= qlo + 32 && q < n_pops) {  // beyond the prefetched 32 (rare)
                qa = offsets[q];
                qb = offsets[q + 1];
            }
            const bool in = q < n_pops && qa < c1;
            if (!__any_sync(0xFFFFFFFFu, in)) break;
            if (in) {
                const int64_t a = qa > c0 ? qa : c0;
                const int64_t b2 = qb < c1 ? qb : c1;
                if (b2 > a) {
                    const uint32_t cnt = (uint32_t)(b2 - a);
                    const uint32_t Mq = (uint32_t)(qb - qa);
                    const uint32_t old = atomic_add_acq_rel(pop_done + q, cnt);
                    if (old + cnt == Mq) {
                        const uint32_t par =
                            draw(seed, RNG_EXCHANGE, sweep, (uint32_t)q, 0u).x & 1u;
                        exb[atomicAdd(s_nex, 1)] = make_int4(q, (int)qa, (int)Mq, (int)par);
                    }
                }
            }
        }
    }
    __syncthreads();
    const int nex = *s_nex;
    if (nex) {
        int total = 0;
        for (int e = 0; e < nex; ++e) total += exchange_npairs(exb[e].z, (uint32_t)exb[e].w);
        uint32_t swaps = 0;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int e = 0, j = t;
            for (;;) {  // entry holding task t (nex is small)
                const int np = exchange_npairs(exb[e].z, (uint32_t)exb[e].w);
                if (j < np) break;
                j -= np;
                ++e;
            }
            const int4 d = exb[e];
            swaps += exchange_pair<K>(theta, ll, Mtot, beta, d.y, d.z, (uint32_t)d.w, d.x, j, Kreal,
                                      seed, sweep, status);
        }
        if (swaps) atomicAdd(s_sw, swaps);
        for (int e = threadIdx.x; e < nex; e += blockDim.x) {
            pop_done[exb[e].x] = 0u;
            atomicAdd(s_try, (uint32_t)exchange_npairs(exb[e].z, (uint32_t)exb[e].w));
        }
    }
}

// Consecutive sweeps use programmatic dependent launch: the next sweep's
// prologue (data staging, random draws, population search: nothing a sweep
// writes) overlaps this one's tail; grid_dep_wait() precedes the chain state.

template <int K, bool EQW>
__global__ void __launch_bounds__(256, SMC_POP_MINB) k_popmcmc_sweep(
    const float* __restrict__ y, int64_t N, float* theta, double* ll, int64_t Mtot,
    const float* __restrict__ beta, const int32_t* __restrict__ offsets, int32_t n_pops,
    float scale, uint64_t seed, uint64_t sweep, unsigned long long* stats, uint32_t* pop_done,
    Gmm1dArgs P, int L, int Kreal, int ychunk, int inline_ex, uint32_t* status) {
    grid_dep_launch();
    // dynamic shared memory: staged data, mbarrier, then two lists of the
    // populations an item completed (at most chains-per-item + 1 each), an
    // entry being {population, first chain, chains, parity}
    extern __shared__ __align__(16) float ys[];
    const int lcap = blockDim.x / L + 1;
    int4* s_exb = reinterpret_cast<int4*>(ys + ychunk + 4);
    __shared__ int s_nex[2];
    __shared__ uint32_t s_mh, s_sw, s_try;
    init_mbar(ychunk_mbar(ys, ychunk));
    if (threadIdx.x == 0) { s_mh = 0; s_sw = 0; s_try = 0; }
    const int lane = threadIdx.x % L;
    const int ppb = blockDim.x / L;
    const int warp = threadIdx.x >> 5;
    const int l32 = threadIdx.x & 31;
    const int64_t nitems = (Mtot + ppb - 1) / ppb;
    uint32_t phase = 0;
    const bool resident = N <= ychunk;  // all data in shared memory: stage once
    if (resident && N > 0)
        stage_y(ys, y, 0, (int)N, ychunk_mbar(ys, ychunk), phase, status, P.wait_limit);
    float lw2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lw2[k] = P.lw2[k];

    // items are equal chunks of ppb consecutive chains, dealt round-robin
    uint32_t iter = 0;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int64_t c0 = item * ppb;
        const int64_t c1 = c0 + ppb < Mtot ? c0 + ppb : Mtot;
        const int64_t c = c0 + threadIdx.x / L;
        const bool active = c < Mtot;
        // ---- work that reads nothing a sweep writes: the move's draws and,
        // in warp 0, the first population overlapping the item (a 32-way
        // parallel search) with the bounds of the next 32 populations
        float z[K];
        uint32_t aw;
        slice_draws<K>(seed, sweep, (uint32_t)(active ? c : 0), lane, L, Kreal, z, aw);
        const float b = active ? beta[c] : 0.0f;
        int qlo = 0;
        int64_t qa = 0, qb = 0;  // bounds of population qlo + l32 (warp 0)
        if (inline_ex && warp == 0) pop_search(offsets, n_pops, c0, l32, qlo, qa, qb);
        // ---- the state of the chains: written by the previous sweep
        if (iter == 0) grid_dep_wait();
        float mu[K], prop[K], nu[K];
        double l = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) mu[k] = 0.0f;
        if (active) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < Kreal) mu[k] = theta[(int64_t)k * Mtot + c];
            l = ll[c];
        }
        // ---- random-walk MH move of chain c
        bool in_box = active;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            prop[k] = k < Kreal ? fmaf(scale, z[k], mu[k]) : 0.0f;
            if (k < Kreal) in_box &= (prop[k] >= P.lo) & (prop[k] <= P.hi);
            nu[k] = -prop[k] * P.r;
        }
        double lp;
        if constexpr (EQW) {
            SliceAccEqW<K> acc;
            if (resident) {
                if (in_box) acc.run(ys, (int)N, lane, L, nu, P.r);
            } else {
                slice_over_data_eq(acc, ys, ychunk, y, N, in_box, lane, L, nu, P.r, phase, status,
                                   P.wait_limit);
            }
            lp = acc.finish(L, P);
        } else {
            SliceAcc<K, false, false> acc;
            if (resident) {
                if (in_box) acc.run(ys, (int)N, lane, L, nu, lw2, P.r);
            } else {
                slice_over_data(acc, ys, ychunk, y, N, in_box, lane, L, nu, lw2, P.r, phase, status,
                                P.wait_limit);
            }
            float gd[K];
            lp = acc.finish(L, P, gd);
        }
        bool ok = false;
        if (in_box && lane == 0) {
            if (lp != lp) raise_status(status, ST_NONFINITE);
            ok = accept(aw, tempered_diff(b, lp, l));
        }
        if (active && lane == 0 && ok) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < Kreal) theta[(int64_t)k * Mtot + c] = prop[k];
            ll[c] = lp;
        }
        const unsigned acc_mask = __ballot_sync(0xFFFFFFFFu, ok);
        if (l32 == 0 && acc_mask) atomicAdd(&s_mh, (uint32_t)__popc(acc_mask));
        ++iter;
        if (!inline_ex) continue;  // the exchanges run in k_popmcmc_exchange
        const int buf = (int)((iter - 1) & 1);  // double-buffered list: no third barrier
        pop_exchange<K>(theta, ll, Mtot, beta, offsets, n_pops, seed, sweep, pop_done, c0, c1,
                        qlo, qa, qb, s_exb + buf * lcap, &s_nex[buf], &s_sw, &s_try, Kreal,
                        status);
    }
    if (iter == 0) grid_dep_wait();  // a block without items still orders its stats
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        if (s_mh) atomicAdd(stats + 0, (unsigned long long)s_mh);
        if (s_sw) atomicAdd(stats + 1, (unsigned long long)s_sw);
        if (s_try) atomicAdd(stats + 2, (unsigned long long)s_try);
    }
}

// ------------------------------------------------------------------ binned population sweep
// The sweep for data sets held whole in shared memory (512 <= N <= 4096,
// K <= 16), with the data sorted into bins once per sweep by every CTA
// (binned.cuh).  A warp's 32 lanes take 32 consecutive chains (a chain
// group) over the same slots of the sorted list, so bins, loop counts and
// shared-memory loads are uniform across the warp.  The work, G groups x H
// pair slots (H = half the list's padded length), is split evenly over the
// CTAs (one 512-thread CTA per SM) as contiguous ranges of the group-major
// order.  A CTA works in rounds of at most 16 groups: its threads draw the
// round's normals (one Box-Muller pair or accept word per task) and propose;
// its warps then take chunks (a piece of one bin of one group: one setup of
// the bin's coefficients each) from a shared-memory queue, largest pieces
// first, so they finish together whatever the warp scheduler favours.  Each
// chunk's partial sum enters its chain's total as an exact 2^-32 fixed-point
// integer, so the totals do not depend on the order chunks finish in.  A
// group cut by a CTA boundary (at most two parts: the grid never has more
// CTAs than groups) stores its part in the context and bumps the group's
// counter; the CTA that brings the counter to two adds the two parts.  The
// group's chains then take their accept decisions, and the exchange stage is
// the same as in k_popmcmc_sweep.
constexpr int kBinThreads = 512;
constexpr int kOffSmem = 4096;   // population offsets staged in shared memory up to this count

__host__ __device__ inline int binned_yb_len(int64_t N) {
    return (int)((N + kClasses + 3) & ~(int64_t)3);
}
__host__ __device__ inline int binned_rk_len(int64_t N) {  // floats holding N uint16 ranks
    return (int)(((N + 1) / 2 + 3) & ~(int64_t)3);
}
// dynamic shared memory: staged data, mbarrier, sorted list, ranks, the
// chains' fixed-point totals [16 groups][32 lanes], then per chain slot: old
// log-likelihood, proposal (normals before it), temperature, accept word,
// in-box flag; the population offsets (when at most kOffSmem + 1); last,
// 16-byte aligned, the cached layout's copy of the data
__host__ __device__ inline size_t binned_smem_bytes(int64_t N, int K, int64_t n_pops) {
    const int yc = ychunk_for(N);
    const size_t off = n_pops + 1 <= kOffSmem ? (size_t)(n_pops + 1) * 4 : 0;
    return ((size_t)yc + 4 + (size_t)binned_yb_len(N) + (size_t)binned_rk_len(N)) * 4 +
           (size_t)kBinThreads * 8 + (size_t)kBinThreads * (8 + 4 * (size_t)K + 12) + off + 16 +
           bcache_ycopy_bytes(N);
}
// shared memory of k_bin_prepare: staged data, mbarrier slot, sorted list, ranks
__host__ __device__ inline size_t bin_prepare_smem_bytes(int64_t N) {
    return ((size_t)ychunk_for(N) + 4 + (size_t)binned_yb_len(N) + (size_t)binned_rk_len(N)) * 4;
}

// The binned layout of a data set (sorted list, table core, pieces) built
// once by one CTA and stored with a copy of the data (binned.cuh), for the
// sweeps that follow.  Launched without programmatic dependent launch and
// never releasing its dependents early, so a sweep that reads the layout
// before its own dependency wait finds it complete.
__global__ void __launch_bounds__(kBinThreads) k_bin_prepare(const float* __restrict__ y, int64_t N,
                                                             float binw, float binw_inv, float cf,
                                                             char* __restrict__ bcache) {
    extern __shared__ __align__(16) float pm[];
    const int yc = ychunk_for(N), ybl = binned_yb_len(N);
    float* ys = pm;
    float* yb = ys + yc + 4;
    uint16_t* rk = reinterpret_cast<uint16_t*>(yb + ybl);
    __shared__ BinTable bt;
    __shared__ __align__(16) int s_piece_w[kPiecesBytes / 4];
    __shared__ int s_np;
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    bin_partition(ys, (int)N, yb, rk, bt, binw, binw_inv, cf);
    bin_pieces(bt, reinterpret_cast<int3*>(s_piece_w), &s_np);
    __syncthreads();
    if (tid == 0) {
        int* h = reinterpret_cast<int*>(bcache);
        h[0] = (int)N;
        h[1] = s_np;
        h[2] = __float_as_int(binw);
        h[3] = __float_as_int(cf);
    }
    float* yc_out = reinterpret_cast<float*>(bcache + 16);
    for (int i = tid; i < (int)(bcache_ycopy_bytes(N) / 4); i += blockDim.x)
        yc_out[i] = i < N ? ys[i] : 0.0f;
    float* yb_out = reinterpret_cast<float*>(bcache + bcache_yb_off(N));
    for (int i = tid; i < ybl; i += blockDim.x) yb_out[i] = yb[i];  // past the list: never read
    const uint32_t* core = reinterpret_cast<const uint32_t*>(&bt);
    uint32_t* core_out = reinterpret_cast<uint32_t*>(bcache + bcache_core_off(N, ybl));
    for (int i = tid; i < (int)(kBinCoreBytes / 4); i += blockDim.x) core_out[i] = core[i];
    int* pc_out = reinterpret_cast<int*>(bcache + bcache_pieces_off(N, ybl));
    for (int i = tid; i < (int)(kPiecesBytes / 4); i += blockDim.x) pc_out[i] = s_piece_w[i];
}

// first pair slot of CTA b's range: floor(b Wt / B)
__device__ __forceinline__ int64_t cta_first(int64_t b, int64_t Wt, int64_t B) {
    return b * Wt / B;
}
// the CTA whose range holds slot x
__device__ __forceinline__ int64_t cta_of(int64_t x, int64_t Wt, int64_t B) {
    int64_t b = x * B / Wt;
    while (b > 0 && cta_first(b, Wt, B) > x) --b;
    while (b + 1 < B && cta_first(b + 1, Wt, B) <= x) ++b;
    return b;
}

template <int K>
__global__ void __launch_bounds__(kBinThreads, 1) k_popmcmc_binned(
    const float* __restrict__ y, int64_t N, float* theta, double* ll, int64_t Mtot,
    const float* __restrict__ beta, const int32_t* __restrict__ offsets, int32_t n_pops,
    float scale, uint64_t seed, uint64_t sweep, unsigned long long* stats, uint32_t* pop_done,
    uint32_t* grp_done, long long* grp_part, Gmm1dArgs P, int Kreal, int inline_ex,
    const char* __restrict__ bcache, uint32_t* status) {
    grid_dep_launch();
    extern __shared__ __align__(16) float sm[];
    constexpr int T = kBinThreads, NW = T / 32;
    const int yc = ychunk_for(N);
    float* ys = sm;
    float* yb = ys + yc + 4;
    uint16_t* rk = reinterpret_cast<uint16_t*>(yb + binned_yb_len(N));
    long long* s_acc = reinterpret_cast<long long*>(yb + binned_yb_len(N) + binned_rk_len(N));
    double* s_lold = reinterpret_cast<double*>(s_acc + T);
    float* s_prop = reinterpret_cast<float*>(s_lold + T);
    float* s_beta = s_prop + K * T;
    uint32_t* s_aw = reinterpret_cast<uint32_t*>(s_beta + T);
    int* s_inb = reinterpret_cast<int*>(s_aw + T);
    int32_t* s_off = reinterpret_cast<int32_t*>(s_inb + T);
    float* s_ycopy = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(s_off + (n_pops + 1 <= kOffSmem ? n_pops + 1 : 0)) + 15) &
        ~(uintptr_t)15);
    __shared__ BinTable bt;
    __shared__ __align__(16) int s_piece_w[kPiecesBytes / 4];
    int3* s_piece = reinterpret_cast<int3*>(s_piece_w);
    __shared__ int4 s_exb[T + 1];
    __shared__ int s_nex, s_next, s_np;
    __shared__ int s_fin[NW];  // a round's groups decided by this CTA
    __shared__ uint32_t s_mh, s_sw, s_try;
    __shared__ uint64_t s_cmb;                  // the cached layout's copies
    __shared__ __align__(16) int s_hdr[4];
    if (threadIdx.x == 0 && bcache) mb_init(&s_cmb, 1);  // (fenced by init_mbar)
    init_mbar(ychunk_mbar(ys, yc));
    if (threadIdx.x == 0) { s_mh = 0; s_sw = 0; s_try = 0; }
    const int tid = (int)threadIdx.x, warp = tid >> 5, l32 = tid & 31;
    // the chain groups of this CTA: [gA, gEnd) with gA = floor(b G / B) and
    // gEnd <= ceil((b + 1) G / B) (both exact whatever H is)
    const int64_t G = (Mtot + 31) >> 5;
    const int64_t B = gridDim.x;
    const int64_t gA = (int64_t)blockIdx.x * G / B;
    const int64_t gEub = ((int64_t)blockIdx.x + 1) * G / B +
                         ((((int64_t)blockIdx.x + 1) * G) % B != 0 ? 1 : 0);
    const int npair = (Kreal + 1) >> 1;  // Box-Muller pairs per chain
    const int nblk = (npair + 1) >> 1;   // Philox blocks (two pairs each) per chain
    // Draws of round g0 (nothing a sweep writes): task t is Box-Muller pair
    // t % (npair + 1) of chain slot t / (npair + 1), or its accept word; the
    // normals wait in s_prop.  Also the temperatures (read-only).
    auto round_draws = [&](int64_t g0, int nslot) {
        const int64_t cfirst = g0 * 32;
        const int64_t cb = cfirst + tid;
        const float bt_c = (tid < nslot && cb < Mtot) ? beta[cb] : 0.0f;  // stored after the draws
        // task j < nblk: Philox block j of the chain's move words, i.e. the
        // Box-Muller pairs 2j (words x, y) and 2j + 1 (z, w); task nblk: the
        // accept word
        for (int t = tid; t < nslot * (nblk + 1); t += T) {
            const int slot = t / (nblk + 1), j = t - slot * (nblk + 1);
            const uint32_t c = (uint32_t)(cfirst + slot);
            if (j == nblk) {
                s_aw[slot] = draw(seed, RNG_ACCEPT, sweep, c, 0u).x;
            } else {
                const uint4 w = draw(seed, RNG_MOVE, sweep, c, (uint32_t)j);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int jp = 2 * j + h;  // the Box-Muller pair
                    if (jp < npair) {
                        float z0, z1;
                        if (h) box_muller(w.z, w.w, z0, z1);
                        else box_muller(w.x, w.y, z0, z1);
                        s_prop[(2 * jp) * T + slot] = z0;
                        if (2 * jp + 1 < K) s_prop[(2 * jp + 1) * T + slot] = z1;
                    }
                }
            }
        }
        s_beta[tid] = bt_c;
    };
    // ---- prologue: the data's bulk copy and the offsets' loads go out first,
    // the first round's draws and an L2 prefetch of its chain states overlap
    // them (a prefetch reads no value; the states are read after the wait)
    uint32_t phase = 0;
    const bool bulk = stage_y_issue(ys, y, 0, (int)N, ychunk_mbar(ys, yc));
    // the cached layout (k_bin_prepare, complete before this launch began):
    // header, data copy, sorted list, table core and pieces, each by one
    // bulk copy into the place the partition below would fill
    const int ybl = binned_yb_len(N);
    if (bcache && tid == 0) {
        const uint32_t ycb = (uint32_t)bcache_ycopy_bytes(N);
        mb_expect_tx(&s_cmb, 16u + ycb + (uint32_t)ybl * 4u + (uint32_t)kBinCoreBytes +
                                 (uint32_t)kPiecesBytes);
        bulk_load(s_hdr, bcache, 16u, &s_cmb);
        bulk_load(s_ycopy, bcache + 16, ycb, &s_cmb);
        bulk_load(yb, bcache + bcache_yb_off(N), (uint32_t)ybl * 4u, &s_cmb);
        bulk_load(&bt, bcache + bcache_core_off(N, ybl), (uint32_t)kBinCoreBytes, &s_cmb);
        bulk_load(s_piece_w, bcache + bcache_pieces_off(N, ybl), (uint32_t)kPiecesBytes, &s_cmb);
    }
    // (each thread's first offset is loaded into a register and stored after
    // the draws, so the thread does not wait for it)
    const int32_t* offs = offsets;
    const bool off_smem = inline_ex && n_pops + 1 <= kOffSmem;
    int32_t off0 = 0;
    if (off_smem) {
        if (tid <= n_pops) off0 = offsets[tid];
        for (int i = tid + T; i <= n_pops; i += T) s_off[i] = offsets[i];
        offs = s_off;
    }
    {
        const int64_t ng0 = (gEub - gA) < NW ? (gEub - gA) : NW;
        const int64_t c = gA * 32 + tid;
        if (tid < ng0 * 32 && c < Mtot) {
            for (int k = 0; k < Kreal; ++k)
                asm volatile("prefetch.global.L2 [%0];" :: "l"(theta + (int64_t)k * Mtot + c));
            asm volatile("prefetch.global.L2 [%0];" :: "l"(ll + c));
        }
        round_draws(gA, (int)(ng0 * 32));
    }
    if (off_smem && tid <= n_pops) s_off[tid] = off0;
    stage_y_wait(bulk, ychunk_mbar(ys, yc), phase, status, P.wait_limit);
    // ---- the data sorted into bins, cut into pieces: the cached layout when
    // it was built from these very data, bin width and c, else partitioned here
    bool fresh = true;
    if (bcache) {
        mb_wait(&s_cmb, 0, status, P.wait_limit);
        bool bad = false;
        for (int i = tid; i < N; i += T) bad |= __float_as_uint(ys[i]) != __float_as_uint(s_ycopy[i]);
        if (tid == 0)
            bad |= s_hdr[0] != (int)N || s_hdr[2] != __float_as_int(P.binw) ||
                   s_hdr[3] != __float_as_int(P.cf) || s_hdr[1] < 1 || s_hdr[1] > kMaxPieces;
        fresh = __syncthreads_or(bad) != 0;
        if (!fresh && tid == 0) s_np = s_hdr[1];
    }
    if (fresh) {
        bin_partition(ys, (int)N, yb, rk, bt, P.binw, P.binw_inv, P.cf);
        bin_pieces(bt, s_piece, &s_np);
    }
    __syncthreads();
    const int np = s_np;
    const int64_t H = bt.start[kClasses] >> 1;
    const int64_t Wt = G * H;
    const int64_t R0 = cta_first(blockIdx.x, Wt, B), R1 = cta_first(blockIdx.x + 1, Wt, B);
    const int64_t gEnd = R1 > R0 ? (R1 - 1) / H + 1 : gA;
    bool first = true;
    for (int64_t g0 = gA; g0 < gEnd; g0 += NW) {
        const int ng = (int)((gEnd - g0) < NW ? (gEnd - g0) : NW);
        const int64_t cfirst = g0 * 32;
        const int nslot = ng * 32;
        if (!first) round_draws(g0, nslot);
        int qlo = 0;
        int64_t qa = 0, qb = 0;
        if (inline_ex && warp == 0) pop_search(offs, n_pops, cfirst, l32, qlo, qa, qb);
        if (threadIdx.x == 0) s_next = 0;
        s_acc[tid] = 0;
        __syncthreads();
        // ---- the chains' states: written by the previous sweep
        if (first) {
            grid_dep_wait();
            first = false;
        }
        {
            const int64_t c = cfirst + tid;
            const bool mine = tid < nslot && c < Mtot;
            bool inb = mine;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float pk = 0.0f;
                if (mine && k < Kreal) {
                    pk = fmaf(scale, s_prop[k * T + tid], theta[(int64_t)k * Mtot + c]);
                    inb &= (pk >= P.lo) & (pk <= P.hi);
                }
                s_prop[k * T + tid] = pk;
            }
            s_lold[tid] = mine ? ll[c] : 0.0;
            s_inb[tid] = inb ? 1 : 0;
        }
        __syncthreads();
        // ---- chunks of the round's slots [P0, P1) from a queue: chunk ci is
        // piece ci / ng of group ci % ng (largest pieces first)
        const int64_t P0 = R0 > g0 * H ? R0 : g0 * H;
        const int64_t P1 = R1 < (g0 + ng) * H ? R1 : (g0 + ng) * H;
#pragma unroll 1
        for (;;) {
            int ci = 0;
            if (l32 == 0) ci = atomicAdd(&s_next, 1);
            ci = __shfl_sync(0xFFFFFFFFu, ci, 0);
            if (ci >= np * ng) break;
            const int j = ci / ng, gs = ci - j * ng;
            const int64_t gb = (g0 + gs) * H;
            const int3 pc = s_piece[j];
            // the piece clipped to this CTA's slots of the group (even bounds)
            int a = pc.x, b = pc.y;
            if (gb * 2 + a < P0 * 2) a = (int)(P0 * 2 - gb * 2);
            if (gb * 2 + b > P1 * 2) b = (int)(P1 * 2 - gb * 2);
            if (b <= a) continue;
            BinnedAcc<K> acc;
            acc.piece(yb, bt, a, b, pc.z, s_prop + gs * 32 + l32, T, P.lw2, P.cf, P.r);
            const float2 pp = acc.partial();
            atomicAdd(reinterpret_cast<unsigned long long*>(s_acc + gs * 32 + l32),
                      (unsigned long long)(fixed32(pp.x) - fixed32(pp.y)));
        }
        __syncthreads();
        // ---- warp gs: the chains of group g0 + gs
        bool ok = false;
        if (warp < ng) {
            const int64_t g = g0 + warp;
            const int64_t x0 = g * H, x1 = x0 + H;
            long long part = s_acc[warp * 32 + l32];
            bool fin = true;
            if (x0 < R0 || x1 > R1) {  // cut by a CTA boundary: two parts
                const int64_t b0 = cta_of(x0, Wt, B);
                const int k = (int)(blockIdx.x - b0);
                grp_part[(g * 2 + k) * 32 + l32] = part;
                __syncwarp();
                uint32_t old = 0;
                if (l32 == 0) old = atomic_add_acq_rel(grp_done + g, 1u);
                old = __shfl_sync(0xFFFFFFFFu, old, 0);
                fin = old == 1u;
                if (fin) {
                    part = __ldcg(grp_part + (g * 2) * 32 + l32) +
                           __ldcg(grp_part + (g * 2 + 1) * 32 + l32);
                    if (l32 == 0) grp_done[g] = 0u;
                }
            }
            const int slot = warp * 32 + l32;
            const int64_t cc = g * 32 + l32;
            if (fin && cc < Mtot && s_inb[slot]) {
                const double lp = ((double)part * 0x1p-32 + bt.dconst) * kLn2 + P.cst;
                if (lp != lp) raise_status(status, ST_NONFINITE);
                ok = accept(s_aw[slot], tempered_diff(s_beta[slot], lp, s_lold[slot]));
                if (ok) {
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (k < Kreal) theta[(int64_t)k * Mtot + cc] = s_prop[k * T + slot];
                    ll[cc] = lp;
                }
            }
            if (l32 == 0) s_fin[warp] = fin ? 1 : 0;
        }
        const unsigned acc_mask = __ballot_sync(0xFFFFFFFFu, ok);
        if (l32 == 0 && acc_mask) atomicAdd(&s_mh, (uint32_t)__popc(acc_mask));
        __syncthreads();
        if (inline_ex) {
            // the groups of this round decided here: a contiguous run (only
            // the first and the last can have been decided by a neighbour)
            int ga = 0, gz = ng;
            while (ga < ng && !s_fin[ga]) ++ga;
            while (gz > ga && !s_fin[gz - 1]) --gz;
            const int64_t c0 = (g0 + ga) * 32;
            int64_t c1 = (g0 + gz) * 32;
            if (c1 > Mtot) c1 = Mtot;
            pop_exchange<K>(theta, ll, Mtot, beta, offs, n_pops, seed, sweep, pop_done, c0,
                            c1 > c0 ? c1 : c0, qlo, qa, qb, s_exb, &s_nex, &s_sw, &s_try, Kreal,
                            status);
        }
        __syncthreads();  // the round's shared arrays are free again
    }
    if (first) grid_dep_wait();  // a block without chains still orders its stats
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        if (s_mh) atomicAdd(stats + 0, (unsigned long long)s_mh);
        if (s_sw) atomicAdd(stats + 1, (unsigned long long)s_sw);
        if (s_try) atomicAdd(stats + 2, (unsigned long long)s_try);
    }
}

// Exchange stage of a sweep as its own grid-wide launch, for populations
// too large for one CTA to exchange after its moves: one thread per chain;
// the thread of a pair's first chain runs that pair (the same pairs, draws
// and swap rule as the in-sweep exchange, so the result is identical).
template <int K>
__global__ void __launch_bounds__(256) k_popmcmc_exchange(
    float* theta, double* ll, int64_t Mtot, const float* __restrict__ beta,
    const int32_t* __restrict__ offsets, int32_t n_pops, uint64_t seed, uint64_t sweep,
    unsigned long long* stats, int Kreal, uint32_t* status) {
    grid_dep_wait();  // the sweep's moves are visible from here on
    grid_dep_launch();
    __shared__ uint32_t s_sw, s_try;
    if (threadIdx.x == 0) { s_sw = 0; s_try = 0; }
    __syncthreads();
    uint32_t sw = 0, tries = 0;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Mtot; c += G) {
        const int q = pop_of(offsets, n_pops, c);
        const int64_t base = __ldg(offsets + q);
        const int Mq = (int)((int64_t)__ldg(offsets + q + 1) - base);
        const int r = (int)(c - base);
        if (Mq < 2) continue;
        const uint32_t par = draw(seed, RNG_EXCHANGE, sweep, (uint32_t)q, 0u).x & 1u;
        int j = -1;
        if (r + 1 < Mq && (uint32_t)(r & 1) == par) j = r >> 1;  // (2j, 2j+1) or (2j+1, 2j+2)
        else if (par == 1u && r == Mq - 1 && (Mq & 1) == 0) j = (Mq - 1) / 2;  // (Mq-1, 0)
        if (j < 0) continue;
        ++tries;
        sw += exchange_pair<K>(theta, ll, Mtot, beta, base, Mq, par, q, j, Kreal, seed, sweep,
                               status);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xFFFFFFFFu, sw, o);
        tries += __shfl_xor_sync(0xFFFFFFFFu, tries, o);
    }
    if ((threadIdx.x & 31) == 0 && (sw | tries)) {
        atomicAdd(&s_sw, sw);
        atomicAdd(&s_try, tries);
    }
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        if (s_sw) atomicAdd(stats + 1, (unsigned long long)s_sw);
        if (s_try) atomicAdd(stats + 2, (unsigned long long)s_try);
    }
}

}  // namespace smc

// bytes of the binned layout buffer at the largest binned data set (the
// context allocates it once, so sweeps captured in a graph can use it)
size_t smc_binned_cache_bytes() {
    return smc::bcache_bytes(smc::kBinnedMaxN, smc::binned_yb_len(smc::kBinnedMaxN));
}

namespace smc_host {

smc_status gmm1d_prepare(const smc_gmm* model, int64_t N, smc::Gmm1dArgs* P, int* Kpad,
                         bool* eqw);

template <int K, bool MALA, bool EQW>
static smc_status launch_move(int blocks, int threads, cudaStream_t s, const float* y, int64_t N,
                              const float* th, const double* l, const float* g, const int32_t* anc,
                              const int32_t* flag, float* tho, double* lo, float* go, int64_t M,
                              const float* beta, int64_t bs, float scale, uint64_t seed,
                              uint64_t step, uint32_t* acc, const smc::Gmm1dArgs& P, int L, int Kr,
                              uint32_t* st) {
    const int yc = smc::ychunk_for(N);
    return launch_pdl(smc::k_mh_move<K, MALA, EQW>, dim3(blocks), dim3(threads),
                      smc::ysmem_bytes(yc), s, y, N, th, l, g, anc, flag, tho, lo, go, M, beta, bs,
                      scale, seed, step, acc, P, L, Kr, yc, st);
}

template <int K>
static smc_status dispatch_move(bool mala, bool eqw, int blocks, int threads, cudaStream_t s,
                                const float* y, int64_t N, const float* th, const double* l,
                                const float* g, const int32_t* anc, const int32_t* flag,
                                float* tho, double* lo, float* go, int64_t M, const float* beta,
                                int64_t bs, float scale, uint64_t seed, uint64_t step,
                                uint32_t* acc, const smc::Gmm1dArgs& P, int L, int Kr,
                                uint32_t* st) {
#define SMC_MV(MA, EQ) \
    launch_move<K, MA, EQ>(blocks, threads, s, y, N, th, l, g, anc, flag, tho, lo, go, M, beta, bs, \
                           scale, seed, step, acc, P, L, Kr, st)
    if (mala) return eqw ? SMC_MV(true, true) : SMC_MV(true, false);
    return eqw ? SMC_MV(false, true) : SMC_MV(false, false);
#undef SMC_MV
}

// Programmatic dependent launch of consecutive sweeps (compile-time knob).
#ifndef SMC_POP_PDL
#define SMC_POP_PDL 1
#endif

// The binned layout of y for the sweep: rebuilt (one small launch, captured
// like any other when the stream is capturing) when the data pointer, N, the
// bin width or c differ from the context's last ones; null (the sweep
// partitions the data itself) without a buffer.  Data changed in place
// under the same pointer are caught by the sweep's own check.
static const char* binned_cache(smc_ctx* ctx, const float* y, int64_t N,
                                const smc::Gmm1dArgs& P, cudaStream_t s) {
    if (!ctx->d_bcache || ctx->bcache_bytes < smc::bcache_bytes(N, smc::binned_yb_len(N)))
        return nullptr;
    uint32_t bw, cf;
    std::memcpy(&bw, &P.binw, 4);
    std::memcpy(&cf, &P.cf, 4);
    if (ctx->bkey_y != y || ctx->bkey_n != N || ctx->bkey_binw != bw || ctx->bkey_cf != cf) {
        ctx->bkey_y = nullptr;
        smc::k_bin_prepare<<<1, smc::kBinThreads, smc::bin_prepare_smem_bytes(N), s>>>(
            y, N, P.binw, P.binw_inv, P.cf, ctx->d_bcache);
        if (cudaGetLastError() != cudaSuccess) return nullptr;
        ctx->bkey_y = y;
        ctx->bkey_n = N;
        ctx->bkey_binw = bw;
        ctx->bkey_cf = cf;
    }
    return ctx->d_bcache;
}

// The binned sweep (data held whole in shared memory): one 512-thread CTA
// per SM, each with an equal share of the work.
template <int K>
static smc_status launch_pop_binned(smc_ctx* ctx, cudaStream_t s, const float* y,
                                    int64_t N, float* th, double* l, int64_t Mt, const float* beta,
                                    const int32_t* off, int32_t n_pops, float scale, uint64_t seed,
                                    uint64_t sweep, uint64_t* stats, const smc::Gmm1dArgs& P,
                                    int Kr, bool inline_ex) {
    auto kern = smc::k_popmcmc_binned<K>;
    const int threads = smc::kBinThreads;
    const size_t smem = smc::binned_smem_bytes(N, K, n_pops);
    SMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // at most one CTA per chain group of 32 (so a group meets at most two CTAs)
    const int64_t groups = (Mt + 31) / 32;
    smc_status st0 = ensure_groups(ctx, groups, s);
    if (st0 != SMC_OK) return st0;
    int64_t grid = ctx->num_sms;
    if (grid > groups) grid = groups;
    const char* bc = binned_cache(ctx, y, N, P, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = SMC_POP_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    smc_status st = cuda_ok(cudaLaunchKernelEx(
        &cfg, kern, y, N, th, l, Mt, beta, off, n_pops, scale, seed, sweep,
        reinterpret_cast<unsigned long long*>(stats), ctx->d_popdone, ctx->d_grpdone,
        reinterpret_cast<long long*>(ctx->d_grppart), P, Kr, inline_ex ? 1 : 0, bc,
        ctx->d_status));
    if (st != SMC_OK || inline_ex) return st;
    int64_t xb = (Mt + 255) / 256;
    if (xb > (int64_t)ctx->num_sms * 8) xb = (int64_t)ctx->num_sms * 8;
    return launch_pdl(smc::k_popmcmc_exchange<K>, dim3((unsigned)xb), dim3(256), 0, s, th, l, Mt,
                      beta, off, n_pops, seed, sweep, reinterpret_cast<unsigned long long*>(stats),
                      Kr, ctx->d_status);
}

template <int K, bool EQW>
static smc_status launch_pop(smc_ctx* ctx, int threads, cudaStream_t s, const float* y,
                             int64_t N, float* th, double* l, int64_t Mt, const float* beta,
                             const int32_t* off, int32_t n_pops, float scale, uint64_t seed,
                             uint64_t sweep, uint64_t* stats, const smc::Gmm1dArgs& P, int L,
                             int Kr, bool inline_ex) {
    if constexpr (K <= 16) {
        if (N >= smc::kBinnedMinN && N <= smc::kBinnedMaxN)
            return launch_pop_binned<K>(ctx, s, y, N, th, l, Mt, beta, off, n_pops, scale, seed,
                                        sweep, stats, P, Kr, inline_ex);
    }
    auto kern = smc::k_popmcmc_sweep<K, EQW>;
    const int yc = smc::ychunk_for(N);
    size_t smem = smc::ysmem_bytes(yc) + 2 * (size_t)(threads / L + 1) * sizeof(int4);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const int ppb = threads / L;
    const int64_t items = (Mt + ppb - 1) / ppb;
    // Items fewer than the resident slots: hold every SM to k = ceil(items /
    // SMs) blocks (by asking for more shared memory), so that no SM runs more
    // than k items whatever order the blocks are placed in.
    const int64_t k = (items + ctx->num_sms - 1) / ctx->num_sms;
    if (k < occ && ctx->smem_per_sm > 0) {
        const size_t pad = (size_t)(ctx->smem_per_sm / (k + 1) - ctx->smem_reserved + 1024) &
                           ~(size_t)1023;
        if (pad > smem) {
            int occ2 = 0;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pad) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, kern, threads, pad) ==
                    cudaSuccess &&
                occ2 == k) {
                smem = pad;
                occ = occ2;
            }
        }
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t grid = (int64_t)ctx->num_sms * occ;
    if (grid > items) grid = items;
    // programmatic serialisation: a sweep following a sweep on this stream
    // runs its prologue while the previous one drains (the kernel waits for
    // it before touching chain state)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = SMC_POP_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    smc_status st = cuda_ok(cudaLaunchKernelEx(
        &cfg, kern, y, N, th, l, Mt, beta, off, n_pops, scale, seed, sweep,
        reinterpret_cast<unsigned long long*>(stats), ctx->d_popdone, P, L, Kr, yc,
        inline_ex ? 1 : 0, ctx->d_status));
    if (st != SMC_OK || inline_ex) return st;
    int64_t xb = (Mt + 255) / 256;
    if (xb > (int64_t)ctx->num_sms * 8) xb = (int64_t)ctx->num_sms * 8;
    return launch_pdl(smc::k_popmcmc_exchange<K>, dim3((unsigned)xb), dim3(256), 0, s, th, l, Mt,
                      beta, off, n_pops, seed, sweep, reinterpret_cast<unsigned long long*>(stats),
                      Kr, ctx->d_status);
}

}  // namespace smc_host

extern "C" smc_status smc_mh_move(smc_ctx* ctx, const smc_gmm* model, const float* y, int64_t N,
                                  const float* theta_in, const double* loglik_in,
                                  const float* grad_in, const int32_t* anc,
                                  const int32_t* do_flag, float* theta_out, double* loglik_out,
                                  float* grad_out, int64_t M, const float* beta,
                                  int64_t beta_stride, float scale, int32_t kind, uint64_t seed,
                                  uint64_t step, uint32_t* accept_count, void* stream) {
    if (!ctx || M < 0 || N < 0 || (kind != SMC_MOVE_RW && kind != SMC_MOVE_MALA)) return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    if (!theta_in || !loglik_in || !theta_out || !loglik_out || !beta || (N > 0 && !y) ||
        beta_stride < 0 || !(scale >= 0.0f) || !std::isfinite(scale))
        return SMC_ERR_ARG;
    if (kind == SMC_MOVE_MALA && (!grad_in || !grad_out)) return SMC_ERR_ARG;
    if (anc && (theta_in == theta_out || loglik_in == loglik_out ||
                (kind == SMC_MOVE_MALA && grad_in == grad_out)))
        return SMC_ERR_ARG;
    smc::Gmm1dArgs P;
    int Kp;
    bool eqw;
    smc_status st = gmm1d_prepare(model, N, &P, &Kp, &eqw);
    if (st != SMC_OK) return st;
    P.wait_limit = ctx->wait_limit;
    st = use_device(ctx);
    if (st != SMC_OK) return st;
    int L, threads;
    launch_shape(ctx, SMC_OP_MOVE, M, N, model->K, &L, &threads);
    int ppb = threads / L;
    int64_t blocks = (M + ppb - 1) / ppb;
    if (blocks > 0x7FFFFFFF) return SMC_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    bool mala = kind == SMC_MOVE_MALA;
    const int Kr = model->K;
#define SMC_DM(KK)                                                                              \
    dispatch_move<KK>(mala, eqw, (int)blocks, threads, s, y, N, theta_in, loglik_in, grad_in,  \
                      anc, do_flag, theta_out, loglik_out, grad_out, M, beta, beta_stride,     \
                      scale, seed, step, accept_count, P, L, Kr, ctx->d_status)
    switch (Kp) {
        case 1: return SMC_DM(1);
        case 2: return SMC_DM(2);
        case 4: return SMC_DM(4);
        case 8: return SMC_DM(8);
        case 16: return SMC_DM(16);
        case 32: return SMC_DM(32);
        default: return SMC_ERR_UNSUPPORTED;
    }
#undef SMC_DM
}

extern "C" smc_status smc_popmcmc_sweep(smc_ctx* ctx, const smc_gmm* model, const float* y,
                                        int64_t N, float* theta, double* loglik, int64_t M_total,
                                        const float* beta, const int32_t* pop_offsets,
                                        int32_t n_pops, float scale,
                                        uint64_t seed, uint64_t sweep, uint64_t* stats,
                                        void* stream) {
    if (!ctx || M_total < 0 || N < 0 || n_pops < 0) return SMC_ERR_ARG;
    if (n_pops == 0 || M_total == 0) return SMC_OK;
    if (!theta || !loglik || !beta || !pop_offsets || (N > 0 && !y) || !(scale >= 0.0f) ||
        !std::isfinite(scale) || M_total > 0x7FFFFFFF)
        return SMC_ERR_ARG;
    smc::Gmm1dArgs P;
    int Kp;
    bool eqw;
    smc_status st = gmm1d_prepare(model, N, &P, &Kp, &eqw);
    if (st != SMC_OK) return st;
    P.wait_limit = ctx->wait_limit;
    st = use_device(ctx);
    if (st != SMC_OK) return st;
    int L, threads;
    launch_shape(ctx, SMC_OP_POPMCMC, M_total, N, model->K, &L, &threads);
    cudaStream_t s = as_stream(stream);
    // Exchanges run inside the sweep (by the CTA that completes a
    // population) while the average population has at most two pairs per
    // thread of a CTA; larger populations take a second, grid-wide launch.
    const bool inline_ex = M_total <= (int64_t)n_pops * 2 * threads;
    if (inline_ex) {
        st = ensure_popdone(ctx, n_pops, s);
        if (st != SMC_OK) return st;
    }
    const int Kr = model->K;
#define SMC_PP(KK, EQ)                                                                       \
    launch_pop<KK, EQ>(ctx, threads, s, y, N, theta, loglik, M_total, beta, pop_offsets,      \
                       n_pops, scale, seed, sweep, stats, P, L, Kr, inline_ex)
    switch (Kp) {
        case 1: return eqw ? SMC_PP(1, true) : SMC_PP(1, false);
        case 2: return eqw ? SMC_PP(2, true) : SMC_PP(2, false);
        case 4: return eqw ? SMC_PP(4, true) : SMC_PP(4, false);
        case 8: return eqw ? SMC_PP(8, true) : SMC_PP(8, false);
        case 16: return eqw ? SMC_PP(16, true) : SMC_PP(16, false);
        case 32: return eqw ? SMC_PP(32, true) : SMC_PP(32, false);
        default: return SMC_ERR_UNSUPPORTED;
    }
#undef SMC_PP
}
