// mrg.cu -- smc_rng_mrg32k3a: the combined multiple recursive generator
// MRG32k3a (L'Ecuyer 1999), parallelised as Section 2.5 describes: every
// thread computes a contiguous block of one overall stream, reaching the
// block's start by skip-ahead in O(log n) matrix-vector products.
//
// Component 1: x_n = (1403580 x_{n-2} - 810728 x_{n-3}) mod m1, m1 = 2^32 - 209
// Component 2: y_n = (527612 y_{n-1} - 1370589 y_{n-3}) mod m2, m2 = 2^32 - 22853
// Output:      z_n = (x_n - y_n) mod m1, taken in [1, m1] (m1 in place of 0);
//              FP64: u_n = z_n / (m1 + 1) (the generator's definition);
//              FP32: u_n = (2 floor(z_n / 2^9) + 1) / 2^24, the same number
//              cut to the 24 bits a float holds, strictly inside (0, 1) and
//              formed from bits (no conversion instruction).
// State (s0, s1, s2 | s3, s4, s5): the last three values of each component,
// oldest first; one step maps (s0, s1, s2) to (s1, s2, new).  As a matrix
// A1 = [0 1 0; 0 0 1; -810728 1403580 0] (mod m1) and
// A2 = [0 1 0; 0 0 1; -1370589 0 527612] (mod m2); n steps multiply the
// state by A^n, formed from the context's table of A^(2^k), k < 64.
#include "ctx.hpp"
#include "device.cuh"

using namespace smc_host;

namespace smc {

constexpr unsigned long long kM1 = 4294967087ull, kM2 = 4294944443ull;
constexpr long long kA12 = 1403580, kA13n = 810728, kA21 = 527612, kA23n = 1370589;
constexpr double kNorm = 2.328306549295727688e-10;  // 1 / (m1 + 1)

// A x mod m for a 3x3 matrix of residues (row-major) and a state of residues
template <unsigned long long MOD>
__device__ __forceinline__ void matvec_mod(const uint32_t* __restrict__ A, uint32_t (&v)[3]) {
    uint32_t r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        unsigned long long acc = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc += (unsigned long long)__ldg(A + 3 * i + k) * v[k] % MOD;  // < 2^32 each
        }
        r[i] = (uint32_t)(acc % MOD);
    }
    v[0] = r[0];
    v[1] = r[1];
    v[2] = r[2];
}

template <bool F32, bool F64>
__global__ void __launch_bounds__(256) k_mrg32k3a(const uint32_t* __restrict__ pow_tab,
                                                  uint4 seed_lo, uint2 seed_hi,
                                                  unsigned long long offset, int64_t n_threads,
                                                  int64_t per_thread, float* __restrict__ out,
                                                  double* __restrict__ out64) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_threads) return;
    uint32_t x[3] = {seed_lo.x, seed_lo.y, seed_lo.z};
    uint32_t y[3] = {seed_lo.w, seed_hi.x, seed_hi.y};
    // skip to offset + t * per_thread (mod 2^64)
    const unsigned long long pos = offset + (unsigned long long)t * (unsigned long long)per_thread;
    for (int b = 0; b < 64; ++b) {
        if ((pos >> b) & 1ull) {
            matvec_mod<kM1>(pow_tab + b * 18, x);
            matvec_mod<kM2>(pow_tab + b * 18 + 9, y);
        }
    }
    long long s0 = x[0], s1 = x[1], s2 = x[2], s3 = y[0], s4 = y[1], s5 = y[2];
    for (int64_t j = 0; j < per_thread; ++j) {
        long long p1 = (kA12 * s1 - kA13n * s0) % (long long)kM1;
        if (p1 < 0) p1 += (long long)kM1;
        s0 = s1;
        s1 = s2;
        s2 = p1;
        long long p2 = (kA21 * s5 - kA23n * s3) % (long long)kM2;
        if (p2 < 0) p2 += (long long)kM2;
        s3 = s4;
        s4 = s5;
        s5 = p2;
        const long long z = p1 > p2 ? p1 - p2 : p1 - p2 + (long long)kM1;
        if (F32) out[j * n_threads + t] = u01((uint32_t)z);  // (2 (z >> 9) + 1) / 2^24
        if (F64) out64[j * n_threads + t] = (double)z * kNorm;
    }
}

}  // namespace smc

namespace smc_host {

// A1^(2^k), A2^(2^k) for k < 64, row-major, [k][component][9]
void mrg_power_table(uint32_t* tab) {
    const unsigned long long m[2] = {smc::kM1, smc::kM2};
    unsigned long long A[2][9] = {
        {0, 1, 0, 0, 0, 1, smc::kM1 - (unsigned long long)smc::kA13n,
         (unsigned long long)smc::kA12, 0},
        {0, 1, 0, 0, 0, 1, smc::kM2 - (unsigned long long)smc::kA23n, 0,
         (unsigned long long)smc::kA21}};
    for (int k = 0; k < 64; ++k) {
        for (int c = 0; c < 2; ++c) {
            for (int i = 0; i < 9; ++i) tab[k * 18 + c * 9 + i] = (uint32_t)A[c][i];
            unsigned long long sq[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    unsigned long long acc = 0;
                    for (int l = 0; l < 3; ++l) acc = (acc + A[c][3 * i + l] * A[c][3 * l + j] % m[c]) % m[c];
                    sq[3 * i + j] = acc;
                }
            for (int i = 0; i < 9; ++i) A[c][i] = sq[i];
        }
    }
}

}  // namespace smc_host

extern "C" smc_status smc_rng_mrg32k3a(smc_ctx* ctx, const uint32_t seed[6], uint64_t offset,
                                       int64_t n_threads, int64_t per_thread, float* out_f32,
                                       double* out_f64, void* stream) {
    if (!ctx || !seed || n_threads < 0 || per_thread < 0) return SMC_ERR_ARG;
    if (n_threads == 0 || per_thread == 0) return SMC_OK;
    if ((!out_f32 && !out_f64) || !ctx->d_mrg_pow) return SMC_ERR_ARG;
    // seeds as in the generator's definition: x-part below m1, y-part below
    // m2, neither part all zero
    if (seed[0] >= smc::kM1 || seed[1] >= smc::kM1 || seed[2] >= smc::kM1 || seed[3] >= smc::kM2 ||
        seed[4] >= smc::kM2 || seed[5] >= smc::kM2 || (seed[0] | seed[1] | seed[2]) == 0 ||
        (seed[3] | seed[4] | seed[5]) == 0)
        return SMC_ERR_ARG;
    if (n_threads > 0x7FFFFFFFLL * 256) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    const int64_t blocks = (n_threads + 255) / 256;
    auto kern = !out_f64 ? smc::k_mrg32k3a<true, false>
                : !out_f32 ? smc::k_mrg32k3a<false, true> : smc::k_mrg32k3a<true, true>;
    return launch_pdl(kern, dim3((unsigned)blocks), dim3(256), 0, as_stream(stream),
                      (const uint32_t*)ctx->d_mrg_pow, make_uint4(seed[0], seed[1], seed[2], seed[3]),
                      make_uint2(seed[4], seed[5]), (unsigned long long)offset, n_threads,
                      per_thread, out_f32, out_f64);
}
