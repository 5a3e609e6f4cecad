// resample.cu -- smc_resample_systematic and smc_gather.
//
// Systematic resampling (Section 3.2: build the empirical CDF of the
// weights, then draw M times from it; Section 4.2 credits the parallel scan
// for the speed of this step) in exact integers:
//   q_j = floor(W_j 2^52)            (integer operations on the FP64 bits)
//   C_j = q_0 + ... + q_j,  S = C_{M-1}
//   F(c) = #{ i in [0,M) : (i 2^32 + u32) S < c M 2^32 }
//   particle j fills output slots [F(C_{j-1}), F(C_j)).
// Pass 1 sums q exactly (integer atomics, order-free) and clears the tile
// descriptors.  Pass 2 is a single-pass scan over tiles of 2048 weights:
// block scan, then decoupled look-back over the predecessors' published
// aggregates / inclusive prefixes (bounded wait), then F at every prefix by
// an estimate and an exact 128-bit fix-up, and a balanced expansion of the
// tile's contiguous output range through shared memory.
#include "ctx.hpp"
#include "device.cuh"
#include "resample.cuh"

using namespace smc_host;

size_t smc_resample_ws_bytes(int64_t M) {
    int64_t tiles = (M + smc::kRsTile - 1) / smc::kRsTile;
    return (size_t)(tiles + 1) * sizeof(unsigned long long) + 256;
}

namespace smc {

__global__ void __launch_bounds__(256) k_gather(const int32_t* __restrict__ anc, int64_t M,
                                                int rows, const float* __restrict__ src,
                                                float* __restrict__ dst,
                                                const double* __restrict__ src64,
                                                double* __restrict__ dst64) {
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        int64_t a = anc ? (int64_t)anc[i] : i;
        for (int r = 0; r < rows; ++r) dst[(int64_t)r * M + i] = src[(int64_t)r * M + a];
        if (src64 && dst64) dst64[i] = src64[a];
    }
}

}  // namespace smc

namespace smc_host {

smc_status resample_launch(int num_sms, const double* W, int64_t M, uint64_t seed, uint64_t step,
                           int32_t* anc, int32_t* counts, const int32_t* do_flag, double* lwreset,
                           const smc::RsScratch& sc, uint32_t* status, cudaStream_t s) {
    int64_t tiles = (M + smc::kRsTile - 1) / smc::kRsTile;
    if (tiles > 0x7FFFFFFF) return SMC_ERR_ARG;
    int64_t b1 = (M + 256 * 8 - 1) / (256 * 8);
    if (b1 > (int64_t)num_sms * 8) b1 = (int64_t)num_sms * 8;
    if (b1 < 1) b1 = 1;
    smc::k_resample_total<<<(unsigned)b1, 256, 0, s>>>(W, M, do_flag, sc, tiles, status);
    SMC_CUDA(cudaGetLastError());
    smc::k_resample_scan<<<(unsigned)tiles, smc::kRsThreads, 0, s>>>(
        W, M, seed, step, do_flag, sc, (uint32_t)tiles, anc, counts, lwreset, status);
    return cuda_ok(cudaGetLastError());
}

}  // namespace smc_host

extern "C" smc_status smc_resample_systematic(smc_ctx* ctx, const double* W, int64_t M,
                                              uint64_t seed, uint64_t step,
                                              int32_t* ancestors_out, int32_t* counts_out,
                                              const int32_t* do_flag, double* logw_reset,
                                              void* stream) {
    if (!ctx || M < 0 || M > 0x7FFFFFFF) return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    if (!W || !ancestors_out) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    st = ensure_ws(ctx, smc_resample_ws_bytes(M), s);
    if (st != SMC_OK) return st;
    smc::RsScratch sc;
    sc.tiles = reinterpret_cast<unsigned long long*>(ctx->ws);
    sc.ticket = ctx->d_counters + CNT_RESAMPLE_TILE;
    sc.sum = ctx->d_counters + CNT_RESAMPLE_SUM;
    sc.done = ctx->d_counters + CNT_RESAMPLE_DONE;
    return resample_launch(ctx->num_sms, W, M, seed, step, ancestors_out, counts_out, do_flag,
                           logw_reset, sc, ctx->d_status, s);
}

extern "C" smc_status smc_gather(smc_ctx* ctx, const int32_t* anc, int64_t M, int32_t rows_f32,
                                 const float* src_f32, float* dst_f32, const double* src_f64,
                                 double* dst_f64, void* stream) {
    if (!ctx || M < 0 || rows_f32 < 0) return SMC_ERR_ARG;
    if (rows_f32 > 0 && (!src_f32 || !dst_f32)) return SMC_ERR_ARG;
    if ((src_f64 == nullptr) != (dst_f64 == nullptr)) return SMC_ERR_ARG;
    if (M == 0) return SMC_OK;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    int64_t b = (M + 255) / 256;
    if (b > (int64_t)ctx->num_sms * 16) b = (int64_t)ctx->num_sms * 16;
    smc::k_gather<<<(unsigned)b, 256, 0, as_stream(stream)>>>(anc, M, rows_f32, src_f32, dst_f32,
                                                              src_f64, dst_f64);
    return cuda_ok(cudaGetLastError());
}

// ------------------------------------------------------------------ no-allocation variant
// Systematic resampling for callers that must not allocate device memory:
// processes whose device memory is all reserved up front by an allocator
// they do not own (a framework's caching pool, a serving runtime with a
// fixed memory budget), and latency-critical loops that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree.  No context is
// created: the scan's scratch (tile descriptors and three counters) lives in
// a file-scope device array that every GPU loading this library holds until
// the process exits.
#include <mutex>

namespace {

constexpr int64_t kNoAllocMaxM = (int64_t)1 << 24;                  // 16,777,216 weights
constexpr int64_t kNoAllocTiles = kNoAllocMaxM / smc::kRsTile;      // 8192 tiles
constexpr int64_t kNoAllocWords = kNoAllocTiles + 8;                // + ticket, sum, done
// 64 KiB + 64 B of scratch per device
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[256] = {};  // device address of the array, per device

// Device address of the scratch array for the current device.  The first
// call on a device looks it up (cudaGetSymbolAddress); host code must not
// use the array's name as a device pointer.
smc_status noalloc_scratch(unsigned long long** out) {
    int dev = -1;
    SMC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return SMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return SMC_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SMC_OK;
}

}  // namespace

extern "C" smc_status smc_resample_systematic_noalloc(const double* W, int64_t M, uint64_t seed,
                                                      uint64_t step, int32_t* ancestors_out,
                                                      int32_t* counts_out, const int32_t* do_flag,
                                                      double* logw_reset, uint32_t* status_out,
                                                      void* stream) {
    if (M < 0) return SMC_ERR_ARG;
    if (M > kNoAllocMaxM) return SMC_ERR_ARG;  // larger than the static scratch
    if (M == 0) return SMC_OK;
    if (!W || !ancestors_out) return SMC_ERR_ARG;
    unsigned long long* scratch = nullptr;
    smc_status st = noalloc_scratch(&scratch);
    if (st != SMC_OK) return st;
    int dev = 0, sms = 0;
    SMC_CUDA(cudaGetDevice(&dev));
    SMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = as_stream(stream);
    smc::RsScratch sc;
    sc.tiles = scratch;
    sc.ticket = scratch + kNoAllocTiles;
    sc.sum = scratch + kNoAllocTiles + 1;
    sc.done = scratch + kNoAllocTiles + 2;
    // the counters must start at zero; an earlier call that stopped on an
    // error may have left them set (the tile words are cleared by pass 1)
    SMC_CUDA(cudaMemsetAsync(sc.ticket, 0, 3 * sizeof(unsigned long long), s));
    return resample_launch(sms, W, M, seed, step, ancestors_out, counts_out, do_flag, logw_reset,
                           sc, status_out, s);
}
