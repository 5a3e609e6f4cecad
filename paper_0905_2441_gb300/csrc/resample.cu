// resample.cu -- smc_resample_systematic and smc_gather.
//
// Systematic resampling (Section 3.2: build the empirical CDF of the
// weights, then draw M times from it; Section 4.2 credits the parallel scan
// for the speed of this step) in exact integers:
//   q_j = floor(W_j 2^52)            (integer operations on the FP64 bits)
//   C_j = q_0 + ... + q_j,  S = C_{M-1}
//   F(c) = #{ i in [0,M) : (i 2^32 + u32) S < c M 2^32 }
//   particle j fills output slots [F(C_{j-1}), F(C_j)).
// Pass 1 sums q exactly per tile of 2048 weights.  One CTA then turns the
// tile sums into exclusive prefixes and forms the call's constants (S, the
// draw u, fixed-point reciprocals of S).  Pass 2 is persistent: per tile a
// block scan, F at every prefix by a fixed-point quotient and an exact
// 128-bit fix-up, and a balanced expansion of the tile's contiguous output
// range through shared memory.  The kernels are chained by programmatic
// dependent launch, so each one's launch overlaps the previous one's tail.
#include "ctx.hpp"
#include "device.cuh"
#include "bounds.cuh"
#include "resample.cuh"

using namespace smc_host;

// scratch of the context entry point: tile sums, constants, the heavy-chunk
// counter and records, and the inclusive F of heavy tiles' items
size_t smc_resample_ws_bytes(int64_t M) {
    return (size_t)(smc::rs_words(M) + 1) * sizeof(unsigned long long) +
           (size_t)smc::rs_heavy_records(M) * sizeof(uint4) + (size_t)M * sizeof(uint32_t) + 512;
}

namespace smc {

__global__ void __launch_bounds__(256) k_gather(const int32_t* __restrict__ anc, int64_t M,
                                                int rows, const float* __restrict__ src,
                                                float* __restrict__ dst,
                                                const double* __restrict__ src64,
                                                double* __restrict__ dst64, uint32_t* status) {
    grid_dep_wait();  // the previous kernel's writes are visible from here on
    grid_dep_launch();
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G) {
        int64_t a = anc ? (int64_t)anc[i] : i;
        if (!SMC_IN_BOUNDS(a >= 0 && a < M, status)) a = i;
        for (int r = 0; r < rows; ++r) dst[(int64_t)r * M + i] = src[(int64_t)r * M + a];
        if (src64 && dst64) dst64[i] = src64[a];
    }
}

}  // namespace smc

namespace smc_host {

// The finalize kernel (one CTA of kRsFinThreads).
smc_status resample_finalize_launch(int64_t M, uint64_t seed, uint64_t step,
                                    const int32_t* do_flag, const smc::RsScratch& sc,
                                    uint32_t* status, cudaStream_t s) {
    return launch_pdl(smc::k_resample_finalize, dim3(1), dim3(smc::kRsFinThreads), 0, s, M, seed,
                      step, do_flag, sc, status);
}

// tiles_ready: the tile sums of pass 1 are already in sc (formed by the
// normalisation pass of smc_reweight_resample, which writes the weights in
// descending tile order, as pass 1 reads them), so pass 1 is skipped
smc_status resample_launch(int num_sms, const double* W, int64_t M, uint64_t seed, uint64_t step,
                           int32_t* anc, int32_t* counts, const int32_t* do_flag, double* lwreset,
                           const smc::RsScratch& sc, uint32_t* status, cudaStream_t s,
                           bool tiles_ready) {
    const int64_t tiles = smc::rs_tiles(M);
    if (tiles > 0x7FFFFFFF) return SMC_ERR_ARG;
    int64_t b1 = tiles;
    if (b1 > (int64_t)num_sms * 4) b1 = (int64_t)num_sms * 4;
    smc_status st = SMC_OK;
    if (!tiles_ready) {
        st = launch_pdl(smc::k_resample_total, dim3((unsigned)b1), dim3(smc::kRsThreads), 0, s, W,
                        M, do_flag, sc, status);
        if (st != SMC_OK) return st;
    }
    st = resample_finalize_launch(M, seed, step, do_flag, sc, status, s);
    if (st != SMC_OK) return st;
    // pass 2 is persistent: as many CTAs as are resident at once (per device)
    static int occ_of_dev[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int occ = occ_of_dev[dev];
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, smc::k_resample_scan,
                                                          smc::kRsThreads, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        occ_of_dev[dev] = occ;
    }
    int64_t g2 = (int64_t)num_sms * occ;
    if (g2 > tiles) g2 = tiles;
    st = launch_pdl(smc::k_resample_scan, dim3((unsigned)g2), dim3(smc::kRsThreads), 0, s, W, M,
                    do_flag, sc, anc, counts, lwreset, status);
    if (st != SMC_OK) return st;
    if (sc.heavy_list) {
        st = launch_pdl(smc::k_resample_heavy, dim3((unsigned)num_sms * 4), dim3(smc::kRsThreads),
                        0, s, do_flag, sc, M, anc, status);
        if (st != SMC_OK) return st;
    }
    return SMC_OK;
}

// scratch layout inside `base`: tile sums, the call constants, then (when
// `heavy`) the heavy-chunk counter, the chunk records and the items'
// inclusive F
smc::RsScratch resample_scratch(unsigned long long* base, int64_t M, bool heavy) {
    smc::RsScratch sc;
    sc.tile_sum = base;
    sc.cst = reinterpret_cast<smc::RsConst*>(base + smc::rs_tiles(M));
    sc.heavy_count = nullptr;
    sc.heavy_list = nullptr;
    sc.fpos = nullptr;
    if (heavy) {
        sc.heavy_count = base + smc::rs_words(M);
        uintptr_t p = reinterpret_cast<uintptr_t>(sc.heavy_count + 1);
        p = (p + 255) & ~(uintptr_t)255;
        sc.heavy_list = reinterpret_cast<uint4*>(p);
        sc.fpos = reinterpret_cast<uint32_t*>(sc.heavy_list + smc::rs_heavy_records(M));
    }
    return sc;
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
    const smc::RsScratch sc =
        resample_scratch(reinterpret_cast<unsigned long long*>(ctx->ws), M, true);
    return resample_launch(ctx->num_sms, W, M, seed, step, ancestors_out, counts_out, do_flag,
                           logw_reset, sc, ctx->d_status, s, false);
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
    return launch_pdl(smc::k_gather, dim3((unsigned)b), dim3(256), 0, as_stream(stream), anc, M,
                      rows_f32, src_f32, dst_f32, src_f64, dst_f64, ctx->d_status);
}

// ------------------------------------------------------------------ no-allocation variant
// Systematic resampling for callers that must not allocate device memory:
// processes whose device memory is all reserved up front by an allocator
// they do not own (a framework's caching pool, a serving runtime with a
// fixed memory budget), and latency-critical loops that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree.  No context is
// created: the scan's scratch (tile sums and constants) lives in a
// file-scope device array that every GPU loading this library holds until
// the process exits.
#include <mutex>

namespace {

constexpr int64_t kNoAllocMaxM = (int64_t)1 << 24;   // 16,777,216 weights
// 8192 tile sums + the call constants: about 64 KiB per device
constexpr int64_t kNoAllocWords = smc::rs_words(kNoAllocMaxM);
static_assert(sizeof(smc::RsConst) <= smc::kRsConstWords * sizeof(unsigned long long),
              "constants fit their words");
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
    // pass 1 overwrites every tile sum it uses; the constants are formed
    // anew by each call
    // no heavy-chunk scratch: a tile with many slots is expanded by its CTA
    const smc::RsScratch sc = resample_scratch(scratch, M, false);
    return resample_launch(sms, W, M, seed, step, ancestors_out, counts_out, do_flag, logw_reset,
                           sc, status_out, s, false);
}
