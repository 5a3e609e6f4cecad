// ctx.cu -- context life cycle, status reporting, launch shapes and the
// raw random-stream entry points of the C ABI.
#include <cstdio>
#include <cstring>
#include <new>

#include "ctx.hpp"
#include "device.cuh"
#include "bounds.cuh"

using namespace smc_host;

namespace smc_host {

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

smc_status use_device(smc_ctx* ctx) {
    int cur = -1;
    SMC_CUDA(cudaGetDevice(&cur));
    if (cur != ctx->device) SMC_CUDA(cudaSetDevice(ctx->device));
    return SMC_OK;
}

smc_status ensure_ws(smc_ctx* ctx, size_t bytes, cudaStream_t s) {
    if (bytes <= ctx->ws_bytes) return SMC_OK;
    if (capturing(s)) return SMC_ERR_ARG;  // reserve before capturing
    size_t nb = bytes + bytes / 4 + 4096;
    SMC_CUDA(cudaStreamSynchronize(s));
    if (ctx->ws) SMC_CUDA(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    SMC_CUDA(cudaMalloc(&ctx->ws, nb));
    SMC_CUDA(cudaMemset(ctx->ws, 0, nb));
    ctx->ws_bytes = nb;
    return SMC_OK;
}

smc_status ensure_popdone(smc_ctx* ctx, int64_t n, cudaStream_t s) {
    if (n <= ctx->popdone_cap) return SMC_OK;
    if (capturing(s)) return SMC_ERR_ARG;
    int64_t cap = n + n / 4 + 64;
    SMC_CUDA(cudaStreamSynchronize(s));
    if (ctx->d_popdone) SMC_CUDA(cudaFree(ctx->d_popdone));
    ctx->d_popdone = nullptr;
    ctx->popdone_cap = 0;
    SMC_CUDA(cudaMalloc(&ctx->d_popdone, (size_t)cap * sizeof(uint32_t)));
    SMC_CUDA(cudaMemset(ctx->d_popdone, 0, (size_t)cap * sizeof(uint32_t)));
    ctx->popdone_cap = cap;
    return SMC_OK;
}

smc_status ensure_groups(smc_ctx* ctx, int64_t n, cudaStream_t s) {
    if (n <= ctx->grp_cap) return SMC_OK;
    if (capturing(s)) return SMC_ERR_ARG;
    int64_t cap = n + n / 4 + 64;
    SMC_CUDA(cudaStreamSynchronize(s));
    if (ctx->d_grpdone) SMC_CUDA(cudaFree(ctx->d_grpdone));
    if (ctx->d_grppart) SMC_CUDA(cudaFree(ctx->d_grppart));
    ctx->d_grpdone = nullptr;
    ctx->d_grppart = nullptr;
    ctx->grp_cap = 0;
    SMC_CUDA(cudaMalloc(&ctx->d_grpdone, (size_t)cap * sizeof(uint32_t)));
    SMC_CUDA(cudaMemset(ctx->d_grpdone, 0, (size_t)cap * sizeof(uint32_t)));
    SMC_CUDA(cudaMalloc(&ctx->d_grppart, (size_t)cap * 64 * sizeof(double)));
    ctx->grp_cap = cap;
    return SMC_OK;
}

void launch_shape(const smc_ctx* ctx, int op, int64_t M, int64_t N, int K, int* lanes,
                  int* threads) {
    if (op >= 0 && op < SMC_OP_COUNT && ctx->lanes[op] > 0) {
        *lanes = ctx->lanes[op];
        *threads = ctx->threads[op] > 0 ? ctx->threads[op] : 256;
        return;
    }
    (void)K;
    if (op == SMC_OP_POPMCMC) {
        // at least two lanes per chain for long data (few items, each long
        // enough to hide the block's fixed latencies); more while the chains
        // do not fill two resident 256-thread blocks per SM, keeping at
        // least 8 pairs of observations per lane
        int L = N >= 128 ? 2 : 1;
        const int64_t slots = (int64_t)ctx->num_sms * 512;
        while (L < 32 && M * L < slots && N / (4 * L) >= 8) L *= 2;
        *lanes = L;
        *threads = 256;
        return;
    }
    // enough resident warps to cover the SMs (about 32 warps each), but
    // keep at least 8 observations per lane
    int64_t target = (int64_t)ctx->num_sms * 1024;
    int L = 1;
    while (L < 32 && M * L < target && N / (2 * L) >= 8) L *= 2;
    *lanes = L;
    *threads = 256;
}

}  // namespace smc_host

// ------------------------------------------------------------------ C ABI

namespace smc_host {
void mrg_power_table(uint32_t* tab);
}

size_t smc_binned_cache_bytes();  // moves.cu

extern "C" smc_status smc_create(smc_ctx** out, int device) {
    if (!out) return SMC_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return SMC_ERR_CUDA;
    smc_ctx* c = new (std::nothrow) smc_ctx();
    if (!c) return SMC_ERR_ARG;
    c->device = device;
    smc_status st = use_device(c);
    if (st != SMC_OK) { delete c; return st; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return SMC_ERR_CUDA; }
    c->num_sms = prop.multiProcessorCount;
    c->max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
    c->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->smem_reserved = (int)prop.reservedSharedMemPerBlock;
    bool ok = cudaMalloc(&c->d_status, sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&c->d_counters, kCounters * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&c->d_partials, (size_t)kMaxPartialBlocks * 8 * sizeof(double)) ==
                  cudaSuccess &&
              cudaMemset(c->d_status, 0, sizeof(uint32_t)) == cudaSuccess &&
              cudaMemset(c->d_counters, 0, kCounters * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&c->d_mrg_pow, 64 * 18 * sizeof(uint32_t)) == cudaSuccess;
    if (ok) {  // the binned sweep's layout buffer, at its largest data set (tens of KB)
        c->bcache_bytes = smc_binned_cache_bytes();
        ok = cudaMalloc(reinterpret_cast<void**>(&c->d_bcache), c->bcache_bytes) == cudaSuccess &&
             cudaMemset(c->d_bcache, 0, c->bcache_bytes) == cudaSuccess;
        if (!ok) c->bcache_bytes = 0;
    }
    if (ok) {
        uint32_t tab[64 * 18];
        mrg_power_table(tab);
        ok = cudaMemcpy(c->d_mrg_pow, tab, sizeof(tab), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        smc_destroy(c);
        return SMC_ERR_CUDA;
    }
    *out = c;
    return SMC_OK;
}

extern "C" smc_status smc_destroy(smc_ctx* ctx) {
    if (!ctx) return SMC_ERR_ARG;
    use_device(ctx);
    cudaDeviceSynchronize();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->d_partials) cudaFree(ctx->d_partials);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_popdone) cudaFree(ctx->d_popdone);
    if (ctx->d_grpdone) cudaFree(ctx->d_grpdone);
    if (ctx->d_grppart) cudaFree(ctx->d_grppart);
    if (ctx->d_bcache) cudaFree(ctx->d_bcache);
    if (ctx->d_mrg_pow) cudaFree(ctx->d_mrg_pow);
    delete ctx;
    return SMC_OK;
}

// bytes of growable workspace the resamplers need for M particles
size_t smc_resample_ws_bytes(int64_t M);
size_t smc_resample_var_ws_bytes(int64_t M);

extern "C" smc_status smc_reserve(smc_ctx* ctx, int64_t max_particles, int32_t max_pops) {
    if (!ctx || max_particles < 0 || max_pops < 0) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    st = ensure_popdone(ctx, max_pops, nullptr);
    if (st != SMC_OK) return st;
    st = ensure_groups(ctx, (max_particles + 31) / 32, nullptr);
    if (st != SMC_OK) return st;
    const size_t a = smc_resample_ws_bytes(max_particles);
    const size_t b = smc_resample_var_ws_bytes(max_particles);
    return ensure_ws(ctx, a > b ? a : b, nullptr);
}

extern "C" smc_status smc_ctx_check(smc_ctx* ctx, void* stream) {
    if (!ctx) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    cudaStream_t s = as_stream(stream);
    SMC_CUDA(cudaStreamSynchronize(s));
    SMC_CUDA(cudaGetLastError());
    uint32_t v = 0;
    SMC_CUDA(cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost));
    if (v) SMC_CUDA(cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
    SMC_CUDA(cudaDeviceSynchronize());
    if (v & smc::ST_BOUNDS) return SMC_ERR_BOUNDS;
    if (v & smc::ST_TIMEOUT) return SMC_ERR_TIMEOUT;
    if (v & smc::ST_NONFINITE) return SMC_ERR_NONFINITE;
    if (v & smc::ST_BADARG) return SMC_ERR_ARG;
    if (v & smc::ST_ZERO_WEIGHT) return SMC_ERR_ZERO_WEIGHT;
    return SMC_OK;
}

extern "C" const char* smc_status_string(smc_status s) {
    switch (s) {
        case SMC_OK: return "ok";
        case SMC_ERR_ARG: return "invalid argument (or workspace growth during graph capture)";
        case SMC_ERR_CUDA: return "CUDA runtime error";
        case SMC_ERR_NONFINITE: return "non-finite log-likelihood or log-weight";
        case SMC_ERR_ZERO_WEIGHT: return "all weights are zero";
        case SMC_ERR_TIMEOUT: return "bounded device wait expired";
        case SMC_ERR_UNSUPPORTED: return "unsupported configuration";
        case SMC_ERR_BOUNDS: return "index out of bounds (debug build)";
    }
    return "unknown status";
}

extern "C" smc_status smc_set_wait_limit(smc_ctx* ctx, uint32_t polls) {
    if (!ctx) return SMC_ERR_ARG;
    ctx->wait_limit = polls;
    return SMC_OK;
}

extern "C" smc_status smc_set_launch(smc_ctx* ctx, int32_t op, int32_t lanes, int32_t threads) {
    if (!ctx || op < 0 || op >= SMC_OP_COUNT) return SMC_ERR_ARG;
    if (lanes == 0) {
        ctx->lanes[op] = 0;
        ctx->threads[op] = 0;
        return SMC_OK;
    }
    // every kernel these shapes launch is compiled for at most 256 threads
    if (lanes < 1 || lanes > 32 || (lanes & (lanes - 1)) || threads < 64 || threads > 256 ||
        threads % 32 || threads % lanes)
        return SMC_ERR_ARG;
    ctx->lanes[op] = lanes;
    ctx->threads[op] = threads;
    return SMC_OK;
}

extern "C" smc_status smc_get_launch(smc_ctx* ctx, int32_t op, int64_t M, int64_t N, int32_t K,
                                     int32_t* lanes, int32_t* threads) {
    if (!ctx || !lanes || !threads || op < 0 || op >= SMC_OP_COUNT) return SMC_ERR_ARG;
    int l, t;
    launch_shape(ctx, op, M, N, K, &l, &t);
    *lanes = l;
    *threads = t;
    return SMC_OK;
}

// ------------------------------------------------------------------ raw streams

__global__ void k_rng_words(uint64_t seed, uint32_t purpose, uint64_t step, uint32_t n_index,
                            uint32_t n_block, uint32_t* out) {
    uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t total = (uint64_t)n_index * n_block;
    if (g >= total) return;
    uint32_t i = (uint32_t)(g / n_block), b = (uint32_t)(g % n_block);
    uint4 w = smc::draw(seed, purpose, step, i, b);
    reinterpret_cast<uint4*>(out)[g] = w;
}

__global__ void k_rng_normals(uint64_t seed, uint32_t purpose, uint64_t step, uint32_t n_index,
                              uint32_t n, float* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_index) return;
    for (uint32_t b = 0; 4 * b < n; ++b) {
        uint4 w = smc::draw(seed, purpose, step, i, b);
        float z[4];
        smc::box_muller(w.x, w.y, z[0], z[1]);
        smc::box_muller(w.z, w.w, z[2], z[3]);
        for (int j = 0; j < 4 && 4 * b + j < n; ++j) out[(size_t)i * n + 4 * b + j] = z[j];
    }
}

extern "C" smc_status smc_rng_words(smc_ctx* ctx, uint64_t seed, uint32_t purpose, uint64_t step,
                                    uint32_t n_index, uint32_t n_block, uint32_t* out,
                                    void* stream) {
    if (!ctx || (!out && n_index && n_block)) return SMC_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    uint64_t total = (uint64_t)n_index * n_block;
    if (total == 0) return SMC_OK;
    unsigned blocks = (unsigned)((total + 255) / 256);
    k_rng_words<<<blocks, 256, 0, as_stream(stream)>>>(seed, purpose, step, n_index, n_block, out);
    return cuda_ok(cudaGetLastError());
}

extern "C" smc_status smc_rng_normals(smc_ctx* ctx, uint64_t seed, uint32_t purpose,
                                      uint64_t step, uint32_t n_index, uint32_t n, float* out,
                                      void* stream) {
    if (!ctx || (!out && n_index && n)) return SMC_ERR_ARG;
    smc_status st = use_device(ctx);
    if (st != SMC_OK) return st;
    if (n_index == 0 || n == 0) return SMC_OK;
    k_rng_normals<<<(n_index + 255) / 256, 256, 0, as_stream(stream)>>>(seed, purpose, step,
                                                                       n_index, n, out);
    return cuda_ok(cudaGetLastError());
}
