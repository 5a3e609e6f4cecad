// ctx.hpp -- host-side context: device status word, workspace, launch
// overrides.  Shared by the host halves of every translation unit.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "smc.h"

struct smc_ctx {
    int device = 0;
    int num_sms = 0;
    int max_threads_per_sm = 0;
    int smem_per_sm = 0;            // shared memory per SM (bytes)
    int smem_optin = 0;             // largest dynamic shared memory one CTA may opt in to
    int smem_reserved = 0;          // shared memory the system reserves per block
    uint32_t* d_status = nullptr;     // latched device errors (bit set)
    // fixed small area: counters and reduction partials
    unsigned long long* d_counters = nullptr;  // [kCounters] zero-initialised
    double* d_partials = nullptr;              // [kMaxPartialBlocks * 8]
    // growable area: resampling tile descriptors, staging buffers
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // per-population completion counters of the population sweep (zeroed)
    uint32_t* d_popdone = nullptr;
    int64_t popdone_cap = 0;
    // binned sweep: per chain group of 32, an arrival counter (zeroed) and
    // the two parts of a group cut by a CTA boundary (double[2][32])
    uint32_t* d_grpdone = nullptr;
    double* d_grppart = nullptr;
    int64_t grp_cap = 0;
    // binned sweep: the binned layout of the last data set seen (built by
    // k_bin_prepare; allocated with the context at the largest N) and the
    // host's key for it; the sweep checks the data against the layout's own
    // copy before using it
    char* d_bcache = nullptr;
    size_t bcache_bytes = 0;
    const void* bkey_y = nullptr;
    int64_t bkey_n = -1;
    uint32_t bkey_binw = 0, bkey_cf = 0;
    // MRG32k3a skip-ahead table: A1^(2^k), A2^(2^k), k < 64 (filled at creation)
    uint32_t* d_mrg_pow = nullptr;
    // polls of the first bounded wait on a bulk data copy before it gives up
    // (ST_TIMEOUT); set by smc_set_wait_limit, a test hook
    uint32_t wait_limit = 4u << 20;
    int32_t lanes[SMC_OP_COUNT] = {0, 0, 0};
    int32_t threads[SMC_OP_COUNT] = {0, 0, 0};
};

namespace smc_host {

// counter slots in d_counters (each call that uses one leaves it at zero)
enum : int {
    CNT_REWEIGHT_TICKET = 0,
    CNT_ESS_TICKET = 1,
    CNT_RESAMPLE_TILE = 2,
    CNT_RESAMPLE_SUM = 3,       // exact uint64 total S of the quantised weights
    CNT_POP_QUEUE = 4,
    CNT_POP_DONE = 5,
    CNT_DIAG_TICKET = 6,
    CNT_RESAMPLE_DONE = 7,
    CNT_IS_TICKET = 8,
    kCounters = 16
};
constexpr int kMaxPartialBlocks = 2048;

// CUDA error -> status, remembering nothing (errors are returned)
inline smc_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? SMC_OK : SMC_ERR_CUDA; }

#define SMC_CUDA(call)                                  \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return SMC_ERR_CUDA;     \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Launch with programmatic stream serialisation: the kernel may begin
// launching while the previous kernel on the stream drains; it calls
// grid_dep_wait() before touching anything that kernel wrote.
template <typename... KArgs, typename... Args>
inline smc_status launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_ok(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

// True while `s` is being captured into a graph.
bool capturing(cudaStream_t s);

// Make sure the growable workspace holds `bytes`; grows only outside capture.
smc_status ensure_ws(smc_ctx* ctx, size_t bytes, cudaStream_t s);

// Make sure there are n zeroed population counters; grows only outside capture.
smc_status ensure_popdone(smc_ctx* ctx, int64_t n, cudaStream_t s);

// Make sure there are n zeroed chain-group counters and their part buffers
// (binned population sweep); grows only outside capture.
smc_status ensure_groups(smc_ctx* ctx, int64_t n, cudaStream_t s);

// Set the context's device current for the calling thread.
smc_status use_device(smc_ctx* ctx);

// Launch shape: lanes per particle and threads per block for `op`.
void launch_shape(const smc_ctx* ctx, int op, int64_t M, int64_t N, int K, int* lanes,
                  int* threads);

}  // namespace smc_host
