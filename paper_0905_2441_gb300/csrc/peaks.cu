// peaks.cu -- issue-rate microbenchmarks for the roofline denominators
// (ex2 / lg2 on the MUFU pipe, FFMA, DFMA).  Each thread runs 8 independent
// dependency chains so that the measured rate is the pipe's throughput.
#include <cuda_runtime.h>

#include "device.cuh"
#include "smc.h"
#include "smc_peaks.h"

namespace {

template <int KIND>
__global__ void __launch_bounds__(256) k_peak(int iters, float seed, float* sink) {
    if constexpr (KIND == SMC_PEAK_DFMA) {
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = (double)seed + threadIdx.x * 1e-9 + j * 1e-3;
        const double b = 0.999999, c = 1e-7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
        }
        double s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) s += a[j];
        if (s == 12345.0) sink[0] = (float)s;
    } else {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + threadIdx.x * 1e-7f + j * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if constexpr (KIND == SMC_PEAK_EX2) a[j] = smc::ex2(-a[j]);          // stays in [0.5, 1]
            if constexpr (KIND == SMC_PEAK_LG2) a[j] = smc::lg2(a[j] + 1.5f);     // stays in [0.58, 1.9]
            if constexpr (KIND == SMC_PEAK_FFMA) a[j] = fmaf(a[j], 0.999999f, 1e-7f);
            if constexpr (KIND == SMC_PEAK_I2F)  // int -> float -> int round trip
                a[j] = (float)(__float_as_int(a[j]) >> 9);
            if constexpr (KIND == SMC_PEAK_FRND) a[j] = rintf(a[j] * 0.5f) + 0.75f;
        }
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.0f) sink[0] = s;
    }
}

template <int KIND>
int run(int blocks, int iters, double* ops, double* ms) {
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return SMC_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_peak<KIND><<<blocks, 256>>>(iters, 0.7f, sink);
    cudaEventRecord(e0);
    k_peak<KIND><<<blocks, 256>>>(iters, 0.7f, sink);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return SMC_ERR_CUDA;
    *ms = t;
    *ops = (double)blocks * 256.0 * 8.0 * (double)iters / (t * 1e-3);
    return SMC_OK;
}

}  // namespace

extern "C" int smc_measure_peak(int32_t kind, int32_t blocks_per_sm, int32_t iters,
                                double* ops_per_s, double* ms) {
    if (!ops_per_s || !ms || blocks_per_sm < 1 || iters < 1) return SMC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SMC_ERR_CUDA;
    int blocks = sms * blocks_per_sm;
    switch (kind) {
        case SMC_PEAK_EX2: return run<SMC_PEAK_EX2>(blocks, iters, ops_per_s, ms);
        case SMC_PEAK_LG2: return run<SMC_PEAK_LG2>(blocks, iters, ops_per_s, ms);
        case SMC_PEAK_FFMA: return run<SMC_PEAK_FFMA>(blocks, iters, ops_per_s, ms);
        case SMC_PEAK_DFMA: return run<SMC_PEAK_DFMA>(blocks, iters, ops_per_s, ms);
        case SMC_PEAK_I2F: return run<SMC_PEAK_I2F>(blocks, iters, ops_per_s, ms);
        case SMC_PEAK_FRND: return run<SMC_PEAK_FRND>(blocks, iters, ops_per_s, ms);
    }
    return SMC_ERR_ARG;
}
