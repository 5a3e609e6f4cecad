// Test helper (not part of the library): runs NVIDIA cuRAND's device-side
// MRG32k3a generator from a given six-word state, so that the oracle's
// generator can be checked against an implementation written by others.
// The state fields are those of curandStateMRG32k3a in curand_kernel.h;
// `rev` stores each component's three words in reversed order.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_mrg(unsigned s10, unsigned s11, unsigned s12, unsigned s20, unsigned s21,
                             unsigned s22, int rev, int n, double* out) {
    curandStateMRG32k3a st;
    const unsigned a[3] = {s10, s11, s12}, b[3] = {s20, s21, s22};
    for (int i = 0; i < 3; ++i) {
        st.s1[i] = a[rev ? 2 - i : i];
        st.s2[i] = b[rev ? 2 - i : i];
    }
    st.boxmuller_flag = 0;
    st.boxmuller_flag_double = 0;
    st.boxmuller_extra = 0.0f;
    st.boxmuller_extra_double = 0.0;
    for (int j = 0; j < n; ++j) out[j] = curand_uniform_double(&st);
}

extern "C" int curand_mrg_run(const unsigned* seed6, int rev, int n, double* host_out) {
    double* d = nullptr;
    if (cudaMalloc(&d, (size_t)n * sizeof(double)) != cudaSuccess) return 1;
    k_curand_mrg<<<1, 1>>>(seed6[0], seed6[1], seed6[2], seed6[3], seed6[4], seed6[5], rev, n, d);
    cudaError_t e = cudaMemcpy(host_out, d, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
