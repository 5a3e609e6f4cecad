// diag_tc.cu -- diagonal d-dimensional mixture log-likelihood with the
// mu . y contraction on the tensor cores (tcgen05, bf16 hi/lo splits).
#include "ctx.hpp"

smc_status smc_diag_tc_loglik(smc_ctx* ctx, const smc_gmm* model, const float* Y, int64_t N,
                              const float* theta, int64_t M, double* out, cudaStream_t s) {
    (void)ctx; (void)model; (void)Y; (void)N; (void)theta; (void)M; (void)out; (void)s;
    return SMC_ERR_UNSUPPORTED;
}
