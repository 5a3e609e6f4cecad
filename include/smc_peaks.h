/*
 * smc_peaks.h -- roofline denominators measured on the running GPU.
 *
 * Issue-rate microbenchmarks used to report the likelihood kernels against
 * the pipe that bounds them (the paper's Section 5 notes the mixture
 * likelihood is arithmetic-bound; on sm_103a the binding pipe is the MUFU
 * unit that evaluates ex2).  Not part of the sampler path.
 */
#ifndef SMC_PEAKS_H
#define SMC_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SMC_PEAK_EX2 = 0, SMC_PEAK_LG2 = 1, SMC_PEAK_FFMA = 2, SMC_PEAK_DFMA = 3,
       SMC_PEAK_I2F = 4,   /* int -> float conversion (plus an integer shift) */
       SMC_PEAK_FRND = 5   /* float round to integer (plus an FMUL and FADD) */ };

/* Run the `kind` issue-rate kernel on the current device over `blocks_per_sm`
 * x (#SMs) blocks of 256 threads, `iters` iterations of 8 independent
 * dependency chains per thread, and return in *ops_per_s the instruction
 * results per second (FMA counted as one operation) and in *ms the kernel
 * time (CUDA events, after one warm-up launch).  Synchronous.  SMC_ERR_ARG
 * for an unknown kind or non-positive sizes; SMC_ERR_CUDA on a CUDA error. */
int smc_measure_peak(int32_t kind, int32_t blocks_per_sm, int32_t iters, double* ops_per_s,
                     double* ms);

#ifdef __cplusplus
}
#endif

#endif
