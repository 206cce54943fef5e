/*
 * dsnu_measure.h -- arithmetic throughput of the current GPU, measured.
 *
 * Not part of the solver (the paper has no counterpart): the denominator of
 * the roofline of the FP64 solver, whose FFT passes are bound by the FP64
 * arithmetic of the GPU rather than by its memory bandwidth.
 */
#ifndef DSNU_MEASURE_H
#define DSNU_MEASURE_H

#include <stdint.h>

#include "dsnufft.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Fused multiply-add throughput of the current device in flop/s (one FMA =
 * 2 flop): a grid of (SMs x resident blocks) blocks of 256 threads, each
 * thread running 8 independent FMA chains, timed with CUDA events on `stream`
 * (cudaStream_t or NULL) after one warm-up launch; the best of three timed
 * launches.  precision: DSNU_FP64 (double FMAs) or DSNU_MIXED (float FMAs).
 * Allocates a small device buffer for the results (freed before returning)
 * and synchronises `stream`; changes no device setting.
 * Errors: DSNU_EINVAL (unknown precision, NULL output), DSNU_ECUDA. */
dsnu_status dsnu_measure_fma_peak(int32_t precision, double* flops_per_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DSNU_MEASURE_H */
