/*
 * kete_peak.h -- ALU peak probe used to state roofline fractions
 * (libkete_peak.so).  Not part of the survey path and not in the paper: the
 * propagation kernel is bound by FP64 (or, in mixed precision, FP32) FMA
 * throughput, whose peak on this GPU is measured rather than assumed.
 */
#ifndef KETE_PEAK_H
#define KETE_PEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Run independent FMA chains on the current CUDA device: `blocks` x `threads`
 * threads, each doing `iters` iterations of 8 independent FMAs in FP64
 * (fp64 != 0) or FP32.  *flops_per_s (host) receives 2 * FMAs / kernel time
 * (CUDA events, best of `reps` launches).  Returns 0, or -5 on a CUDA error. */
int kete_peak_fma(int fp64, int64_t iters, int blocks, int threads, int reps,
                  double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif
