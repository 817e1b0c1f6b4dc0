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
 * (CUDA events, best of `reps` launches).  threads must be a multiple of 32.
 * Returns 0, -1 on a bad argument, or -5 on a CUDA error. */
int kete_peak_fma(int fp64, int64_t iters, int blocks, int threads, int reps,
                  double *flops_per_s);

/* The same chains run by only the first `active_lanes` (1..32) lanes of every
 * warp; *warp_inst_per_s (host) receives FMA warp-instructions per second.
 * Shows whether an instruction's cost depends on its active lanes (on GB300
 * the FP64 rate does not).  threads must be a multiple of 32.  Returns 0, -1
 * on a bad argument, or -5 on a CUDA error. */
int kete_peak_fma_lanes(int fp64, int active_lanes, int64_t iters, int blocks, int threads,
                        int reps, double *warp_inst_per_s);

#ifdef __cplusplus
}
#endif
#endif
