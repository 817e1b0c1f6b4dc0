// kete_peak.cu -- FMA-chain probe of the FP64 / FP32 ALU peak (include/kete_peak.h).
#include <cuda_runtime.h>

#include "../../include/kete_peak.h"

// lanes below `active` of every warp run the chains; the others skip them
template <typename T>
__global__ void k_fma_chain(int64_t iters, T seed, T *sink, int active)
{
    T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    const T b = (T)0.999999, c = (T)1e-7;
    const int64_t n = ((int)(threadIdx.x & 31) < active) ? iters : 0;
    for (int64_t i = 0; i < n; i++) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == (T)-12345.0) sink[0] = s;   // never true; keeps the chains alive
}

template <typename T>
static int run(int64_t iters, int blocks, int threads, int reps, int active, double *out)
{
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return -5;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < reps + 1; r++) {
        cudaEventRecord(e0);
        k_fma_chain<T><<<blocks, threads>>>(iters, (T)0.5, sink, active);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;   // first launch is warm-up
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return -5;
    *out = 8.0 * (double)iters * blocks * (threads / 32) / (best * 1e-3);   // warp FMA instr/s
    return 0;
}

extern "C" int kete_peak_fma(int fp64, int64_t iters, int blocks, int threads, int reps,
                             double *flops_per_s)
{
    if (!flops_per_s || iters < 1 || blocks < 1 || threads < 32 || threads % 32 || reps < 1)
        return -1;
    double wi = 0.0;
    int rc = fp64 ? run<double>(iters, blocks, threads, reps, 32, &wi)
                  : run<float>(iters, blocks, threads, reps, 32, &wi);
    if (rc == 0) *flops_per_s = wi * 32.0 * 2.0;
    return rc;
}

extern "C" int kete_peak_fma_lanes(int fp64, int active_lanes, int64_t iters, int blocks,
                                   int threads, int reps, double *warp_inst_per_s)
{
    if (!warp_inst_per_s || active_lanes < 1 || active_lanes > 32 || iters < 1 || blocks < 1 ||
        threads < 32 || threads % 32 || reps < 1)
        return -1;
    return fp64 ? run<double>(iters, blocks, threads, reps, active_lanes, warp_inst_per_s)
                : run<float>(iters, blocks, threads, reps, active_lanes, warp_inst_per_s);
}
