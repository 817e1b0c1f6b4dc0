// kete_order.cu -- the order in which the propagation kernels take bodies.
//
// On GB300 an FP64 warp instruction costs the same pipe time whatever the
// number of its active lanes, so a warp whose lanes hold bodies of very
// different step counts wastes most of what it issues.  Bodies are taken most
// expensive first, so that a warp's lanes hold bodies of similar cost and the
// longest chains start early.  The cost of a body is estimated from its
// heliocentric conic: the Gauss-Radau step the step control settles on
// scales with the local dynamical time r^1.5 / sqrt(mu), so the number of
// steps over [t, t_end] is about  integral dt / (c r^1.5),  evaluated at 8
// epochs of the two-body motion.  A stable counting sort on 256 log-spaced
// buckets gives the order.  With non-gravitational terms the bodies are first
// grouped by class (thermal-lag terms, which cost a two-body solve per force
// evaluation; other terms; none), so that a warp's lanes take the extra work
// together or not at all: 3 x 256 buckets.  The order changes only which lane
// takes which body: every body's arithmetic, and so every result, is
// unchanged.
#include <cuda_runtime.h>

#include <cmath>

#include "kete_device.cuh"
#include "kete_fov.h"
#include "kete_order.h"

namespace kete {

constexpr int kCostBuckets = 256;               // per class
constexpr int kMaxClasses = 3;
constexpr int kMaxBuckets = kCostBuckets * kMaxClasses;
constexpr int kOrderTile = 1024;   // elements per block of the counting sort

static int n_classes(const kete_nongrav *ng) { return ng ? kMaxClasses : 1; }

// key of body i: class (lagged terms, other terms, none) first, then cost,
// most expensive first (ascending key)
__global__ void k_order_keys(EphemDev E, const double *__restrict__ w, int64_t stride,
                             const double *__restrict__ epochs, int64_t n, double t_end,
                             const double *__restrict__ t_end_i, const kete_nongrav *__restrict__ ng,
                             uint16_t *__restrict__ key)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t0 = epochs[i];
    const double t1 = t_end_i ? t_end_i[i] : t_end;
    double cost = 0.0;
    Seg g;
    if (isfinite(t0) && isfinite(t1) && ephem_seg(E, t0, 0.0, g)) {
        double sp[3], sv[3], r0[3], v0[3];
        cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, sp, sv);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            r0[c] = w[c * stride + i] - sp[c];
            v0[c] = w[(3 + c) * stride + i] - sv[c];
        }
        const double mu = E.gm[0], sqmu = sqrt(mu);
        const double span = fabs(t1 - t0), dts = (t1 - t0) / 8.0;
        double chi = 0.0;
        for (int k = 0; k < 8; k++) {
            double r[3], v[3];
            kepler_uv(mu, sqmu, r0, v0, ((double)k + 0.5) * dts, chi, r, v);
            const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            cost += (span / 8.0) * sqmu / (rn * sqrt(rn));
        }
    }
    // log-spaced buckets, 16 per octave above cost 2^-4
    int b = 0;
    if (cost > 0.0 && isfinite(cost)) b = (int)floor(16.0 * (log2(cost) + 4.0));
    b = b < 0 ? 0 : (b > kCostBuckets - 1 ? kCostBuckets - 1 : b);
    int cls = 0;   // 0: thermal-lag terms, 1: other terms, 2: none (without ng: 0)
    if (ng) {
        const kete_nongrav p = ng[i];
        const bool jpl = p.a1 != 0.0 || p.a2 != 0.0 || p.a3 != 0.0;
        cls = (jpl && p.dt != 0.0) ? 0 : ((jpl || p.beta != 0.0) ? 1 : 2);
    }
    key[i] = (uint16_t)(cls * kCostBuckets + (kCostBuckets - 1 - b));
}

// hist[key][tile]: the keys of each tile of kOrderTile bodies
__global__ void k_order_hist(const uint16_t *__restrict__ key, int64_t n, int n_buckets,
                             int32_t *__restrict__ hist, int64_t n_tiles)
{
    __shared__ int32_t cnt[kMaxBuckets];
    for (int b = threadIdx.x; b < n_buckets; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kOrderTile;
    for (int j = threadIdx.x; j < kOrderTile; j += blockDim.x)
        if (base + j < n) atomicAdd(&cnt[key[base + j]], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < n_buckets; b += blockDim.x)
        hist[(int64_t)b * n_tiles + blockIdx.x] = cnt[b];
}

// stable scatter: within a tile, bodies of equal key keep their index order
// (warps in turn, lanes by rank among equal keys)
__global__ void __launch_bounds__(256)
k_order_scatter(const uint16_t *__restrict__ key, int64_t n, int n_buckets,
                const int64_t *__restrict__ off, int64_t n_tiles, int32_t *__restrict__ order)
{
    __shared__ int64_t next[kMaxBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (int b = threadIdx.x; b < n_buckets; b += blockDim.x)
        next[b] = off[(int64_t)b * n_tiles + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kOrderTile;
    for (int r = 0; r < kOrderTile; r += blockDim.x) {
        const int64_t j = base + r + threadIdx.x;
        const bool valid = (r + (int)threadIdx.x < kOrderTile) && j < n;
        const int k = valid ? (int)key[j] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int lead = __ffs(peers) - 1;
        for (int w = 0; w < n_warps; w++) {
            if (w == warp && valid) order[next[k] + rank] = (int32_t)j;
            __syncthreads();
            if (w == warp && valid && lane == lead) next[k] += __popc(peers);
            __syncthreads();
        }
    }
}

cudaError_t order_by_cost(const EphemDev &E, const double *states, int64_t stride,
                          const double *epochs, int64_t n, double t_end, const double *t_end_i,
                          const kete_nongrav *ng, OrderScratch s, int32_t *order, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t n_tiles = (n + kOrderTile - 1) / kOrderTile;
    const int nb = kCostBuckets * n_classes(ng);
    k_order_keys<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(E, states, stride, epochs, n, t_end,
                                                              t_end_i, ng, s.key);
    k_order_hist<<<(unsigned)n_tiles, 256, 0, st>>>(s.key, n, nb, s.hist, n_tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(s.hist, (int64_t)nb * n_tiles, s.off, s.scan_tmp, st);
    if (e != cudaSuccess) return e;
    k_order_scatter<<<(unsigned)n_tiles, 256, 0, st>>>(s.key, n, nb, s.off, n_tiles, order);
    return cudaGetLastError();
}

int order_launches(int64_t n, const kete_nongrav *ng)
{
    if (n <= 0) return 0;
    const int64_t n_tiles = (n + kOrderTile - 1) / kOrderTile;
    return 3 + scan_launches((int64_t)kCostBuckets * n_classes(ng) * n_tiles);
}

size_t order_hist_elems(int64_t n)
{
    return (size_t)kMaxBuckets * (size_t)((n + kOrderTile - 1) / kOrderTile);
}

}  // namespace kete
