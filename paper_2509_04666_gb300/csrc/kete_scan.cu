// kete_scan.cu -- exclusive prefix sums used to build the CSR layouts of the
// FoV stage (sky cells, candidates per exposure, hits per frame).
#include <cuda_runtime.h>

#include "kete_fov.h"

namespace kete {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = kScanThreads * kScanItems;

// each block scans one tile of m = n + 1 elements (element n is 0, so the
// last output is the total) and writes the tile total to sums
template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_tile(const T *__restrict__ in, int64_t n, int64_t *__restrict__ out, int64_t *__restrict__ sums)
{
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t idx = base + j;
        v[j] = (idx < n) ? (int64_t)in[idx] : 0;
        s += v[j];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    int64_t run = incl - s + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t idx = base + j;
        if (idx <= n) out[idx] = run;
        run += v[j];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t m, const int64_t *__restrict__ off)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] += off[i / kScanTile];
}

static int64_t tiles_of(int64_t n) { return (n + 1 + kScanTile - 1) / kScanTile; }

size_t scan_tmp_elems(int64_t n)
{
    int64_t nb = tiles_of(n);
    if (nb <= 1) return 1;
    return (size_t)(nb + nb + 1) + scan_tmp_elems(nb);
}

template <typename T>
static cudaError_t scan_impl(const T *in, int64_t n, int64_t *out, int64_t *tmp, cudaStream_t st)
{
    int64_t nb = tiles_of(n);
    k_scan_tile<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nb <= 1) return e;
    int64_t *sums = tmp, *offs = tmp + nb, *rest = tmp + 2 * nb + 1;
    e = scan_impl<int64_t>(sums, nb, offs, rest, st);
    if (e != cudaSuccess) return e;
    int64_t m = n + 1;
    k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(out, m, offs);
    return cudaGetLastError();
}

int scan_launches(int64_t n)
{
    int64_t nb = tiles_of(n);
    return nb <= 1 ? 1 : 2 + scan_launches(nb);
}

cudaError_t exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *tmp,
                           cudaStream_t st)
{
    return scan_impl<int32_t>(in, n, out, tmp, st);
}

}  // namespace kete
