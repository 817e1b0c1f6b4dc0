// kete_noalloc.cu -- kete_propagate_noalloc: propagation without any device
// allocation (declared in include/kete.h).
//
// kete_propagate keeps each body's chain state (position, velocity, epoch,
// step size, status) in scratch the library allocates with cudaMalloc on first
// use.  Some callers cannot allocate device memory while they run: an
// application that hands the whole GPU memory to its own pool at start-up, a
// host thread with a real-time deadline that must not block in the driver's
// allocator, or an embedding framework that forbids allocation outside its
// set-up phase.  This variant takes that scratch from a fixed array in the
// library's own device data instead, so the call allocates nothing.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it (about 4.5 MB) until the process exits.  In host code its
// name is only a host-side stand-in, never a device address, so the first call
// on each device resolves the real address with cudaGetSymbolAddress (that
// first call may load the module's device data; make it before any stream
// capture) and passes the address to the kernels.
//
// Every call on a device shares the one array: calls whose work overlaps on
// the GPU (two streams, two host threads) race on it, so order them on one
// stream or serialize them.  The array keeps the last call's contents; the
// counters the kernels accumulate into are cleared at the start of each call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "kete_impl.h"

namespace kete {

constexpr int64_t kNoallocMaxBodies = KETE_NOALLOC_MAX_BODIES;

struct NoallocScratch {
    double work[8 * kNoallocMaxBodies];   // chain state [8][n]
    int32_t status[kNoallocMaxBodies];
    double stop;                          // the single target epoch
    DevCounters ctr;                      // cleared at the start of each call
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;
static NoallocScratch *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Resolve the device address of the array for `device` (must be current).
static cudaError_t noalloc_scratch(int device, NoallocScratch **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = (NoallocScratch *)p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

__global__ void k_noalloc_begin(NoallocScratch *s, double t_target)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->stop = t_target;
        memset(&s->ctr, 0, sizeof(DevCounters));
    }
}

int noalloc_propagate(int device, cudaStream_t st, const EphemDev &E, const ForceDev &F,
                      double *states, double *epochs, int64_t n, double t_target,
                      int32_t *status, const char **why)
{
    *why = "";
    if (n > kNoallocMaxBodies) {
        *why = "n exceeds KETE_NOALLOC_MAX_BODIES";
        return KETE_ERR_BAD_ARG;
    }
    if (n == 0) return KETE_OK;
    NoallocScratch *s = nullptr;
    cudaError_t e = noalloc_scratch(device, &s);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return KETE_ERR_CUDA;
    }
    ChainState cs;
    cs.w = s->work;
    cs.status = s->status;
    cs.n = n;
    k_noalloc_begin<<<1, 32, 0, st>>>(s, t_target);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return KETE_ERR_CUDA;
    }
    if ((e = launch_chain_init(cs, states, epochs, F, st)) == cudaSuccess &&
        (e = launch_propagate(E, F, cs, &s->stop, 1, states, n, true, &s->ctr, st)) == cudaSuccess)
        e = launch_chain_finish(cs, states, epochs, status, st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return KETE_ERR_CUDA;
    }
    return KETE_OK;
}

}  // namespace kete
