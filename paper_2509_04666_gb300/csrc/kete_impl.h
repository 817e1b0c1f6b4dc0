// kete_impl.h -- internal types shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kete.h"

namespace kete {

// physical constants (App. A.1 units: AU, TDB days)
constexpr double kKmPerAu = 149597870.7;
constexpr double kC = 299792.458 * 86400.0 / kKmPerAu;   // speed of light, AU/day
constexpr double kInvC2 = 1.0 / (kC * kC);
constexpr double kInvC = 1.0 / kC;

// device view of the loaded Chebyshev table
struct EphemDev {
    const double *coef;      // [body][seg][3][n_coef]
    const float *coef32;     // the same table in FP32 (mixed-precision planets)
    double t_start, t_end, seg_len, inv_seg;
    int n_seg, n_coef, n_bodies, pad;
    double gm[KETE_MAX_BODIES];
};

// device view of a force model (derived quantities precomputed on the host)
struct ForceDev {
    uint32_t active_mask;    // body_mask with massless bodies removed
    uint32_t gr_mask, j2_mask;
    int32_t precision;
    double j2k[KETE_MAX_BODIES];        // 1.5 * J2 * mu * R^2
    double pole[KETE_MAX_BODIES][3];    // unit pole, ecliptic J2000
    // per-mass factors of the GR and J2 terms, formed once here (each saves
    // an FP64 multiply per mass and force evaluation): 4 mu, mu / c^2,
    // 4 mu / c^2 and -2 x the pole
    double gm4[KETE_MAX_BODIES], grk[KETE_MAX_BODIES], gr4k[KETE_MAX_BODIES];
    double pole_m2[KETE_MAX_BODIES][3];
    double eps, eps_pc, safety, dt_init;
    int32_t max_iter, pad;
    int64_t max_steps;
    // FP32 copies for the mixed-precision planetary terms (rounded once here)
    float gm32[KETE_MAX_BODIES];
    float j2k32[KETE_MAX_BODIES];
    float pole32[KETE_MAX_BODIES][3];
    float gm4_32[KETE_MAX_BODIES], grk32[KETE_MAX_BODIES], gr4k32[KETE_MAX_BODIES];
    float pole_m2_32[KETE_MAX_BODIES][3];
    const kete_nongrav *nongrav;        // per-body non-gravitational terms or null
};

// device counters accumulated by the kernels
struct DevCounters {
    unsigned long long steps, rejected, force_evals, iterations;
    unsigned long long candidates, hits;
    unsigned long long node_evals;   // force evaluations served by batch node rows
    unsigned long long deferred;     // bodies set aside for the split second phase
    int error_flags;         // bit 0: unsorted epochs, 1: exposure mismatch, 2: bad observer,
                             // 3: bad n_edges, 4: non-finite frame, 5: batch epoch outside table
    int pad;
};

// planet states at the 8 Gauss-Radau node epochs of each leg of a chain of
// stops (leg k runs from t0[k] to t0[k] + h[k]); h[k] is NaN when the leg
// cannot use the rows (a node outside the table)
struct NodeTable {
    const double *t0, *h;
    const double *row64;   // [leg][8][n_bodies][6] FP64 barycentric pos, vel
    const float *row32;    // [leg][8][n_bodies][6] FP32 heliocentric pos, vel
    int n_legs, nb;
};

// per-body working state of a propagation chain: [8][n] = x,y,z,vx,vy,vz,t,dt;
// kstop[n] (may be null): the stop a set-aside body resumes at
struct ChainState {
    double *w;
    int32_t *status;
    int64_t n;
    int32_t *kstop = nullptr;
};

// where a propagation launch takes its bodies from (see k_propagate)
struct PropQueue {
    const int32_t *list = nullptr;               // bodies to take; null: 0..n-1
    const unsigned long long *list_n = nullptr;  // how many (device)
    int resume = 0;                              // bodies resume at cs.kstop (else stop 0)
    int32_t *defer = nullptr;                    // set-aside bodies are appended here
    unsigned long long *defer_n = nullptr;
    int budget = 0;                              // step attempts per stop reached
};

// scratch of the two-phase (split) launch
struct PropDefer {
    int32_t *list;                 // [n]
    unsigned long long *count;     // set-aside bodies
    unsigned long long *next;      // work-stealing counter of the second phase
};

// launch helpers implemented in the .cu files ---------------------------------
void upload_radau_tables(cudaStream_t st);            // kete_prop.cu
cudaError_t launch_ephem_eval(const EphemDev &E, const double *t, int64_t n, int body,
                              double *pos, double *vel, cudaStream_t st);
cudaError_t launch_chain_init(ChainState cs, const double *states, const double *epochs,
                              const ForceDev &F, cudaStream_t st);
cudaError_t launch_node_table(const EphemDev &E, const double *stops_dev, int n_stops,
                              const double *epoch0, double *t0, double *h, double *row64,
                              float *row32, cudaStream_t st);
// how the propagation kernel is launched (chosen by the autotuner)
enum PropKind { PROP_STATIC = 0, PROP_WORK_STEALING = 1 };
struct PropVariant {
    int kind;         // PropKind
    int block;        // threads per block (<= 128)
    int split = 0;    // lanes per body for long bodies (4, 8, 16; 0 or 1: none)
    int budget = 0;   // step attempts per stop after which a body is set aside
    int order = 0;    // take bodies most expensive first (kete_order.cu)
    double grid_scale = 1.0;   // persistent grids scaled by this (<= 1: a sample of the
                               // bodies run with as many bodies per lane as the whole)
};
cudaError_t launch_propagate(const EphemDev &E, const ForceDev &F, ChainState cs,
                             const double *stops_dev, int n_stops, double *out,
                             int64_t out_stride, bool keep_on_fail, DevCounters *ctr,
                             cudaStream_t st, const NodeTable *nt = nullptr, int leg0 = 0,
                             PropVariant var = PropVariant{PROP_STATIC, 128},
                             unsigned long long *next_body = nullptr,
                             PropDefer *defer = nullptr, const int32_t *order = nullptr,
                             const unsigned long long *order_n = nullptr, bool out_aos = false);
int propagate_ws_blocks(int block, int mode);
cudaError_t launch_gather_bodies(const double *st, const double *ep, int64_t n, int64_t m,
                                 double *dst, double *dep, cudaStream_t s);
cudaError_t launch_chain_finish(ChainState cs, double *states, double *epochs,
                                int32_t *status, cudaStream_t st);
// kete_noalloc.cu: propagation with the chain scratch in a fixed device array
int noalloc_propagate(int device, cudaStream_t st, const EphemDev &E, const ForceDev &F,
                      double *states, double *epochs, int64_t n, double t_target,
                      int32_t *status, const char **why);

}  // namespace kete
