// kete_adjoint.h -- device buffers and launchers of the adjoint (kete_adjoint.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kete_impl.h"

namespace kete {

// one record per accepted step: t_start, t_end, then the symmetric Newtonian
// da/dx (xx, xy, xz, yy, yz, zz) at the step's 8 Gauss-Radau nodes; a final
// record (t_end = t_start) holds da/dx at the last state in node 0's place
constexpr int kAdjRec = 2 + 8 * 6;
// the full-model extension of a record: 8 nodes x (da/dx beyond Newton, da/dv)
constexpr int kAdjRecX = 8 * 18;
// checkpoint stops per body before the chain gives up (KETE_BODY_STEP_CAP)
constexpr int kAdjMaxCkpt = 1 << 16;

// the problem (caller's arrays; states and grad are [6][n], obs [n][m])
struct AdjProblem {
    const double *states, *epochs;
    int64_t n;
    const kete_obs *obs;
    int32_t m;
    double span, ckpt;
    double cos_eps, sin_eps;
    double *loss, *grad, *pred;
    double *jac;       // [n][m][2][6] d(RA, Dec)/d(x0, v0) per observation, or null
    int32_t *status;
    DevCounters *ctr;
};

// library scratch for one chunk of nc bodies
struct AdjBuffers {
    double *rec;       // [nc][cap][kAdjRec]
    int32_t cap;       // records per body
    int32_t *n_rec;    // [nc] records written (0: no gradient)
    int32_t *nbat;     // [nc] batches
    int32_t *bidx;     // [nc][m] steps taken when batch k's midpoint was reached
    double *yref;      // [nc][m][6] state at batch k's midpoint
    double *gjump;     // [nc][m][6] dL/dy(t_ref) of batch k
    double *phi;       // [nc][m][36] state-transition matrix at batch k's midpoint
                       // (row-major, d y_r(t_ref) / d y0_c; only with P.jac)
    double *recx;      // [nc][cap][8][18] per record and node: da/dx beyond the Newtonian
                       // part (9, row-major) and da/dv (9) -- the full force model's
                       // Jacobian (calls with non-gravitational terms); null: the
                       // Newtonian da/dx of rec alone
    int32_t *rich;     // [nc] (with recx) 1: the body has non-gravitational terms and
                       // its records carry recx; 0: a body without terms, Newtonian
                       // records only
    int32_t *status;   // [nc]
};

cudaError_t upload_adjoint_tables(cudaStream_t st);
// next != null: persistent grid with work stealing from the counter *next;
// order != null: lanes take the chunk's bodies in that order
cudaError_t launch_adjoint_forward(const EphemDev &E, const ForceDev &F, const AdjBuffers &B,
                                   const AdjProblem &P, int64_t i0, int64_t nc,
                                   unsigned long long *next, cudaStream_t st,
                                   const int32_t *order = nullptr);
// t_end[i] = the last observation epoch of chunk body i (its epoch if none)
cudaError_t launch_adjoint_last_epoch(const AdjProblem &P, int64_t i0, int64_t nc, double *t_end,
                                      cudaStream_t st);
cudaError_t launch_adjoint_observe(const EphemDev &E, const AdjBuffers &B, const AdjProblem &P,
                                   int64_t i0, int64_t nc, cudaStream_t st);
cudaError_t launch_adjoint_backward(const AdjBuffers &B, const AdjProblem &P, int64_t i0,
                                    int64_t nc, cudaStream_t st);
// the state-transition matrix at every batch midpoint (B.phi), integrated
// forward over the recorded steps
cudaError_t launch_adjoint_stm(const AdjBuffers &B, const AdjProblem &P, int64_t i0, int64_t nc,
                               cudaStream_t st);

}  // namespace kete
