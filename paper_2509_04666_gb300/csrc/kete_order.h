// kete_order.h -- cost order of the bodies taken by the propagation kernels
// (kete_order.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kete_impl.h"

namespace kete {

struct OrderScratch {
    uint16_t *key;      // [n]
    int32_t *hist;      // [order_hist_elems(n)]
    int64_t *off;       // [order_hist_elems(n) + 1]
    int64_t *scan_tmp;  // [scan_tmp_elems(order_hist_elems(n))]
};

size_t order_hist_elems(int64_t n);   // histogram capacity for n bodies (any class count)
int order_launches(int64_t n, const kete_nongrav *ng);   // launches of order_by_cost

// order[0..n) = the n bodies (states [6][stride] SoA, epochs [n]) most
// expensive first over [epoch, t_end] (t_end_i: per-body end epochs, or null
// for t_end).  ng (per-body non-gravitational terms, or null): group the
// bodies by the class of their terms first.
cudaError_t order_by_cost(const EphemDev &E, const double *states, int64_t stride,
                          const double *epochs, int64_t n, double t_end, const double *t_end_i,
                          const kete_nongrav *ng, OrderScratch s, int32_t *order,
                          cudaStream_t st);

}  // namespace kete
