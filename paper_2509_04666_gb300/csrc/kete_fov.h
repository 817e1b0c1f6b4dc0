// kete_fov.h -- device arrays and launchers of the FoV stage (Sec. 2, Sec. 3.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kete_impl.h"

namespace kete {

// per exposure (a union of sub-field polygons sharing epoch and observer)
struct ExpArrays {
    double *epoch;     // [E]
    double *obs;       // [E][3]
    double *cen;       // [E][3] unit centre of the covering cap
    double *rad;       // [E] cap radius, rad (pi = covers everything)
    float2 *cs;        // [E] (cos r, sin r) of the cap, cos = -2 when r = pi
    float4 *cenf;      // [E] the centre in FP32 for the candidate search (w unused)
    int32_t *batch;    // [E]
    double *sun;       // [E][6] Sun position and velocity at the exposure epoch
    float4 *obs_rel;   // [E] observer minus its batch's mean observer (FP32), w unused
};

// per batch of exposures (<= span in time, Sec. 2)
struct BatchArrays {
    int32_t *first;    // [K+1] first exposure of each batch
    double *t_ref;     // [K] batch midpoint: the n-body stop
    double *O;         // [K][3] mean observer
    double *robs;      // [K] max distance of an exposure's observer from O
    double *tspan;     // [K] max |t_e - t_ref|
    double *rmax;      // [K] max exposure cap radius
    double *sun;       // [K][6] Sun position and velocity at t_ref
};

// latitude-band sky cells
struct CellGrid {
    const int32_t *band_off;   // [n_bands+1] first cell of each band
    const int32_t *band_n;     // [n_bands] cells in each band
    double hb;                 // band height, rad
    int32_t n_bands, n_cells;
};

struct CandArgs {
    ExpArrays X;
    BatchArrays B;
    CellGrid G;
    const double *stop_states;   // [nk][n][6] per-body records of the chunk's batches
    int64_t n;
    int32_t k0, nk;
    const int64_t *cell_start;
    const int32_t *cell_exp;
    uint2 *cand;
    unsigned long long cap;
    int32_t *exp_cnt;
    DevCounters *ctr;
    double mu_sun;
};

struct ExactArgs {
    EphemDev E;
    ExpArrays X;
    BatchArrays B;
    const kete_frame *frames;
    const float4 *faux;
    const double *stop_states;   // [nk][n][6] per-body records of the chunk's batches
    int64_t n;
    int32_t k0, e_begin, e_end;
    const int64_t *exp_off;
    int64_t n_cand;            // candidates of the chunk
    const int32_t *cand_body;
    const int32_t *exp_first;
    kete_hit *hits;
    unsigned long long cap;
    int32_t *frame_cnt;
    int32_t *status;
    DevCounters *ctr;
    const kete_mag_params *mag = nullptr;   // [n] magnitude models, or null
    // scratch of the prefilter pass (null: no prefilter): the indices of the
    // candidates it keeps ([n_cand]) and their count
    uint32_t *keep = nullptr;
    unsigned long long *n_keep = nullptr;
};

cudaError_t fov_frame_prep(const kete_frame *frames, int64_t nf, int64_t n_obs, int32_t *is_start,
                           double *fcen, float4 *faux, DevCounters *ctr, cudaStream_t st);
cudaError_t fov_exposure_first(const int32_t *is_start, const int64_t *ex, int64_t nf,
                               int32_t *exp_first, cudaStream_t st);
cudaError_t fov_exposure_prep(const EphemDev &E, const kete_frame *frames, int64_t nf,
                              const double *observers, const double *fcen,
                              const int32_t *exp_first, int64_t ne, ExpArrays X,
                              unsigned int *max_rad_bits, DevCounters *ctr, cudaStream_t st);
cudaError_t fov_batches(const double *ep, int64_t ne, double span, int32_t *next, BatchArrays B,
                        int32_t *n_batches, cudaStream_t st);
cudaError_t fov_batch_info(const EphemDev &E, ExpArrays X, BatchArrays B, int32_t nb,
                           DevCounters *ctr, cudaStream_t st);
cudaError_t fov_cell_keys(ExpArrays X, CellGrid G, int32_t e0, int32_t e1, int32_t k0,
                          int32_t *key, int32_t *cnt, cudaStream_t st);
cudaError_t fov_cell_scatter(int32_t e0, int32_t e1, const int32_t *key, const int64_t *start,
                             int32_t *cursor, int32_t *cell_exp, cudaStream_t st);
cudaError_t fov_candidates(const CandArgs &a, cudaStream_t st);
cudaError_t fov_cand_scatter(const uint2 *cand, unsigned long long nc, const int64_t *exp_off,
                             int32_t e_begin, int32_t *cursor, int32_t *cand_body, cudaStream_t st);
cudaError_t fov_exact(const ExactArgs &a, int n_sm, cudaStream_t st);
cudaError_t fov_order_hits(const kete_hit *tmp, unsigned long long nh, const int64_t *frame_off,
                           int64_t nf, int32_t *cursor, kete_hit *grouped, kete_hit *out,
                           int n_sm, cudaStream_t st);

// Extended exposures: validate the caller's frames against their durations
// (device, [nf]) and n_sub, and write nf * n_sub sub-frames and each one's
// parent frame.  Flags in ctr->error_flags: bits 0-2 as fov_frame_prep, bit 6
// a bad duration.
cudaError_t fov_ext_expand(const kete_frame *frames, const double *dur, int64_t nf, int n_sub,
                           int64_t n_obs, int32_t *is_start, int64_t *ex, int64_t *scan_tmp,
                           int32_t *exp_first, kete_frame *sub, int32_t *parent, DevCounters *ctr,
                           cudaStream_t st);
// Union of the sub-frames' hits per parent frame: count (scatter = false) or
// scatter into groups by parent (scatter = true, offsets from the counts);
// then mark the earliest sub-frame's hit of every body and count them; then
// place those in body order, renamed to the parent frame.
cudaError_t fov_merge_count(const kete_hit *h, unsigned long long nh, const int32_t *parent,
                            int32_t *cnt, const int64_t *off, int32_t *cur, kete_hit *grouped,
                            bool scatter, cudaStream_t st);
cudaError_t fov_merge_keep(const kete_hit *grouped, const int64_t *off, int64_t np, int8_t *keep,
                           int32_t *kept_cnt, int n_sm, cudaStream_t st);
cudaError_t fov_merge_place(const kete_hit *grouped, const int64_t *off, const int8_t *keep,
                            const int64_t *kept_off, int64_t np, kete_hit *out, int n_sm,
                            cudaStream_t st);

// kete_scan.cu: exclusive prefix sum of int32 counts into int64 offsets
// (out has n+1 entries; out[n] = total).  tmp must hold scan_tmp_elems(n).
size_t scan_tmp_elems(int64_t n);
int scan_launches(int64_t n);   // kernel launches of exclusive_scan over n
cudaError_t exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *tmp,
                           cudaStream_t st);

}  // namespace kete
