// kete_fov.cu -- the FoV stage of the survey path (Sec. 2, Sec. 3.1, App. A.1).
//
//   frame prep   validate frames, find exposure boundaries, circumscribed cap
//                of every polygon (from its vertices, found in any edge order)
//   exposures    epoch, observer, cap covering all sub-fields
//   batching     greedy <= span batches over epoch-sorted exposures, t_ref =
//                midpoint of first and last epoch (Sec. 2)
//   batch info   mean observer, observer spread, time spread, Sun state at t_ref
//   sky cells    per batch, exposures bucketed by the sky cell of their centre
//   candidates   per (body, batch): conservative motion + parallax radius,
//                enumerate nearby cells, cap test against each exposure
//   exact test   per candidate: heliocentric universal-variable two-body from
//                t_ref, light-delay iteration, polygon test of every
//                sub-field (strict n.u > 0), RA/Dec
//   ordering     hits grouped by frame, sorted by body within a frame
#include <cuda_runtime.h>

#include <cmath>

#include "kete_device.cuh"
#include "kete_fov.h"

namespace kete {

constexpr float kPadF = 2e-4f;        // radians added to every float cap test
constexpr double kSunSpeedMax = 5e-5; // bound on the barycentric Sun speed, AU/day

// Cosine bound of a frame's FP32 cap test in k_exact: cos(rad + kPadF) taken
// in FP64, less an absolute slack above the rounding of the FP32 dot product
// of two unit vectors (components rounded to FP32, three products and two
// sums: below 4e-7).  Taken in FP32 instead, cos(rad + pad) of a frame under
// ~3e-4 rad rounds to 1 and a body at its centre could fail the cap test.
__device__ __forceinline__ float cap_cos(double rad)
{
    return (rad >= kPi) ? -2.0f : (float)(cos(rad + (double)kPadF) - 2e-6);
}

__device__ __forceinline__ void set_flag(DevCounters *c, int bit) { atomicOr(&c->error_flags, 1 << bit); }

__device__ __forceinline__ double dot3(const double *a, const double *b)
{
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// warp-aggregated append: returns this lane's slot
__device__ __forceinline__ unsigned long long agg_append(unsigned long long *ctr)
{
    unsigned mask = __activemask();
    int leader = __ffs(mask) - 1;
    int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------------------
// frames
// ---------------------------------------------------------------------------
__global__ void k_frame_prep(const kete_frame *__restrict__ fr, int64_t nf, int64_t n_obs,
                             int32_t *__restrict__ is_start, double *__restrict__ fcen,
                             float4 *__restrict__ faux, DevCounters *ctr)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const kete_frame f = fr[i];
    bool start = (i == 0) || (fr[i - 1].exposure_id != f.exposure_id);
    is_start[i] = start ? 1 : 0;
    if (i > 0) {
        double pe = fr[i - 1].epoch;
        if (!(f.epoch >= pe)) set_flag(ctr, 0);
        if (!start && (pe != f.epoch || fr[i - 1].observer_idx != f.observer_idx)) set_flag(ctr, 1);
    }
    if (f.observer_idx < 0 || f.observer_idx >= n_obs) set_flag(ctr, 2);
    int ne = f.n_edges;
    if (ne != KETE_FRAME_CONE && (ne < 3 || ne > KETE_MAX_EDGES)) {
        set_flag(ctr, 3);
        ne = 3;
    }
    if (!isfinite(f.epoch)) set_flag(ctr, 4);
    if (f.n_edges == KETE_FRAME_CONE) {
        // cone: its own centre and radius
        const double cn = sqrt(dot3(f.normals[0], f.normals[0]));
        const double rho = f.normals[1][0];
        double cen[3] = {1.0, 0.0, 0.0}, rad = kPi;
        if (!(cn > 0.0) || !isfinite(cn) || !(rho > 0.0 && rho < kPi)) {
            set_flag(ctr, 4);
        } else {
            for (int c = 0; c < 3; c++) cen[c] = f.normals[0][c] / cn;
            rad = rho > 1.4 ? kPi : rho;   // as for polygons: wide cones cover everything
        }
        fcen[3 * i + 0] = cen[0];
        fcen[3 * i + 1] = cen[1];
        fcen[3 * i + 2] = cen[2];
        fcen[3 * nf + i] = rad;
        faux[i] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], cap_cos(rad));
        return;
    }
    // vertices: intersections n_a x n_b (either sign) that satisfy every
    // other half-space; independent of the order the edges are listed in
    double cen[3] = {0, 0, 0};
    double vx[2 * KETE_MAX_EDGES * (KETE_MAX_EDGES - 1) / 2][3];
    int nv = 0;
    bool bad = false;
    for (int a = 0; a < ne; a++) {
        double na = sqrt(dot3(f.normals[a], f.normals[a]));
        if (!(na > 0.0) || !isfinite(na)) bad = true;
        for (int b = a + 1; b < ne; b++) {
            const double *A = f.normals[a], *Bn = f.normals[b];
            double v[3] = {A[1] * Bn[2] - A[2] * Bn[1], A[2] * Bn[0] - A[0] * Bn[2],
                           A[0] * Bn[1] - A[1] * Bn[0]};
            double vn = sqrt(dot3(v, v));
            if (!(vn > 0.0)) continue;
            for (int sgn = 0; sgn < 2; sgn++) {
                double w[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
                if (sgn) { w[0] = -w[0]; w[1] = -w[1]; w[2] = -w[2]; }
                bool ok = true;
                for (int c = 0; c < ne; c++) {
                    if (c == a || c == b) continue;
                    double nc = sqrt(dot3(f.normals[c], f.normals[c]));
                    if (dot3(f.normals[c], w) < -1e-12 * nc) ok = false;
                }
                if (ok && nv < 2 * KETE_MAX_EDGES * (KETE_MAX_EDGES - 1) / 2) {
                    for (int q = 0; q < 3; q++) { vx[nv][q] = w[q]; cen[q] += w[q]; }
                    nv++;
                }
            }
        }
    }
    if (nv < 3) bad = true;
    double cn = sqrt(dot3(cen, cen));
    double rad = 0.0;
    if (bad || !(cn > 0.0)) {
        set_flag(ctr, 4);
        cen[0] = 1.0; cen[1] = 0.0; cen[2] = 0.0;
        rad = kPi;
    } else {
        for (int c = 0; c < 3; c++) cen[c] /= cn;
        for (int k = 0; k < nv; k++) {
            double d = fmin(1.0, fmax(-1.0, dot3(cen, vx[k])));
            rad = fmax(rad, acos(d));
        }
        // a polygon wider than ~80 deg is treated as covering everything
        if (rad > 1.4) rad = kPi;
    }
    fcen[3 * i + 0] = cen[0];
    fcen[3 * i + 1] = cen[1];
    fcen[3 * i + 2] = cen[2];
    fcen[3 * nf + i] = rad;
    faux[i] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], cap_cos(rad));
}

__global__ void k_exposure_first(const int32_t *__restrict__ is_start,
                                 const int64_t *__restrict__ ex, int64_t nf,
                                 int32_t *__restrict__ exp_first)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    if (is_start[i]) exp_first[ex[i]] = (int32_t)i;
    if (i == nf - 1) exp_first[ex[i] + is_start[i]] = (int32_t)nf;
}

__global__ void k_exposure_prep(EphemDev E, const kete_frame *__restrict__ fr, int64_t nf,
                                const double *__restrict__ observers,
                                const double *__restrict__ fcen, const int32_t *__restrict__ exp_first,
                                int64_t ne, ExpArrays X, unsigned int *max_rad_bits,
                                DevCounters *ctr)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int32_t f0 = exp_first[e], f1 = exp_first[e + 1];
    const kete_frame &f = fr[f0];
    X.epoch[e] = f.epoch;
    // the Sun at the exposure epoch: every candidate of the exposure re-adds it
    Seg g;
    double sp[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
    if (ephem_seg(E, f.epoch, 0.0, g))
        cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, sp, sv);
    else
        set_flag(ctr, 5);
    for (int c = 0; c < 3; c++) {
        X.sun[6 * e + c] = sp[c];
        X.sun[6 * e + 3 + c] = sv[c];
    }
    int64_t oi = f.observer_idx;
    for (int c = 0; c < 3; c++) X.obs[3 * e + c] = observers[3 * oi + c];
    double s[3] = {0, 0, 0};
    bool huge = false;
    for (int32_t k = f0; k < f1; k++) {
        for (int c = 0; c < 3; c++) s[c] += fcen[3 * k + c];
        if (fcen[3 * nf + k] >= kPi) huge = true;
    }
    double sn = sqrt(dot3(s, s));
    double rad = 0.0;
    if (!(sn > 0.0)) huge = true;
    else {
        for (int c = 0; c < 3; c++) s[c] /= sn;
        for (int32_t k = f0; k < f1; k++) {
            double d = fmin(1.0, fmax(-1.0, dot3(s, fcen + 3 * k)));
            rad = fmax(rad, acos(d) + fcen[3 * nf + k]);
        }
    }
    if (huge || rad > 1.4) {
        rad = kPi;
        s[0] = 1.0; s[1] = 0.0; s[2] = 0.0;
    }
    for (int c = 0; c < 3; c++) X.cen[3 * e + c] = s[c];
    X.cenf[e] = make_float4((float)s[0], (float)s[1], (float)s[2], 0.0f);
    X.rad[e] = rad;
    float r = (float)rad;
    X.cs[e] = make_float2(rad >= kPi ? -2.0f : cosf(r), rad >= kPi ? 0.0f : sinf(r));
    atomicMax(max_rad_bits, __float_as_uint(r));
}

// next[e]: first exposure that cannot join a batch starting at e (Sec. 2)
__global__ void k_batch_next(const double *__restrict__ ep, int64_t ne, double span,
                             int32_t *__restrict__ next)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double t0 = ep[e];
    int64_t lo = e + 1, hi = ne;   // first j in [lo, hi) with !(ep[j]==t0 || ep[j]-t0 < span)
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        double tj = ep[mid];
        bool joins = (tj == t0) || (tj - t0 < span);
        if (joins) lo = mid + 1;
        else hi = mid;
    }
    next[e] = (int32_t)lo;
}

__global__ void k_batch_walk(const double *__restrict__ ep, const int32_t *__restrict__ next,
                             int64_t ne, int32_t *__restrict__ batch_first,
                             double *__restrict__ t_ref, int32_t *n_batches)
{
    int32_t e = 0, k = 0;
    while (e < ne) {
        int32_t nx = next[e];
        batch_first[k] = e;
        t_ref[k] = 0.5 * (ep[e] + ep[nx - 1]);
        k++;
        e = nx;
    }
    batch_first[k] = (int32_t)ne;
    *n_batches = k;
}

// one block per batch: observer mean/spread, time spread, Sun state at t_ref
__global__ void k_batch_info(EphemDev E, ExpArrays X, BatchArrays B, int32_t n_batches,
                             DevCounters *ctr)
{
    const int k = blockIdx.x;
    if (k >= n_batches) return;
    const int32_t e0 = B.first[k], e1 = B.first[k + 1];
    const double tr = B.t_ref[k];
    __shared__ double red[4][32];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        s0 += X.obs[3 * e + 0];
        s1 += X.obs[3 * e + 1];
        s2 += X.obs[3 * e + 2];
        X.batch[e] = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; }
    __syncthreads();
    __shared__ double O[3];
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int q = 0; q < nw; q++) { a += red[0][q]; b += red[1][q]; c += red[2][q]; }
        double inv = 1.0 / (double)(e1 - e0);
        O[0] = a * inv; O[1] = b * inv; O[2] = c * inv;
    }
    __syncthreads();
    double robs = 0, tsp = 0, rmax = 0;
    for (int32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double d0 = X.obs[3 * e] - O[0], d1 = X.obs[3 * e + 1] - O[1], d2 = X.obs[3 * e + 2] - O[2];
        X.obs_rel[e] = make_float4((float)d0, (float)d1, (float)d2, 0.f);
        robs = fmax(robs, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
        tsp = fmax(tsp, fabs(X.epoch[e] - tr));
        rmax = fmax(rmax, X.rad[e]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        robs = fmax(robs, __shfl_xor_sync(0xffffffffu, robs, o));
        tsp = fmax(tsp, __shfl_xor_sync(0xffffffffu, tsp, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    __syncthreads();
    if (l == 0) { red[0][w] = robs; red[1][w] = tsp; red[2][w] = rmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int q = 0; q < nw; q++) {
            a = fmax(a, red[0][q]); b = fmax(b, red[1][q]); c = fmax(c, red[2][q]);
        }
        for (int q = 0; q < 3; q++) B.O[3 * k + q] = O[q];
        B.robs[k] = a * (1.0 + 1e-12) + 1e-12;
        B.tspan[k] = b;
        B.rmax[k] = c;
        Seg g;
        double p[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        if (ephem_seg(E, tr, 0.0, g)) {
            cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, p, v);
        } else {
            set_flag(ctr, 5);
        }
        for (int q = 0; q < 3; q++) { B.sun[6 * k + q] = p[q]; B.sun[6 * k + 3 + q] = v[q]; }
    }
}

// ---------------------------------------------------------------------------
// sky cells: latitude bands of height hb, n_j cells of longitude per band
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_of(const CellGrid &G, double lat, double lon)
{
    int j = (int)floor((lat + 0.5 * kPi) / G.hb);
    j = j < 0 ? 0 : (j >= G.n_bands ? G.n_bands - 1 : j);
    int nj = G.band_n[j];
    int i = (int)floor(lon / (kTwoPi / nj));
    i = i < 0 ? 0 : (i >= nj ? nj - 1 : i);
    return G.band_off[j] + i;
}

__global__ void k_cell_keys(ExpArrays X, CellGrid G, int32_t e_begin, int32_t e_end, int32_t k0,
                            int32_t *__restrict__ key, int32_t *__restrict__ cnt)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t e = e_begin + (int32_t)q;
    if (e >= e_end) return;
    const double *c = X.cen + 3 * e;
    double lat = asin(fmin(1.0, fmax(-1.0, c[2])));
    double lon = atan2(c[1], c[0]);
    if (lon < 0.0) lon += kTwoPi;
    int kk = (X.batch[e] - k0) * G.n_cells + cell_of(G, lat, lon);
    key[q] = kk;
    atomicAdd(&cnt[kk], 1);
}

__global__ void k_cell_scatter(int32_t e_begin, int32_t e_end, const int32_t *__restrict__ key,
                               const int64_t *__restrict__ start, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ cell_exp)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t e = e_begin + (int32_t)q;
    if (e >= e_end) return;
    int kk = key[q];
    int pos = atomicAdd(&cursor[kk], 1);
    cell_exp[start[kk] + pos] = e;
}

// ---------------------------------------------------------------------------
// candidates: an item is one (body, batch of the chunk); a warp shares the
// tests of its 32 items
// ---------------------------------------------------------------------------
struct CandCtx {
    ExpArrays X;
    BatchArrays B;
    CellGrid G;
    const double *stop_states;   // [C][n][6]: body i's state at batch k0 + kl
    int64_t n;
    int32_t k0, nk;              // chunk batches [k0, k0+nk)
    const int64_t *cell_start;   // [nk * n_cells + 1]
    const int32_t *cell_exp;
    uint2 *cand;                 // (exposure, body)
    unsigned long long cap;
    int32_t *exp_cnt;            // per exposure (global index)
    DevCounters *ctr;
    double mu_sun;
};

// Cap test of one exposure for a body at pb = p - O (FP32, relative to the
// batch's mean observer O): the body's apparent direction from the exposure's
// observer can move by at most asin(s/Q) during the batch, so the exposure is
// a candidate iff angle(pb - (o - O), centre) <= r + asin(s/Q) (+ padding for
// the FP32 rounding of the offsets, ~1e-7 of a few AU).
__device__ __forceinline__ void test_exposure(const CandCtx &C, int32_t e, const float pb[3],
                                              float s, int32_t body)
{
    const float4 o = C.X.obs_rel[e];
    const float q0 = pb[0] - o.x, q1 = pb[1] - o.y, q2 = pb[2] - o.z;
    const float Q = sqrtf(q0 * q0 + q1 * q1 + q2 * q2);
    const float2 cs = C.X.cs[e];
    bool pass;
    const float sig = s / Q;
    if (cs.x < -1.5f || sig >= 0.999f) {
        pass = true;
    } else {
        const float4 c = C.X.cenf[e];
        const float cosang = (q0 * c.x + q1 * c.y + q2 * c.z) / Q;
        const float cd = sqrtf(1.0f - sig * sig);
        const float lim = cs.x * cd - cs.y * sig;                 // cos(r + delta)
        pass = cosang >= lim - kPadF * (cs.y * cd + cs.x * sig) - 2e-6f - kPadF;
    }
    if (pass) {
        unsigned long long slot = agg_append(&C.ctr->candidates);
        if (slot < C.cap) C.cand[slot] = make_uint2((unsigned)e, (unsigned)body);
        atomicAdd(&C.exp_cnt[e], 1);
    }
}

// The runs of one item: contiguous ranges of exposure indices to test, either
// the whole batch (direct) or, band by band, the cells within R of the body's
// direction (indices into cell_exp).  A lane steps through its item's runs
// one at a time.
struct CandRuns {
    int mode;            // 0: none left, 1: direct range, 2: cell ranges
    int64_t a, b;        // current run [a, b)
    int j, jhi, r, nr;   // band, last band, piece of the band, pieces
    int rl0, rh0, rl1, rh1;   // cell index ranges of the band's pieces
    float lon, dlon;
    int64_t base;        // first cell key of the item's batch
};

// next non-empty run (or mode 0)
__device__ __forceinline__ void cand_next_run(const CandCtx &C, CandRuns &u)
{
    const CellGrid &G = C.G;
    while (u.mode == 2 && u.a >= u.b) {
        if (u.r >= u.nr) {
            if (++u.j > u.jhi) {
                u.mode = 0;
                break;
            }
            const int nj = G.band_n[u.j];
            const float w = (float)kTwoPi / nj;
            const int ilo = (int)floorf((u.lon - u.dlon) / w), ihi = (int)floorf((u.lon + u.dlon) / w);
            if (u.dlon >= (float)kPi || ihi - ilo + 1 >= nj) {
                u.rl0 = 0; u.rh0 = nj - 1; u.nr = 1;
            } else if (ilo < 0) {
                u.rl0 = 0; u.rh0 = ihi; u.rl1 = ilo + nj; u.rh1 = nj - 1; u.nr = 2;
            } else if (ihi >= nj) {
                u.rl0 = ilo; u.rh0 = nj - 1; u.rl1 = 0; u.rh1 = ihi - nj; u.nr = 2;
            } else {
                u.rl0 = ilo; u.rh0 = ihi; u.nr = 1;
            }
            u.r = 0;
        }
        const int64_t k0 = u.base + G.band_off[u.j];
        const int lo = u.r == 0 ? u.rl0 : u.rl1, hi = u.r == 0 ? u.rh0 : u.rh1;
        u.a = C.cell_start[k0 + lo];
        u.b = C.cell_start[k0 + hi + 1];
        u.r++;
    }
    if (u.mode == 1 && u.a >= u.b) u.mode = 0;
}

// Each lane sets up its item (the body's batch state, the conservative
// search radius, its runs); then the warp takes the tests of all 32 items 32
// at a time: slot q of a round goes to the lane whose pending tests cover it
// (a prefix sum over the lanes' counts and a 5-step search), so the lanes stay
// busy whatever the spread of the items' test counts -- a body near the
// observer that tests every exposure of its batch is shared by the warp.
// Every (item, exposure) pair is tested once, with its own item's geometry:
// the candidates are those of a thread-per-item scan.
__global__ void __launch_bounds__(256) k_candidates(CandCtx C)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_items = C.n * C.nk;
    if (idx - lane >= n_items) return;   // whole warps past the end
    CandRuns u;
    u.mode = 0;
    u.a = u.b = 0;
    float pb[3] = {0.0f, 0.0f, 0.0f}, s_eff = 0.0f;
    int32_t body = 0;
    if (idx < n_items) {
        const int32_t kl = (int32_t)(idx / C.n);
        const int32_t i = (int32_t)(idx - (int64_t)kl * C.n);
        const int32_t k = C.k0 + kl;
        body = i;
        const double *st = C.stop_states + ((int64_t)kl * C.n + i) * 6;
        const double p[3] = {st[0], st[1], st[2]};
        if (isfinite(p[0])) {
            const double v[3] = {st[3], st[4], st[5]};
            const double *O = C.B.O + 3 * k;
            const double *sun = C.B.sun + 6 * k;
            const float robs = (float)C.B.robs[k];
            // FP32 from here on: a conservative prefilter, padded for its rounding
            const float d[3] = {(float)(p[0] - O[0]), (float)(p[1] - O[1]), (float)(p[2] - O[2])};
            const float D = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const float h[3] = {(float)(p[0] - sun[0]), (float)(p[1] - sun[1]), (float)(p[2] - sun[2])};
            const float vh[3] = {(float)(v[0] - sun[3]), (float)(v[1] - sun[4]), (float)(v[2] - sun[5])};
            const float rh = sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
            const float vn = sqrtf(vh[0] * vh[0] + vh[1] * vh[1] + vh[2] * vh[2]);
            // time offsets from t_ref: frame epochs within tspan, light time below tau_max
            const float T = (float)C.B.tspan[k] + (D + robs + 1.0f) * (float)kInvC;
            // heliocentric displacement bound, valid while the body stays beyond rh/2
            const float disp = vn * T + 2.0f * (float)C.mu_sun * T * T / (rh * rh);
            const float s = (disp + (float)kSunSpeedMax * T) * 1.0001f + 1e-6f;
            const bool all = (disp > 0.5f * rh) || (s + robs >= 0.99f * D) || (D < 0.05f);
            const float rho = all ? (float)kPi : asinf((s + robs) / D);
            const float R = rho + (float)C.B.rmax[k] + 4.0f * kPadF;
            pb[0] = d[0]; pb[1] = d[1]; pb[2] = d[2];
            s_eff = all ? 1e30f : s;
            if (all || R >= 1.2f) {   // every exposure of the batch
                u.mode = 1;
                u.a = C.B.first[k];
                u.b = C.B.first[k + 1];
            } else {   // the cells within R of the body's direction from the mean observer
                const CellGrid &G = C.G;
                const float lat = asinf(fminf(1.0f, fmaxf(-1.0f, d[2] / D)));
                float lon = atan2f(d[1], d[0]);
                if (lon < 0.0f) lon += (float)kTwoPi;
                const float hb = (float)G.hb;
                int jlo = (int)floorf((lat - R + 0.5f * (float)kPi) / hb);
                int jhi = (int)floorf((lat + R + 0.5f * (float)kPi) / hb);
                jlo = jlo < 0 ? 0 : jlo;
                jhi = jhi >= G.n_bands ? G.n_bands - 1 : jhi;
                u.lon = lon;
                if (fabsf(lat) + R >= 0.5f * (float)kPi - 1e-4f) u.dlon = (float)kPi;
                else u.dlon = asinf(fminf(1.0f, sinf(R) / cosf(lat))) + 4.0f * kPadF;
                u.mode = 2;
                u.j = jlo - 1;
                u.jhi = jhi;
                u.r = u.nr = 0;
                u.base = (int64_t)kl * G.n_cells;
            }
        }
    }
    for (;;) {
        cand_next_run(C, u);
        const int cnt = u.mode ? (int)min(u.b - u.a, (int64_t)32) : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        if (total == 0) break;
        const int excl = incl - cnt;
        // owner of slot `lane`: the first lane whose inclusive count exceeds it
        int own = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int v = __shfl_sync(FULL, incl, own + step - 1);
            if (v <= lane) own += step;
        }
        own = own > 31 ? 31 : own;
        const int off = lane - __shfl_sync(FULL, excl, own);
        const int64_t a_o = __shfl_sync(FULL, u.a, own);
        const int mode_o = __shfl_sync(FULL, u.mode, own);
        const float q[3] = {__shfl_sync(FULL, pb[0], own), __shfl_sync(FULL, pb[1], own),
                            __shfl_sync(FULL, pb[2], own)};
        const float s_o = __shfl_sync(FULL, s_eff, own);
        const int32_t body_o = __shfl_sync(FULL, body, own);
        if (lane < total) {
            const int32_t e = mode_o == 1 ? (int32_t)(a_o + off) : C.cell_exp[a_o + off];
            test_exposure(C, e, q, s_o, body_o);
        }
        // each lane's tests taken in this pass of the loop
        const int taken = min(max(32 - excl, 0), cnt);
        u.a += taken;
    }
}

__global__ void k_cand_scatter(const uint2 *__restrict__ cand, unsigned long long nc,
                               const int64_t *__restrict__ exp_off, int32_t e_begin,
                               int32_t *__restrict__ cursor, int32_t *__restrict__ cand_body)
{
    unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    uint2 c = cand[q];
    int32_t el = (int32_t)c.x - e_begin;
    int pos = atomicAdd(&cursor[el], 1);
    cand_body[exp_off[el] + pos] = (int32_t)c.y;
}

// ---------------------------------------------------------------------------
// exact test: one thread per candidate (exposure, body) pair
// ---------------------------------------------------------------------------
struct ExactCtx {
    EphemDev E;
    ExpArrays X;
    BatchArrays B;
    const kete_frame *frames;
    const float4 *faux;
    const double *stop_states;
    int64_t n;
    int32_t k0, e_begin, e_end;
    const int64_t *exp_off;      // chunk-relative
    int64_t n_cand;              // candidates of the chunk (exp_off[e_end - e_begin])
    const int32_t *cand_body;
    const int32_t *exp_first;
    kete_hit *hits;
    unsigned long long cap;
    int32_t *frame_cnt;
    int32_t *status;
    DevCounters *ctr;
    double cos_eps, sin_eps;
    const kete_mag_params *mag;
    uint32_t *keep;                     // candidates kept by the prefilter (null: all)
    unsigned long long *n_keep;
};

// The exposure, batch and body of candidate q and the body's heliocentric
// batch state (shared by the prefilter and the exact test).
struct CandSetup {
    int32_t e, k, kl, f0, f1, i;
    double dt_obs, o[3], sun_obs[6], hr[3], hv[3];
};

__device__ __forceinline__ void cand_setup(const ExactCtx &C, int64_t q, CandSetup &S)
{
    const int32_t nexp = C.e_end - C.e_begin;
    // the exposure of candidate q: the last el with exp_off[el] <= q
    int32_t lo = 0, hi = nexp - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(C.exp_off + mid) <= q) lo = mid;
        else hi = mid - 1;
    }
    const int32_t e = C.e_begin + lo;
    S.e = e;
    S.k = C.X.batch[e];
    S.kl = S.k - C.k0;
    S.dt_obs = C.X.epoch[e] - C.B.t_ref[S.k];
#pragma unroll
    for (int c = 0; c < 3; c++) S.o[c] = C.X.obs[3 * e + c];
#pragma unroll
    for (int c = 0; c < 6; c++) S.sun_obs[c] = C.X.sun[6 * e + c];
    S.f0 = C.exp_first[e];
    S.f1 = C.exp_first[e + 1];
    S.i = C.cand_body[q];
    const double *st = C.stop_states + ((int64_t)S.kl * C.n + S.i) * 6;
    const double *sun = C.B.sun + 6 * S.k;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        S.hr[c] = st[c] - sun[c];
        S.hv[c] = st[3 + c] - sun[3 + c];
    }
}

// Apparent magnitude (Sec. 3.3; comet appendix) from the heliocentric
// position p of the body at emission and the apparent vector u (|u| = dl):
// H-G V = H + 5 log10(r dl) - 2.5 log10((1-G) Phi1 + G Phi2) with
// Phi_i = exp(-A_i tan(alpha/2)^B_i), A = (3.33, 1.87), B = (0.63, 1.22);
// comets M + 5 log10(dl) + K log10(r) (+ 0.035 per degree of phase for the
// nucleus).  The half-angle tangent comes from the FP64 cross and dot
// products, tan(alpha/2) = |p x u| / (r dl + p.u): an FP32 arc cosine of the
// cosine would lose alpha to ~3e-4 rad near opposition, where the H-G phase
// function is steepest (its slope in tan(alpha/2) is unbounded at zero).  The
// laws themselves run in FP32 (a magnitude needs ~1e-4).
__device__ __forceinline__ float apparent_mag(const kete_mag_params &P, const double p[3],
                                              const double u[3], double dl)
{
    if (P.kind < KETE_MAG_HG || P.kind > KETE_MAG_COMET_NUCLEUS)
        return __int_as_float(0x7fc00000);
    const double r = sqrt(dot3(p, p));
    const double cx = p[1] * u[2] - p[2] * u[1], cy = p[2] * u[0] - p[0] * u[2],
                 cz = p[0] * u[1] - p[1] * u[0];
    const float t = (float)(sqrt(cx * cx + cy * cy + cz * cz) / fma(r, dl, dot3(p, u)));
    const float lr = log10f((float)r), ld = log10f((float)dl);
    const float p1 = (float)P.p1, p2 = (float)P.p2;
    if (P.kind == KETE_MAG_HG) {
        const float phi1 = expf(-3.33f * powf(t, 0.63f));
        const float phi2 = expf(-1.87f * powf(t, 1.22f));
        return p1 + 5.f * (lr + ld) - 2.5f * log10f((1.f - p2) * phi1 + p2 * phi2);
    }
    float m = p1 + 5.f * ld + p2 * lr;
    if (P.kind == KETE_MAG_COMET_NUCLEUS) m += 0.035f * (2.f * atanf(t) * (180.f / (float)kPi));
    return m;
}

// Position at t_ref + dt_obs - tau.  The heliocentric two-body state is
// solved once, at dt_obs (universal variables from the batch state); the
// light-time iterations move it back by tau with its Taylor expansion,
//   r(dt_obs - tau) = r - v tau + a tau^2 / 2 - j tau^3 / 6,
// a = -mu r / |r|^3, j = da/dt.  The first neglected term is tau^4 |r4| / 24;
// differentiating a twice more with |r.v| <= |r||v| and d(r.v)/dt = v^2 -
// mu/|r| bounds the fourth derivative by |r4| <= 4 mu (mu/|r| + 6 v^2) / |r|^4.
// With twice that bound (the expansion point moves by v tau) the term is
// below tau^4 mu (mu / |r| + 6 v^2) / (3 |r|^4); main-belt bodies give ~1e-17
// AU, bodies at 0.2 AU from the Sun ~1e-13 AU, a sungrazer at 0.01 AU ~1e-7
// AU.  Where the bound exceeds kTaylorMaxAu (lt_taylor_poor), k_exact solves
// the two-body problem at every light-time iterate instead, as the definition
// does.  The Sun at t_obs -
// tau comes from its state at the exposure epoch, S - V tau (the neglected
// term, a_sun tau^2 / 2 with |a_sun| ~ 1e-8 AU/day^2, stays below 2e-11 AU
// for tau < 0.06 day).
constexpr double kTaylorMaxAu = 1e-13;
struct TwoBodyLT {
    double r[3], mv[3], a2[3], mj6[3];   // r, -v, a/2, -j/6 at dt_obs
    double ri;                           // 1 / |r|
};

// the bound above exceeds kTaylorMaxAu (compared without the division)
__device__ __forceinline__ bool lt_taylor_poor(double mu, const TwoBodyLT &T, double tau)
{
    const double rr = dot3(T.r, T.r);
    const double vv = dot3(T.mv, T.mv);
    const double t2 = tau * tau;
    return t2 * t2 * mu * fma(mu, T.ri, 6.0 * vv) > (3.0 * kTaylorMaxAu) * (rr * rr);
}

__device__ __forceinline__ bool twobody_at(double mu, double sqmu, const double hr[3],
                                           const double hv[3], double dt_obs, double &chi,
                                           TwoBodyLT &T)
{
    double v[3];
    const bool ok = kepler_uv(mu, sqmu, hr, hv, dt_obs, chi, T.r, v);
    const double rr = dot3(T.r, T.r);
    const double ri = rsqrt(rr), ri2 = ri * ri;
    T.ri = ri;
    const double k = -mu * ri2 * ri;
    const double q = 3.0 * dot3(T.r, v) * ri2;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T.mv[c] = -v[c];
        T.a2[c] = 0.5 * k * T.r[c];
        T.mj6[c] = -(k / 6.0) * fma(-q, T.r[c], v[c]);
    }
    return ok;
}

__device__ __forceinline__ void twobody_pos(const TwoBodyLT &T, const double *sun_obs, double tau,
                                            double pos[3])
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double p = fma(fma(fma(T.mj6[c], tau, T.a2[c]), tau, T.mv[c]), tau, T.r[c]);
        pos[c] = fma(-tau, sun_obs[3 + c], sun_obs[c]) + p;
    }
}

// Candidates are grouped by exposure (CSR exp_off), so neighbouring threads
// mostly share an exposure and its data; every lane has a candidate of its
// own whatever the exposures' candidate counts.
// FP32 prefilter of a candidate before its two-body solve.  From the
// body's heliocentric batch state (hr, hv) a second-order Taylor step gives
// its position at the exposure epoch, retarded by the light time as the exact
// path does (p(t - tau) ~ p(t) - tau v(t), the Sun moved by -tau v_sun).  The
// distance E to the exact position is bounded by
//   J s^3 / 6 + a_max tau^2 / 2           (Taylor remainder, s = |dt| + tau;
//                                          J = 4 mu v_max / r_min^3 bounds
//                                          |da/dt| of two-body motion)
// + FP32 rounding (and the light time's own error, a relative 1e-3 of it),
// valid while the body stays beyond r_min = r/2 (displacement within the
// interval below r/2; otherwise no cheap bound and the candidate goes on).
// The predicted direction is then within theta = E / (|u| - E) of the exact
// one, so a candidate whose predicted direction misses every sub-field's
// FP32 cap by more than theta (plus the FP32 dot products' rounding) fails
// the exact path's cap test too, and is not a hit.
// An exposure of several sub-fields is tested first against its covering cap
// (radius rad >= angle(centre, c_k) + r_k for every sub-field k): a direction
// that passes sub-field k's FP32 test is within r_k + kPadF + 3e-3 of c_k
// (the test's 2e-6 cosine slack plus FP32 rounding widen the angle by at most
// sqrt(2 x 2.4e-6) < 3e-3), hence within rad + kPadF + 3e-3 of the centre, and
// the predicted direction within theta more.
__device__ __forceinline__ bool exact_prefilter(const ExactCtx &C, int32_t e, const double hr[3],
                                                const double hv[3], double dt,
                                                const double sun_obs[6], const double o[3],
                                                int32_t f0, int32_t f1, double mu)
{
    const float muf = (float)mu;
    const float r[3] = {(float)hr[0], (float)hr[1], (float)hr[2]};
    const float v[3] = {(float)hv[0], (float)hv[1], (float)hv[2]};
    const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const float rn = sqrtf(rr);
    const float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float adt = fabsf((float)dt);
    const float so[3] = {(float)(sun_obs[0] - o[0]), (float)(sun_obs[1] - o[1]),
                         (float)(sun_obs[2] - o[2])};
    const float son = sqrtf(so[0] * so[0] + so[1] * so[1] + so[2] * so[2]);
    // light time bound: the body is within rn + son + motion of the observer
    const float tmax = (rn + son + vn * adt + 1.0f) * (float)kInvC * 1.01f;
    const float s = adt + tmax;
    const float rmin = 0.5f * rn;
    const float amax = muf / (rmin * rmin);
    if (!(vn * s + 0.5f * amax * s * s <= rmin)) return true;   // no cheap bound
    const float vmax = vn + amax * s;
    const float J = 4.0f * muf * vmax / (rmin * rmin * rmin);
    // position at the exposure epoch (heliocentric, FP32)
    const float dtf = (float)dt;
    const float k = -muf / (rr * rn);                  // a = k r
    const float h2 = 0.5f * dtf * dtf * k;
    float p[3], vt[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        p[c] = fmaf(v[c], dtf, fmaf(h2, r[c], r[c]));
        vt[c] = fmaf(k * dtf, r[c], v[c]) + (float)sun_obs[3 + c];   // body + Sun velocity
    }
    float u[3] = {so[0] + p[0], so[1] + p[1], so[2] + p[2]};
    float tau = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * (float)kInvC;
#pragma unroll
    for (int it = 0; it < 2; it++) {
        float w[3];
#pragma unroll
        for (int c = 0; c < 3; c++) w[c] = fmaf(-tau, vt[c], u[c]);
        tau = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]) * (float)kInvC;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fmaf(-tau, vt[c], u[c]);
    const float un = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    // bound on the distance to the exact retarded position; the light time's
    // own error (that distance over c) moves the position by at most
    // |v| / c < 1e-3 of it, hence the factor
    const float E = 1.001f * (J * s * s * s * (1.0f / 6.0f) + 0.5f * amax * tmax * tmax +
                              2e-6f * (rn + son + un + vn * adt)) + 1e-9f;
    if (!(E < 0.5f * un)) return true;
    const float theta = E / (un - E) + 2e-6f;
    const float iu = 1.0f / un;
    const float uh[3] = {u[0] * iu, u[1] * iu, u[2] * iu};
    if (f1 - f0 > 1) {
        const float2 cs = C.X.cs[e];
        if (cs.x > -1.5f) {
            const float phi = kPadF + 3e-3f + theta;
            const float lim = cs.x * cosf(phi) - cs.y * sinf(phi) - 2e-6f;   // cos(rad + phi)
            const float4 c = C.X.cenf[e];
            if (c.x * uh[0] + c.y * uh[1] + c.z * uh[2] < lim) return false;
        }
    }
    for (int32_t f = f0; f < f1; f++) {
        const float4 a = __ldg(C.faux + f);
        if (a.x * uh[0] + a.y * uh[1] + a.z * uh[2] >= a.w - theta) return true;
    }
    return false;
}

// The prefilter pass: thread per candidate; the candidates it keeps are
// appended to C.keep (warp-aggregated), so that the exact pass runs them with
// full lanes (an FP64 warp instruction costs the same whatever its active
// lanes: a rejection inside the exact pass would save nothing).
__global__ void __launch_bounds__(128) k_exact_prefilter(ExactCtx C)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= C.n_cand) return;
    CandSetup S;
    cand_setup(C, q, S);
    if (exact_prefilter(C, S.e, S.hr, S.hv, S.dt_obs, S.sun_obs, S.o, S.f0, S.f1, C.E.gm[0])) {
        const unsigned long long slot = agg_append(C.n_keep);
        C.keep[slot] = (uint32_t)q;
    }
}

__global__ void __launch_bounds__(128) k_exact(ExactCtx C)
{
    const double mu = C.E.gm[0];
    const double sqmu = sqrt(mu);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_work = C.keep ? (int64_t)*C.n_keep : C.n_cand;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_work; j += stride) {
        const int64_t q = C.keep ? (int64_t)C.keep[j] : j;
        CandSetup S;
        cand_setup(C, q, S);
        const int32_t f0 = S.f0, f1 = S.f1, i = S.i;
        const double dt_obs = S.dt_obs;
        const double *o = S.o, *sun_obs = S.sun_obs, *hr = S.hr, *hv = S.hv;
        {
            // light delay (Sec. 2): tau0 = |r(t)-o|/c, three fixed iterations
            double chi = 0.0, pos[3];
            TwoBodyLT T;
            bool ok = twobody_at(mu, sqmu, hr, hv, dt_obs, chi, T);
            // twobody_pos at tau = 0
#pragma unroll
            for (int c = 0; c < 3; c++) pos[c] = sun_obs[c] + T.r[c];
            double u[3] = {pos[0] - o[0], pos[1] - o[1], pos[2] - o[2]};
            double tau = sqrt(dot3(u, u)) * kInvC;
            // near the Sun the cubic is not good enough: solve at every iterate
            const bool exact_lt = lt_taylor_poor(mu, T, 1.01 * tau);
            for (int it = 0; it < 4; it++) {
                if (exact_lt) {
                    double rk[3], vk[3];
                    ok = kepler_uv(mu, sqmu, hr, hv, dt_obs - tau, chi, rk, vk) && ok;
#pragma unroll
                    for (int c = 0; c < 3; c++) pos[c] = fma(-tau, sun_obs[3 + c], sun_obs[c]) + rk[c];
                } else {
                    twobody_pos(T, sun_obs, tau, pos);
                }
                u[0] = pos[0] - o[0]; u[1] = pos[1] - o[1]; u[2] = pos[2] - o[2];
                if (it < 3) tau = sqrt(dot3(u, u)) * kInvC;
            }
            if (!ok) {
                if (C.status) atomicCAS(&C.status[i], KETE_BODY_OK, KETE_BODY_KEPLER_CAP);
                continue;   // next candidate of this thread
            }
            const double uu = dot3(u, u);
            const double un = sqrt(uu);
            const double iun = rsqrt(uu);   // for the FP32 direction only
            const float uf[3] = {(float)(u[0] * iun), (float)(u[1] * iun), (float)(u[2] * iun)};
            bool have_radec = false;
            double ra = 0.0, dec = 0.0;
            // Sub-fields 64 at a time: first the FP32 cap tests of all of them
            // into a mask, then the exact tests of this lane's passing ones
            // only -- each pass of the second loop gives every lane a
            // sub-field of its own, where a loop over the sub-fields would run
            // the FP64 test whenever any lane of the warp passed a cap.
            for (int32_t fb = f0; fb < f1; fb += 64) {
                const int32_t nfb = min(64, f1 - fb);
                unsigned long long pass = 0ull;
                for (int32_t j = 0; j < nfb; j++) {
                    const float4 a = __ldg(C.faux + fb + j);
                    if (a.x * uf[0] + a.y * uf[1] + a.z * uf[2] >= a.w) pass |= 1ull << j;
                }
                while (pass) {
                    const int32_t f = fb + __ffsll((long long)pass) - 1;
                    pass &= pass - 1ull;
                    const kete_frame &fr = C.frames[f];
                    bool inside = true;
                    if (fr.n_edges == KETE_FRAME_CONE) {
                        // angle(u, centre) < r  <=>  c.u > |c| |u| cos r
                        const double *cv = fr.normals[0];
                        const double cn = sqrt(dot3(cv, cv));
                        inside = fma(cv[0], u[0], fma(cv[1], u[1], cv[2] * u[2])) >
                                 cos(fr.normals[1][0]) * cn * un;
                    }
                    for (int kq = 0; kq < fr.n_edges; kq++) {
                        const double *nv = fr.normals[kq];
                        if (!(fma(nv[0], u[0], fma(nv[1], u[1], nv[2] * u[2])) > 0.0)) inside = false;
                    }
                    if (!inside) continue;
                    if (!have_radec) {
                        radec(u, C.cos_eps, C.sin_eps, ra, dec);
                        have_radec = true;
                    }
                    unsigned long long slot = agg_append(&C.ctr->hits);
                    if (slot < C.cap) {
                        kete_hit hh;
                        hh.frame = f;
                        hh.body = i;
                        hh.mag = __int_as_float(0x7fc00000);
                        if (C.mag) {
                            // heliocentric position at emission: pos minus the Sun there
                            const double ph[3] = {pos[0] - fma(-tau, sun_obs[3], sun_obs[0]),
                                                  pos[1] - fma(-tau, sun_obs[4], sun_obs[1]),
                                                  pos[2] - fma(-tau, sun_obs[5], sun_obs[2])};
                            hh.mag = apparent_mag(C.mag[i], ph, u, un);
                        }
                        hh.ra = ra;
                        hh.dec = dec;
                        C.hits[slot] = hh;
                    }
                    atomicAdd(&C.frame_cnt[f], 1);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// ordering: group hits by frame, sort each frame's hits by body
// ---------------------------------------------------------------------------
__global__ void k_hit_scatter(const kete_hit *__restrict__ src, unsigned long long nh,
                              const int64_t *__restrict__ frame_off, int32_t *__restrict__ cursor,
                              kete_hit *__restrict__ dst)
{
    unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nh) return;
    kete_hit h = src[q];
    int pos = atomicAdd(&cursor[h.frame], 1);
    dst[frame_off[h.frame] + pos] = h;
}

// warp per frame: rank of each hit = number of hits of the frame with a
// smaller body index (body indices are unique within a frame)
__global__ void k_hit_rank(const kete_hit *__restrict__ src, const int64_t *__restrict__ frame_off,
                           int64_t nf, kete_hit *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t f = warp; f < nf; f += nwarps) {
        const int64_t a = frame_off[f], b = frame_off[f + 1];
        const int64_t m = b - a;
        if (m == 0) continue;
        if (m == 1) {
            if (lane == 0) dst[a] = src[a];
            continue;
        }
        for (int64_t j = lane; j < m; j += 32) {
            const int32_t bj = src[a + j].body;
            int64_t rank = 0;
            for (int64_t q = 0; q < m; q++) rank += (src[a + q].body < bj) ? 1 : 0;
            dst[a + rank] = src[a + j];
        }
    }
}

// ---------------------------------------------------------------------------
// extended exposures (Sec. 3.1: an exposure of finite length is approximated
// by several instantaneous observations along it)
// ---------------------------------------------------------------------------
// Exposure starts of the caller's frames, and their checks: bit 0 epochs not
// sorted, bit 1 an exposure's frames differ in epoch, observer or duration,
// bit 2 observer rows out of range, bit 6 a negative or non-finite duration.
__global__ void k_ext_starts(const kete_frame *__restrict__ fr, const double *__restrict__ dur,
                             int64_t nf, int n_sub, int64_t n_obs, int32_t *__restrict__ is_start,
                             DevCounters *ctr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const double ep = fr[i].epoch, d = dur[i];
    const int64_t oi = fr[i].observer_idx;
    const bool start = (i == 0) || (fr[i - 1].exposure_id != fr[i].exposure_id);
    is_start[i] = start ? 1 : 0;
    if (i > 0) {
        if (!(ep >= fr[i - 1].epoch)) set_flag(ctr, 0);
        if (!start && (fr[i - 1].epoch != ep || fr[i - 1].observer_idx != oi || dur[i - 1] != d))
            set_flag(ctr, 1);
    }
    if (oi < 0 || oi > n_obs - n_sub) set_flag(ctr, 2);
    if (!(d >= 0.0) || !isfinite(d)) set_flag(ctr, 6);
}

// Sub-frame k of frame f (exposure starting at frame f0, S frames): index
// f0 n_sub + k S + (f - f0), epoch t + ((k + 1/2) d) / n_sub, observer row
// observer_idx + k, exposure f0 n_sub + k -- so the sub-frames of sub-interval
// k of one exposure form one contiguous exposure, in epoch order.
__global__ void k_ext_expand(const kete_frame *__restrict__ fr, const double *__restrict__ dur,
                             int64_t nf, int n_sub, const int32_t *__restrict__ is_start,
                             const int64_t *__restrict__ ex, const int32_t *__restrict__ exp_first,
                             kete_frame *__restrict__ sub, int32_t *__restrict__ parent)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int64_t e = ex[f] + is_start[f] - 1;   // starts up to and including f, less one
    const int64_t f0 = exp_first[e], S = exp_first[e + 1] - f0;
    const int64_t base = f0 * n_sub;
    const kete_frame src = fr[f];
    const double d = dur[f];
    for (int k = 0; k < n_sub; k++) {
        kete_frame o = src;
        o.epoch = src.epoch + ((k + 0.5) * d) / (double)n_sub;
        o.observer_idx = src.observer_idx + k;
        o.exposure_id = base + k;
        const int64_t j = base + (int64_t)k * S + (f - f0);
        sub[j] = o;
        parent[j] = (int32_t)f;
    }
}

// hits of the sub-frames per parent frame
__global__ void k_merge_count(const kete_hit *__restrict__ h, unsigned long long nh,
                              const int32_t *__restrict__ parent, int32_t *__restrict__ cnt)
{
    const unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nh) return;
    atomicAdd(&cnt[parent[h[q].frame]], 1);
}

__global__ void k_merge_scatter(const kete_hit *__restrict__ h, unsigned long long nh,
                                const int32_t *__restrict__ parent, const int64_t *__restrict__ off,
                                int32_t *__restrict__ cur, kete_hit *__restrict__ grouped)
{
    const unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nh) return;
    const kete_hit x = h[q];
    const int32_t p = parent[x.frame];
    grouped[off[p] + atomicAdd(&cur[p], 1)] = x;   // frame still names the sub-frame
}

// Warp per parent frame: a hit is kept iff no hit of the same body comes from
// an earlier sub-frame (sub-frame indices grow with time within a frame).
__global__ void k_merge_keep(const kete_hit *__restrict__ g, const int64_t *__restrict__ off,
                             int64_t np, int8_t *__restrict__ keep, int32_t *__restrict__ kept_cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < np; p += nwarps) {
        const int64_t a = off[p], m = off[p + 1] - a;
        int32_t c = 0;
        for (int64_t j = lane; j < m; j += 32) {
            const int32_t bj = g[a + j].body;
            const int64_t sj = g[a + j].frame;
            bool first = true;
            for (int64_t q = 0; q < m; q++)
                if (g[a + q].body == bj && g[a + q].frame < sj) first = false;
            keep[a + j] = first ? 1 : 0;
            c += first ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) kept_cnt[p] = c;
    }
}

// Warp per parent frame: kept hits in body order at out[kept_off[p] + rank],
// renamed to the parent frame.
__global__ void k_merge_place(const kete_hit *__restrict__ g, const int64_t *__restrict__ off,
                              const int8_t *__restrict__ keep, const int64_t *__restrict__ kept_off,
                              int64_t np, kete_hit *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < np; p += nwarps) {
        const int64_t a = off[p], m = off[p + 1] - a;
        for (int64_t j = lane; j < m; j += 32) {
            if (!keep[a + j]) continue;
            const int32_t bj = g[a + j].body;
            int64_t rank = 0;
            for (int64_t q = 0; q < m; q++) rank += (keep[a + q] && g[a + q].body < bj) ? 1 : 0;
            kete_hit x = g[a + j];
            x.frame = p;
            out[kept_off[p] + rank] = x;
        }
    }
}

// ---------------------------------------------------------------------------
static unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

#define KLAUNCH(...)                            \
    do {                                        \
        __VA_ARGS__;                            \
        cudaError_t _e = cudaGetLastError();    \
        if (_e != cudaSuccess) return _e;       \
    } while (0)

cudaError_t fov_frame_prep(const kete_frame *frames, int64_t nf, int64_t n_obs, int32_t *is_start,
                           double *fcen, float4 *faux, DevCounters *ctr, cudaStream_t st)
{
    if (nf > 0) KLAUNCH(k_frame_prep<<<grid_for(nf, 128), 128, 0, st>>>(frames, nf, n_obs, is_start, fcen, faux, ctr));
    return cudaSuccess;
}

cudaError_t fov_exposure_first(const int32_t *is_start, const int64_t *ex, int64_t nf,
                               int32_t *exp_first, cudaStream_t st)
{
    if (nf > 0) KLAUNCH(k_exposure_first<<<grid_for(nf, 256), 256, 0, st>>>(is_start, ex, nf, exp_first));
    return cudaSuccess;
}

cudaError_t fov_exposure_prep(const EphemDev &E, const kete_frame *frames, int64_t nf,
                              const double *observers, const double *fcen,
                              const int32_t *exp_first, int64_t ne, ExpArrays X,
                              unsigned int *max_rad_bits, DevCounters *ctr, cudaStream_t st)
{
    if (ne > 0) KLAUNCH(k_exposure_prep<<<grid_for(ne, 128), 128, 0, st>>>(E, frames, nf, observers, fcen, exp_first, ne, X, max_rad_bits, ctr));
    return cudaSuccess;
}

cudaError_t fov_batches(const double *ep, int64_t ne, double span, int32_t *next,
                        BatchArrays B, int32_t *n_batches, cudaStream_t st)
{
    if (ne <= 0) return cudaSuccess;
    KLAUNCH(k_batch_next<<<grid_for(ne, 256), 256, 0, st>>>(ep, ne, span, next));
    KLAUNCH(k_batch_walk<<<1, 1, 0, st>>>(ep, next, ne, B.first, B.t_ref, n_batches));
    return cudaSuccess;
}

cudaError_t fov_batch_info(const EphemDev &E, ExpArrays X, BatchArrays B, int32_t nb,
                           DevCounters *ctr, cudaStream_t st)
{
    if (nb > 0) KLAUNCH(k_batch_info<<<nb, 256, 0, st>>>(E, X, B, nb, ctr));
    return cudaSuccess;
}

cudaError_t fov_cell_keys(ExpArrays X, CellGrid G, int32_t e0, int32_t e1, int32_t k0,
                          int32_t *key, int32_t *cnt, cudaStream_t st)
{
    if (e1 > e0) KLAUNCH(k_cell_keys<<<grid_for(e1 - e0, 256), 256, 0, st>>>(X, G, e0, e1, k0, key, cnt));
    return cudaSuccess;
}

cudaError_t fov_cell_scatter(int32_t e0, int32_t e1, const int32_t *key, const int64_t *start,
                             int32_t *cursor, int32_t *cell_exp, cudaStream_t st)
{
    if (e1 > e0) KLAUNCH(k_cell_scatter<<<grid_for(e1 - e0, 256), 256, 0, st>>>(e0, e1, key, start, cursor, cell_exp));
    return cudaSuccess;
}

cudaError_t fov_candidates(const CandArgs &a, cudaStream_t st)
{
    CandCtx C;
    C.X = a.X; C.B = a.B; C.G = a.G; C.stop_states = a.stop_states; C.n = a.n; C.k0 = a.k0;
    C.nk = a.nk; C.cell_start = a.cell_start; C.cell_exp = a.cell_exp; C.cand = a.cand;
    C.cap = a.cap; C.exp_cnt = a.exp_cnt; C.ctr = a.ctr; C.mu_sun = a.mu_sun;
    int64_t tot = a.n * (int64_t)a.nk;
    if (tot > 0) KLAUNCH(k_candidates<<<grid_for(tot, 256), 256, 0, st>>>(C));
    return cudaSuccess;
}

cudaError_t fov_cand_scatter(const uint2 *cand, unsigned long long nc, const int64_t *exp_off,
                             int32_t e_begin, int32_t *cursor, int32_t *cand_body, cudaStream_t st)
{
    if (nc > 0) KLAUNCH(k_cand_scatter<<<grid_for((int64_t)nc, 256), 256, 0, st>>>(cand, nc, exp_off, e_begin, cursor, cand_body));
    return cudaSuccess;
}

cudaError_t fov_exact(const ExactArgs &a, int n_sm, cudaStream_t st)
{
    ExactCtx C;
    C.E = a.E; C.X = a.X; C.B = a.B; C.frames = a.frames; C.faux = a.faux;
    C.stop_states = a.stop_states; C.n = a.n; C.k0 = a.k0; C.e_begin = a.e_begin;
    C.e_end = a.e_end; C.exp_off = a.exp_off; C.n_cand = a.n_cand; C.cand_body = a.cand_body;
    C.exp_first = a.exp_first; C.hits = a.hits; C.cap = a.cap; C.frame_cnt = a.frame_cnt;
    C.status = a.status; C.ctr = a.ctr; C.mag = a.mag;
    // the prefilter stores 32-bit candidate indices
    const bool pre = a.keep && a.n_keep && a.n_cand <= (int64_t)UINT32_MAX;
    C.keep = pre ? a.keep : nullptr;
    C.n_keep = pre ? a.n_keep : nullptr;
    const double eps = 84381.448 / 3600.0 * (kPi / 180.0);
    C.cos_eps = cos(eps);
    C.sin_eps = sin(eps);
    int64_t nexp = a.e_end - a.e_begin;
    if (nexp <= 0 || a.n_cand <= 0) return cudaSuccess;
    if (pre) {
        const cudaError_t e = cudaMemsetAsync(a.n_keep, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        KLAUNCH(k_exact_prefilter<<<(unsigned)((a.n_cand + 127) / 128), 128, 0, st>>>(C));
    }
    int64_t blocks = (a.n_cand + 127) / 128;
    int64_t cap_blocks = (int64_t)n_sm * 16;
    if (blocks > cap_blocks) blocks = cap_blocks;
    KLAUNCH(k_exact<<<(unsigned)blocks, 128, 0, st>>>(C));
    return cudaSuccess;
}

cudaError_t fov_order_hits(const kete_hit *tmp, unsigned long long nh, const int64_t *frame_off,
                           int64_t nf, int32_t *cursor, kete_hit *grouped, kete_hit *out,
                           int n_sm, cudaStream_t st)
{
    if (nh == 0) return cudaSuccess;
    KLAUNCH(k_hit_scatter<<<grid_for((int64_t)nh, 256), 256, 0, st>>>(tmp, nh, frame_off, cursor, grouped));
    int64_t blocks = (nf * 32 + 255) / 256;
    if (blocks > (int64_t)n_sm * 32) blocks = (int64_t)n_sm * 32;
    KLAUNCH(k_hit_rank<<<(unsigned)blocks, 256, 0, st>>>(grouped, frame_off, nf, out));
    return cudaSuccess;
}

cudaError_t fov_ext_expand(const kete_frame *frames, const double *dur, int64_t nf, int n_sub,
                           int64_t n_obs, int32_t *is_start, int64_t *ex, int64_t *scan_tmp,
                           int32_t *exp_first, kete_frame *sub, int32_t *parent, DevCounters *ctr,
                           cudaStream_t st)
{
    if (nf <= 0) return cudaSuccess;
    KLAUNCH(k_ext_starts<<<grid_for(nf, 256), 256, 0, st>>>(frames, dur, nf, n_sub, n_obs, is_start, ctr));
    cudaError_t e = exclusive_scan(is_start, nf, ex, scan_tmp, st);
    if (e != cudaSuccess) return e;
    KLAUNCH(k_exposure_first<<<grid_for(nf, 256), 256, 0, st>>>(is_start, ex, nf, exp_first));
    KLAUNCH(k_ext_expand<<<grid_for(nf, 128), 128, 0, st>>>(frames, dur, nf, n_sub, is_start, ex, exp_first, sub, parent));
    return cudaSuccess;
}

cudaError_t fov_merge_count(const kete_hit *h, unsigned long long nh, const int32_t *parent,
                            int32_t *cnt, const int64_t *off, int32_t *cur, kete_hit *grouped,
                            bool scatter, cudaStream_t st)
{
    if (nh == 0) return cudaSuccess;
    if (!scatter) KLAUNCH(k_merge_count<<<grid_for((int64_t)nh, 256), 256, 0, st>>>(h, nh, parent, cnt));
    else KLAUNCH(k_merge_scatter<<<grid_for((int64_t)nh, 256), 256, 0, st>>>(h, nh, parent, off, cur, grouped));
    return cudaSuccess;
}

cudaError_t fov_merge_keep(const kete_hit *grouped, const int64_t *off, int64_t np, int8_t *keep,
                           int32_t *kept_cnt, int n_sm, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    int64_t blocks = (np * 32 + 255) / 256;
    if (blocks > (int64_t)n_sm * 32) blocks = (int64_t)n_sm * 32;
    KLAUNCH(k_merge_keep<<<(unsigned)blocks, 256, 0, st>>>(grouped, off, np, keep, kept_cnt));
    return cudaSuccess;
}

cudaError_t fov_merge_place(const kete_hit *grouped, const int64_t *off, const int8_t *keep,
                            const int64_t *kept_off, int64_t np, kete_hit *out, int n_sm,
                            cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    int64_t blocks = (np * 32 + 255) / 256;
    if (blocks > (int64_t)n_sm * 32) blocks = (int64_t)n_sm * 32;
    KLAUNCH(k_merge_place<<<(unsigned)blocks, 256, 0, st>>>(grouped, off, keep, kept_off, np, out));
    return cudaSuccess;
}

}  // namespace kete
