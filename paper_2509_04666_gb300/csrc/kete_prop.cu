// kete_prop.cu -- n-body propagation of massless bodies (Sec. 3.2, App. A, App. A.6).
//
// Each lane integrates one body at a time along its chain of stops (the
// body's epoch, then every stop in order).  Each step is a 15th-order Gauss-Radau step in the
// IAS15 form (Newton-basis coefficients g, power-basis coefficients b, 8
// spacings), with the predictor removed: every step starts from b = 0 and the
// corrector iterates until max|db6|/max|a| < eps_pc, the error stops falling
// (after 3 iterations) or max_iter is reached.  Step control follows IAS15:
// dt_new = dt (eps / (max|b6|/max|a|))^(1/7), reject below safety*dt, grow at
// most 1/safety.  Every loop is bounded: max_iter corrector iterations,
// max_steps step attempts per leg, after which the body gets a status code.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "kete_device.cuh"

namespace kete {

__constant__ RadauTables g_rt;

// Gauss-Radau spacings on [0, 1] (Everhart 1985, 30 published digits)
static const double kRadauH[8] = {
    0.0,
    0.0562625605369221464656521910318,
    0.180240691736892364987579942780,
    0.352624717113169637373907769648,
    0.547153626330555383001448554766,
    0.734210177215410531523210605558,
    0.885320946839095768090359771030,
    0.977520613561287501891174488626,
};

void upload_radau_tables(cudaStream_t st)
{
    RadauTables t;
    std::memset(&t, 0, sizeof(t));
    for (int n = 0; n < 8; n++) t.h[n] = kRadauH[n];
    for (int n = 0; n < 8; n++)
        for (int k = 0; k < n; k++) t.rinv[n][k] = 1.0 / (kRadauH[n] - kRadauH[k]);
    // Newton basis N_n(s) = s (s-h_1)...(s-h_{n-1}); c[n][m] = coefficient of
    // s^(m+1) in N_n, built by the recurrence N_n = N_{n-1} (s - h_{n-1}).
    double poly[8] = {1, 0, 0, 0, 0, 0, 0, 0};   // coefficients of prod (s-h_i), s^0 first
    for (int n = 1; n <= 7; n++) {
        if (n >= 2) {
            double nxt[8] = {0};
            for (int p = 0; p < 7; p++) {
                nxt[p + 1] += poly[p];
                nxt[p] -= kRadauH[n - 1] * poly[p];
            }
            std::memcpy(poly, nxt, sizeof(poly));
        }
        for (int m = 0; m < 7; m++) t.c[n][m] = (m < n) ? poly[m] : 0.0;
    }
    // leading coefficient of the interpolant through the 8 nodes
    for (int n = 0; n < 8; n++) {
        double p = 1.0;
        for (int k = 0; k < 8; k++)
            if (k != n) p *= (kRadauH[n] - kRadauH[k]);
        t.w7[n] = 1.0 / p;
    }
    cudaMemcpyToSymbolAsync(g_rt, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
}

struct Cnt {
    unsigned long long steps, rejected, evals, iters, node_evals;
};

// Rows of the node table for leg kg, or null when the step (t, h) does not span
// that whole leg.
struct LegRows {
    const double *r64;
    const float *r32;
    int stride64;   // doubles per node
};

// Force evaluation dispatch by precision mode.
// detect: the evaluation at a step start, which also finds the planets near
// the body (see accel_fp64 / accel_mixed).
template <int MODE>
__device__ __forceinline__ int accel(const EphemDev &E, const ForceDev &F, double t0, double off,
                                     const double *row64, const float *row32, uint32_t &close,
                                     const double x[3], const double v[3], double a[3],
                                     double as[3], Encounter &enc, const double dx[3], bool detect)
{
    if (MODE == KETE_MIXED)
        return accel_mixed(E, F, t0, off, row64, row32, close, x, v, a, as, enc, dx, detect);
    int st = accel_fp64(E, F, t0, off, row64, x, v, a, enc, dx, detect);
    as[0] = a[0]; as[1] = a[1]; as[2] = a[2];
    return st;
}

// One Gauss-Radau attempt of size h from (t, x0, v0) with a0 = a(t, x0, v0)
// (as0: its FP64 part).  rows != null: the step spans the whole leg and the
// planets come from the node rows (node n at rows.r64 + n * stride).
template <int MODE>
__device__ __forceinline__ int radau_attempt(const EphemDev &E, const ForceDev &F, double t,
                                             const double x0[3], const double v0[3],
                                             const double a0[3], const double as0[3],
                                             uint32_t close, Encounter enc, double h,
                                             LegRows rows, double x1[3], double v1[3],
                                             double &err, Cnt &cnt)
{
    double b[7][3], g[7][3];
#pragma unroll
    for (int m = 0; m < 7; m++)
#pragma unroll
        for (int i = 0; i < 3; i++) b[m][i] = g[m][i] = 0.0;
    double amax = 0.0, pc_prev = 0.0;
    double gs7[3] = {0.0, 0.0, 0.0};   // b6 of the FP64 part (mixed precision)
    for (int it = 1; it <= F.max_iter; it++) {
        double b6o[3] = {b[6][0], b[6][1], b[6][2]};
        double F7[3];
        if (MODE == KETE_MIXED) {
#pragma unroll
            for (int i = 0; i < 3; i++) gs7[i] = g_rt.w7[0] * as0[i];
        }
#pragma unroll
        for (int n = 1; n <= 7; n++) {
            const double s = g_rt.h[n];
            const double sh = s * h;
            double xn[3], vn[3], dxn[3];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                // x(s) = x0 + s h v0 + (s h)^2 [a0/2 + s(b0/6 + s(b1/12 + ... + s b6/72))]
                double px = b[6][i] * (1.0 / 72.0);
                px = fma(px, s, b[5][i] * (1.0 / 56.0));
                px = fma(px, s, b[4][i] * (1.0 / 42.0));
                px = fma(px, s, b[3][i] * (1.0 / 30.0));
                px = fma(px, s, b[2][i] * (1.0 / 20.0));
                px = fma(px, s, b[1][i] * (1.0 / 12.0));
                px = fma(px, s, b[0][i] * (1.0 / 6.0));
                px = fma(px, s, a0[i] * 0.5);
                dxn[i] = fma(sh * sh, px, sh * v0[i]);   // displacement since the step start
                xn[i] = x0[i] + dxn[i];
                // v(s) = v0 + s h [a0 + s(b0/2 + s(b1/3 + ... + s b6/8))]
                double pv = b[6][i] * 0.125;
                pv = fma(pv, s, b[5][i] * (1.0 / 7.0));
                pv = fma(pv, s, b[4][i] * (1.0 / 6.0));
                pv = fma(pv, s, b[3][i] * 0.2);
                pv = fma(pv, s, b[2][i] * 0.25);
                pv = fma(pv, s, b[1][i] * (1.0 / 3.0));
                pv = fma(pv, s, b[0][i] * 0.5);
                pv = fma(pv, s, a0[i]);
                vn[i] = fma(sh, pv, v0[i]);
            }
            double Fn[3], Fs[3];
            const double *r64 = rows.r64 ? rows.r64 + n * rows.stride64 : nullptr;
            const float *r32 = rows.r32 ? rows.r32 + n * rows.stride64 : nullptr;
            int st = accel<MODE>(E, F, t, sh, r64, r32, close, xn, vn, Fn, Fs, enc, dxn, false);
            cnt.evals++;
            if (r64) cnt.node_evals++;
            if (st != KETE_BODY_OK) return st;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                double gn = (Fn[i] - a0[i]) * g_rt.rinv[n][0];
#pragma unroll
                for (int k = 1; k < n; k++) gn = (gn - g[k - 1][i]) * g_rt.rinv[n][k];
                double dg = gn - g[n - 1][i];
                g[n - 1][i] = gn;
#pragma unroll
                for (int m = 0; m < n; m++) b[m][i] = fma(g_rt.c[n][m], dg, b[m][i]);
                if (n == 7) F7[i] = Fn[i];
                if (MODE == KETE_MIXED) gs7[i] = fma(g_rt.w7[n], Fs[i], gs7[i]);
            }
        }
        cnt.iters++;
        double db = 0.0;
        amax = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            db = fmax(db, fabs(b[6][i] - b6o[i]));
            amax = fmax(amax, fabs(F7[i]));
        }
        double pc = db / amax;
        if (!isfinite(pc)) return KETE_BODY_NONFINITE;
        if (pc < F.eps_pc) break;
        if (it >= 3 && pc >= pc_prev) break;
        pc_prev = pc;
    }
    // step-size error estimate: max|b6| / max|a|; in mixed precision b6 of the
    // smooth FP64 part (FP32 rounding is not smooth and b6 would amplify it)
    double bmax = (MODE == KETE_MIXED)
                      ? fmax(fabs(gs7[0]), fmax(fabs(gs7[1]), fabs(gs7[2])))
                      : fmax(fabs(b[6][0]), fmax(fabs(b[6][1]), fabs(b[6][2])));
    err = bmax / amax;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double px = fma(b[6][i], 1.0 / 72.0, b[5][i] * (1.0 / 56.0));
        px = fma(b[4][i], 1.0 / 42.0, px);
        px = fma(b[3][i], 1.0 / 30.0, px);
        px = fma(b[2][i], 1.0 / 20.0, px);
        px = fma(b[1][i], 1.0 / 12.0, px);
        px = fma(b[0][i], 1.0 / 6.0, px);
        px = fma(a0[i], 0.5, px);
        double pv = fma(b[6][i], 0.125, b[5][i] * (1.0 / 7.0));
        pv = fma(b[4][i], 1.0 / 6.0, pv);
        pv = fma(b[3][i], 0.2, pv);
        pv = fma(b[2][i], 0.25, pv);
        pv = fma(b[1][i], 1.0 / 3.0, pv);
        pv = fma(b[0][i], 0.5, pv);
        pv = pv + a0[i];
        x1[i] = fma(h * h, px, fma(h, v0[i], x0[i]));
        v1[i] = fma(h, pv, v0[i]);
    }
    if (!(isfinite(x1[0]) && isfinite(x1[1]) && isfinite(x1[2]) && isfinite(v1[0]) &&
          isfinite(v1[1]) && isfinite(v1[2])))
        return KETE_BODY_NONFINITE;
    return KETE_BODY_OK;
}

// Per-body integrator state between step attempts.
struct StepState {
    double a0[3], as0[3];   // acceleration at the step start (and its FP64 part)
    uint32_t close;         // planets near the body at the step start (mixed precision)
    Encounter enc;          // nearest planet within kEncounterAu (close-encounter path)
    double t_stop;          // end of the step's range: the target, or the next table
                            // segment boundary during an encounter
    bool have_a0;           // a0 valid for (x, v, t): kept across a rejection
};

// Node-table view of leg kg (null pointers: no rows).
struct LegView {
    double t0, h;
    const double *r64;
    const float *r32;
    int stride;
};

__device__ __forceinline__ LegView leg_view(const NodeTable *nt, int kg)
{
    LegView L;
    L.t0 = 0.0;
    L.h = __longlong_as_double(0x7ff8000000000000ll);
    L.r64 = nullptr;
    L.r32 = nullptr;
    L.stride = 0;
    if (nt) {
        L.stride = nt->nb * 6;
        L.t0 = __ldg(nt->t0 + kg);
        L.h = __ldg(nt->h + kg);
        L.r64 = nt->row64 + (size_t)kg * 8 * L.stride;
        L.r32 = nt->row32 + (size_t)kg * 8 * L.stride;
    }
    return L;
}

// One step attempt of (x, v, t) toward `target` (t != target).  Accepted: the
// state advances and dt holds the next proposal.  Rejected: dt shrinks and a0
// is kept.  Returns a KETE_BODY_* status.
template <int MODE>
__device__ __forceinline__ int step_once(const EphemDev &E, const ForceDev &F, const LegView &L,
                                         double x[3], double v[3], double &t, double &dt,
                                         double target, StepState &S, Cnt &cnt)
{
    // rows of node 0 serve a0 whenever the step starts at the leg start
    const bool at_start = L.r64 && (t == L.t0) && isfinite(L.h);
    if (!S.have_a0) {
        const double zero[3] = {0.0, 0.0, 0.0};
        int st = accel<MODE>(E, F, t, 0.0, at_start ? L.r64 : nullptr, at_start ? L.r32 : nullptr,
                             S.close, x, v, S.a0, S.as0, S.enc, zero, true);
        cnt.evals++;
        if (at_start) cnt.node_evals++;
        if (st != KETE_BODY_OK) return st;
        // during an encounter no step straddles a boundary of the planet polynomials
        S.t_stop = target;
        if (S.enc.m >= 0) {
            const double k = floor((t - E.t_start) * E.inv_seg);
            double b = (target > t) ? E.t_start + (k + 1.0) * E.seg_len : E.t_start + k * E.seg_len;
            if (target < t && b == t) b = E.t_start + (k - 1.0) * E.seg_len;
            if ((target > t && b < target) || (target < t && b > target)) S.t_stop = b;
        }
        S.have_a0 = true;
    }
    const double remaining = S.t_stop - t;
    const bool clamped = fabs(dt) >= fabs(remaining);
    // the step is the exact difference of the representable epochs it joins
    const double t_new = clamped ? S.t_stop : t + dt;
    const double h = t_new - t;
    if (h == 0.0) return KETE_BODY_STEP_CAP;   // step below the epoch resolution
    LegRows rows = {nullptr, nullptr, L.stride};
    if (at_start && h == L.h) {
        rows.r64 = L.r64;
        rows.r32 = L.r32;
    }
    double x1[3], v1[3], err;
    int st = radau_attempt<MODE>(E, F, t, x, v, S.a0, S.as0, S.close, S.enc, h, rows, x1, v1,
                                 err, cnt);
    if (st != KETE_BODY_OK) return st;
    double dt_new;
    if (isfinite(err) && err >= 2.2250738585072014e-308)
        dt_new = pow(F.eps / err, 1.0 / 7.0) * h;
    else
        dt_new = h / F.safety;
    if (fabs(dt_new / h) < F.safety) {   // reject: retry from the same a0
        dt = dt_new;
        cnt.rejected++;
        return KETE_BODY_OK;
    }
    if (fabs(dt_new / h) > 1.0 / F.safety) dt_new = h / F.safety;
    dt = dt_new;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        x[i] = x1[i];
        v[i] = v1[i];
    }
    t = t_new;
    S.have_a0 = false;
    cnt.steps++;
    return KETE_BODY_OK;
}

// orient the carried step toward the next stop (|dt| kept; dt_init to start)
__device__ __forceinline__ void aim_step(const ForceDev &F, double t, double target, double &dt)
{
    const double dir = (target >= t) ? 1.0 : -1.0;
    if (dt == 0.0 || ((dt > 0.0) != (dir > 0.0))) dt = dir * fabs(dt == 0.0 ? F.dt_init : dt);
}

__device__ __forceinline__ void flush_counters(const Cnt &c, DevCounters *ctr)
{
    unsigned long long s = c.steps, r = c.rejected, e = c.evals, it = c.iters, ne = c.node_evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
        it += __shfl_xor_sync(0xffffffffu, it, o);
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctr->steps, s);
        atomicAdd(&ctr->rejected, r);
        atomicAdd(&ctr->force_evals, e);
        atomicAdd(&ctr->iterations, it);
        atomicAdd(&ctr->node_evals, ne);
    }
}

#ifndef KETE_PROP_MIN_BLOCKS
#define KETE_PROP_MIN_BLOCKS 1   // resident blocks per SM asked of the register allocator
#endif

// The propagation kernel.  Each lane owns one body at a time and advances it
// one step attempt per loop iteration along its chain of stops, writing the
// state at every stop to out[k][c][i] (stride out_stride between rows) and the
// chain state back when it is done.  Stop k of this launch is leg leg0 + k of
// the node table (if any).
//   refill = 0 (static): lane j of the grid takes body j and then idles;
//   refill = 1 (work stealing, persistent grid): a lane whose body is done
//   takes the next one from an atomic counter (warp-aggregated), so a body
//   needing hundreds of steps no longer idles the other 31 lanes of its warp.
// Both schedules run the same instructions per body: results are identical.
template <int MODE>
__global__ void __launch_bounds__(128, KETE_PROP_MIN_BLOCKS)
k_propagate(EphemDev E, ForceDev F, ChainState cs, const double *__restrict__ stops,
            int n_stops, double *__restrict__ out, int64_t out_stride, int keep_on_fail,
            DevCounters *ctr, NodeTable nt, int use_nt, int leg0,
            unsigned long long *__restrict__ next_body, int refill)
{
    const int64_t n = cs.n;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    Cnt cnt = {0, 0, 0, 0, 0};
    int64_t i = -1;           // current body (-1: none; n: no work left)
    int k = 0;                // next stop of the body
    double x[3], v[3], t = 0.0, dt = 0.0;
    int status = KETE_BODY_OK;
    long long attempts = 0;
    StepState S;
    S.have_a0 = false;
    LegView L = leg_view(nullptr, 0);
    bool first = true;
    for (;;) {
        // lanes without a body take the next ones
        const bool need = (i < 0);
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (refill) {
                if (lane == leader) base = atomicAdd(next_body, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
            }
            if (need) {
                unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
                if (!refill)   // static: one body per lane, taken on the first pass
                    mine = first ? (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x
                                 : (unsigned long long)n;
                if (mine < (unsigned long long)n) {
                    i = (int64_t)mine;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x[c] = cs.w[c * n + i];
                        v[c] = cs.w[(3 + c) * n + i];
                    }
                    t = cs.w[6 * n + i];
                    dt = cs.w[7 * n + i];
                    status = cs.status[i];
                    k = 0;
                    attempts = 0;
                    S.have_a0 = false;
                    L = leg_view(use_nt ? &nt : nullptr, leg0);
                    if (status == KETE_BODY_OK && n_stops > 0) aim_step(F, t, stops[0], dt);
                } else {
                    i = n;   // drained
                }
            }
        }
        first = false;
        const bool active = (i >= 0 && i < n);
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;
        if (k < n_stops && status == KETE_BODY_OK && t != stops[k]) {
            if (++attempts > F.max_steps) status = KETE_BODY_STEP_CAP;
            else status = step_once<MODE>(E, F, L, x, v, t, dt, stops[k], S, cnt);
            if (status == KETE_BODY_OK && t != stops[k]) continue;
        }
        // the body is at stop k (or failed): record it and move on
        while (k < n_stops && (status != KETE_BODY_OK || t == stops[k])) {
            double *o = out + (int64_t)k * 6 * out_stride;
            if (status == KETE_BODY_OK) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    o[c * out_stride + i] = x[c];
                    o[(3 + c) * out_stride + i] = v[c];
                }
            } else if (!keep_on_fail) {
#pragma unroll
                for (int c = 0; c < 6; c++) o[c * out_stride + i] = __longlong_as_double(0x7ff8000000000000ll);
            }
            k++;
            attempts = 0;
            S.have_a0 = false;
            if (k < n_stops) {
                L = leg_view(use_nt ? &nt : nullptr, leg0 + k);
                if (status == KETE_BODY_OK) aim_step(F, t, stops[k], dt);
            }
        }
        if (k < n_stops) continue;
        // all stops done: write the chain state back and free the lane
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cs.w[c * n + i] = x[c];
            cs.w[(3 + c) * n + i] = v[c];
        }
        cs.w[6 * n + i] = t;
        cs.w[7 * n + i] = dt;
        cs.status[i] = status;
        i = -1;
    }
    flush_counters(cnt, ctr);
}

// Node table: thread per (leg k, node n, body m).  Leg 0 starts at the first
// body's epoch (*epoch0, device), leg k > 0 at stops[k-1]; h is their exact
// difference, as the integrator forms it.
__global__ void k_node_table(EphemDev E, const double *__restrict__ stops, int n_stops,
                             const double *__restrict__ epoch0, double *__restrict__ t0,
                             double *__restrict__ hh,
                             double *__restrict__ row64, float *__restrict__ row32)
{
    const int nb = E.n_bodies;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_stops * 8 * nb) return;
    const int m = (int)(idx % nb);
    const int n = (int)((idx / nb) % 8);
    const int k = (int)(idx / (8 * nb));
    const double ts = (k == 0) ? epoch0[0] : stops[k - 1];
    const double h = stops[k] - ts;
    const double off = g_rt.h[n] * h;
    Seg g;
    double st[6], sun[6];
    const bool ok = ephem_seg(E, ts, off, g);
    double *o64 = row64 + (((int64_t)k * 8 + n) * nb + m) * 6;
    float *o32 = row32 + (((int64_t)k * 8 + n) * nb + m) * 6;
    if (ok) {
        cheb_pos_vel(ephem_coef(E, m, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, st, st + 3);
        cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, sun, sun + 3);
        for (int q = 0; q < 6; q++) o64[q] = st[q];
        for (int q = 0; q < 3; q++) {
            o32[q] = (float)(st[q] - sun[q]);
            o32[3 + q] = (float)st[3 + q];
        }
    }
    if (m == 0 && n == 0) {
        t0[k] = ts;
        hh[k] = h;
    }
    // any node of the leg outside the table: the leg uses the per-thread path
    __syncwarp(__activemask());
    if (!ok) hh[k] = __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void k_chain_init(ChainState cs, const double *__restrict__ states,
                             const double *__restrict__ epochs)
{
    const int64_t n = cs.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    for (int c = 0; c < 6; c++) {
        double q = states[c * n + i];
        cs.w[c * n + i] = q;
        ok = ok && isfinite(q);
    }
    double t = epochs[i];
    cs.w[6 * n + i] = t;
    cs.w[7 * n + i] = 0.0;
    cs.status[i] = (ok && isfinite(t)) ? KETE_BODY_OK : KETE_BODY_NONFINITE;
}

__global__ void k_chain_finish(ChainState cs, double *__restrict__ epochs,
                               int32_t *__restrict__ status)
{
    const int64_t n = cs.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = cs.status[i];
    if (epochs && s == KETE_BODY_OK) epochs[i] = cs.w[6 * n + i];
    if (status) status[i] = s;
}

__global__ void k_ephem_eval(EphemDev E, const double *__restrict__ t, int64_t n, int body,
                             double *__restrict__ pos, double *__restrict__ vel)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Seg g;
    double p[3], v[3];
    if (!ephem_seg(E, t[i], 0.0, g)) {
        for (int c = 0; c < 3; c++) {
            pos[3 * i + c] = __longlong_as_double(0x7ff8000000000000ll);
            if (vel) vel[3 * i + c] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return;
    }
    cheb_pos_vel(ephem_coef(E, body, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, p, v);
    for (int c = 0; c < 3; c++) {
        pos[3 * i + c] = p[c];
        if (vel) vel[3 * i + c] = v[c];
    }
}

// strided sample of bodies: dst[c][j] = src[c][j * stride] (autotuner)
__global__ void k_gather_bodies(const double *__restrict__ st, const double *__restrict__ ep,
                                int64_t n, int64_t stride, int64_t m, double *__restrict__ dst,
                                double *__restrict__ dep)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t i = j * stride;
    for (int c = 0; c < 6; c++) dst[c * m + j] = st[c * n + i];
    dep[j] = ep[i];
}

static unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

cudaError_t launch_ephem_eval(const EphemDev &E, const double *t, int64_t n, int body,
                              double *pos, double *vel, cudaStream_t st)
{
    if (n > 0) k_ephem_eval<<<grid_for(n, 256), 256, 0, st>>>(E, t, n, body, pos, vel);
    return cudaGetLastError();
}

cudaError_t launch_chain_init(ChainState cs, const double *states, const double *epochs,
                              const ForceDev &, cudaStream_t st)
{
    if (cs.n > 0) k_chain_init<<<grid_for(cs.n, 256), 256, 0, st>>>(cs, states, epochs);
    return cudaGetLastError();
}

cudaError_t launch_node_table(const EphemDev &E, const double *stops_dev, int n_stops,
                              const double *epoch0, double *t0, double *h, double *row64,
                              float *row32, cudaStream_t st)
{
    int64_t tot = (int64_t)n_stops * 8 * E.n_bodies;
    if (tot > 0) k_node_table<<<grid_for(tot, 128), 128, 0, st>>>(E, stops_dev, n_stops, epoch0, t0, h, row64, row32);
    return cudaGetLastError();
}

int propagate_ws_blocks(int block, int mode)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (mode == KETE_MIXED)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate<KETE_MIXED>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate<KETE_FP64>, block, 0);
    return (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_propagate(const EphemDev &E, const ForceDev &F, ChainState cs,
                             const double *stops_dev, int n_stops, double *out,
                             int64_t out_stride, bool keep_on_fail, DevCounters *ctr,
                             cudaStream_t st, const NodeTable *nt, int leg0, PropVariant var,
                             unsigned long long *next_body)
{
    if (cs.n <= 0 || n_stops <= 0) return cudaGetLastError();
    NodeTable t{};
    if (nt) t = *nt;
    const int kof = keep_on_fail ? 1 : 0, unt = nt ? 1 : 0;
    const int block = (var.block > 0 && var.block <= 128) ? var.block : 128;
    int refill = 0;
    int64_t grid = (cs.n + block - 1) / block;
    if (var.kind == PROP_WORK_STEALING && next_body) {
        cudaError_t e = cudaMemsetAsync(next_body, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        refill = 1;
        int64_t persistent = propagate_ws_blocks(block, F.precision);
        if (grid > persistent) grid = persistent;
    }
    if (F.precision == KETE_MIXED)
        k_propagate<KETE_MIXED><<<(unsigned)grid, block, 0, st>>>(E, F, cs, stops_dev, n_stops, out, out_stride, kof, ctr, t, unt, leg0, next_body, refill);
    else
        k_propagate<KETE_FP64><<<(unsigned)grid, block, 0, st>>>(E, F, cs, stops_dev, n_stops, out, out_stride, kof, ctr, t, unt, leg0, next_body, refill);
    return cudaGetLastError();
}

cudaError_t launch_gather_bodies(const double *st, const double *ep, int64_t n, int64_t stride,
                                 int64_t m, double *dst, double *dep, cudaStream_t s)
{
    if (m > 0) k_gather_bodies<<<grid_for(m, 256), 256, 0, s>>>(st, ep, n, stride, m, dst, dep);
    return cudaGetLastError();
}

cudaError_t launch_chain_finish(ChainState cs, double *states, double *epochs, int32_t *status,
                                cudaStream_t st)
{
    (void)states;
    if (cs.n > 0) k_chain_finish<<<grid_for(cs.n, 256), 256, 0, st>>>(cs, epochs, status);
    return cudaGetLastError();
}

}  // namespace kete
