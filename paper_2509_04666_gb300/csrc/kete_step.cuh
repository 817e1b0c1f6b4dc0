// kete_step.cuh -- one Gauss-Radau 15th-order step in the IAS15 form with the
// predictor removed (Sec. 3.2, App. A.6), shared by the propagation kernel and
// the adjoint's forward pass.
//
// Each translation unit that includes this header holds its own copy of the
// node tables g_rt in constant memory and must fill it with
// upload_step_tables() before its first launch.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "kete_device.cuh"

namespace kete {
static __constant__ RadauTables g_rt;

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

static inline void fill_radau_tables(RadauTables &t)
{
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
        for (int m = 0; m < 7; m++) {
            t.c[n][m] = (m < n) ? poly[m] : 0.0;
            t.cf[n][m] = (float)t.c[n][m];
        }
    }
    // predictor weights of the power-basis coefficients at each node
    for (int n = 0; n < 8; n++) {
        double sp = kRadauH[n];
        for (int k = 0; k < 7; k++) {
            t.wx[n][k] = sp / ((k + 2.0) * (k + 3.0));
            t.wv[n][k] = sp / (k + 2.0);
            t.wvf[n][k] = (float)t.wv[n][k];
            sp *= kRadauH[n];
        }
    }
    // leading coefficient of the interpolant through the 8 nodes
    for (int n = 0; n < 8; n++) {
        double p = 1.0;
        for (int k = 0; k < 8; k++)
            if (k != n) p *= (kRadauH[n] - kRadauH[k]);
        t.w7[n] = 1.0 / p;
    }
}

// fill this translation unit's copy of g_rt
static inline cudaError_t upload_step_tables(cudaStream_t st)
{
    RadauTables t;
    fill_radau_tables(t);
    return cudaMemcpyToSymbolAsync(g_rt, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
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
// JAC (FP64 only): also store the Newtonian da/dx at this point to jout[0..5].
// G: lanes per body (LaneGroup).
template <int MODE, bool JAC = false, int G = 1>
__device__ __forceinline__ int accel(const EphemDev &E, const ForceDev &F, double t0, double off,
                                     const double *row64, const float *row32, uint32_t &close,
                                     const double x[3], const double v[3], double a[3],
                                     double as[3], Encounter &enc, const double dx[3], bool detect,
                                     double *jout = nullptr, const kete_nongrav *ng = nullptr,
                                     const float *vf = nullptr, double *ng_chi = nullptr)
{
    static_assert(!(JAC && MODE == KETE_MIXED), "Jacobian capture is FP64 only");
    if (MODE == KETE_MIXED)
        return accel_mixed<G>(E, F, t0, off, row64, row32, close, x, v, a, as, enc, dx, detect, ng,
                              vf, ng_chi);
    double J[6];
    int st = accel_fp64<JAC, G>(E, F, t0, off, row64, x, v, a, enc, dx, detect, J, ng, ng_chi);
    as[0] = a[0]; as[1] = a[1]; as[2] = a[2];
    if (JAC) {
#pragma unroll
        for (int q = 0; q < 6; q++) jout[q] = J[q];
    }
    return st;
}

// Corrector state of one Gauss-Radau step attempt of size h (from t to
// t_new) between corrector sweeps; one sweep is one corrector iteration over
// the 7 substep nodes.  rows.r64 != null: the step spans the whole leg and
// the planets come from the node rows (node n at rows.r64 + n * stride).
struct Attempt {
    double b[7][3], g[7][3];
    float bf[7][3];         // mixed precision: b in FP32, for the node velocity
    double gs7[3];          // mixed precision: b6 of the FP64 part, last sweep
    double amax, pc_prev;   // max|a| at the last node and the last convergence measure
    double h, t_new;
    LegRows rows;
    int it;                 // sweeps done
};

__device__ __forceinline__ void attempt_begin(Attempt &A, double h, double t_new, LegRows rows)
{
#pragma unroll
    for (int m = 0; m < 7; m++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            A.b[m][i] = A.g[m][i] = 0.0;
            A.bf[m][i] = 0.0f;
        }
    A.gs7[0] = A.gs7[1] = A.gs7[2] = 0.0;
    A.amax = 0.0;
    A.pc_prev = 0.0;
    A.h = h;
    A.t_new = t_new;
    A.rows = rows;
    A.it = 0;
}

// The corrector update at node N (compile-time): Newton divided difference
// g_{N-1} from the node's force and the earlier g, then the power-basis
// coefficients b.
template <int MODE, int N, bool V32 = false>
__device__ __forceinline__ void node_update(Attempt &A, const double Fn[3], const double Fs[3],
                                            const double a0[3], double F7[3])
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double gn = (Fn[i] - a0[i]) * g_rt.rinv[N][0];
#pragma unroll
        for (int k = 1; k < N; k++) gn = (gn - A.g[k - 1][i]) * g_rt.rinv[N][k];
        double dg = gn - A.g[N - 1][i];
        A.g[N - 1][i] = gn;
#pragma unroll
        for (int m = 0; m < N; m++) A.b[m][i] = fma(g_rt.c[N][m], dg, A.b[m][i]);
        if (MODE == KETE_MIXED && V32) {
            const float dgf = (float)dg;
#pragma unroll
            for (int m = 0; m < N; m++) A.bf[m][i] = fmaf(g_rt.cf[N][m], dgf, A.bf[m][i]);
        }
        if (N == 7) F7[i] = Fn[i];
        if (MODE == KETE_MIXED) A.gs7[i] = fma(g_rt.w7[N], Fs[i], A.gs7[i]);
    }
}

// One corrector sweep of the attempt from (t, x0, v0) with a0 = a(t, x0, v0)
// (as0: its FP64 part).  V32: see vel32 below.  Sets done when the corrector has converged
// (max|db6|/max|a| < eps_pc), stopped improving (from the third sweep) or
// reached max_iter sweeps.  JAC: every node evaluation also stores da/dx at
// node n to jrec[6n..6n+5]; the last sweep's values remain.
template <int MODE, bool JAC = false, int G = 1, bool V32 = false>
__device__ __forceinline__ int attempt_sweep(const EphemDev &E, const ForceDev &F, double t,
                                             const double x0[3], const double v0[3],
                                             const double a0[3], const double as0[3],
                                             uint32_t close, Encounter enc, Attempt &A, bool &done,
                                             Cnt &cnt, double *jrec = nullptr,
                                             const kete_nongrav *ng = nullptr,
                                             double *ng_chi = nullptr)
{
    const double h = A.h;
    double b6o[3] = {A.b[6][0], A.b[6][1], A.b[6][2]};
    double F7[3];
    // V32 (mixed precision, launches with node rows): without non-gravitational
    // terms the node velocity feeds only FP32 terms, so it is predicted in FP32
    // from A.bf (kept only in these launches: the extra registers cost the
    // per-thread-ephemeris launches more than the FP64 work they save)
    const bool vel32 = (MODE == KETE_MIXED) && V32 && !ng;
    float v0f[3], a0f[3];
    if (MODE == KETE_MIXED) {
#pragma unroll
        for (int i = 0; i < 3; i++) A.gs7[i] = g_rt.w7[0] * as0[i];
        if (vel32) {
#pragma unroll
            for (int i = 0; i < 3; i++) {
                v0f[i] = (float)v0[i];
                a0f[i] = (float)a0[i];
            }
        }
    }
    // one copy of the force evaluation: the node index is the same for every
    // lane of the sweep (uniform table reads, uniform guards below)
#pragma unroll 1
    for (int n = 1; n <= 7; n++) {
        const double s = g_rt.h[n];
        const double sh = s * h;
        double xn[3], vn[3], dxn[3];
        float vnf[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            // x(s) = x0 + s h v0 + (s h)^2 [a0/2 + sum_k b_k s^(k+1) / ((k+2)(k+3))]
            // v(s) = v0 + s h [a0 + sum_k b_k s^(k+1) / (k+2)]
            // with the node's weights from the table (smallest terms first)
            double px = A.b[6][i] * g_rt.wx[n][6];
#pragma unroll
            for (int k = 5; k >= 0; k--) px = fma(A.b[k][i], g_rt.wx[n][k], px);
            px = fma(a0[i], 0.5, px);
            dxn[i] = fma(sh * sh, px, sh * v0[i]);   // displacement since the step start
            xn[i] = x0[i] + dxn[i];
            if (vel32) {
                float pv = A.bf[6][i] * g_rt.wvf[n][6];
#pragma unroll
                for (int k = 5; k >= 0; k--) pv = fmaf(A.bf[k][i], g_rt.wvf[n][k], pv);
                vnf[i] = fmaf((float)sh, pv + a0f[i], v0f[i]);
                vn[i] = 0.0;
            } else {
                double pv = A.b[6][i] * g_rt.wv[n][6];
#pragma unroll
                for (int k = 5; k >= 0; k--) pv = fma(A.b[k][i], g_rt.wv[n][k], pv);
                pv = pv + a0[i];
                vn[i] = fma(sh, pv, v0[i]);
            }
        }
        double Fn[3], Fs[3];
        const double *r64 = A.rows.r64 ? A.rows.r64 + n * A.rows.stride64 : nullptr;
        const float *r32 = A.rows.r32 ? A.rows.r32 + n * A.rows.stride64 : nullptr;
        int st = accel<MODE, JAC, G>(E, F, t, sh, r64, r32, close, xn, vn, Fn, Fs, enc, dxn,
                                     false, JAC ? jrec + 6 * n : nullptr, ng,
                                     vel32 ? vnf : nullptr, ng_chi);
        cnt.evals++;
        if (r64) cnt.node_evals++;
        if (st != KETE_BODY_OK) return st;
        switch (n) {
        case 1: node_update<MODE, 1, V32>(A, Fn, Fs, a0, F7); break;
        case 2: node_update<MODE, 2, V32>(A, Fn, Fs, a0, F7); break;
        case 3: node_update<MODE, 3, V32>(A, Fn, Fs, a0, F7); break;
        case 4: node_update<MODE, 4, V32>(A, Fn, Fs, a0, F7); break;
        case 5: node_update<MODE, 5, V32>(A, Fn, Fs, a0, F7); break;
        case 6: node_update<MODE, 6, V32>(A, Fn, Fs, a0, F7); break;
        default: node_update<MODE, 7, V32>(A, Fn, Fs, a0, F7); break;
        }
    }
    cnt.iters++;
    A.it++;
    double db = 0.0, amax = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        db = fmax(db, fabs(A.b[6][i] - b6o[i]));
        amax = fmax(amax, fabs(F7[i]));
    }
    A.amax = amax;
    const double pc = db / amax;
    if (!isfinite(pc)) return KETE_BODY_NONFINITE;
    done = (pc < F.eps_pc) || (A.it >= 3 && pc >= A.pc_prev) || (A.it >= F.max_iter);
    A.pc_prev = pc;
    return KETE_BODY_OK;
}

// The attempt's end state and its IAS15 error estimate max|b6| / max|a| (in
// mixed precision b6 of the smooth FP64 part: FP32 rounding is not smooth and
// b6 would amplify it).
template <int MODE>
__device__ __forceinline__ int attempt_end(const Attempt &A, const double x0[3], const double v0[3],
                                           const double a0[3], double x1[3], double v1[3],
                                           double &err)
{
    const double h = A.h;
    double bmax = (MODE == KETE_MIXED)
                      ? fmax(fabs(A.gs7[0]), fmax(fabs(A.gs7[1]), fabs(A.gs7[2])))
                      : fmax(fabs(A.b[6][0]), fmax(fabs(A.b[6][1]), fabs(A.b[6][2])));
    err = bmax / A.amax;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double px = fma(A.b[6][i], 1.0 / 72.0, A.b[5][i] * (1.0 / 56.0));
        px = fma(A.b[4][i], 1.0 / 42.0, px);
        px = fma(A.b[3][i], 1.0 / 30.0, px);
        px = fma(A.b[2][i], 1.0 / 20.0, px);
        px = fma(A.b[1][i], 1.0 / 12.0, px);
        px = fma(A.b[0][i], 1.0 / 6.0, px);
        px = fma(a0[i], 0.5, px);
        double pv = fma(A.b[6][i], 0.125, A.b[5][i] * (1.0 / 7.0));
        pv = fma(A.b[4][i], 1.0 / 6.0, pv);
        pv = fma(A.b[3][i], 0.2, pv);
        pv = fma(A.b[2][i], 0.25, pv);
        pv = fma(A.b[1][i], 1.0 / 3.0, pv);
        pv = fma(A.b[0][i], 0.5, pv);
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
    const kete_nongrav *ng; // the body's non-gravitational terms (null: none)
    double ng_chi;          // the thermal lag's last two-body solution (0: none yet)
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

// Start a step attempt of (x, v, t) toward `target` (t != target): the
// acceleration at the step start if it is not known yet (kept across a
// rejection), the step size and its node rows, the corrector state A.
// Returns a KETE_BODY_* status.  JAC: as attempt_sweep (jrec[0..5] at t).
template <int MODE, bool JAC = false, int G = 1>
__device__ __forceinline__ int step_begin(const EphemDev &E, const ForceDev &F, const LegView &L,
                                          const double x[3], const double v[3], double t,
                                          double dt, double target, StepState &S, Attempt &A,
                                          Cnt &cnt, double *jrec = nullptr)
{
    // rows of node 0 serve a0 whenever the step starts at the leg start
    const bool at_start = L.r64 && (t == L.t0) && isfinite(L.h);
    if (!S.have_a0) {
        const double zero[3] = {0.0, 0.0, 0.0};
        int st = accel<MODE, JAC, G>(E, F, t, 0.0, at_start ? L.r64 : nullptr,
                                     at_start ? L.r32 : nullptr, S.close, x, v, S.a0, S.as0,
                                     S.enc, zero, true, jrec, S.ng, nullptr, &S.ng_chi);
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
    attempt_begin(A, h, t_new, rows);
    return KETE_BODY_OK;
}

// End a step attempt whose corrector is done: IAS15 step control.  Accepted:
// the state advances and dt holds the next proposal.  Rejected: dt shrinks and
// a0 is kept.  Returns a KETE_BODY_* status.
template <int MODE>
__device__ __forceinline__ int step_end(const ForceDev &F, const Attempt &A, double x[3],
                                        double v[3], double &t, double &dt, StepState &S, Cnt &cnt)
{
    double x1[3], v1[3], err;
    int st = attempt_end<MODE>(A, x, v, S.a0, x1, v1, err);
    if (st != KETE_BODY_OK) return st;
    const double h = A.h;
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
    t = A.t_new;
    S.have_a0 = false;
    cnt.steps++;
    return KETE_BODY_OK;
}

// One whole step attempt of (x, v, t) toward `target` (t != target):
// step_begin, corrector sweeps until done, step_end.
// JAC: da/dx at the 8 nodes of the attempt go to jrec[6n..6n+5]; after an
// accepted step they describe that step.
template <int MODE, bool JAC = false, int G = 1>
__device__ __forceinline__ int step_once(const EphemDev &E, const ForceDev &F, const LegView &L,
                                         double x[3], double v[3], double &t, double &dt,
                                         double target, StepState &S, Cnt &cnt,
                                         double *jrec = nullptr)
{
    Attempt A;
    int st = step_begin<MODE, JAC, G>(E, F, L, x, v, t, dt, target, S, A, cnt, jrec);
    if (st != KETE_BODY_OK) return st;
    for (;;) {
        bool done = false;
        st = attempt_sweep<MODE, JAC, G>(E, F, t, x, v, S.a0, S.as0, S.close, S.enc, A, done, cnt,
                                         jrec, S.ng, &S.ng_chi);
        if (st != KETE_BODY_OK) return st;
        if (done) break;
    }
    return step_end<MODE>(F, A, x, v, t, dt, S, cnt);
}

// orient the carried step toward the next stop (|dt| kept; dt_init to start)
__device__ __forceinline__ void aim_step(const ForceDev &F, double t, double target, double &dt)
{
    const double dir = (target >= t) ? 1.0 : -1.0;
    if (dt == 0.0 || ((dt > 0.0) != (dir > 0.0))) dt = dir * fabs(dt == 0.0 ? F.dt_init : dt);
}

// warp sums of the lanes' counters into ctr; with G lanes per body only the
// rank-0 lane of a group counts
template <int G = 1>
__device__ __forceinline__ void flush_counters(const Cnt &c, DevCounters *ctr)
{
    const unsigned long long w = (LaneGroup<G>::rank() == 0) ? 1ull : 0ull;
    unsigned long long s = w * c.steps, r = w * c.rejected, e = w * c.evals, it = w * c.iters,
                       ne = w * c.node_evals;
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


}  // namespace kete
