// kete_adjoint.cu -- orbit-fit loss and its gradient with respect to each
// body's initial state by the adjoint method (differentiation of the path of
// Sec. 2: n-body propagation of App. A, two-body + light time, RA/Dec).
//
// Three kernels per chunk of bodies:
//   k_adj_forward   one lane per body at a time (work stealing).  The body's
//                   observations are batched
//                   by the <= span rule (Sec. 2); the chain visits the batch
//                   midpoints and the checkpoint grid in ascending order with
//                   the same Gauss-Radau steps as the propagation kernel.
//                   Every accepted step leaves a record in device memory: its
//                   start and end epochs and the Newtonian da/dx at its 8
//                   Gauss-Radau nodes, taken from the force evaluations the
//                   step already makes.  The state at each batch midpoint is
//                   kept for the sky projection.
//   k_adj_observe   one warp per body, one lane per observation: prediction,
//                   residual, loss term and dL/dy(t_ref) through RA/Dec, the
//                   light-time fixed point (implicit derivative) and the
//                   universal-variable two-body map (forward-mode dual numbers
//                   at the converged universal anomaly).
//   k_adj_backward  one lane per body: mu = lambda_v obeys mu'' = J(t) mu
//                   (lambda_x = -mu'), integrated backward over every recorded
//                   step by collocation on the step's 9 sample epochs (its 8
//                   nodes and its end); dL/dy(t_ref) is added at each batch
//                   midpoint.  dL/dx0 = -mu'(t0), dL/dv0 = mu(t0).
//   k_adj_stm       (per-observation sky partials) one lane per body: the six
//                   columns of the state-transition matrix obey dx'' = J(t) dx,
//                   integrated forward over the recorded steps by the same
//                   collocation; the matrix is kept at every batch midpoint and
//                   k_adj_observe multiplies each observation's RA and Dec
//                   partials by it.
// The backward and state-transition passes evaluate no force and read no
// ephemeris: every Jacobian they need was recorded by the forward pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "kete_adjoint.h"
#include "kete_step.cuh"

namespace kete {

// ---------------------------------------------------------------------------
// backward collocation weights
// ---------------------------------------------------------------------------
// Sample points of one step in the backward variable s = (t_end - t) / h:
// sig[0] = 0 (the step end), sig[n] = 1 - h_{8-n} (forward node 8-n),
// sig[8] = 1 (the step start).  With F(s) interpolated through the 9 points,
//   mu(sig_n)  = mu_0 + sig_n mu'_0 + sum_k W2[n][k] F_k
//   mu'(sig_n) = mu'_0 + sum_k W1[n][k] F_k
// where W1[n][k] = int_0^sig_n l_k(s) ds, W2[n][k] = int_0^sig_n (sig_n - s) l_k(s) ds.
// The forward pass of the state-transition matrix uses the same weights for
// the forward variable s = (t - t_start) / h on the samples (node 0, ..., node
// 7, step end): W1f, W2f.
struct AdjTables {
    double sig[9];
    double W1[9][9];
    double W2[9][9];
    double sigf[9];
    double W1f[9][9];
    double W2f[9][9];
};
static __constant__ AdjTables g_adj;

// Lagrange-basis integrals on 9 sample points sg (see AdjTables)
static void fill_colloc(const long double sg[9], double sig[9], double W1[9][9], double W2[9][9])
{
    for (int n = 0; n < 9; n++) sig[n] = (double)sg[n];
    for (int k = 0; k < 9; k++) {
        // l_k(s) = prod_{j != k} (s - sg_j) / (sg_k - sg_j), power basis
        long double c[9] = {1.0L, 0, 0, 0, 0, 0, 0, 0, 0};
        long double den = 1.0L;
        int deg = 0;
        for (int j = 0; j < 9; j++) {
            if (j == k) continue;
            for (int p = deg + 1; p >= 1; p--) c[p] = c[p - 1] - sg[j] * c[p];
            c[0] = -sg[j] * c[0];
            deg++;
            den *= (sg[k] - sg[j]);
        }
        for (int n = 0; n < 9; n++) {
            long double w1 = 0.0L, w2 = 0.0L, sp = sg[n];
            for (int p = 0; p <= 8; p++) {
                w1 += c[p] * sp / (p + 1);
                w2 += c[p] * sp * sg[n] / ((p + 1) * (p + 2));
                sp *= sg[n];
            }
            W1[n][k] = (double)(w1 / den);
            W2[n][k] = (double)(w2 / den);
        }
    }
}

static void fill_adj_tables(AdjTables &T)
{
    RadauTables rt;
    fill_radau_tables(rt);
    long double sg[9];
    sg[0] = 0.0L;
    for (int n = 1; n <= 7; n++) sg[n] = 1.0L - (long double)rt.h[8 - n];
    sg[8] = 1.0L;
    fill_colloc(sg, T.sig, T.W1, T.W2);
    for (int n = 0; n <= 7; n++) sg[n] = (long double)rt.h[n];
    sg[8] = 1.0L;
    fill_colloc(sg, T.sigf, T.W1f, T.W2f);
}

cudaError_t upload_adjoint_tables(cudaStream_t st)
{
    cudaError_t e = upload_step_tables(st);
    if (e != cudaSuccess) return e;
    static AdjTables T;
    static bool filled = false;
    if (!filled) {
        fill_adj_tables(T);
        filled = true;
    }
    return cudaMemcpyToSymbolAsync(g_adj, &T, sizeof(T), 0, cudaMemcpyHostToDevice, st);
}

// ---------------------------------------------------------------------------
// batches of one body's observations (the <= span rule of Sec. 2)
// ---------------------------------------------------------------------------
// The batch starting at j0 ends before the returned index; tref = midpoint.
__device__ __forceinline__ int next_batch(const kete_obs *o, int mi, int j0, double span,
                                          double &tref)
{
    const double e0 = o[j0].epoch;
    int j = j0;
    while (j + 1 < mi) {
        const double e = o[j + 1].epoch;
        if (!(e == e0 || e - e0 < span)) break;
        j++;
    }
    tref = 0.5 * (e0 + o[j].epoch);
    return j + 1;
}

// observations in use: those before the first non-finite epoch
__device__ __forceinline__ int obs_count(const kete_obs *o, int m)
{
    int mi = 0;
    while (mi < m && isfinite(o[mi].epoch)) mi++;
    return mi;
}

// ---------------------------------------------------------------------------
// forward-mode dual numbers
// ---------------------------------------------------------------------------
// forward-mode dual number with 6 tangents (d/d r0, d/d v0)
struct D6 {
    double v, d[6];
};
__device__ __forceinline__ D6 dconst(double a)
{
    D6 r;
    r.v = a;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = 0.0;
    return r;
}
__device__ __forceinline__ D6 operator+(const D6 &a, const D6 &b)
{
    D6 r;
    r.v = a.v + b.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = a.d[q] + b.d[q];
    return r;
}
__device__ __forceinline__ D6 operator-(const D6 &a, const D6 &b)
{
    D6 r;
    r.v = a.v - b.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = a.d[q] - b.d[q];
    return r;
}
__device__ __forceinline__ D6 operator*(const D6 &a, const D6 &b)
{
    D6 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = fma(a.d[q], b.v, a.v * b.d[q]);
    return r;
}
__device__ __forceinline__ D6 operator*(double s, const D6 &a)
{
    D6 r;
    r.v = s * a.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = s * a.d[q];
    return r;
}
__device__ __forceinline__ D6 operator+(double s, const D6 &a)
{
    D6 r = a;
    r.v = s + a.v;
    return r;
}
__device__ __forceinline__ D6 dinv(const D6 &a)
{
    D6 r;
    r.v = 1.0 / a.v;
    const double k = -r.v * r.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = k * a.d[q];
    return r;
}
__device__ __forceinline__ D6 dsqrt(const D6 &a)
{
    D6 r;
    r.v = sqrt(a.v);
    const double k = 0.5 / r.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = k * a.d[q];
    return r;
}

// dC/dz, dS/dz of the Stumpff functions: power series for |z| < 1
// (sum_k>=1 (-1)^k k z^(k-1) / (2k+2)!, resp. / (2k+3)!), else
// (1 - zS - 2C) / 2z and (C - 3S) / 2z.
__device__ __forceinline__ void stumpff_dz(double z, double C, double S, double &dC, double &dS)
{
    if (fabs(z) < 1.0) {
        double tc = -1.0 / 24.0, ts = -1.0 / 120.0;
        dC = tc;
        dS = ts;
        for (int k = 1; k < 14; k++) {
            const double kk = (double)k;
            tc *= -z * (kk + 1.0) / (kk * (2.0 * kk + 3.0) * (2.0 * kk + 4.0));
            ts *= -z * (kk + 1.0) / (kk * (2.0 * kk + 4.0) * (2.0 * kk + 5.0));
            dC += tc;
            dS += ts;
        }
    } else {
        dC = (1.0 - z * S - 2.0 * C) / (2.0 * z);
        dS = (C - 3.0 * S) / (2.0 * z);
    }
}

__device__ __forceinline__ void stumpff_dual(const D6 &z, D6 &C, D6 &S)
{
    double c, s, dc, ds;
    stumpff(z.v, c, s);
    stumpff_dz(z.v, c, s, dc, ds);
    C.v = c;
    S.v = s;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        C.d[q] = dc * z.d[q];
        S.d[q] = ds * z.d[q];
    }
}

// Jr[i][c] = d r_i(dt) / d(r0, v0)_c of the universal-variable solution, at
// fixed dt, from the converged universal anomaly chi: one Newton step of
// Kepler's equation in dual numbers starting at chi carries the implicit
// derivative of chi.
__device__ void kepler_jacobian(double mu, double sqmu, const double r0[3], const double v0[3],
                                double dt, double chi, double Jr[3][6])
{
    D6 R[3], V[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        R[c] = dconst(r0[c]);
        R[c].d[c] = 1.0;
        V[c] = dconst(v0[c]);
        V[c].d[3 + c] = 1.0;
    }
    const D6 rn0 = dsqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    const D6 vv = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const D6 rv = R[0] * V[0] + R[1] * V[1] + R[2] * V[2];
    const D6 alpha = 2.0 * dinv(rn0) - (1.0 / mu) * vv;
    const D6 A = (1.0 / sqmu) * rv;
    const D6 B = 1.0 + (-1.0) * (alpha * rn0);
    // Kepler's equation at fixed chi: F = A chi^2 C + B chi^3 S + rn0 chi - sqmu dt
    const double x2 = chi * chi;
    D6 C, S;
    stumpff_dual(x2 * alpha, C, S);
    const D6 Fk = (-sqmu * dt) + (x2 * (A * C) + (x2 * chi) * (B * S) + chi * rn0);
    const double z = x2 * alpha.v;
    const double dF = A.v * chi * (1.0 - z * S.v) + B.v * x2 * C.v + rn0.v;
    D6 X = (-1.0 / dF) * Fk;
    X.v = chi;   // the value stays the converged root; the tangent is -F_p / F_chi
    const D6 X2 = X * X;
    D6 C2, S2;
    stumpff_dual(X2 * alpha, C2, S2);
    const D6 f = 1.0 + (-1.0) * (X2 * C2 * dinv(rn0));
    const D6 g = dt + (-1.0 / sqmu) * (X2 * X * S2);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const D6 ri = f * R[i] + g * V[i];
#pragma unroll
        for (int c = 0; c < 6; c++) Jr[i][c] = ri.d[c];
    }
}

__device__ __forceinline__ D6 operator*(const D6 &a, double s) { return s * a; }
__device__ __forceinline__ D6 ddot(const D6 a[3], const D6 b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
// a^p, d(a^p) = p a^(p-1) da
__device__ __forceinline__ D6 dpow(const D6 &a, double p)
{
    D6 r;
    r.v = pow(a.v, p);
    const double k = p * r.v / a.v;
#pragma unroll
    for (int q = 0; q < 6; q++) r.d[q] = k * a.d[q];
    return r;
}
__device__ __forceinline__ void dcross(const D6 a[3], const D6 b[3], D6 c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// The universal-variable two-body map of a state (R0, V0) in dual numbers
// (any tangents) over a fixed dt: chi from the plain solve, its tangent from one
// Newton step of Kepler's equation at the converged root (see
// kepler_jacobian), then r = f R0 + g V0, v = fdot R0 + gdot V0.
__device__ bool kepler_dual(double mu, double sqmu, const D6 R0[3], const D6 V0[3], double dt,
                            D6 R[3], D6 V[3])
{
    const double r0v[3] = {R0[0].v, R0[1].v, R0[2].v}, v0v[3] = {V0[0].v, V0[1].v, V0[2].v};
    double chi = 0.0, rr[3], vr[3];
    const bool ok = kepler_uv(mu, sqmu, r0v, v0v, dt, chi, rr, vr);
    const D6 rn0 = dsqrt(ddot(R0, R0));
    const D6 vv = ddot(V0, V0);
    const D6 rv = ddot(R0, V0);
    const D6 alpha = 2.0 * dinv(rn0) - (1.0 / mu) * vv;
    const D6 A = (1.0 / sqmu) * rv;
    const D6 B = 1.0 + (-1.0) * (alpha * rn0);
    const double x2 = chi * chi;
    D6 C, S;
    stumpff_dual(x2 * alpha, C, S);
    const D6 Fk = (-sqmu * dt) + (x2 * (A * C) + (x2 * chi) * (B * S) + chi * rn0);
    const double z = x2 * alpha.v;
    const double dF = A.v * chi * (1.0 - z * S.v) + B.v * x2 * C.v + rn0.v;
    D6 X = (-1.0 / dF) * Fk;
    X.v = chi;
    const D6 X2 = X * X;
    const D6 Z = X2 * alpha;
    D6 C2, S2;
    stumpff_dual(Z, C2, S2);
    const D6 f = 1.0 + (-1.0) * (X2 * C2 * dinv(rn0));
    const D6 g = dt + (-1.0 / sqmu) * (X2 * X * S2);
#pragma unroll
    for (int i = 0; i < 3; i++) R[i] = f * R0[i] + g * V0[i];
    const D6 rn = dsqrt(ddot(R, R));
    const D6 fd = sqmu * (dinv(rn * rn0) * (((-1.0) + Z * S2) * X));
    const D6 gd = 1.0 + (-1.0) * (X2 * C2 * dinv(rn));
#pragma unroll
    for (int i = 0; i < 3; i++) V[i] = fd * R0[i] + gd * V0[i];
    return ok;
}

// da/dx and da/dv (row-major 3x3, a_i by x_c) of the force terms beyond the
// Newtonian point masses at (t0 + off, x, v): the GR term (Eq. A.3) and the J2
// term (Eq. A.4) of every mass that carries them, and the body's
// non-gravitational terms (App. A.4-A.5: radiation pressure with drag, the JPL
// comet model with its thermal lag through the two-body map), by forward-mode
// dual numbers with the six tangents of (x, v).  The Newtonian da/dx
// (newton_jacobian, symmetric) is added by the caller.
__device__ int extra_jacobian(const EphemDev &E, const ForceDev &F, double t0, double off,
                              const double x[3], const double v[3], const kete_nongrav *ng,
                              double Ax[9], double Av[9])
{
    Seg g;
    if (!ephem_seg(E, t0, off, g)) return KETE_BODY_OUT_OF_SPAN;
    D6 X[3], V[3], a[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        X[c] = dconst(x[c]);
        X[c].d[c] = 1.0;
        V[c] = dconst(v[c]);
        V[c].d[3 + c] = 1.0;
        a[c] = dconst(0.0);
    }
    for (int m = 0; m < E.n_bodies; m++) {
        if (!((F.active_mask >> m) & 1u)) continue;
        const bool gr = (F.gr_mask >> m) & 1u, j2 = (F.j2_mask >> m) & 1u;
        if (!gr && !j2) continue;
        double st[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        cheb_state64(E, m, g.s, g.tau, st, gr);
        D6 r[3], w[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            r[c] = (-st[c]) + X[c];
            w[c] = (-st[3 + c]) + V[c];
        }
        const double mu = E.gm[m];
        const D6 ri = dinv(dsqrt(ddot(r, r)));
        const D6 ri2 = ri * ri, ri3 = ri2 * ri;
        if (gr) {   // mu / (c^2 r^3) [(4 mu / r - w^2) r + 4 (r.w) w]
            const D6 k = (mu * kInvC2) * ri3;
            const D6 f = k * ((4.0 * mu) * ri + (-1.0) * ddot(w, w));
            const D6 fw = 4.0 * (k * ddot(r, w));
#pragma unroll
            for (int c = 0; c < 3; c++) a[c] = a[c] + f * r[c] + fw * w[c];
        }
        if (j2) {   // -psi [(1 - 5 z^2 / r^2) r + 2 z p], psi = 1.5 J2 mu R^2 / r^5
            const double *P = F.pole[m];
            const D6 z = P[0] * r[0] + P[1] * r[1] + P[2] * r[2];
            const D6 psi = F.j2k[m] * (ri3 * ri2);
            const D6 q = 5.0 * (z * z * ri2);
            const D6 f = (-1.0) * (psi * (1.0 + (-1.0) * q));
            const D6 fp = -2.0 * (psi * z);
#pragma unroll
            for (int c = 0; c < 3; c++) a[c] = a[c] + f * r[c] + fp * P[c];
        }
    }
    if (ng) {
        const kete_nongrav p = *ng;
        const double mu = E.gm[0];
        double sun[6];
        cheb_state64(E, 0, g.s, g.tau, sun, true);
        D6 r[3], w[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            r[c] = (-sun[c]) + X[c];
            w[c] = (-sun[3 + c]) + V[c];
        }
        if (p.beta != 0.0) {   // beta mu / r^2 [(1 - rdot / c) rhat - w / c]
            const D6 rr = ddot(r, r);
            const D6 rin = dinv(dsqrt(rr));
            const D6 rdot = ddot(r, w) * rin;
            const D6 f = (p.beta * mu) * dinv(rr);
            const D6 kr = f * (1.0 + (-kInvC) * rdot) * rin;
            const D6 kw = kInvC * f;
#pragma unroll
            for (int c = 0; c < 3; c++) a[c] = a[c] + kr * r[c] + (-1.0) * (kw * w[c]);
        }
        if (p.a1 != 0.0 || p.a2 != 0.0 || p.a3 != 0.0) {
            D6 rl[3], wl[3];
            if (p.dt != 0.0) {
                if (!kepler_dual(mu, sqrt(mu), r, w, -p.dt, rl, wl)) return KETE_BODY_KEPLER_CAP;
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++) { rl[c] = r[c]; wl[c] = w[c]; }
            }
            const D6 rn = dsqrt(ddot(rl, rl));
            const D6 q = (1.0 / p.r0) * rn;
            D6 gq = p.alpha * dpow(q, -p.m);
            if (p.k != 0.0) gq = gq * dpow(1.0 + dpow(q, p.n), -p.k);
            const D6 irn = dinv(rn);
            D6 rh[3], h[3], nh[3], th[3];
#pragma unroll
            for (int c = 0; c < 3; c++) rh[c] = rl[c] * irn;
            dcross(rl, wl, h);
            const D6 ihn = dinv(dsqrt(ddot(h, h)));
#pragma unroll
            for (int c = 0; c < 3; c++) nh[c] = h[c] * ihn;
            dcross(nh, rh, th);
#pragma unroll
            for (int c = 0; c < 3; c++)
                a[c] = a[c] + gq * (p.a1 * rh[c] + p.a2 * th[c] + p.a3 * nh[c]);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            Ax[3 * i + c] = a[i].d[c];
            Av[3 * i + c] = a[i].d[3 + c];
        }
    return KETE_BODY_OK;
}

// The full model's Jacobian at the 8 nodes of an accepted step (t0, x0, v0,
// a0, the attempt's final corrector coefficients A.b and size A.h): node n at
// x(s) = x0 + s h v0 + (s h)^2 [a0/2 + sum_k b_k s^(k+1) / ((k+2)(k+3))],
// v(s) = v0 + s h [a0 + sum_k b_k s^(k+1) / (k+2)], da/dx beyond the Newtonian
// part and da/dv from extra_jacobian, to out[18 n .. 18 n + 17].
__device__ __noinline__ int record_extra(const EphemDev &E, const ForceDev &F, double t0,
                                         const double x0[3], const double v0[3],
                                         const double a0[3], const Attempt &A,
                                         const kete_nongrav *ng, double *out)
{
    for (int n = 0; n < 8; n++) {
        const double sh = g_rt.h[n] * A.h;
        double xn[3], vn[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double px = A.b[6][i] * g_rt.wx[n][6];
            double pv = A.b[6][i] * g_rt.wv[n][6];
#pragma unroll
            for (int k = 5; k >= 0; k--) {
                px = fma(A.b[k][i], g_rt.wx[n][k], px);
                pv = fma(A.b[k][i], g_rt.wv[n][k], pv);
            }
            px = fma(a0[i], 0.5, px);
            pv = pv + a0[i];
            xn[i] = x0[i] + fma(sh * sh, px, sh * v0[i]);
            vn[i] = fma(sh, pv, v0[i]);
        }
        const int st = extra_jacobian(E, F, t0, sh, xn, vn, ng, out + 18 * n, out + 18 * n + 9);
        if (st != KETE_BODY_OK) return st;
    }
    return KETE_BODY_OK;
}

// ---------------------------------------------------------------------------
// forward pass
// ---------------------------------------------------------------------------
// Per-lane walk over one body's stops: the batch midpoints and the checkpoint
// grid epoch0 + k ckpt (before the last midpoint), merged in ascending order.
struct StopWalk {
    int mi, nb;          // observations in use, batches
    int kb, j1;          // next batch, end of its observations
    double tref;         // its midpoint
    int kc;              // next checkpoint index
    double tc, t_last;   // its epoch, the last midpoint
    bool ckpt_ok;        // tc is a stop
};

// the next stop of the walk (call only while w.kb < w.nb); mid: a midpoint
__device__ __forceinline__ double walk_target(const StopWalk &w, bool &mid)
{
    mid = !(w.ckpt_ok && w.tc < w.tref);
    return mid ? w.tref : w.tc;
}

__device__ __forceinline__ void walk_next_ckpt(StopWalk &w, double epoch0, double ckpt)
{
    w.kc++;
    w.tc = epoch0 + (double)w.kc * ckpt;
    w.ckpt_ok = w.tc < w.t_last;
}

// One lane per body at a time, one step attempt per loop iteration (lanes of a
// warp stay in step while their bodies sit at different stops).  refill = 1:
// persistent grid, a lane whose body is done takes the next one from *next.
// RICH: a body with non-gravitational terms has them in its force, and each
// of its records gets the full model's Jacobian (B.recx) besides the
// Newtonian da/dx; a body whose terms are all zero keeps the Newtonian
// records (B.rich[i] tells which).
template <bool RICH>
__global__ void __launch_bounds__(128)
k_adj_forward(EphemDev E, ForceDev F, AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc,
              unsigned long long *__restrict__ next, int refill, const int32_t *__restrict__ order)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    Cnt cnt = {0, 0, 0, 0, 0};
    int64_t i = -1;   // current body (chunk index); -1: none; nc: no work left
    double x[3], v[3], t = 0.0, dt = 0.0, epoch0 = 0.0, ts = 0.0;
    bool mid = false, capped = false;
    int status = KETE_BODY_OK, count = 0;
    long long attempts = 0;
    const kete_obs *o = nullptr;
    StopWalk W;
    StepState S;
    S.have_a0 = false;
    S.ng = nullptr;   // set per body on the full-model path
    S.ng_chi = 0.0;
    const LegView L = leg_view(nullptr, 0);
    double *rec = nullptr, *recx = nullptr;   // recx: null for a body without terms
    bool first = true;
    for (;;) {
        const bool need = (i < 0);
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (refill) {
                if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
            }
            if (need) {
                unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
                if (!refill)
                    mine = first ? (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x
                                 : (unsigned long long)nc;
                if (mine < (unsigned long long)nc) {
                    i = order ? (int64_t)order[mine] : (int64_t)mine;
                    const int64_t gi = i0 + i;
                    o = P.obs + gi * P.m;
                    bool fin = true;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x[c] = P.states[c * P.n + gi];
                        v[c] = P.states[(3 + c) * P.n + gi];
                        fin = fin && isfinite(x[c]) && isfinite(v[c]);
                    }
                    epoch0 = P.epochs[gi];
                    t = epoch0;
                    dt = 0.0;
                    status = (fin && isfinite(epoch0)) ? KETE_BODY_OK : KETE_BODY_NONFINITE;
                    W.mi = obs_count(o, P.m);
                    for (int j = 1; j < W.mi; j++)
                        if (o[j].epoch < o[j - 1].epoch) {
                            atomicOr(&P.ctr->error_flags, 1 << 6);
                            status = KETE_BODY_NONFINITE;
                        }
                    // batches and the last midpoint (the checkpoint grid ends there)
                    W.nb = 0;
                    W.t_last = epoch0;
                    for (int j0 = 0; j0 < W.mi; W.nb++) j0 = next_batch(o, W.mi, j0, P.span, W.t_last);
                    W.kb = 0;
                    W.j1 = (W.mi > 0) ? next_batch(o, W.mi, 0, P.span, W.tref) : 0;
                    W.kc = 1;
                    W.tc = epoch0 + P.ckpt;
                    W.ckpt_ok = P.ckpt > 0.0 && W.tc < W.t_last;
                    rec = B.rec + (size_t)i * B.cap * kAdjRec;
                    if (RICH) {
                        const kete_nongrav *p = F.nongrav ? F.nongrav + gi : nullptr;
                        const bool terms = p && (p->a1 != 0.0 || p->a2 != 0.0 ||
                                                 p->a3 != 0.0 || p->beta != 0.0);
                        recx = terms ? B.recx + (size_t)i * B.cap * kAdjRecX : nullptr;
                        S.ng = terms ? p : nullptr;
                        S.ng_chi = 0.0;
                    }
                    count = 0;
                    capped = false;
                    attempts = 0;
                    S.have_a0 = false;
                    if (W.kb < W.nb) {
                        ts = walk_target(W, mid);
                        aim_step(F, t, ts, dt);
                    }
                } else {
                    i = nc;
                }
            }
        }
        first = false;
        const bool active = (i >= 0 && i < nc);
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;
        if (status == KETE_BODY_OK && W.kb < W.nb && t != ts) {
            if (++attempts > F.max_steps) {
                status = KETE_BODY_STEP_CAP;
            } else {
                const int slot = count < B.cap - 1 ? count : B.cap - 2;
                double *r = rec + (size_t)slot * kAdjRec;
                const double t_prev = t;
                if (RICH && recx) {   // the accepted attempt's coefficients give the node states
                    const double x0[3] = {x[0], x[1], x[2]}, v0[3] = {v[0], v[1], v[2]};
                    Attempt A;
                    status = step_begin<KETE_FP64, true>(E, F, L, x, v, t, dt, ts, S, A, cnt, r + 2);
                    while (status == KETE_BODY_OK) {
                        bool done = false;
                        status = attempt_sweep<KETE_FP64, true>(E, F, t, x, v, S.a0, S.as0,
                                                                S.close, S.enc, A, done, cnt,
                                                                r + 2, S.ng, &S.ng_chi);
                        if (done) break;
                    }
                    if (status == KETE_BODY_OK)
                        status = step_end<KETE_FP64>(F, A, x, v, t, dt, S, cnt);
                    if (status == KETE_BODY_OK && t != t_prev)
                        status = record_extra(E, F, t_prev, x0, v0, S.a0, A, S.ng,
                                              recx + (size_t)slot * kAdjRecX);
                } else {
                    status = step_once<KETE_FP64, true>(E, F, L, x, v, t, dt, ts, S, cnt, r + 2);
                }
                if (status == KETE_BODY_OK && t != t_prev) {
                    r[0] = t_prev;
                    r[1] = t;
                    if (count < B.cap - 1) count++;
                    else capped = true;
                }
            }
            if (status == KETE_BODY_OK && t != ts) continue;
        }
        // at the stop ts (or failed): bookkeeping, then the next stop
        if (status == KETE_BODY_OK && W.kb < W.nb) {
            if (mid) {
                double *y = B.yref + ((size_t)i * P.m + W.kb) * 6;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    y[c] = x[c];
                    y[3 + c] = v[c];
                }
                B.bidx[(size_t)i * P.m + W.kb] = count;
                if (W.ckpt_ok && W.tc == W.tref) walk_next_ckpt(W, epoch0, P.ckpt);   // one stop
                W.kb++;
                if (W.kb < W.nb) W.j1 = next_batch(o, W.mi, W.j1, P.span, W.tref);
            } else if (W.kc >= kAdjMaxCkpt) {   // bounded work per body
                status = KETE_BODY_STEP_CAP;
            } else {
                walk_next_ckpt(W, epoch0, P.ckpt);
            }
            if (status == KETE_BODY_OK && W.kb < W.nb) {
                ts = walk_target(W, mid);
                aim_step(F, t, ts, dt);
                S.have_a0 = false;
                attempts = 0;
                continue;
            }
        }
        // the body is done
        if (status == KETE_BODY_OK && !capped) {
            // terminal record: da/dx at the final state closes the last step
            double *r = rec + (size_t)count * kAdjRec;
            double a[3], J[6];
            Encounter enc;
            const double zero[3] = {0.0, 0.0, 0.0};
            status = accel_fp64<true>(E, F, t, 0.0, nullptr, x, v, a, enc, zero, true, J, S.ng,
                                      &S.ng_chi);
            cnt.evals++;
            r[0] = t;
            r[1] = t;
#pragma unroll
            for (int q = 0; q < 6; q++) r[2 + q] = J[q];
            if (RICH && recx && status == KETE_BODY_OK) {
                double *rx = recx + (size_t)count * kAdjRecX;
                status = extra_jacobian(E, F, t, 0.0, x, v, S.ng, rx, rx + 9);
            }
            count++;
        }
        if (status == KETE_BODY_OK && capped) status = KETE_BODY_ADJ_CAP;
        B.n_rec[i] = (status == KETE_BODY_OK) ? count : 0;
        B.nbat[i] = W.nb;
        B.status[i] = status;
        if (RICH) B.rich[i] = recx ? 1 : 0;
        i = -1;
    }
    flush_counters(cnt, P.ctr);
}

// ---------------------------------------------------------------------------
// observation operator and its partials
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool sun_at(const EphemDev &E, double t0, double off, double p[3],
                                       double v[3])
{
    Seg g;
    if (!ephem_seg(E, t0, off, g)) return false;
    cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, p, v);
    return true;
}

__device__ __forceinline__ double wrap_pi(double a)
{
    while (a > kPi) a -= kTwoPi;
    while (a <= -kPi) a += kTwoPi;
    return a;
}

// warp per body, lane per observation (m <= 32)
__global__ void __launch_bounds__(128)
k_adj_observe(EphemDev E, AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc)
{
    __shared__ double sh[4][32][7];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= nc) return;   // whole warp
    const int64_t gi = i0 + i;
    const kete_obs *o = P.obs + gi * P.m;
    const int mi = obs_count(o, P.m);
    int st = B.status[i];
    // this lane's batch
    int kb = -1, j0 = 0, j1 = 0;
    double tref = 0.0;
    {
        int b = 0, s0 = 0;
        while (s0 < mi) {
            double tr;
            const int s1 = next_batch(o, mi, s0, P.span, tr);
            if (lane >= s0 && lane < s1) {
                kb = b;
                j0 = s0;
                j1 = s1;
                tref = tr;
            }
            s0 = s1;
            b++;
        }
    }
    double Lj = 0.0, gj[6] = {0, 0, 0, 0, 0, 0};
    double ra = __longlong_as_double(0x7ff8000000000000ll), dec = ra;
    bool bad = false, jac_done = false;
    const bool mine = (lane < mi) && (st == KETE_BODY_OK || st == KETE_BODY_ADJ_CAP);
    if (mine) {
        const double *y = B.yref + ((size_t)i * P.m + kb) * 6;
        const kete_obs ob = o[lane];
        double sp[3], sv[3], hr[3], hv[3];
        bool ok = sun_at(E, tref, 0.0, sp, sv);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            hr[c] = y[c] - sp[c];
            hv[c] = y[3 + c] - sv[c];
        }
        const double mu = E.gm[0], sqmu = sqrt(mu);
        const double dt_obs = ob.epoch - tref;   // intervals before absolute epochs
        double chi = 0.0, r[3], vh[3], pos[3], su[3], svel[3], tau = 0.0;
        // position at the epoch t_ref + d: Sun there plus the two-body offset
        auto at = [&](double d) {
            bool good = sun_at(E, tref, d, su, svel);
            good = kepler_uv(mu, sqmu, hr, hv, d, chi, r, vh) && good;
#pragma unroll
            for (int c = 0; c < 3; c++) pos[c] = su[c] + r[c];
            return good;
        };
        auto dist = [&]() {
            const double d0 = pos[0] - ob.obs[0], d1 = pos[1] - ob.obs[1], d2 = pos[2] - ob.obs[2];
            return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        };
        ok = at(dt_obs) && ok;
        tau = dist() * kInvC;
        for (int it = 0; it < 3; it++) {
            ok = at(dt_obs - tau) && ok;
            tau = dist() * kInvC;
        }
        const double dfin = dt_obs - tau;
        ok = at(dfin) && ok;
        if (!ok) {
            bad = true;
        } else {
            const double u[3] = {pos[0] - ob.obs[0], pos[1] - ob.obs[1], pos[2] - ob.obs[2]};
            radec(u, P.cos_eps, P.sin_eps, ra, dec);
            const double cd = cos(ob.dec);
            const double r0 = wrap_pi(ra - ob.ra) * cd, r1 = dec - ob.dec;
            Lj = r0 * r0 + r1 * r1;
            // partials of RA and Dec with respect to u: in the equatorial frame,
            // dRA = (-Y, X, 0) / rxy^2, dDec = (-X Z, -Y Z, rxy^2) / (|u|^2 rxy),
            // rotated back to the ecliptic
            const double X = u[0];
            const double Y = P.cos_eps * u[1] - P.sin_eps * u[2];
            const double Z = P.sin_eps * u[1] + P.cos_eps * u[2];
            const double rxy2 = X * X + Y * Y, rxy = sqrt(rxy2), uu = rxy2 + Z * Z;
            const double ia = 1.0 / rxy2, id = 1.0 / (uu * rxy);
            const double aY = X * ia;
            const double dY = -Y * Z * id, dZ = rxy2 * id;
            double wa[3] = {-Y * ia, P.cos_eps * aY, -P.sin_eps * aY};
            double wd[3] = {-X * Z * id, P.cos_eps * dY + P.sin_eps * dZ,
                            -P.sin_eps * dY + P.cos_eps * dZ};
            // light time: u = P(t_obs - tau) - obs with tau = |u| / c, so
            // du = P_y dy - Pdot dtau, dtau = rho.P_y dy / (c + rho.Pdot)
            const double un = sqrt(uu);
            const double rh[3] = {u[0] / un, u[1] / un, u[2] / un};
            const double pd[3] = {vh[0] + svel[0], vh[1] + svel[1], vh[2] + svel[2]};
            const double den = kC + (rh[0] * pd[0] + rh[1] * pd[1] + rh[2] * pd[2]);
            const double pa = (wa[0] * pd[0] + wa[1] * pd[1] + wa[2] * pd[2]) / den;
            const double pdd = (wd[0] * pd[0] + wd[1] * pd[1] + wd[2] * pd[2]) / den;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                wa[c] -= pa * rh[c];
                wd[c] -= pdd * rh[c];
            }
            double Jr[3][6];
            kepler_jacobian(mu, sqmu, hr, hv, dfin, chi, Jr);
            double ga[6], gd[6];   // d RA / d y(t_ref), d Dec / d y(t_ref)
#pragma unroll
            for (int c = 0; c < 6; c++) {
                ga[c] = wa[0] * Jr[0][c] + wa[1] * Jr[1][c] + wa[2] * Jr[2][c];
                gd[c] = wd[0] * Jr[0][c] + wd[1] * Jr[1][c] + wd[2] * Jr[2][c];
                gj[c] = fma(2.0 * r0 * cd, ga[c], 2.0 * r1 * gd[c]);
            }
            if (P.jac && st == KETE_BODY_OK) {
                // rows of the orbit-fit Jacobian: d(RA, Dec)/d y(t_ref) Phi
                const double *phi = B.phi + ((size_t)i * P.m + kb) * 36;
                double *jr = P.jac + (gi * P.m + lane) * 12;
#pragma unroll
                for (int c0 = 0; c0 < 6; c0++) {
                    double sa = 0.0, sd = 0.0;
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        const double p = phi[c * 6 + c0];
                        sa = fma(ga[c], p, sa);
                        sd = fma(gd[c], p, sd);
                    }
                    jr[c0] = sa;
                    jr[6 + c0] = sd;
                }
                jac_done = true;
            }
        }
        if (P.pred) {
            P.pred[(gi * P.m + lane) * 2] = ra;
            P.pred[(gi * P.m + lane) * 2 + 1] = dec;
        }
    } else if (P.pred && lane < P.m) {
        P.pred[(gi * P.m + lane) * 2] = ra;
        P.pred[(gi * P.m + lane) * 2 + 1] = dec;
    }
    if (P.jac && lane < P.m && !jac_done) {   // unused slot or failed body: NaN rows
        double *jr = P.jac + (gi * P.m + lane) * 12;
        for (int q = 0; q < 12; q++) jr[q] = __longlong_as_double(0x7ff8000000000000ll);
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (P.jac && any_bad && lane < P.m) {   // a failed body has no Jacobian
        double *jr = P.jac + (gi * P.m + lane) * 12;
        for (int q = 0; q < 12; q++) jr[q] = __longlong_as_double(0x7ff8000000000000ll);
    }
    sh[w][lane][0] = Lj;
#pragma unroll
    for (int c = 0; c < 6; c++) sh[w][lane][1 + c] = gj[c];
    __syncwarp();
    // loss in observation order; gradient jumps summed per batch in order
    if (lane == 0) {
        double L = 0.0;
        for (int j = 0; j < mi; j++) L += sh[w][j][0];
        const bool ok = (st == KETE_BODY_OK || st == KETE_BODY_ADJ_CAP) && !any_bad;
        if (any_bad && st == KETE_BODY_OK) st = KETE_BODY_KEPLER_CAP;
        if (P.loss) P.loss[gi] = ok ? L : __longlong_as_double(0x7ff8000000000000ll);
        B.status[i] = st;
        if (P.status) P.status[gi] = st;
    }
    if (mine && lane == j0) {
        double g[6] = {0, 0, 0, 0, 0, 0};
        for (int j = j0; j < j1; j++)
#pragma unroll
            for (int c = 0; c < 6; c++) g[c] += sh[w][j][1 + c];
        double *dst = B.gjump + ((size_t)i * P.m + kb) * 6;
#pragma unroll
        for (int c = 0; c < 6; c++) dst[c] = g[c];
    }
}

// ---------------------------------------------------------------------------
// backward pass
// ---------------------------------------------------------------------------
// sample k of a step in the backward order (see AdjTables): J at sig[k]
__device__ __forceinline__ const double *jac_sample(const double *r, const double *r_next, int k)
{
    if (k == 0) return r_next + 2;            // step end = next record's node 0
    return r + 2 + 6 * (8 - k);               // forward node 8-k (k = 8: node 0)
}

__device__ __forceinline__ void jmul(const double *J, const double m[3], double out[3])
{
    const double j0 = __ldg(J), j1 = __ldg(J + 1), j2 = __ldg(J + 2), j3 = __ldg(J + 3),
                 j4 = __ldg(J + 4), j5 = __ldg(J + 5);
    out[0] = fma(j0, m[0], fma(j1, m[1], j2 * m[2]));
    out[1] = fma(j1, m[0], fma(j3, m[1], j4 * m[2]));
    out[2] = fma(j2, m[0], fma(j4, m[1], j5 * m[2]));
}

__global__ void __launch_bounds__(128)
k_adj_backward(AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int64_t gi = i0 + i;
    const int st = B.status[i];
    if (st != KETE_BODY_OK) {
        for (int c = 0; c < 6; c++) P.grad[c * P.n + gi] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int count = B.n_rec[i];
    int kb = B.nbat[i] - 1;
    const double *rec = B.rec + (size_t)i * B.cap * kAdjRec;
    const int32_t *bidx = B.bidx + (size_t)i * P.m;
    const double *gjump = B.gjump + (size_t)i * P.m * 6;
    double mu[3] = {0, 0, 0}, mud[3] = {0, 0, 0};   // lambda_v and d lambda_v / dt
    for (int s = count - 2; s >= -1; s--) {
        // jumps of the batches whose midpoint the chain reached after s+1 steps
        while (kb >= 0 && bidx[kb] == s + 1) {
            const double *g = gjump + kb * 6;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                mud[c] -= g[c];       // lambda_x += dL/dx
                mu[c] += g[3 + c];    // lambda_v += dL/dv
            }
            kb--;
        }
        if (s < 0) break;
        if (mu[0] == 0.0 && mu[1] == 0.0 && mu[2] == 0.0 && mud[0] == 0.0 && mud[1] == 0.0 &&
            mud[2] == 0.0)
            continue;
        const double *r = rec + (size_t)s * kAdjRec;
        const double *rn = r + kAdjRec;
        const double h = __ldg(r + 1) - __ldg(r);
        const double h2 = h * h;
        // s-derivative at the step end: d mu / ds = -h d mu / dt
        const double q0[3] = {-h * mud[0], -h * mud[1], -h * mud[2]};
        double Fk[9][3], mk[9][3];
#pragma unroll
        for (int k = 0; k < 9; k++) {
#pragma unroll
            for (int c = 0; c < 3; c++) mk[k][c] = fma(g_adj.sig[k], q0[c], mu[c]);
            jmul(jac_sample(r, rn, k), mk[k], Fk[k]);
#pragma unroll
            for (int c = 0; c < 3; c++) Fk[k][c] *= h2;
        }
        // Picard iteration of the collocation equations (a linear system with
        // contraction ~ h^2 |J|); at most 12 sweeps
        for (int it = 0; it < 12; it++) {
            double delta = 0.0, size = 0.0;
#pragma unroll
            for (int k = 1; k < 9; k++) {
                double nm[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    double acc = fma(g_adj.sig[k], q0[c], mu[c]);
#pragma unroll
                    for (int j = 0; j < 9; j++) acc = fma(g_adj.W2[k][j], Fk[j][c], acc);
                    nm[c] = acc;
                }
                if (k == 8) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        delta = fmax(delta, fabs(nm[c] - mk[8][c]));
                        size = fmax(size, fabs(nm[c]));
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; c++) mk[k][c] = nm[c];
            }
#pragma unroll
            for (int k = 1; k < 9; k++) {
                jmul(jac_sample(r, rn, k), mk[k], Fk[k]);
#pragma unroll
                for (int c = 0; c < 3; c++) Fk[k][c] *= h2;
            }
            if (delta <= 1e-16 * size) break;
        }
        double q8[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double acc = q0[c];
#pragma unroll
            for (int j = 0; j < 9; j++) acc = fma(g_adj.W1[8][j], Fk[j][c], acc);
            q8[c] = acc;
            mu[c] = mk[8][c];
            mud[c] = -q8[c] / h;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        P.grad[c * P.n + gi] = -mud[c];
        P.grad[(3 + c) * P.n + gi] = mu[c];
    }
}

// ---------------------------------------------------------------------------
// state-transition matrix at the batch midpoints
// ---------------------------------------------------------------------------
// sample k of a step in the forward order: J at node k (k <= 7), at the step
// end (k = 8: the next record's node 0)
__device__ __forceinline__ const double *jac_sample_fwd(const double *r, const double *r_next, int k)
{
    return k == 8 ? r_next + 2 : r + 2 + 6 * k;
}

// One lane per body: the six columns (dx, dv) of Phi obey dx'' = J(t) dx.  Over
// a recorded step of size h, with s = (t - t_start) / h and F_k = h^2 J_k dx_k
// at the samples s_k (node 0..7, end):
//   dx(s_n) = dx_0 + s_n h dv_0 + sum_k W2f[n][k] F_k,
//   dv(1)   = dv_0 + (1/h) sum_k W1f[8][k] F_k,
// solved by Picard iteration (contraction ~ h^2 |J|, at most 12 sweeps).
// Phi is stored at each batch midpoint when the chain reaches it.
__global__ void __launch_bounds__(128)
k_adj_stm(AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int st = B.status[i];
    if (st != KETE_BODY_OK) return;   // the observation kernel writes NaN rows
    const int count = B.n_rec[i];
    const int nb = B.nbat[i];
    const double *rec = B.rec + (size_t)i * B.cap * kAdjRec;
    const int32_t *bidx = B.bidx + (size_t)i * P.m;
    double *phi_out = B.phi + (size_t)i * P.m * 36;
    for (int c0 = 0; c0 < 6; c0++) {
        double dx[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
        if (c0 < 3) dx[c0] = 1.0;
        else dv[c0 - 3] = 1.0;
        int kb = 0;
        for (int s = 0; s <= count - 1; s++) {
            // batches whose midpoint the chain reached after s steps
            while (kb < nb && bidx[kb] == s) {
                double *ph = phi_out + (size_t)kb * 36;
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    ph[r * 6 + c0] = dx[r];
                    ph[(3 + r) * 6 + c0] = dv[r];
                }
                kb++;
            }
            if (s == count - 1) break;
            const double *r = rec + (size_t)s * kAdjRec;
            const double *rn = r + kAdjRec;
            const double h = __ldg(r + 1) - __ldg(r);
            const double h2 = h * h;
            double xk[9][3], Fk[9][3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
#pragma unroll
                for (int c = 0; c < 3; c++) xk[k][c] = fma(g_adj.sigf[k] * h, dv[c], dx[c]);
                jmul(jac_sample_fwd(r, rn, k), xk[k], Fk[k]);
#pragma unroll
                for (int c = 0; c < 3; c++) Fk[k][c] *= h2;
            }
            for (int it = 0; it < 12; it++) {
                double delta = 0.0, size = 0.0;
#pragma unroll
                for (int k = 1; k < 9; k++) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        double acc = fma(g_adj.sigf[k] * h, dv[c], dx[c]);
#pragma unroll
                        for (int j = 0; j < 9; j++) acc = fma(g_adj.W2f[k][j], Fk[j][c], acc);
                        if (k == 8) {
                            delta = fmax(delta, fabs(acc - xk[8][c]));
                            size = fmax(size, fabs(acc));
                        }
                        xk[k][c] = acc;
                    }
                }
#pragma unroll
                for (int k = 1; k < 9; k++) {
                    jmul(jac_sample_fwd(r, rn, k), xk[k], Fk[k]);
#pragma unroll
                    for (int c = 0; c < 3; c++) Fk[k][c] *= h2;
                }
                if (delta <= 1e-16 * size) break;
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < 9; j++) acc = fma(g_adj.W1f[8][j], Fk[j][c], acc);
                dv[c] += acc / h;
                dx[c] = xk[8][c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the full force model: da/dx beyond the Newtonian part and da/dv
// ---------------------------------------------------------------------------
// extension (Ex, Av) of backward sample k (see jac_sample)
__device__ __forceinline__ const double *jacx_sample(const double *rx, const double *rx_next, int k)
{
    if (!rx) return nullptr;   // a body without terms
    return k == 0 ? rx_next : rx + 18 * (8 - k);
}

// extension of forward sample k (see jac_sample_fwd)
__device__ __forceinline__ const double *jacx_sample_fwd(const double *rx, const double *rx_next,
                                                         int k)
{
    if (!rx) return nullptr;   // a body without terms
    return k == 8 ? rx_next : rx + 18 * k;
}

// adjoint right-hand sides: G = h^2 (J + Ex)^T m, H = h Av^T m (J symmetric,
// Ex and Av row-major a_i by x_c; X null: a body without terms, Ex = Av = 0)
__device__ __forceinline__ void adj_rhs_full(const double *J, const double *X, double h,
                                             const double m[3], double G[3], double H[3])
{
    double jm[3];
    jmul(J, m, jm);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double ex = 0.0, av = 0.0;
        if (X) {
            ex = fma(__ldg(X + c), m[0], fma(__ldg(X + 3 + c), m[1], __ldg(X + 6 + c) * m[2]));
            av = fma(__ldg(X + 9 + c), m[0], fma(__ldg(X + 12 + c), m[1], __ldg(X + 15 + c) * m[2]));
        }
        G[c] = h * h * (jm[c] + ex);
        H[c] = h * av;
    }
}

// variational right-hand side: F = h^2 ((J + Ex) dx + Av dv) (X null: Ex = Av = 0)
__device__ __forceinline__ void var_rhs_full(const double *J, const double *X, double h,
                                             const double dx[3], const double dv[3], double F[3])
{
    double jx[3];
    jmul(J, dx, jx);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double ex = 0.0, av = 0.0;
        if (X) {
            const double *e = X + 3 * c, *a = X + 9 + 3 * c;
            ex = fma(__ldg(e), dx[0], fma(__ldg(e + 1), dx[1], __ldg(e + 2) * dx[2]));
            av = fma(__ldg(a), dv[0], fma(__ldg(a + 1), dv[1], __ldg(a + 2) * dv[2]));
        }
        F[c] = h * h * (jx[c] + ex + av);
    }
}

// Backward pass of the full model.  The adjoints (lx, mu) = (lambda_x,
// lambda_v) obey lx' = -Ax^T mu, mu' = -lx - Av^T mu.  In the backward variable
// s = (t_end - t) / h of a recorded step, with G_k = h^2 Ax^T mu_k and
// H_k = h Av^T mu_k at the samples sig_k:
//   mu(sig_n) = mu_0 + sig_n h lx_0 + sum_k (W2[n][k] G_k + W1[n][k] H_k),
//   lx(1)     = lx_0 + (1/h) sum_k W1[8][k] G_k,
// solved by Gauss-Seidel sweeps over the samples (contraction ~ h^2 |Ax| +
// h |Av|, at most 16 sweeps).  Without the extension this is k_adj_backward.
__global__ void __launch_bounds__(128)
k_adj_backward_full(AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int64_t gi = i0 + i;
    if (B.status[i] != KETE_BODY_OK) {
        for (int c = 0; c < 6; c++) P.grad[c * P.n + gi] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int count = B.n_rec[i];
    int kb = B.nbat[i] - 1;
    const double *rec = B.rec + (size_t)i * B.cap * kAdjRec;
    const double *recx = B.rich[i] ? B.recx + (size_t)i * B.cap * kAdjRecX : nullptr;
    const int32_t *bidx = B.bidx + (size_t)i * P.m;
    const double *gjump = B.gjump + (size_t)i * P.m * 6;
    double mu[3] = {0, 0, 0}, lx[3] = {0, 0, 0};
    for (int s = count - 2; s >= -1; s--) {
        while (kb >= 0 && bidx[kb] == s + 1) {
            const double *g = gjump + kb * 6;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                lx[c] += g[c];
                mu[c] += g[3 + c];
            }
            kb--;
        }
        if (s < 0) break;
        if (mu[0] == 0.0 && mu[1] == 0.0 && mu[2] == 0.0 && lx[0] == 0.0 && lx[1] == 0.0 &&
            lx[2] == 0.0)
            continue;
        const double *r = rec + (size_t)s * kAdjRec;
        const double *rn = r + kAdjRec;
        const double *rx = recx ? recx + (size_t)s * kAdjRecX : nullptr;
        const double *rxn = recx ? rx + kAdjRecX : nullptr;
        const double h = __ldg(r + 1) - __ldg(r);
        const double q0[3] = {h * lx[0], h * lx[1], h * lx[2]};
        double G[9][3], H[9][3], m8[3];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double m[3];
#pragma unroll
            for (int c = 0; c < 3; c++) m[c] = fma(g_adj.sig[k], q0[c], mu[c]);
            adj_rhs_full(jac_sample(r, rn, k), jacx_sample(rx, rxn, k), h, m, G[k], H[k]);
            if (k == 8)
#pragma unroll
                for (int c = 0; c < 3; c++) m8[c] = m[c];
        }
        for (int it = 0; it < 16; it++) {
            double delta = 0.0, size = 0.0;
#pragma unroll
            for (int n = 1; n < 9; n++) {
                double m[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    double acc = fma(g_adj.sig[n], q0[c], mu[c]);
#pragma unroll
                    for (int j = 0; j < 9; j++)
                        acc = fma(g_adj.W2[n][j], G[j][c], fma(g_adj.W1[n][j], H[j][c], acc));
                    m[c] = acc;
                }
                if (n == 8) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        delta = fmax(delta, fabs(m[c] - m8[c]));
                        size = fmax(size, fabs(m[c]));
                        m8[c] = m[c];
                    }
                }
                adj_rhs_full(jac_sample(r, rn, n), jacx_sample(rx, rxn, n), h, m, G[n], H[n]);
            }
            if (delta <= 1e-16 * size) break;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < 9; j++) acc = fma(g_adj.W1[8][j], G[j][c], acc);
            lx[c] += acc / h;
            mu[c] = m8[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        P.grad[c * P.n + gi] = lx[c];
        P.grad[(3 + c) * P.n + gi] = mu[c];
    }
}

// State-transition matrix of the full model: the columns (dx, dv) obey
// dx' = dv, dv' = Ax dx + Av dv.  In the forward variable of a recorded step,
// with F_k = h^2 (Ax dx_k + Av dv_k) at the samples (node 0..7, step end):
//   dx(s_n) = dx_0 + s_n h dv_0 + sum_k W2f[n][k] F_k,
//   dv(s_n) = dv_0 + (1/h) sum_k W1f[n][k] F_k,
// Gauss-Seidel sweeps as in k_adj_backward_full.
__global__ void __launch_bounds__(128)
k_adj_stm_full(AdjBuffers B, AdjProblem P, int64_t i0, int64_t nc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    if (B.status[i] != KETE_BODY_OK) return;   // the observation kernel writes NaN rows
    const int count = B.n_rec[i];
    const int nb = B.nbat[i];
    const double *rec = B.rec + (size_t)i * B.cap * kAdjRec;
    const double *recx = B.rich[i] ? B.recx + (size_t)i * B.cap * kAdjRecX : nullptr;
    const int32_t *bidx = B.bidx + (size_t)i * P.m;
    double *phi_out = B.phi + (size_t)i * P.m * 36;
    for (int c0 = 0; c0 < 6; c0++) {
        double dx[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
        if (c0 < 3) dx[c0] = 1.0;
        else dv[c0 - 3] = 1.0;
        int kb = 0;
        for (int s = 0; s <= count - 1; s++) {
            while (kb < nb && bidx[kb] == s) {
                double *ph = phi_out + (size_t)kb * 36;
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    ph[q * 6 + c0] = dx[q];
                    ph[(3 + q) * 6 + c0] = dv[q];
                }
                kb++;
            }
            if (s == count - 1) break;
            const double *r = rec + (size_t)s * kAdjRec;
            const double *rn = r + kAdjRec;
            const double *rx = recx ? recx + (size_t)s * kAdjRecX : nullptr;
            const double *rxn = recx ? rx + kAdjRecX : nullptr;
            const double h = __ldg(r + 1) - __ldg(r);
            const double ih = 1.0 / h;
            double F[9][3], x8[3], v8[3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                double xk[3];
#pragma unroll
                for (int c = 0; c < 3; c++) xk[c] = fma(g_adj.sigf[k] * h, dv[c], dx[c]);
                var_rhs_full(jac_sample_fwd(r, rn, k), jacx_sample_fwd(rx, rxn, k), h, xk, dv,
                             F[k]);
                if (k == 8)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x8[c] = xk[c];
                        v8[c] = dv[c];
                    }
            }
            for (int it = 0; it < 16; it++) {
                double delta = 0.0, size = 0.0;
#pragma unroll
                for (int n = 1; n < 9; n++) {
                    double xn[3], vn[3];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        double ax = fma(g_adj.sigf[n] * h, dv[c], dx[c]), av = 0.0;
#pragma unroll
                        for (int j = 0; j < 9; j++) {
                            ax = fma(g_adj.W2f[n][j], F[j][c], ax);
                            av = fma(g_adj.W1f[n][j], F[j][c], av);
                        }
                        xn[c] = ax;
                        vn[c] = fma(av, ih, dv[c]);
                    }
                    if (n == 8) {
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            delta = fmax(delta, fmax(fabs(xn[c] - x8[c]), fabs(h * (vn[c] - v8[c]))));
                            size = fmax(size, fmax(fabs(xn[c]), fabs(h * vn[c])));
                            x8[c] = xn[c];
                            v8[c] = vn[c];
                        }
                    }
                    var_rhs_full(jac_sample_fwd(r, rn, n), jacx_sample_fwd(rx, rxn, n), h, xn, vn,
                                 F[n]);
                }
                if (delta <= 1e-16 * size) break;
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < 9; j++) acc = fma(g_adj.W1f[8][j], F[j][c], acc);
                dv[c] = fma(acc, ih, dv[c]);
                dx[c] = x8[c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// last observation epoch of each body of the chunk (its chain's end)
__global__ void k_adj_last_epoch(AdjProblem P, int64_t i0, int64_t nc, double *__restrict__ t_end)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const kete_obs *o = P.obs + (i0 + i) * P.m;
    const int mi = obs_count(o, P.m);
    t_end[i] = mi > 0 ? o[mi - 1].epoch : P.epochs[i0 + i];
}

cudaError_t launch_adjoint_last_epoch(const AdjProblem &P, int64_t i0, int64_t nc, double *t_end,
                                      cudaStream_t st)
{
    if (nc > 0) k_adj_last_epoch<<<blocks_for(nc, 256), 256, 0, st>>>(P, i0, nc, t_end);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_forward(const EphemDev &E, const ForceDev &F, const AdjBuffers &B,
                                   const AdjProblem &P, int64_t i0, int64_t nc,
                                   unsigned long long *next, cudaStream_t st,
                                   const int32_t *order)
{
    if (nc <= 0) return cudaGetLastError();
    int64_t grid = blocks_for(nc, 128);
    int refill = 0;
    if (next) {   // persistent grid with work stealing
        cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (B.recx) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_forward<true>, 128, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_forward<false>, 128, 0);
        const int64_t persistent = (int64_t)(sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
        if (grid > persistent) grid = persistent;
        refill = 1;
    }
    if (B.recx) k_adj_forward<true><<<(unsigned)grid, 128, 0, st>>>(E, F, B, P, i0, nc, next, refill, order);
    else k_adj_forward<false><<<(unsigned)grid, 128, 0, st>>>(E, F, B, P, i0, nc, next, refill, order);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_observe(const EphemDev &E, const AdjBuffers &B, const AdjProblem &P,
                                   int64_t i0, int64_t nc, cudaStream_t st)
{
    if (nc > 0) k_adj_observe<<<blocks_for(nc, 4), 128, 0, st>>>(E, B, P, i0, nc);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_stm(const AdjBuffers &B, const AdjProblem &P, int64_t i0, int64_t nc,
                               cudaStream_t st)
{
    if (nc <= 0) return cudaGetLastError();
    if (B.recx) k_adj_stm_full<<<blocks_for(nc, 128), 128, 0, st>>>(B, P, i0, nc);
    else k_adj_stm<<<blocks_for(nc, 128), 128, 0, st>>>(B, P, i0, nc);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_backward(const AdjBuffers &B, const AdjProblem &P, int64_t i0,
                                    int64_t nc, cudaStream_t st)
{
    if (nc <= 0) return cudaGetLastError();
    if (B.recx) k_adj_backward_full<<<blocks_for(nc, 128), 128, 0, st>>>(B, P, i0, nc);
    else k_adj_backward<<<blocks_for(nc, 128), 128, 0, st>>>(B, P, i0, nc);
    return cudaGetLastError();
}

}  // namespace kete
