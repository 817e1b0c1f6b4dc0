// kete_device.cuh -- device-side building blocks of the survey path.
//
// Ephemeris lookup (Sec. 3.2 / App. A), force model (Eq. A.1 with the GR term
// of Eq. A.3 and the J2 term of Eq. A.4), Gauss-Radau 15th-order step with
// IAS15 corrector convergence and step control, predictor removed (App. A.6),
// universal-variable two-body propagation and light-delay correction (Sec. 2),
// spherical-polygon test (Sec. 3.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kete_impl.h"

namespace kete {

// ---------------------------------------------------------------------------
// physical constants (App. A.1 units: AU, TDB days)
// ---------------------------------------------------------------------------
constexpr double kKmPerAu = 149597870.7;
constexpr double kC = 299792.458 * 86400.0 / kKmPerAu;   // speed of light, AU/day
constexpr double kInvC2 = 1.0 / (kC * kC);
constexpr double kInvC = 1.0 / kC;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

// Gauss-Radau spacings (Everhart 1985), h_0 = 0
struct RadauTables {
    double h[8];
    double rinv[8][8];   // 1 / (h_n - h_k), k < n
    double c[8][7];      // c[n][m]: d b_m / d g_n  (Newton -> power basis)
};

// ---------------------------------------------------------------------------
// Ephemeris: uniform segments, Clenshaw summation
// ---------------------------------------------------------------------------
struct Seg {
    int s;
    double tau;
};

// Segment and Chebyshev argument at the epoch t0 + off.  tau is formed as
// 2((t0 - t_mid) + off)/L so that a small offset (a substep, a light-time
// interval) is never rounded to the resolution of an absolute Julian date.
__device__ __forceinline__ bool ephem_seg(const EphemDev &E, double t0, double off, Seg &g)
{
    const double t = t0 + off;
    if (!(t >= E.t_start && t <= E.t_end)) return false;
    int s = (int)floor((t - E.t_start) * E.inv_seg);
    s = s < 0 ? 0 : (s > E.n_seg - 1 ? E.n_seg - 1 : s);
    double t_mid = E.t_start + ((double)s + 0.5) * E.seg_len;
    g.s = s;
    g.tau = 2.0 * ((t0 - t_mid) + off) * E.inv_seg;
    return true;
}

// position of one body: sum_k c_k T_k(tau) by Clenshaw's recurrence
__device__ __forceinline__ void cheb_pos(const double *__restrict__ c, int nc, double tau,
                                         double p[3])
{
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double *cd = c + d * nc;
        double b1 = 0.0, b2 = 0.0;
        for (int k = nc - 1; k >= 1; k--) {
            double b0 = fma(2.0 * tau, b1, __ldg(cd + k) - b2);
            b2 = b1;
            b1 = b0;
        }
        p[d] = fma(tau, b1, __ldg(cd) - b2);
    }
}

// position and d/dtau (T_k' = k U_{k-1}, Clenshaw on the U series)
__device__ __forceinline__ void cheb_pos_vel(const double *__restrict__ c, int nc, double tau,
                                             double dtau_dt, double p[3], double v[3])
{
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double *cd = c + d * nc;
        double b1 = 0.0, b2 = 0.0, u1 = 0.0, u2 = 0.0;
        for (int k = nc - 1; k >= 1; k--) {
            double ck = __ldg(cd + k);
            double b0 = fma(2.0 * tau, b1, ck - b2);
            double u0 = fma(2.0 * tau, u1, (double)k * ck - u2);
            b2 = b1;
            b1 = b0;
            u2 = u1;
            u1 = u0;
        }
        p[d] = fma(tau, b1, __ldg(cd) - b2);
        v[d] = u1 * dtau_dt;
    }
}

__device__ __forceinline__ const double *ephem_coef(const EphemDev &E, int body, int s)
{
    return E.coef + ((size_t)body * E.n_seg + s) * 3 * E.n_coef;
}

// ---------------------------------------------------------------------------
// Force model (Eq. A.1): for each active mass m with r = x - x_m, v = v - v_m:
//   Newton  -mu r / |r|^3
//   GR      mu / (c^2 |r|^3) [ (4 mu/|r| - |v|^2) r + 4 (r.v) v ]       (Eq. A.3)
//   J2      -(3/2) J2 mu R^2 / |r|^5 [ (1 - 5 z^2/|r|^2) r + 2 z p ]     (Eq. A.4,
//           z = r.p with p the body's pole; the same vector written in the
//           body's equatorial frame is the component form of Eq. A.4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int accel_fp64(const EphemDev &E, const ForceDev &F, double t0,
                                          double off, const double x[3], const double v[3],
                                          double a[3])
{
    Seg g;
    a[0] = a[1] = a[2] = 0.0;
    if (!ephem_seg(E, t0, off, g)) return KETE_BODY_OUT_OF_SPAN;
    const double dtau_dt = 2.0 * E.inv_seg;
    for (int m = 0; m < E.n_bodies; m++) {
        if (!((F.active_mask >> m) & 1u)) continue;
        const double mu = E.gm[m];
        const double *c = ephem_coef(E, m, g.s);
        const bool gr = (F.gr_mask >> m) & 1u;
        double p[3], pv[3];
        if (gr)
            cheb_pos_vel(c, E.n_coef, g.tau, dtau_dt, p, pv);
        else
            cheb_pos(c, E.n_coef, g.tau, p);
        double r0 = x[0] - p[0], r1 = x[1] - p[1], r2 = x[2] - p[2];
        double rr = fma(r0, r0, fma(r1, r1, r2 * r2));
        double ri = rsqrt(rr);
        double ri2 = ri * ri;
        double ri3 = ri2 * ri;
        double f = -mu * ri3;
        if (gr) {
            double w0 = v[0] - pv[0], w1 = v[1] - pv[1], w2 = v[2] - pv[2];
            double ww = fma(w0, w0, fma(w1, w1, w2 * w2));
            double rw = fma(r0, w0, fma(r1, w1, r2 * w2));
            double k = mu * ri3 * kInvC2;
            double fr = k * fma(4.0 * mu, ri, -ww);
            double fw = 4.0 * k * rw;
            f += fr;
            a[0] = fma(fw, w0, a[0]);
            a[1] = fma(fw, w1, a[1]);
            a[2] = fma(fw, w2, a[2]);
        }
        if ((F.j2_mask >> m) & 1u) {
            const double *P = F.pole[m];
            double z = fma(r0, P[0], fma(r1, P[1], r2 * P[2]));
            double psi = F.j2k[m] * ri3 * ri2;   // 1.5 J2 mu R^2 / r^5
            double q = 5.0 * z * z * ri2;
            f = fma(-psi, 1.0 - q, f);
            double fp = -2.0 * psi * z;
            a[0] = fma(fp, P[0], a[0]);
            a[1] = fma(fp, P[1], a[1]);
            a[2] = fma(fp, P[2], a[2]);
        }
        a[0] = fma(f, r0, a[0]);
        a[1] = fma(f, r1, a[1]);
        a[2] = fma(f, r2, a[2]);
    }
    return KETE_BODY_OK;
}

// ---------------------------------------------------------------------------
// universal-variable two-body propagation
// ---------------------------------------------------------------------------
// Stumpff C(z), S(z): nested (Horner) form of the power series for |z| < 1,
// closed trigonometric / hyperbolic forms otherwise.
__device__ __forceinline__ void stumpff(double z, double &C, double &S)
{
    if (fabs(z) < 1.0) {
        // C = 1/2 (1 - z/(3.4) (1 - z/(5.6) (1 - ...)))
        double c = 1.0, s = 1.0;
        c = fma(-z * (1.0 / (23.0 * 24.0)), c, 1.0);
        c = fma(-z * (1.0 / (21.0 * 22.0)), c, 1.0);
        c = fma(-z * (1.0 / (19.0 * 20.0)), c, 1.0);
        c = fma(-z * (1.0 / (17.0 * 18.0)), c, 1.0);
        c = fma(-z * (1.0 / (15.0 * 16.0)), c, 1.0);
        c = fma(-z * (1.0 / (13.0 * 14.0)), c, 1.0);
        c = fma(-z * (1.0 / (11.0 * 12.0)), c, 1.0);
        c = fma(-z * (1.0 / (9.0 * 10.0)), c, 1.0);
        c = fma(-z * (1.0 / (7.0 * 8.0)), c, 1.0);
        c = fma(-z * (1.0 / (5.0 * 6.0)), c, 1.0);
        c = fma(-z * (1.0 / (3.0 * 4.0)), c, 1.0);
        C = 0.5 * c;
        // S = 1/6 (1 - z/(4.5) (1 - z/(6.7) (1 - ...)))
        s = fma(-z * (1.0 / (24.0 * 25.0)), s, 1.0);
        s = fma(-z * (1.0 / (22.0 * 23.0)), s, 1.0);
        s = fma(-z * (1.0 / (20.0 * 21.0)), s, 1.0);
        s = fma(-z * (1.0 / (18.0 * 19.0)), s, 1.0);
        s = fma(-z * (1.0 / (16.0 * 17.0)), s, 1.0);
        s = fma(-z * (1.0 / (14.0 * 15.0)), s, 1.0);
        s = fma(-z * (1.0 / (12.0 * 13.0)), s, 1.0);
        s = fma(-z * (1.0 / (10.0 * 11.0)), s, 1.0);
        s = fma(-z * (1.0 / (8.0 * 9.0)), s, 1.0);
        s = fma(-z * (1.0 / (6.0 * 7.0)), s, 1.0);
        s = fma(-z * (1.0 / (4.0 * 5.0)), s, 1.0);
        S = s * (1.0 / 6.0);
    } else if (z > 0.0) {
        double q = sqrt(z), sn, cs;
        sincos(q, &sn, &cs);
        C = (1.0 - cs) / z;
        S = (q - sn) / (z * q);
    } else {
        double q = sqrt(-z);
        C = (cosh(q) - 1.0) / (-z);
        S = (sinh(q) - q) / (-z * q);
    }
}

// Heliocentric state (r0, v0) advanced by dt under mu.  chi is the universal
// anomaly: in = initial guess (0 = none), out = solution (warm start).
// Returns false if Newton's iteration did not converge.
__device__ __forceinline__ bool kepler_uv(double mu, double sqmu, const double r0[3],
                                          const double v0[3], double dt, double &chi,
                                          double r[3], double v[3])
{
    double rn0 = sqrt(fma(r0[0], r0[0], fma(r0[1], r0[1], r0[2] * r0[2])));
    double vv = fma(v0[0], v0[0], fma(v0[1], v0[1], v0[2] * v0[2]));
    double rv = fma(r0[0], v0[0], fma(r0[1], v0[1], r0[2] * v0[2]));
    double alpha = 2.0 / rn0 - vv / mu;
    double A = rv / sqmu;
    double B = 1.0 - alpha * rn0;
    double target = sqmu * dt;
    if (chi == 0.0) chi = target / rn0;
    double C = 0.5, S = 1.0 / 6.0, z = 0.0;
    bool ok = false;
    for (int it = 0; it < 64; it++) {
        double x2 = chi * chi;
        z = alpha * x2;
        stumpff(z, C, S);
        double Fv = fma(A * x2, C, fma(B * x2 * chi, S, fma(rn0, chi, -target)));
        double dF = fma(A * chi, fma(-z, S, 1.0), fma(B * x2, C, rn0));
        double step = Fv / dF;
        // keep the iterate on the solution's side of zero and bounded in growth
        double nxt = chi - step;
        if ((nxt > 0.0) != (dt > 0.0) && dt != 0.0) nxt = 0.5 * chi;
        chi = nxt;
        if (fabs(step) <= 1e-15 * fabs(chi) || Fv == 0.0) {
            ok = true;
            break;
        }
    }
    double x2 = chi * chi;
    z = alpha * x2;
    stumpff(z, C, S);
    double f = 1.0 - x2 / rn0 * C;
    double gg = dt - x2 * chi * S / sqmu;
    r[0] = fma(f, r0[0], gg * v0[0]);
    r[1] = fma(f, r0[1], gg * v0[1]);
    r[2] = fma(f, r0[2], gg * v0[2]);
    double rn = sqrt(fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2])));
    double fd = sqmu / (rn * rn0) * fma(z, S, -1.0) * chi;
    double gd = 1.0 - x2 / rn * C;
    v[0] = fma(fd, r0[0], gd * v0[0]);
    v[1] = fma(fd, r0[1], gd * v0[1]);
    v[2] = fma(fd, r0[2], gd * v0[2]);
    return ok;
}

// RA/Dec (equatorial J2000) of an ecliptic vector
__device__ __forceinline__ void radec(const double u[3], double cos_eps, double sin_eps,
                                      double &ra, double &dec)
{
    double x = u[0];
    double y = cos_eps * u[1] - sin_eps * u[2];
    double z = sin_eps * u[1] + cos_eps * u[2];
    double a = atan2(y, x);
    if (a < 0.0) a += kTwoPi;
    if (a >= kTwoPi) a = 0.0;
    ra = a;
    dec = atan2(z, sqrt(x * x + y * y));
}

}  // namespace kete
