/*
 * kete_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Built with -O2 -ffp-contract=off.  Every function is written for a reader
 * checking it against the paper by eye; speed is not a goal.  The CUDA path
 * never includes, links or calls this file.
 *
 * Readings of the paper (where it is silent, ambiguous or garbled):
 *  R1 (Eq. A.1/A.3/A.4 sign convention): r = r_body - r_m, v = v_body - v_m;
 *     Newton a = -mu r/|r|^3, GR as printed in Eq. A.3 with that r and v,
 *     J2 = -psi [(1-5z^2/r^2)x, (1-5z^2/r^2)y, (3-5z^2/r^2)z] in the body's
 *     equatorial frame.
 *  R2 (App. A.2/A.3): GR for Sun, Jupiter and Earth; J2 for Sun and Jupiter.
 *  R4 (App. A.6, predictor removed): every step starts its corrector from
 *     b = 0 and iterates until converged or the cap.
 *  R5 (App. A.6, "tuned" constants): IAS15's step control eps 1e-9, safety
 *     factor 0.25, cap 12 iterations, stop early when the error stops
 *     decreasing; the corrector threshold on max|db6|/max|a| is tuned to 1e-10
 *     (IAS15 uses 1e-16): b6 enters a position as h^2 b6/72, so the looser
 *     threshold drops the iteration that only confirms convergence at
 *     round-off, moving one-year positions by < 5e-14 AU (measured over main
 *     belt, NEOs, Trojans, comets to e = 0.99 and 0.002 AU Earth encounters).
 *  R6 (Sec. 2, batches): greedy batches over epoch-sorted FoVs, a batch holds
 *     the epochs t with t - t_first < span; t_ref = (t_first + t_last)/2.
 *  R7 (Sec. 2, two-body): heliocentric, mu = GM_sun, Sun position re-added at
 *     the target time.
 *  R8 (Sec. 2, light delay): tau0 = |r(t)-o|/c, then three fixed iterations
 *     tau <- |r(t-tau)-o|/c; apparent vector u = r(t-tau)-o.  No aberration.
 *  R9 (Sec. 3.1): inside iff every n_i.u > 0 (strict).
 *  R10 (time bookkeeping, not in the paper): epochs are absolute TDB Julian
 *     dates, so every step is taken as the exact difference of the two
 *     representable epochs it joins; the last step of a leg lands exactly on
 *     the target epoch.  Two-body intervals are formed as (t_obs - t_ref) - tau
 *     before any absolute epoch is rounded, and the planets are evaluated at
 *     (epoch, offset) pairs: the Chebyshev argument is 2((t0 - t_mid) + off)/L,
 *     so substep epochs carry no rounding of the absolute date (which would
 *     otherwise add noise the corrector's b6 estimate amplifies near planets).
 *     A step that rounds to zero length ends the leg with KO_STEP_CAP.
 *  R12 (close encounters, not in the paper): with a planet within 0.1 AU at
 *     the step start, the body-planet vector at a substep is formed as
 *     (x0 - p(t0)) + (dx - dp) from the displacements since the step start
 *     (dp by a recurrence on Chebyshev differences), and the step ends at the
 *     next table segment boundary.  The force is unchanged; its rounding noise
 *     (~1e-16 AU of ~1 AU coordinates, large relative to a 0.001 AU distance)
 *     no longer reaches b6, which would otherwise shrink the step forever.
 *  R11 (Sec. 2, chain of batch midpoints): a body is integrated from its epoch
 *     to the first batch midpoint, then from each midpoint to the next; the
 *     proposed step size is carried along the chain.
 */
#include "kete_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- constants (App. A.1 units: AU, TDB days) ---------------------------- */
static const double KM_PER_AU = 149597870.7;
static double c_au_per_day(void) { return 299792.458 * 86400.0 / KM_PER_AU; }
static double deg2rad(double d) { return d * (M_PI / 180.0); }
static double obliquity(void) { return deg2rad(84381.448 / 3600.0); }

void ko_force_model_default(ko_force_model *fm)
{
    memset(fm, 0, sizeof(*fm));
    fm->body_mask = 0x1FF;                          /* Sun + 8 planets */
    fm->gr_mask = (1u << 0) | (1u << 3) | (1u << 5); /* Sun, Earth, Jupiter */
    fm->j2_mask = (1u << 0) | (1u << 5);             /* Sun, Jupiter */
    fm->max_iter = 12;
    /* Sun */
    fm->j2[0] = 2.1961e-7;
    fm->radius[0] = 696000.0 / KM_PER_AU;
    fm->pole_ra[0] = deg2rad(286.13);
    fm->pole_dec[0] = deg2rad(63.87);
    /* Jupiter */
    fm->j2[5] = 0.014736;
    fm->radius[5] = 71492.0 / KM_PER_AU;
    fm->pole_ra[5] = deg2rad(268.056595);
    fm->pole_dec[5] = deg2rad(64.495303);
    fm->eps = 1e-9;
    fm->eps_pc = 1e-10;
    fm->safety = 0.25;
    fm->dt_init = 4.0;
    fm->max_steps = 100000;
}

/* ---- ephemeris table (App. A: SPICE-like segment lookup) ----------------- */
int ko_ephem_load(ko_ephem *e, const void *buf, size_t n)
{
    const unsigned char *p = (const unsigned char *)buf;
    int32_t hdr[4];
    double td[2];
    memset(e, 0, sizeof(*e));
    if (n < 256 || memcmp(p, "KETECHB1", 8) != 0) return -1;
    memcpy(hdr, p + 8, sizeof(hdr));
    memcpy(td, p + 24, sizeof(td));
    /* at most 64 coefficients: the recurrences below keep T_k, U_k, D_k in
     * arrays of 64 */
    if (hdr[0] != 1 || hdr[1] < 1 || hdr[1] > KO_MAX_BODIES || hdr[2] < 1 || hdr[2] > 64 ||
        hdr[3] < 1)
        return -1;
    e->n_bodies = hdr[1];
    e->n_coef = hdr[2];
    e->n_seg = hdr[3];
    e->t_start = td[0];
    e->seg_len = td[1];
    memcpy(e->gm, p + 48, sizeof(double) * KO_MAX_BODIES);
    size_t nc = (size_t)e->n_bodies * e->n_seg * 3 * e->n_coef;
    if (n < 256 + nc * sizeof(double) || !(e->seg_len > 0)) return -1;
    e->coef = (double *)malloc(nc * sizeof(double));
    if (!e->coef) return -1;
    memcpy(e->coef, p + 256, nc * sizeof(double));
    return 0;
}

void ko_ephem_free(ko_ephem *e)
{
    free(e->coef);
    e->coef = NULL;
}

/* Position (and velocity) of table body `body` at t0 + off: sum_k c_k T_k(tau)
 * with T_k from the textbook three-term recurrence; velocity from dT_k/dtau =
 * k U_{k-1}(tau) and dtau/dt = 2/L.  The Chebyshev argument is formed as
 * 2((t0 - t_mid) + off)/L so that a small offset from an epoch is not rounded
 * to the resolution of an absolute Julian date (R10). */
static int ephem_eval_off(const ko_ephem *e, int body, double t0, double off, double pos[3],
                          double vel[3])
{
    double t = t0 + off;
    double t_end = e->t_start + e->n_seg * e->seg_len;
    if (!(t >= e->t_start && t <= t_end)) return KO_OUT_OF_SPAN;
    int64_t s = (int64_t)floor((t - e->t_start) / e->seg_len);
    if (s < 0) s = 0;
    if (s > e->n_seg - 1) s = e->n_seg - 1;
    double t_mid = e->t_start + ((double)s + 0.5) * e->seg_len;
    double tau = 2.0 * ((t0 - t_mid) + off) / e->seg_len;
    double T[64], U[64];
    int nc = e->n_coef;
    T[0] = 1.0;
    T[1] = tau;
    U[0] = 1.0;
    U[1] = 2.0 * tau;
    for (int k = 2; k < nc; k++) {
        T[k] = 2.0 * tau * T[k - 1] - T[k - 2];
        U[k] = 2.0 * tau * U[k - 1] - U[k - 2];
    }
    for (int c = 0; c < 3; c++) {
        const double *cf = e->coef + (((size_t)body * e->n_seg + s) * 3 + c) * nc;
        double sp = 0.0, sv = 0.0;
        for (int k = 0; k < nc; k++) sp += cf[k] * T[k];
        for (int k = 1; k < nc; k++) sv += cf[k] * (double)k * U[k - 1];
        pos[c] = sp;
        if (vel) vel[c] = sv * 2.0 / e->seg_len;
    }
    return KO_OK;
}

int ko_ephem_eval(const ko_ephem *e, int body, double t, double pos[3], double vel[3])
{
    return ephem_eval_off(e, body, t, 0.0, pos, vel);
}

/* p(t0 + off) - p(t0) of table body `body`, both read from the segment that
 * holds t0 (R12): sum_k c_k (T_k(tau1) - T_k(tau0)) with the differences from
 * D_1 = tau1 - tau0, D_{k+1} = 2 tau1 D_k - D_{k-1} + 2 (tau1 - tau0) T_k(tau0),
 * so that a small displacement is not formed as the difference of two rounded
 * positions of size ~1 AU. */
static int ephem_delta(const ko_ephem *e, int body, double t0, double off, double dp[3])
{
    double t_end = e->t_start + e->n_seg * e->seg_len;
    if (!(t0 >= e->t_start && t0 <= t_end)) return KO_OUT_OF_SPAN;
    int64_t s = (int64_t)floor((t0 - e->t_start) / e->seg_len);
    if (s < 0) s = 0;
    if (s > e->n_seg - 1) s = e->n_seg - 1;
    double t_mid = e->t_start + ((double)s + 0.5) * e->seg_len;
    double tau0 = 2.0 * (t0 - t_mid) / e->seg_len;
    double dtau = 2.0 * off / e->seg_len;
    double tau1 = tau0 + dtau;
    int nc = e->n_coef;
    double T[64], D[64];
    T[0] = 1.0;
    T[1] = tau0;
    for (int k = 2; k < nc; k++) T[k] = 2.0 * tau0 * T[k - 1] - T[k - 2];
    D[0] = 0.0;
    D[1] = dtau;
    for (int k = 1; k + 1 < nc; k++) D[k + 1] = 2.0 * tau1 * D[k] - D[k - 1] + 2.0 * dtau * T[k];
    for (int c = 0; c < 3; c++) {
        const double *cf = e->coef + (((size_t)body * e->n_seg + s) * 3 + c) * nc;
        double sum = 0.0;
        for (int k = 1; k < nc; k++) sum += cf[k] * D[k];
        dp[c] = sum;
    }
    return KO_OK;
}

/* Close encounter (R12): the planet nearest the body at the step start, if it
 * is within KO_CLOSE_AU; its relative position at a substep is
 * (x0 - p(t0)) + (dx - dp) with dx, dp the body's and the planet's
 * displacements since the step start. */
#define KO_CLOSE_AU 0.1
typedef struct {
    int m;               /* table body, -1: none */
    double t0;           /* step start */
    double d0[3];        /* x0 - p_m(t0) */
    double dx[3];        /* body displacement x(t0 + off) - x0 of the current call */
} ko_close;

/* ---- optional non-gravitational terms (App. A.4, A.5) --------------------- */
static int ng_active(const ko_nongrav *p)
{
    return p->beta != 0.0 || p->a1 != 0.0 || p->a2 != 0.0 || p->a3 != 0.0;
}

/* Added to a: the non-gravitational acceleration of a body at heliocentric
 * position r and velocity w (mu = the Sun's GM).
 *   Eq. A.6 (radiation pressure + Poynting-Robertson drag), read as
 *     beta mu / |r|^2 [(1 - rdot/c) rhat - w/c],  rdot = rhat . w
 *   (the printed "(1 - v/c)" factor of the radial term is the radial speed).
 *   Eq. A.7 (JPL comet model): g(r') (A1 rhat' + A2 that' + A3 nhat') with
 *   (r', w') the two-body state dt days earlier, nhat' = r' x w' / |r' x w'|,
 *   that' = nhat' x rhat' (along the motion). */
static int nongrav_add(const ko_nongrav *p, double mu, const double r[3], const double w[3],
                       double a[3])
{
    const double c = c_au_per_day();
    if (p->beta != 0.0) {
        double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double rdot = (r[0] * w[0] + r[1] * w[1] + r[2] * w[2]) / rn;
        double f = p->beta * mu / (rn * rn);
        for (int i = 0; i < 3; i++) a[i] += f * ((1.0 - rdot / c) * r[i] / rn - w[i] / c);
    }
    if (p->a1 != 0.0 || p->a2 != 0.0 || p->a3 != 0.0) {
        double rl[3], wl[3];
        if (p->dt != 0.0) {
            int s = ko_kepler(mu, r, w, -p->dt, rl, wl);
            if (s != KO_OK) return s;
        } else {
            memcpy(rl, r, sizeof(rl));
            memcpy(wl, w, sizeof(wl));
        }
        double rn = sqrt(rl[0] * rl[0] + rl[1] * rl[1] + rl[2] * rl[2]);
        double q = rn / p->r0;
        double g = p->alpha * pow(q, -p->m) * pow(1.0 + pow(q, p->n), -p->k);
        double rh[3] = {rl[0] / rn, rl[1] / rn, rl[2] / rn};
        double h[3] = {rl[1] * wl[2] - rl[2] * wl[1], rl[2] * wl[0] - rl[0] * wl[2],
                       rl[0] * wl[1] - rl[1] * wl[0]};
        double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
        double nh[3] = {h[0] / hn, h[1] / hn, h[2] / hn};
        double th[3] = {nh[1] * rh[2] - nh[2] * rh[1], nh[2] * rh[0] - nh[0] * rh[2],
                        nh[0] * rh[1] - nh[1] * rh[0]};
        for (int i = 0; i < 3; i++) a[i] += g * (p->a1 * rh[i] + p->a2 * th[i] + p->a3 * nh[i]);
    }
    return KO_OK;
}

/* ---- force model: Eq. A.1 = sum over masses of Newton + A.3 + A.4 -------- */
static void pole_vector(double ra, double dec, double p[3])
{
    double eq[3] = {cos(dec) * cos(ra), cos(dec) * sin(ra), sin(dec)};
    double ce = cos(obliquity()), se = sin(obliquity());
    p[0] = eq[0];                      /* equatorial -> ecliptic */
    p[1] = ce * eq[1] + se * eq[2];
    p[2] = -se * eq[1] + ce * eq[2];
}

/* acceleration at epoch t0 + off (Eq. A.1); see ephem_eval_off for the offset */
static int accel_off_cl(const ko_ephem *e, const ko_force_model *fm, double t0, double off,
                        const double x[3], const double v[3], double a[3], const ko_close *cl);

static int accel_off(const ko_ephem *e, const ko_force_model *fm, double t0, double off,
                     const double x[3], const double v[3], double a[3])
{
    return accel_off_cl(e, fm, t0, off, x, v, a, NULL);
}

static int accel_off_cl(const ko_ephem *e, const ko_force_model *fm, double t0, double off,
                        const double x[3], const double v[3], double a[3], const ko_close *cl)
{
    const double c = c_au_per_day();
    a[0] = a[1] = a[2] = 0.0;
    for (int m = 0; m < e->n_bodies; m++) {
        if (!((fm->body_mask >> m) & 1u) || e->gm[m] == 0.0) continue;
        double pm[3], vm[3];
        int st = ephem_eval_off(e, m, t0, off, pm, vm);
        if (st != KO_OK) return st;
        double mu = e->gm[m];
        double r[3] = {x[0] - pm[0], x[1] - pm[1], x[2] - pm[2]};
        if (cl && cl->m == m) {
            double dp[3];
            st = ephem_delta(e, m, cl->t0, off, dp);
            if (st != KO_OK) return st;
            for (int i = 0; i < 3; i++) r[i] = cl->d0[i] + (cl->dx[i] - dp[i]);
        }
        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double rn = sqrt(r2);
        double r3 = r2 * rn;
        /* Newtonian point mass */
        for (int i = 0; i < 3; i++) a[i] += -mu * r[i] / r3;
        /* Eq. A.3: test-particle GR correction */
        if ((fm->gr_mask >> m) & 1u) {
            double w[3] = {v[0] - vm[0], v[1] - vm[1], v[2] - vm[2]};
            double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            double rw = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
            double k = mu / (c * c * r3);
            for (int i = 0; i < 3; i++)
                a[i] += k * ((4.0 * mu / rn - w2) * r[i] + 4.0 * rw * w[i]);
        }
        /* Eq. A.4: J2 in the body's equatorial frame, rotated back */
        if ((fm->j2_mask >> m) & 1u) {
            double p[3], e1[3], e2[3];
            pole_vector(fm->pole_ra[m], fm->pole_dec[m], p);
            /* e1 = normalize(z_ecl x p) (any axis in the equator will do) */
            e1[0] = -p[1];
            e1[1] = p[0];
            e1[2] = 0.0;
            double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
            if (n1 < 1e-12) { e1[0] = 1.0; e1[1] = 0.0; n1 = 1.0; }
            e1[0] /= n1;
            e1[1] /= n1;
            e2[0] = p[1] * e1[2] - p[2] * e1[1];
            e2[1] = p[2] * e1[0] - p[0] * e1[2];
            e2[2] = p[0] * e1[1] - p[1] * e1[0];
            double xb = r[0] * e1[0] + r[1] * e1[1] + r[2] * e1[2];
            double yb = r[0] * e2[0] + r[1] * e2[1] + r[2] * e2[2];
            double zb = r[0] * p[0] + r[1] * p[1] + r[2] * p[2];
            double psi = 1.5 * fm->j2[m] * mu * fm->radius[m] * fm->radius[m] / (r2 * r2 * rn);
            double q = 5.0 * zb * zb / r2;
            double ab[3] = {-psi * (1.0 - q) * xb, -psi * (1.0 - q) * yb, -psi * (3.0 - q) * zb};
            for (int i = 0; i < 3; i++) a[i] += ab[0] * e1[i] + ab[1] * e2[i] + ab[2] * p[i];
        }
    }
    if (ng_active(&fm->ng)) {
        /* heliocentric state: relative to table body 0, the Sun */
        double ps[3], vs[3];
        int st = ephem_eval_off(e, 0, t0, off, ps, vs);
        if (st != KO_OK) return st;
        double r[3] = {x[0] - ps[0], x[1] - ps[1], x[2] - ps[2]};
        double w[3] = {v[0] - vs[0], v[1] - vs[1], v[2] - vs[2]};
        st = nongrav_add(&fm->ng, e->gm[0], r, w, a);
        if (st != KO_OK) return st;
    }
    return KO_OK;
}

int ko_accel(const ko_ephem *e, const ko_force_model *fm, double t, const double x[3],
             const double v[3], double a[3])
{
    return accel_off(e, fm, t, 0.0, x, v, a);
}

/* ---- Gauss-Radau spacings: roots of P7(x)+P8(x) on [-1,1], h=(x+1)/2 ----- */
static double legendre(int n, double x)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) return p0;
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

static double radau_poly(double x) { return legendre(7, x) + legendre(8, x); }

void ko_radau_nodes(double h[8])
{
    /* x = -1 is a root; the other seven are bracketed on a fine grid and
     * bisected to the last bit. */
    int found = 0;
    h[found++] = 0.0;
    const int N = 40000;
    double xa = -1.0 + 1e-9, fa = radau_poly(xa);
    for (int i = 1; i <= N && found < 8; i++) {
        double xb = -1.0 + 1e-9 + (2.0 - 2e-9) * i / N, fb = radau_poly(xb);
        if ((fa < 0) != (fb < 0)) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi);
                if (mid == lo || mid == hi) break;
                double fm_ = radau_poly(mid);
                if ((fm_ < 0) == (flo < 0)) { lo = mid; flo = fm_; } else hi = mid;
            }
            h[found++] = 0.5 * (0.5 * (lo + hi) + 1.0);
        }
        xa = xb;
        fa = fb;
    }
}

/* ---- IAS15 tables computed from the spacings at first use ---------------- */
typedef struct {
    double h[8];
    double C[8][7];   /* C[j][m]: coefficient of s^(m+1) in s*prod_{i=1}^{j-1}(s-h_i), j=1..7 */
} ko_radau;

static ko_radau g_radau;
static pthread_once_t g_radau_once = PTHREAD_ONCE_INIT;

static void radau_init(void)
{
    ko_radau_nodes(g_radau.h);
    memset(g_radau.C, 0, sizeof(g_radau.C));
    for (int j = 1; j <= 7; j++) {
        /* poly[p] = coefficient of s^p of prod_{i=1}^{j-1}(s - h_i) */
        double poly[8] = {0};
        poly[0] = 1.0;
        int deg = 0;
        for (int i = 1; i <= j - 1; i++) {
            double nxt[8] = {0};
            for (int p = 0; p <= deg; p++) {
                nxt[p + 1] += poly[p];
                nxt[p] -= g_radau.h[i] * poly[p];
            }
            deg++;
            memcpy(poly, nxt, sizeof(poly));
        }
        /* multiply by s: coefficient of s^(p+1) is poly[p]; b index m = p */
        for (int p = 0; p <= deg; p++) g_radau.C[j][p] = poly[p];
    }
}

static const ko_radau *radau(void)
{
    pthread_once(&g_radau_once, radau_init);
    return &g_radau;
}

static int finite3(const double *x)
{
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

/* One attempt of a Gauss-Radau step of size dt from (t, x0, v0) with a0 given.
 * Fills x1, v1 and the IAS15 error estimate max|b6|/max|a|. */
static int radau_attempt(const ko_ephem *e, const ko_force_model *fm, double t,
                         const double x0[3], const double v0[3], const double a0[3],
                         double dt, double x1[3], double v1[3], double *err,
                         ko_stats *stats, ko_close *cl)
{
    const ko_radau *R = radau();
    double g[8][3], b[7][3], F[8][3];
    memset(g, 0, sizeof(g));
    memset(b, 0, sizeof(b));                /* R4: predictor removed, b = 0 */
    for (int i = 0; i < 3; i++) F[0][i] = a0[i];
    double pc_prev = 0.0;
    double amax = 0.0;
    for (int it = 1; it <= fm->max_iter; it++) {
        double b6_old[3] = {b[6][0], b[6][1], b[6][2]};
        for (int n = 1; n <= 7; n++) {
            double s = R->h[n];
            double xn[3], vn[3];
            for (int i = 0; i < 3; i++) {
                /* x(s) = x0 + v0 dt s + dt^2 (a0 s^2/2 + sum_k b_k s^(k+3)/((k+2)(k+3))) */
                double acc = a0[i] * s * s / 2.0;
                double vacc = a0[i] * s;
                double sp = s * s;  /* s^(k+2) */
                for (int k = 0; k < 7; k++) {
                    acc += b[k][i] * sp * s / ((k + 2.0) * (k + 3.0));
                    vacc += b[k][i] * sp / (k + 2.0);
                    sp *= s;
                }
                double dxn = v0[i] * dt * s + dt * dt * acc;
                xn[i] = x0[i] + dxn;
                vn[i] = v0[i] + dt * vacc;
                if (cl) cl->dx[i] = dxn;
            }
            int st = accel_off_cl(e, fm, t, s * dt, xn, vn, F[n], cl);
            if (stats) stats->force_evals++;
            if (st != KO_OK) return st;
            /* Newton divided difference g_n from F_0..F_n and g_1..g_{n-1} */
            for (int i = 0; i < 3; i++) {
                double d = (F[n][i] - F[0][i]) / (R->h[n] - R->h[0]);
                for (int k = 1; k < n; k++) d = (d - g[k][i]) / (R->h[n] - R->h[k]);
                g[n][i] = d;
            }
            /* power-basis coefficients b = C g */
            for (int m = 0; m < 7; m++)
                for (int i = 0; i < 3; i++) {
                    double sum = 0.0;
                    for (int j = m + 1; j <= 7; j++) sum += R->C[j][m] * g[j][i];
                    b[m][i] = sum;
                }
        }
        if (stats) stats->iterations++;
        double db = 0.0;
        amax = 0.0;
        for (int i = 0; i < 3; i++) {
            double d = fabs(b[6][i] - b6_old[i]);
            if (d > db) db = d;
            if (fabs(F[7][i]) > amax) amax = fabs(F[7][i]);
        }
        double pc = db / amax;
        if (!isfinite(pc)) return KO_NONFINITE;
        if (pc < fm->eps_pc) break;
        if (it >= 3 && pc >= pc_prev) break;
        pc_prev = pc;
    }
    double bmax = 0.0;
    for (int i = 0; i < 3; i++)
        if (fabs(b[6][i]) > bmax) bmax = fabs(b[6][i]);
    *err = bmax / amax;
    for (int i = 0; i < 3; i++) {
        double acc = a0[i] / 2.0, vacc = a0[i];
        for (int k = 0; k < 7; k++) {
            acc += b[k][i] / ((k + 2.0) * (k + 3.0));
            vacc += b[k][i] / (k + 2.0);
        }
        x1[i] = x0[i] + v0[i] * dt + dt * dt * acc;
        v1[i] = v0[i] + dt * vacc;
    }
    if (!finite3(x1) || !finite3(v1)) return KO_NONFINITE;
    return KO_OK;
}

/* Encounter set-up at a step start (R12): the nearest active planet within
 * KO_CLOSE_AU, and, if there is one, the step limit moved to the next table
 * segment boundary in the direction of motion (no step of an encounter
 * straddles a boundary of the piecewise planet polynomials). */
static int find_close(const ko_ephem *e, const ko_force_model *fm, double t, const double x[3],
                      double dir, ko_close *cl, double *t_stop, double t_target)
{
    cl->m = -1;
    cl->t0 = t;
    double best = KO_CLOSE_AU;
    for (int m = 1; m < e->n_bodies; m++) {
        if (!((fm->body_mask >> m) & 1u) || e->gm[m] == 0.0) continue;
        double p[3];
        int st = ko_ephem_eval(e, m, t, p, NULL);
        if (st != KO_OK) return st;
        double d = sqrt((x[0] - p[0]) * (x[0] - p[0]) + (x[1] - p[1]) * (x[1] - p[1]) +
                        (x[2] - p[2]) * (x[2] - p[2]));
        if (d < best) {
            best = d;
            cl->m = m;
            for (int i = 0; i < 3; i++) cl->d0[i] = x[i] - p[i];
        }
    }
    *t_stop = t_target;
    if (cl->m >= 0) {
        double k = floor((t - e->t_start) / e->seg_len);
        double b = (dir > 0) ? e->t_start + (k + 1.0) * e->seg_len : e->t_start + k * e->seg_len;
        if (dir < 0 && b == t) b = e->t_start + (k - 1.0) * e->seg_len;
        if ((dir > 0 && b < t_target) || (dir < 0 && b > t_target)) *t_stop = b;
    }
    return KO_OK;
}

/* Exported for the pins of R12: the planet displacement of ephem_delta and the
 * encounter set-up of find_close (nearest planet *m, -1: none; *d0 = x -
 * p_m(t); *t_stop = where a step starting at t toward t_target must end). */
int ko_ephem_delta(const ko_ephem *e, int body, double t0, double off, double dp[3])
{
    return ephem_delta(e, body, t0, off, dp);
}

int ko_find_close(const ko_ephem *e, const ko_force_model *fm, double t, const double x[3],
                  double t_target, int *m, double d0[3], double *t_stop)
{
    ko_close cl;
    int st = find_close(e, fm, t, x, (t_target >= t) ? 1.0 : -1.0, &cl, t_stop, t_target);
    *m = cl.m;
    for (int i = 0; i < 3; i++) d0[i] = (cl.m >= 0) ? cl.d0[i] : 0.0;
    return st;
}

/* Integrate (st, *t) to t_target exactly; *dt is the proposed step (carried). */
int ko_propagate(const ko_ephem *e, const ko_force_model *fm, double st[6], double *t,
                 double t_target, double *dt, ko_stats *stats)
{
    int64_t attempts = 0;
    double dir = (t_target >= *t) ? 1.0 : -1.0;
    if (*dt == 0.0 || (*dt > 0) != (dir > 0)) *dt = dir * fabs(*dt == 0.0 ? fm->dt_init : *dt);
    while (*t != t_target) {
        double x0[3] = {st[0], st[1], st[2]}, v0[3] = {st[3], st[4], st[5]}, a0[3];
        ko_close cl;
        double t_stop = t_target;
        int s0 = find_close(e, fm, *t, x0, dir, &cl, &t_stop, t_target);
        if (s0 != KO_OK) return s0;
        for (int i = 0; i < 3; i++) cl.dx[i] = 0.0;
        s0 = accel_off_cl(e, fm, *t, 0.0, x0, v0, a0, cl.m >= 0 ? &cl : NULL);
        if (stats) stats->force_evals++;
        if (s0 != KO_OK) return s0;
        for (;;) {
            if (++attempts > fm->max_steps) return KO_STEP_CAP;
            double remaining = t_stop - *t;
            int clamped = fabs(*dt) >= fabs(remaining);
            /* the step is the exact difference of the two representable epochs
             * it joins, so that the sum of the steps equals the elapsed time */
            double t_new = clamped ? t_stop : *t + *dt;
            double h = t_new - *t;
            if (h == 0.0) return KO_STEP_CAP;   /* step below the epoch resolution */
            double x1[3], v1[3], err;
            int s1 = radau_attempt(e, fm, *t, x0, v0, a0, h, x1, v1, &err, stats,
                                   cl.m >= 0 ? &cl : NULL);
            if (s1 != KO_OK) return s1;
            /* IAS15 step-size control */
            double dt_new;
            if (isnormal(err))
                dt_new = pow(fm->eps / err, 1.0 / 7.0) * h;
            else
                dt_new = h / fm->safety;
            if (fabs(dt_new / h) < fm->safety) {     /* reject and retry */
                *dt = dt_new;
                if (stats) stats->rejected++;
                continue;
            }
            if (fabs(dt_new / h) > 1.0 / fm->safety) dt_new = h / fm->safety;
            *dt = dt_new;
            for (int i = 0; i < 3; i++) { st[i] = x1[i]; st[3 + i] = v1[i]; }
            *t = t_new;
            if (stats) stats->steps++;
            break;
        }
    }
    return KO_OK;
}

/* Chain of stops (Sec. 2: n-body integration between the median times of
 * consecutive batches, R11): from the epoch to stops[0], then from each stop to
 * the next in the given order.  The proposed step is carried along the chain,
 * which starts from dt_init; a failed body gets NaN from its failing stop on. */
int ko_propagate_stops(const ko_ephem *e, const ko_force_model *fm, const double st0[6],
                       double epoch, const double *stops, int64_t n_stops, double *out,
                       ko_stats *stats)
{
    int status = KO_OK;
    double st[6], t = epoch, dt = 0.0;
    memcpy(st, st0, sizeof(st));
    for (int64_t k = 0; k < n_stops; k++) {
        if (status == KO_OK) status = ko_propagate(e, fm, st, &t, stops[k], &dt, stats);
        for (int i = 0; i < 6; i++) out[k * 6 + i] = (status == KO_OK) ? st[i] : NAN;
    }
    return status;
}

/* ---- threads over bodies ------------------------------------------------- */
typedef struct {
    const ko_ephem *e;
    const ko_force_model *fm;
    double *states, *epochs;
    int64_t n;
    double t_target;
    int32_t *status;
    int tid, nt;
    ko_stats stats;
    const ko_nongrav *ng;
} prop_job;

static void *prop_worker(void *arg)
{
    prop_job *j = (prop_job *)arg;
    for (int64_t i = j->tid; i < j->n; i += j->nt) {
        double st[6], t = j->epochs[i], dt = 0.0;
        for (int c = 0; c < 6; c++) st[c] = j->states[c * j->n + i];
        ko_force_model fmb = *j->fm;
        if (j->ng) fmb.ng = j->ng[i];
        int s = ko_propagate(j->e, &fmb, st, &t, j->t_target, &dt, &j->stats);
        if (j->status) j->status[i] = s;
        if (s == KO_OK) {
            for (int c = 0; c < 6; c++) j->states[c * j->n + i] = st[c];
            j->epochs[i] = t;
        }
    }
    return NULL;
}

int ko_propagate_many(const ko_ephem *e, const ko_force_model *fm, double *states,
                      double *epochs, int64_t n, double t_target, int32_t *status,
                      int n_threads, ko_stats *stats, const ko_nongrav *ng_bodies)
{
    if (n_threads < 1) n_threads = 1;
    prop_job *jobs = (prop_job *)calloc(n_threads, sizeof(prop_job));
    pthread_t *th = (pthread_t *)calloc(n_threads, sizeof(pthread_t));
    for (int k = 0; k < n_threads; k++) {
        prop_job j = {e, fm, states, epochs, n, t_target, status, k, n_threads, {0, 0, 0, 0},
                      ng_bodies};
        jobs[k] = j;
        pthread_create(&th[k], NULL, prop_worker, &jobs[k]);
    }
    for (int k = 0; k < n_threads; k++) {
        pthread_join(th[k], NULL);
        if (stats) {
            stats->steps += jobs[k].stats.steps;
            stats->rejected += jobs[k].stats.rejected;
            stats->force_evals += jobs[k].stats.force_evals;
            stats->iterations += jobs[k].stats.iterations;
        }
    }
    free(jobs);
    free(th);
    return 0;
}

/* ---- universal-variable two-body propagation (Sec. 2, R7) ---------------- */
/* Stumpff functions C(z) = c2, S(z) = c3: their power series for |z| < 1,
 * the closed trigonometric / hyperbolic forms otherwise. */
void ko_stumpff(double z, double *c2, double *c3)
{
    if (fabs(z) < 1.0) {
        double t2 = 0.5, t3 = 1.0 / 6.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < 40; k++) {
            s2 += t2;
            s3 += t3;
            t2 *= -z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));
            t3 *= -z / ((2.0 * k + 4.0) * (2.0 * k + 5.0));
            if (fabs(t2) < 1e-19 && fabs(t3) < 1e-19) break;
        }
        *c2 = s2;
        *c3 = s3;
    } else if (z > 0) {
        double sz = sqrt(z);
        *c2 = (1.0 - cos(sz)) / z;
        *c3 = (sz - sin(sz)) / (sz * sz * sz);
    } else {
        double sz = sqrt(-z);
        *c2 = (cosh(sz) - 1.0) / (-z);
        *c3 = (sinh(sz) - sz) / (sz * sz * sz);
    }
}

int ko_kepler(double mu, const double r0v[3], const double v0v[3], double dt, double r[3],
              double v[3])
{
    if (dt == 0.0) {
        memcpy(r, r0v, 3 * sizeof(double));
        memcpy(v, v0v, 3 * sizeof(double));
        return KO_OK;
    }
    double smu = sqrt(mu);
    double r0 = sqrt(r0v[0] * r0v[0] + r0v[1] * r0v[1] + r0v[2] * r0v[2]);
    double v02 = v0v[0] * v0v[0] + v0v[1] * v0v[1] + v0v[2] * v0v[2];
    double rv = r0v[0] * v0v[0] + r0v[1] * v0v[1] + r0v[2] * v0v[2];
    double alpha = 2.0 / r0 - v02 / mu;
    double A = rv / smu;              /* r0 vr0 / sqrt(mu) */
    double B = 1.0 - alpha * r0;
    /* F(chi) = A chi^2 C + B chi^3 S + r0 chi - sqrt(mu) dt, F' = r > 0 */
    double target = smu * dt;
    double lo, hi;
    double chi = smu * dt / r0;
    /* bracket: F is increasing in chi and F(0) = -target */
    if (dt > 0) { lo = 0.0; hi = chi; } else { hi = 0.0; lo = chi; }
    for (int k = 0; k < 200; k++) {
        double x = (dt > 0) ? hi : lo;
        double z = alpha * x * x, c2, c3;
        ko_stumpff(z, &c2, &c3);
        double F = A * x * x * c2 + B * x * x * x * c3 + r0 * x - target;
        if ((dt > 0 && F >= 0) || (dt < 0 && F <= 0)) break;
        if (dt > 0) { lo = hi; hi *= 2.0; } else { hi = lo; lo *= 2.0; }
        if (k == 199) return KO_KEPLER_FAIL;
    }
    int ok = 0;
    for (int it = 0; it < 200; it++) {
        double z = alpha * chi * chi, c2, c3;
        ko_stumpff(z, &c2, &c3);
        double F = A * chi * chi * c2 + B * chi * chi * chi * c3 + r0 * chi - target;
        double dF = A * chi * (1.0 - z * c3) + B * chi * chi * c2 + r0;
        if (F < 0) lo = chi; else hi = chi;
        double nxt = chi - F / dF;
        if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);   /* bisection fallback */
        double d = fabs(nxt - chi);
        chi = nxt;
        if (d <= 1e-16 * fabs(chi) || lo == hi) { ok = 1; break; }
    }
    if (!ok) return KO_KEPLER_FAIL;
    double z = alpha * chi * chi, c2, c3;
    ko_stumpff(z, &c2, &c3);
    double f = 1.0 - chi * chi / r0 * c2;
    double g = dt - chi * chi * chi * c3 / smu;
    for (int i = 0; i < 3; i++) r[i] = f * r0v[i] + g * v0v[i];
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double fdot = smu / (rn * r0) * (z * c3 - 1.0) * chi;
    double gdot = 1.0 - chi * chi / rn * c2;
    for (int i = 0; i < 3; i++) v[i] = fdot * r0v[i] + gdot * v0v[i];
    return KO_OK;
}

/* Two-body position at t_ref + dt from the heliocentric batch state (R7). */
static int twobody_pos(const ko_ephem *e, const double helio[6], double t_ref, double dt,
                       double pos[3])
{
    double sun[3], r[3], v[3];
    int s = ephem_eval_off(e, 0, t_ref, dt, sun, NULL);
    if (s != KO_OK) return s;
    s = ko_kepler(e->gm[0], helio, helio + 3, dt, r, v);
    if (s != KO_OK) return s;
    for (int i = 0; i < 3; i++) pos[i] = sun[i] + r[i];
    return KO_OK;
}

static double dist3(const double a[3], const double b[3])
{
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

/* Light-delay corrected apparent vector (Sec. 2, R8). */
int ko_apparent(const ko_ephem *e, const double st_ref[6], double t_ref, double t_obs,
                const double obs[3], double u[3], double *tau_out)
{
    const double c = c_au_per_day();
    double sp[3], sv[3], helio[6], pos[3];
    int s = ko_ephem_eval(e, 0, t_ref, sp, sv);
    if (s != KO_OK) return s;
    for (int i = 0; i < 3; i++) {
        helio[i] = st_ref[i] - sp[i];
        helio[3 + i] = st_ref[3 + i] - sv[i];
    }
    /* intervals are formed before absolute epochs (R10) */
    double dt_obs = t_obs - t_ref;
    s = twobody_pos(e, helio, t_ref, dt_obs, pos);
    if (s != KO_OK) return s;
    double tau = dist3(pos, obs) / c;
    for (int it = 0; it < 3; it++) {
        s = twobody_pos(e, helio, t_ref, dt_obs - tau, pos);
        if (s != KO_OK) return s;
        tau = dist3(pos, obs) / c;
    }
    s = twobody_pos(e, helio, t_ref, dt_obs - tau, pos);
    if (s != KO_OK) return s;
    for (int i = 0; i < 3; i++) u[i] = pos[i] - obs[i];
    if (tau_out) *tau_out = tau;
    return KO_OK;
}

/* Apparent magnitudes (Sec. 3.3: V by the H-G system of Bowell et al. 1989 in
 * its two-exponential form; appendix: the comet total and nucleus
 * magnitudes).  Geometry from the light-time corrected apparent vector. */
int ko_magnitude(const ko_ephem *e, const double st_ref[6], double t_ref, double t_obs,
                 const double obs[3], const ko_mag *p, double *mag, double *r_h,
                 double *delta, double *alpha_deg)
{
    double u[3], tau, sun[3];
    int s = ko_apparent(e, st_ref, t_ref, t_obs, obs, u, &tau);
    if (s != KO_OK) return s;
    /* body and Sun at the emission epoch t_obs - tau */
    s = ephem_eval_off(e, 0, t_ref, (t_obs - t_ref) - tau, sun, NULL);
    if (s != KO_OK) return s;
    double rv[3];
    for (int i = 0; i < 3; i++) rv[i] = (obs[i] + u[i]) - sun[i];
    const double rh = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    const double dl = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    /* angle at the body between the directions to the Sun (-rv) and to the
     * observer (-u) */
    double ca = (rv[0] * u[0] + rv[1] * u[1] + rv[2] * u[2]) / (rh * dl);
    if (ca > 1.0) ca = 1.0;
    if (ca < -1.0) ca = -1.0;
    const double alpha = acos(ca);
    double m = NAN;
    if (p && p->kind == 1) {
        const double t = tan(0.5 * alpha);
        const double phi1 = exp(-3.33 * pow(t, 0.63));
        const double phi2 = exp(-1.87 * pow(t, 1.22));
        m = p->p1 + 5.0 * log10(rh * dl) - 2.5 * log10((1.0 - p->p2) * phi1 + p->p2 * phi2);
    } else if (p && p->kind == 2) {
        m = p->p1 + 5.0 * log10(dl) + p->p2 * log10(rh);
    } else if (p && p->kind == 3) {
        m = p->p1 + 5.0 * log10(dl) + p->p2 * log10(rh) + 0.035 * (alpha * 180.0 / M_PI);
    }
    if (mag) *mag = m;
    if (r_h) *r_h = rh;
    if (delta) *delta = dl;
    if (alpha_deg) *alpha_deg = alpha * 180.0 / M_PI;
    return KO_OK;
}

/* RA/Dec of an ecliptic vector: rotate by the obliquity to equatorial J2000. */
void ko_radec(const double u[3], double *ra, double *dec)
{
    double ce = cos(obliquity()), se = sin(obliquity());
    double x = u[0];
    double y = ce * u[1] - se * u[2];
    double z = se * u[1] + ce * u[2];
    double a = atan2(y, x);
    if (a < 0) a += 2.0 * M_PI;
    *ra = a;
    *dec = atan2(z, sqrt(x * x + y * y));
}

/* Sec. 3.1: inside iff every inward normal has a positive dot product (R9). */
int ko_in_polygon(const ko_frame *f, const double u[3], double *margin)
{
    int inside = 1;
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double mg = INFINITY;
    if (f->n_edges == 0) {
        /* cone (Sec. 3.1): inside iff the angle between u and the centre
         * normals[0] is below the radius normals[1][0] */
        const double *cv = f->normals[0];
        const double rho = f->normals[1][0];
        double cn = sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
        double d = cv[0] * u[0] + cv[1] * u[1] + cv[2] * u[2];
        inside = d > cos(rho) * cn * un;
        if (margin) *margin = rho - acos(fmax(-1.0, fmin(1.0, d / (cn * un))));
        return inside;
    }
    for (int k = 0; k < f->n_edges; k++) {
        const double *nv = f->normals[k];
        double d = nv[0] * u[0] + nv[1] * u[1] + nv[2] * u[2];
        if (!(d > 0.0)) inside = 0;
        double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        double ang = asin(fmax(-1.0, fmin(1.0, d / (nn * un))));
        if (ang < mg) mg = ang;
    }
    if (margin) *margin = mg;
    return inside;
}

/* ---- batching (Sec. 2, R6) ------------------------------------------------ */
int64_t ko_make_batches(const double *ep, int64_t n, double batch_span, double twobody_max,
                        int64_t *batch_start, double *t_ref)
{
    double span = batch_span;
    if (2.0 * twobody_max < span) span = 2.0 * twobody_max;
    int64_t nb = 0, i = 0;
    while (i < n) {
        int64_t j = i;
        while (j + 1 < n && (ep[j + 1] == ep[i] || ep[j + 1] - ep[i] < span)) j++;
        if (batch_start) batch_start[nb] = i;
        if (t_ref) t_ref[nb] = 0.5 * (ep[i] + ep[j]);
        nb++;
        i = j + 1;
    }
    return nb;
}

/* ---- survey driver (Sec. 2) ------------------------------------------------ */
typedef struct {
    ko_hit *h;
    int64_t n, cap;
} hitbuf;

static void hit_push(hitbuf *b, const ko_hit *x)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 256;
        b->h = (ko_hit *)realloc(b->h, b->cap * sizeof(ko_hit));
    }
    b->h[b->n++] = *x;
}

typedef struct {
    const ko_ephem *e;
    const ko_force_model *fm;
    const double *states, *epochs;
    int64_t n;
    const ko_frame *frames;
    const int64_t *order;        /* frames sorted by epoch */
    const double *observers;
    const ko_survey_opts *opt;
    const int32_t *subset;
    int64_t n_subset;
    int64_t nb;
    const int64_t *bstart;
    const double *tref;
    int64_t n_frames;
    int32_t *status;
    int tid, nt;
    hitbuf out;
    ko_stats stats;
    double (*centre)[4];         /* frame centre (unit) + circumradius */
    const ko_nongrav *ng;        /* per-body non-gravitational terms or NULL */
} fov_job;

static void *fov_worker(void *arg)
{
    fov_job *j = (fov_job *)arg;
    const double c = c_au_per_day();
    double *st_stops = (double *)malloc(sizeof(double) * 6 * (j->nb ? j->nb : 1));
    for (int64_t q = j->tid; q < j->n_subset; q += j->nt) {
        int32_t bi = j->subset ? j->subset[q] : (int32_t)q;
        double st0[6];
        for (int k = 0; k < 6; k++) st0[k] = j->states[(int64_t)k * j->n + bi];
        ko_force_model fmb = *j->fm;
        if (j->ng) fmb.ng = j->ng[bi];
        int s = ko_propagate_stops(j->e, &fmb, st0, j->epochs[bi], j->tref, j->nb, st_stops,
                                   &j->stats);
        if (j->status) j->status[bi] = s;
        for (int64_t k = 0; k < j->nb; k++) {
            const double *sk = st_stops + 6 * k;
            if (!isfinite(sk[0])) continue;
            int64_t f0 = j->bstart[k], f1 = (k + 1 < j->nb) ? j->bstart[k + 1] : j->n_frames;
            for (int64_t fi = f0; fi < f1; fi++) {
                int64_t fid = j->order[fi];
                const ko_frame *fr = &j->frames[fid];
                const double *o = j->observers + 3 * fr->observer_idx;
                if (j->opt->prefilter_deg > 0) {
                    /* plain conservative prefilter: angle from the observer to
                     * the batch-epoch position vs frame centre, padded by a
                     * bound on the motion over |t - t_ref| + light time. */
                    double d[3] = {sk[0] - o[0], sk[1] - o[1], sk[2] - o[2]};
                    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    double vn = sqrt(sk[3] * sk[3] + sk[4] * sk[4] + sk[5] * sk[5]);
                    double T = fabs(fr->epoch - j->tref[k]) + (dn + 1.0) / c;
                    double sm = 2.0 * vn * T + 0.01 * T * T + 1e-4;
                    if (sm < 0.5 * dn) {
                        const double *cc = j->centre[fid];
                        double cosang = (d[0] * cc[0] + d[1] * cc[1] + d[2] * cc[2]) / dn;
                        double lim = cc[3] + deg2rad(j->opt->prefilter_deg) + asin(sm / dn);
                        if (lim < M_PI && cosang < cos(lim)) continue;
                    }
                }
                double u[3], tau, margin;
                int sa = ko_apparent(j->e, sk, j->tref[k], fr->epoch, o, u, &tau);
                if (sa != KO_OK) {
                    if (j->status && j->status[bi] == KO_OK) j->status[bi] = sa;
                    continue;
                }
                if (ko_in_polygon(fr, u, &margin)) {
                    ko_hit h;
                    h.frame = fid;
                    h.body = bi;
                    h.status = 0;
                    ko_radec(u, &h.ra, &h.dec);
                    h.margin = margin;
                    h.tau = tau;
                    hit_push(&j->out, &h);
                }
            }
        }
    }
    free(st_stops);
    return NULL;
}

static const double *g_sort_ep;
static int cmp_epoch(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, k = *(const int64_t *)b;
    double x = g_sort_ep[i], y = g_sort_ep[k];
    if (x < y) return -1;
    if (x > y) return 1;
    return (i < k) ? -1 : (i > k);
}

static int cmp_hit(const void *a, const void *b)
{
    const ko_hit *x = (const ko_hit *)a, *y = (const ko_hit *)b;
    if (x->frame != y->frame) return (x->frame < y->frame) ? -1 : 1;
    return (x->body < y->body) ? -1 : (x->body > y->body);
}

int ko_fov_check(const ko_ephem *e, const ko_force_model *fm, const double *states,
                 const double *epochs, int64_t n, const ko_frame *frames, int64_t n_frames,
                 const double *observers, int64_t n_obs, const ko_survey_opts *opt,
                 const int32_t *body_subset, int64_t n_subset, ko_hit *hits, int64_t capacity,
                 int64_t *n_hits, int32_t *status, int n_threads, ko_stats *stats,
                 const ko_nongrav *ng_bodies)
{
    (void)n_obs;
    if (n_threads < 1) n_threads = 1;
    /* sort FoVs by epoch (Sec. 2: "grouping the FoVs into batches based on time") */
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (n_frames ? n_frames : 1));
    double *ep_all = (double *)malloc(sizeof(double) * (n_frames ? n_frames : 1));
    for (int64_t i = 0; i < n_frames; i++) { order[i] = i; ep_all[i] = frames[i].epoch; }
    g_sort_ep = ep_all;
    qsort(order, n_frames, sizeof(int64_t), cmp_epoch);
    double *ep = (double *)malloc(sizeof(double) * (n_frames ? n_frames : 1));
    for (int64_t i = 0; i < n_frames; i++) ep[i] = ep_all[order[i]];
    int64_t *bstart = (int64_t *)malloc(sizeof(int64_t) * (n_frames ? n_frames : 1));
    double *tref = (double *)malloc(sizeof(double) * (n_frames ? n_frames : 1));
    int64_t nb = ko_make_batches(ep, n_frames, opt->batch_span, opt->twobody_max, bstart, tref);
    /* frame centres for the optional prefilter: the polygon's vertices are the
     * intersections n_a x n_b (either sign) lying in every other half-space;
     * centre = normalized sum of the vertices, radius = largest vertex angle */
    double (*centre)[4] = (double (*)[4])malloc(sizeof(double) * 4 * (n_frames ? n_frames : 1));
    for (int64_t i = 0; i < n_frames; i++) {
        const ko_frame *f = &frames[i];
        if (f->n_edges == 0) {          /* cone: its own centre and radius */
            const double *cv = f->normals[0];
            double cn = sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
            for (int c = 0; c < 3; c++) centre[i][c] = cv[c] / cn;
            centre[i][3] = f->normals[1][0];
            continue;
        }
        double vs[2 * KO_MAX_EDGES * KO_MAX_EDGES][3], cs[3] = {0, 0, 0};
        int ne = f->n_edges, nv = 0;
        for (int a = 0; a < ne; a++)
            for (int b = a + 1; b < ne; b++) {
                const double *p = f->normals[a], *q = f->normals[b];
                double x[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2],
                               p[0] * q[1] - p[1] * q[0]};
                double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                if (!(xn > 0)) continue;
                for (int sg = -1; sg <= 1; sg += 2) {
                    int ok = 1;
                    for (int c = 0; c < ne; c++) {
                        if (c == a || c == b) continue;
                        const double *m = f->normals[c];
                        if (sg * (m[0] * x[0] + m[1] * x[1] + m[2] * x[2]) < 0) ok = 0;
                    }
                    if (!ok) continue;
                    for (int c = 0; c < 3; c++) { vs[nv][c] = sg * x[c] / xn; cs[c] += vs[nv][c]; }
                    nv++;
                }
            }
        double cn = sqrt(cs[0] * cs[0] + cs[1] * cs[1] + cs[2] * cs[2]);
        double rad = 0.0;
        if (nv < 3 || !(cn > 0)) {
            centre[i][0] = 1.0; centre[i][1] = 0.0; centre[i][2] = 0.0;
            centre[i][3] = M_PI;
            continue;
        }
        for (int c = 0; c < 3; c++) centre[i][c] = cs[c] / cn;
        for (int k = 0; k < nv; k++) {
            double dd = vs[k][0] * centre[i][0] + vs[k][1] * centre[i][1] + vs[k][2] * centre[i][2];
            double ang = acos(fmax(-1.0, fmin(1.0, dd)));
            if (ang > rad) rad = ang;
        }
        centre[i][3] = rad;
    }
    int64_t nsub = body_subset ? n_subset : n;
    fov_job *jobs = (fov_job *)calloc(n_threads, sizeof(fov_job));
    pthread_t *th = (pthread_t *)calloc(n_threads, sizeof(pthread_t));
    for (int k = 0; k < n_threads; k++) {
        fov_job *j = &jobs[k];
        j->e = e; j->fm = fm; j->states = states; j->epochs = epochs; j->n = n;
        j->frames = frames; j->order = order; j->observers = observers; j->opt = opt;
        j->subset = body_subset; j->n_subset = nsub; j->nb = nb; j->bstart = bstart;
        j->tref = tref; j->n_frames = n_frames; j->status = status; j->tid = k;
        j->nt = n_threads; j->centre = centre; j->ng = ng_bodies;
        pthread_create(&th[k], NULL, fov_worker, j);
    }
    int64_t total = 0;
    for (int k = 0; k < n_threads; k++) {
        pthread_join(th[k], NULL);
        total += jobs[k].out.n;
        if (stats) {
            stats->steps += jobs[k].stats.steps;
            stats->rejected += jobs[k].stats.rejected;
            stats->force_evals += jobs[k].stats.force_evals;
            stats->iterations += jobs[k].stats.iterations;
        }
    }
    ko_hit *all = (ko_hit *)malloc(sizeof(ko_hit) * (total ? total : 1));
    int64_t pos = 0;
    for (int k = 0; k < n_threads; k++) {
        memcpy(all + pos, jobs[k].out.h, jobs[k].out.n * sizeof(ko_hit));
        pos += jobs[k].out.n;
        free(jobs[k].out.h);
    }
    qsort(all, total, sizeof(ko_hit), cmp_hit);
    *n_hits = total;
    int rc = 0;
    if (total > capacity) rc = -3;
    else if (hits) memcpy(hits, all, total * sizeof(ko_hit));
    free(all); free(jobs); free(th); free(order); free(ep_all); free(ep); free(bstart);
    free(tref); free(centre);
    return rc;
}

/* ---- variational equations and the orbit-fit loss (adjoint reference) ---- */

/* Jacobians J_x = da/dx, J_v = da/dv of Eq. A.1 at (t0 + off, x, v) by central
 * differences (steps 1e-7 AU, 1e-9 AU/day). */
static int accel_jacobian(const ko_ephem *e, const ko_force_model *fm, double t0, double off,
                          const double x[3], const double v[3], double Jx[3][3], double Jv[3][3])
{
    const double hx = 1e-7, hv = 1e-9;
    for (int k = 0; k < 3; k++) {
        double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
        double vp[3] = {v[0], v[1], v[2]}, vm[3] = {v[0], v[1], v[2]};
        double ap[3], am[3];
        xp[k] += hx;
        xm[k] -= hx;
        int s = accel_off(e, fm, t0, off, xp, v, ap);
        if (s == KO_OK) s = accel_off(e, fm, t0, off, xm, v, am);
        if (s != KO_OK) return s;
        for (int i = 0; i < 3; i++) Jx[i][k] = (ap[i] - am[i]) / (2.0 * hx);
        vp[k] += hv;
        vm[k] -= hv;
        s = accel_off(e, fm, t0, off, x, vp, ap);
        if (s == KO_OK) s = accel_off(e, fm, t0, off, x, vm, am);
        if (s != KO_OK) return s;
        for (int i = 0; i < 3; i++) Jv[i][k] = (ap[i] - am[i]) / (2.0 * hv);
    }
    return KO_OK;
}

/* One Gauss-Radau attempt of the body (identical arithmetic to radau_attempt)
 * carrying the 6 columns of Phi as variational particles: column c has
 * position Phi[0..2][c], velocity Phi[3..5][c] and acceleration
 * J_x dx + J_v dv at the body's substep state.  The body alone decides
 * convergence and the error estimate. */
static int radau_attempt_stm(const ko_ephem *e, const ko_force_model *fm, double t,
                             const double x0[3], const double v0[3], const double a0[3],
                             const double P0[36], const double Pa0[18], double dt,
                             double x1[3], double v1[3], double P1[36], double *err,
                             ko_stats *stats, ko_close *cl)
{
    const ko_radau *R = radau();
    double g[8][3], b[7][3], F[8][3];
    double gv[8][18], bv[7][18], Fv[8][18];   /* variational: 6 columns x 3 */
    memset(g, 0, sizeof(g));
    memset(b, 0, sizeof(b));
    memset(gv, 0, sizeof(gv));
    memset(bv, 0, sizeof(bv));
    for (int i = 0; i < 3; i++) F[0][i] = a0[i];
    for (int q = 0; q < 18; q++) Fv[0][q] = Pa0[q];
    double pc_prev = 0.0, amax = 0.0;
    for (int it = 1; it <= fm->max_iter; it++) {
        double b6_old[3] = {b[6][0], b[6][1], b[6][2]};
        for (int n = 1; n <= 7; n++) {
            double s = R->h[n];
            double xn[3], vn[3];
            for (int i = 0; i < 3; i++) {
                double acc = a0[i] * s * s / 2.0;
                double vacc = a0[i] * s;
                double sp = s * s;
                for (int k = 0; k < 7; k++) {
                    acc += b[k][i] * sp * s / ((k + 2.0) * (k + 3.0));
                    vacc += b[k][i] * sp / (k + 2.0);
                    sp *= s;
                }
                double dxn = v0[i] * dt * s + dt * dt * acc;
                xn[i] = x0[i] + dxn;
                vn[i] = v0[i] + dt * vacc;
                if (cl) cl->dx[i] = dxn;
            }
            /* variational particles at the substep */
            double dxn[18], dvn[18];
            for (int c = 0; c < 6; c++)
                for (int i = 0; i < 3; i++) {
                    int q = 3 * c + i;
                    double acc = Pa0[q] * s * s / 2.0, vacc = Pa0[q] * s, sp = s * s;
                    for (int k = 0; k < 7; k++) {
                        acc += bv[k][q] * sp * s / ((k + 2.0) * (k + 3.0));
                        vacc += bv[k][q] * sp / (k + 2.0);
                        sp *= s;
                    }
                    dxn[q] = P0[i * 6 + c] + P0[(3 + i) * 6 + c] * dt * s + dt * dt * acc;
                    dvn[q] = P0[(3 + i) * 6 + c] + dt * vacc;
                }
            int st = accel_off_cl(e, fm, t, s * dt, xn, vn, F[n], cl);
            if (stats) stats->force_evals++;
            if (st != KO_OK) return st;
            double Jx[3][3], Jv[3][3];
            st = accel_jacobian(e, fm, t, s * dt, xn, vn, Jx, Jv);
            if (st != KO_OK) return st;
            for (int c = 0; c < 6; c++)
                for (int i = 0; i < 3; i++) {
                    double a = 0.0;
                    for (int k = 0; k < 3; k++)
                        a += Jx[i][k] * dxn[3 * c + k] + Jv[i][k] * dvn[3 * c + k];
                    Fv[n][3 * c + i] = a;
                }
            for (int i = 0; i < 3; i++) {
                double d = (F[n][i] - F[0][i]) / (R->h[n] - R->h[0]);
                for (int k = 1; k < n; k++) d = (d - g[k][i]) / (R->h[n] - R->h[k]);
                g[n][i] = d;
            }
            for (int q = 0; q < 18; q++) {
                double d = (Fv[n][q] - Fv[0][q]) / (R->h[n] - R->h[0]);
                for (int k = 1; k < n; k++) d = (d - gv[k][q]) / (R->h[n] - R->h[k]);
                gv[n][q] = d;
            }
            for (int mm = 0; mm < 7; mm++) {
                for (int i = 0; i < 3; i++) {
                    double sum = 0.0;
                    for (int j = mm + 1; j <= 7; j++) sum += R->C[j][mm] * g[j][i];
                    b[mm][i] = sum;
                }
                for (int q = 0; q < 18; q++) {
                    double sum = 0.0;
                    for (int j = mm + 1; j <= 7; j++) sum += R->C[j][mm] * gv[j][q];
                    bv[mm][q] = sum;
                }
            }
        }
        if (stats) stats->iterations++;
        double db = 0.0;
        amax = 0.0;
        for (int i = 0; i < 3; i++) {
            double d = fabs(b[6][i] - b6_old[i]);
            if (d > db) db = d;
            if (fabs(F[7][i]) > amax) amax = fabs(F[7][i]);
        }
        double pc = db / amax;
        if (!isfinite(pc)) return KO_NONFINITE;
        if (pc < fm->eps_pc) break;
        if (it >= 3 && pc >= pc_prev) break;
        pc_prev = pc;
    }
    double bmax = 0.0;
    for (int i = 0; i < 3; i++)
        if (fabs(b[6][i]) > bmax) bmax = fabs(b[6][i]);
    *err = bmax / amax;
    for (int i = 0; i < 3; i++) {
        double acc = a0[i] / 2.0, vacc = a0[i];
        for (int k = 0; k < 7; k++) {
            acc += b[k][i] / ((k + 2.0) * (k + 3.0));
            vacc += b[k][i] / (k + 2.0);
        }
        x1[i] = x0[i] + v0[i] * dt + dt * dt * acc;
        v1[i] = v0[i] + dt * vacc;
    }
    for (int c = 0; c < 6; c++)
        for (int i = 0; i < 3; i++) {
            int q = 3 * c + i;
            double acc = Pa0[q] / 2.0, vacc = Pa0[q];
            for (int k = 0; k < 7; k++) {
                acc += bv[k][q] / ((k + 2.0) * (k + 3.0));
                vacc += bv[k][q] / (k + 2.0);
            }
            P1[i * 6 + c] = P0[i * 6 + c] + P0[(3 + i) * 6 + c] * dt + dt * dt * acc;
            P1[(3 + i) * 6 + c] = P0[(3 + i) * 6 + c] + dt * vacc;
        }
    if (!finite3(x1) || !finite3(v1)) return KO_NONFINITE;
    return KO_OK;
}

int ko_propagate_stm(const ko_ephem *e, const ko_force_model *fm, double st[6], double phi[36],
                     double *t, double t_target, double *dt, ko_stats *stats)
{
    int64_t attempts = 0;
    double dir = (t_target >= *t) ? 1.0 : -1.0;
    if (*dt == 0.0 || (*dt > 0) != (dir > 0)) *dt = dir * fabs(*dt == 0.0 ? fm->dt_init : *dt);
    while (*t != t_target) {
        double x0[3] = {st[0], st[1], st[2]}, v0[3] = {st[3], st[4], st[5]}, a0[3];
        ko_close cl;
        double t_stop = t_target;
        int s0 = find_close(e, fm, *t, x0, dir, &cl, &t_stop, t_target);
        if (s0 != KO_OK) return s0;
        for (int i = 0; i < 3; i++) cl.dx[i] = 0.0;
        s0 = accel_off_cl(e, fm, *t, 0.0, x0, v0, a0, cl.m >= 0 ? &cl : NULL);
        if (stats) stats->force_evals++;
        if (s0 != KO_OK) return s0;
        double Jx[3][3], Jv[3][3], Pa0[18];
        s0 = accel_jacobian(e, fm, *t, 0.0, x0, v0, Jx, Jv);
        if (s0 != KO_OK) return s0;
        for (int c = 0; c < 6; c++)
            for (int i = 0; i < 3; i++) {
                double a = 0.0;
                for (int k = 0; k < 3; k++)
                    a += Jx[i][k] * phi[k * 6 + c] + Jv[i][k] * phi[(3 + k) * 6 + c];
                Pa0[3 * c + i] = a;
            }
        for (;;) {
            if (++attempts > fm->max_steps) return KO_STEP_CAP;
            double remaining = t_stop - *t;
            int clamped = fabs(*dt) >= fabs(remaining);
            double t_new = clamped ? t_stop : *t + *dt;
            double h = t_new - *t;
            if (h == 0.0) return KO_STEP_CAP;
            double x1[3], v1[3], P1[36], err;
            int s1 = radau_attempt_stm(e, fm, *t, x0, v0, a0, phi, Pa0, h, x1, v1, P1, &err, stats,
                                       cl.m >= 0 ? &cl : NULL);
            if (s1 != KO_OK) return s1;
            double dt_new;
            if (isnormal(err))
                dt_new = pow(fm->eps / err, 1.0 / 7.0) * h;
            else
                dt_new = h / fm->safety;
            if (fabs(dt_new / h) < fm->safety) {
                *dt = dt_new;
                if (stats) stats->rejected++;
                continue;
            }
            if (fabs(dt_new / h) > 1.0 / fm->safety) dt_new = h / fm->safety;
            *dt = dt_new;
            for (int i = 0; i < 3; i++) { st[i] = x1[i]; st[3 + i] = v1[i]; }
            memcpy(phi, P1, sizeof(P1));
            *t = t_new;
            if (stats) stats->steps++;
            break;
        }
    }
    return KO_OK;
}

static double wrap_pi(double a)
{
    while (a > M_PI) a -= 2.0 * M_PI;
    while (a <= -M_PI) a += 2.0 * M_PI;
    return a;
}

/* residual (wrap(RA - RA_obs) cos Dec_obs, Dec - Dec_obs) of one observation
 * predicted from the batch state y at t_ref */
static int obs_residual(const ko_ephem *e, const double y[6], double t_ref, const ko_obs *o,
                        double res[2], double *ra_out, double *dec_out)
{
    double u[3], tau, ra, dec;
    int s = ko_apparent(e, y, t_ref, o->epoch, o->obs, u, &tau);
    if (s != KO_OK) return s;
    ko_radec(u, &ra, &dec);
    res[0] = wrap_pi(ra - o->ra) * cos(o->dec);
    res[1] = dec - o->dec;
    if (ra_out) *ra_out = ra;
    if (dec_out) *dec_out = dec;
    return KO_OK;
}

static int cmp_dbl(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y);
}

int ko_body_loss(const ko_ephem *e, const ko_force_model *fm, const double st0[6], double epoch0,
                 const ko_obs *obs, int m, double batch_span, double twobody_max,
                 double ckpt_days, double *loss, double *pred, double grad_var[6])
{
    for (int j = 1; j < m; j++)
        if (obs[j].epoch < obs[j - 1].epoch) return -1;
    double *ep = (double *)malloc(sizeof(double) * (m ? m : 1));
    int64_t *bs = (int64_t *)malloc(sizeof(int64_t) * (m ? m : 1));
    double *tref = (double *)malloc(sizeof(double) * (m ? m : 1));
    for (int j = 0; j < m; j++) ep[j] = obs[j].epoch;
    int64_t nb = ko_make_batches(ep, m, batch_span, twobody_max, bs, tref);
    /* stops: batch midpoints and the checkpoint grid up to the last midpoint */
    int cap = (int)nb + 4096;
    double *stops = (double *)malloc(sizeof(double) * cap);
    int ns = 0;
    for (int64_t k = 0; k < nb; k++) stops[ns++] = tref[k];
    if (nb > 0 && ckpt_days > 0)
        for (int k = 1; epoch0 + k * ckpt_days < tref[nb - 1] && ns < cap; k++)
            stops[ns++] = epoch0 + k * ckpt_days;
    qsort(stops, ns, sizeof(double), cmp_dbl);
    double y[6], phi[36], t = epoch0, dt = 0.0, L = 0.0;
    memcpy(y, st0, sizeof(y));
    for (int r = 0; r < 36; r++) phi[r] = (r % 7 == 0) ? 1.0 : 0.0;
    if (grad_var) memset(grad_var, 0, 6 * sizeof(double));
    int status = KO_OK;
    int64_t kb = 0;
    for (int q = 0; q < ns && status == KO_OK; q++) {
        if (grad_var) status = ko_propagate_stm(e, fm, y, phi, &t, stops[q], &dt, NULL);
        else status = ko_propagate(e, fm, y, &t, stops[q], &dt, NULL);
        if (status != KO_OK) break;
        if (kb < nb && stops[q] == tref[kb]) {
            int64_t j0 = bs[kb], j1 = (kb + 1 < nb) ? bs[kb + 1] : m;
            for (int64_t j = j0; j < j1 && status == KO_OK; j++) {
                double res[2], ra, dec;
                status = obs_residual(e, y, tref[kb], &obs[j], res, &ra, &dec);
                if (status != KO_OK) break;
                L += res[0] * res[0] + res[1] * res[1];
                if (pred) { pred[2 * j] = ra; pred[2 * j + 1] = dec; }
                if (!grad_var) continue;
                /* d res / d y(t_ref) by central differences, step 1e-7 in
                 * position (AU) and velocity (AU/day): |t_obs - t_ref| is at
                 * most a few days, so the velocity step moves the apparent
                 * position by < 1e-6 AU (truncation < 1e-12 relative) while
                 * the rounding of an RA difference (~1e-15 rad) stays below
                 * 1e-8 of the partial */
                double dr[2][6];
                for (int c = 0; c < 6; c++) {
                    double h = 1e-7;
                    double yp[6], ym[6], rp[2], rm[2];
                    memcpy(yp, y, sizeof(yp));
                    memcpy(ym, y, sizeof(ym));
                    yp[c] += h;
                    ym[c] -= h;
                    status = obs_residual(e, yp, tref[kb], &obs[j], rp, NULL, NULL);
                    if (status == KO_OK) status = obs_residual(e, ym, tref[kb], &obs[j], rm, NULL, NULL);
                    if (status != KO_OK) break;
                    dr[0][c] = wrap_pi(rp[0] - rm[0]) / (2.0 * h);
                    dr[1][c] = (rp[1] - rm[1]) / (2.0 * h);
                }
                /* dL/dy0 += 2 res^T (dres/dy) Phi */
                for (int c0 = 0; c0 < 6; c0++) {
                    double acc = 0.0;
                    for (int c = 0; c < 6; c++)
                        acc += (2.0 * res[0] * dr[0][c] + 2.0 * res[1] * dr[1][c]) * phi[c * 6 + c0];
                    grad_var[c0] += acc;
                }
            }
            kb++;
        }
    }
    *loss = L;
    free(ep); free(bs); free(tref); free(stops);
    return status;
}

/* Per-observation sky partials of one body: jac[j][0][c] = d RA_j / d y0_c and
 * jac[j][1][c] = d Dec_j / d y0_c, y0 = (x0, v0), for every observation j:
 * the rows of the orbit-fit Jacobian (whose J^T J gives the covariance).  The
 * forward model is ko_body_loss's; each row is the state-transition matrix
 * from the variational equations at the observation's batch midpoint chained
 * with central-difference partials of RA and Dec with respect to the state
 * there (the same steps as ko_body_loss's gradient).  pred (may be NULL):
 * [m][2] predicted RA, Dec. */
int ko_body_sky_jacobian(const ko_ephem *e, const ko_force_model *fm, const double st0[6],
                         double epoch0, const ko_obs *obs, int m, double batch_span,
                         double twobody_max, double ckpt_days, double *pred, double *jac)
{
    for (int j = 1; j < m; j++)
        if (obs[j].epoch < obs[j - 1].epoch) return -1;
    double *ep = (double *)malloc(sizeof(double) * (m ? m : 1));
    int64_t *bs = (int64_t *)malloc(sizeof(int64_t) * (m ? m : 1));
    double *tref = (double *)malloc(sizeof(double) * (m ? m : 1));
    for (int j = 0; j < m; j++) ep[j] = obs[j].epoch;
    int64_t nb = ko_make_batches(ep, m, batch_span, twobody_max, bs, tref);
    int cap = (int)nb + 4096;
    double *stops = (double *)malloc(sizeof(double) * cap);
    int ns = 0;
    for (int64_t k = 0; k < nb; k++) stops[ns++] = tref[k];
    if (nb > 0 && ckpt_days > 0)
        for (int k = 1; epoch0 + k * ckpt_days < tref[nb - 1] && ns < cap; k++)
            stops[ns++] = epoch0 + k * ckpt_days;
    qsort(stops, ns, sizeof(double), cmp_dbl);
    double y[6], phi[36], t = epoch0, dt = 0.0;
    memcpy(y, st0, sizeof(y));
    for (int r = 0; r < 36; r++) phi[r] = (r % 7 == 0) ? 1.0 : 0.0;
    int status = KO_OK;
    int64_t kb = 0;
    for (int q = 0; q < ns && status == KO_OK; q++) {
        status = ko_propagate_stm(e, fm, y, phi, &t, stops[q], &dt, NULL);
        if (status != KO_OK) break;
        if (kb < nb && stops[q] == tref[kb]) {
            int64_t j0 = bs[kb], j1 = (kb + 1 < nb) ? bs[kb + 1] : m;
            for (int64_t j = j0; j < j1 && status == KO_OK; j++) {
                double res[2], ra, dec;
                status = obs_residual(e, y, tref[kb], &obs[j], res, &ra, &dec);
                if (status != KO_OK) break;
                if (pred) { pred[2 * j] = ra; pred[2 * j + 1] = dec; }
                /* d(RA, Dec) / d y(t_ref) by central differences (the steps of
                 * ko_body_loss's observation partials) */
                double dr[2][6];
                for (int c = 0; c < 6; c++) {
                    double h = 1e-7;
                    double yp[6], ym[6], rp[2], rm[2], rap, decp, ram, decm;
                    memcpy(yp, y, sizeof(yp));
                    memcpy(ym, y, sizeof(ym));
                    yp[c] += h;
                    ym[c] -= h;
                    status = obs_residual(e, yp, tref[kb], &obs[j], rp, &rap, &decp);
                    if (status == KO_OK) status = obs_residual(e, ym, tref[kb], &obs[j], rm, &ram, &decm);
                    if (status != KO_OK) break;
                    dr[0][c] = wrap_pi(rap - ram) / (2.0 * h);
                    dr[1][c] = (decp - decm) / (2.0 * h);
                }
                /* rows: d(RA, Dec)/d y(t_ref) Phi */
                for (int a = 0; a < 2; a++)
                    for (int c0 = 0; c0 < 6; c0++) {
                        double acc = 0.0;
                        for (int c = 0; c < 6; c++) acc += dr[a][c] * phi[c * 6 + c0];
                        jac[(j * 2 + a) * 6 + c0] = acc;
                    }
            }
            kb++;
        }
    }
    free(ep); free(bs); free(tref); free(stops);
    return status;
}
