/*
 * kete_oracle.h -- plain, slow, FP64 CPU oracle of the survey-prediction path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path; the two meet only on the seeded input files.
 *
 * What it computes (each function cites the passage it follows):
 *   - planetary ephemeris lookup: Chebyshev series per segment (App. A, Sec. 3.2)
 *   - acceleration: Newton + GR (Eq. A.3) + J2 (Eq. A.4), summed as Eq. A.1,
 *     plus the optional non-gravitational terms: radiation pressure with
 *     Poynting-Robertson drag (Eq. A.6) and the JPL comet model with its
 *     thermal lag (Eq. A.7)
 *   - Gauss-Radau 15th-order step with IAS15 corrector convergence and step
 *     control, predictor removed (Sec. 3.2, App. A.6)
 *   - universal-variable two-body propagation + light-delay iteration (Sec. 2)
 *   - FoV test: spherical polygons by inward normals, and cones (Sec. 3.1)
 *   - apparent magnitudes: H-G V for asteroids, comet total and nucleus
 *     magnitudes (Sec. 3.3, App. B)
 *   - orbit-fit loss and its gradient by the variational equations
 *   - time batching of FoVs into <= 3-day groups with n-body to the batch
 *     midpoint (Sec. 2)
 *   - RA/Dec in equatorial J2000 (App. A.1)
 *
 * Parity pins: see tests/test_oracle_*.py (closed-form Kepler, conservation
 * laws, time reversal, GR perihelion advance, J2 nodal regression, light-time
 * closed forms, gnomonic FoV test, brute-force FoV, batching rules; the
 * non-gravitational terms against Kepler with a weakened Sun, Gauss's rate
 * for a transverse force, the angular-momentum decay and Wyatt & Whipple's
 * secular rate of Poynting-Robertson drag, and Galilean invariance).
 * The full force model with planets on is "parity unpinned" by the paper:
 * no worked example exists; it is held only by the invariants above.
 */
#ifndef KETE_ORACLE_H
#define KETE_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KO_MAX_BODIES 16
#define KO_MAX_EDGES 4

/* status codes (per body) */
#define KO_OK 0
#define KO_STEP_CAP 1
#define KO_OUT_OF_SPAN 2
#define KO_NONFINITE 3
#define KO_KEPLER_FAIL 4

typedef struct {
    int n_bodies, n_coef, n_seg;
    double t_start, seg_len;
    double gm[KO_MAX_BODIES];
    double *coef;           /* [body][seg][3][coef] */
} ko_ephem;

/* Non-gravitational parameters of one body (App. A.4-A.5).  All zero: none.
 *   beta: radiation pressure / solar gravity ratio (Eq. A.6)
 *   a1, a2, a3: radial, transverse, normal JPL coefficients, AU/day^2, with
 *   g(r) = alpha (r/r0)^-m (1 + (r/r0)^n)^-k (Eq. A.7), evaluated, with the
 *   directions, at the two-body heliocentric state dt days earlier. */
typedef struct {
    double a1, a2, a3;
    double alpha, r0, m, n, k;
    double dt;
    double beta;
} ko_nongrav;

typedef struct {
    uint32_t body_mask;     /* bodies whose gravity acts (bit b = table body b) */
    uint32_t gr_mask;       /* bodies with the GR term of Eq. A.3 */
    uint32_t j2_mask;       /* bodies with the J2 term of Eq. A.4 */
    int32_t max_iter;       /* corrector iteration cap */
    double j2[KO_MAX_BODIES];
    double radius[KO_MAX_BODIES];    /* AU */
    double pole_ra[KO_MAX_BODIES];   /* radians, equatorial J2000 */
    double pole_dec[KO_MAX_BODIES];
    double eps;             /* IAS15 step-size control parameter */
    double eps_pc;          /* corrector convergence threshold */
    double safety;          /* IAS15 safety factor */
    double dt_init;         /* first step of every propagation chain, days */
    int64_t max_steps;      /* step attempts per leg */
    ko_nongrav ng;          /* this body's non-gravitational terms (zero: none) */
} ko_force_model;

typedef struct {
    double epoch;
    int64_t observer_idx;
    int64_t exposure_id;
    int32_t n_edges;
    int32_t reserved;
    double normals[KO_MAX_EDGES][3];
} ko_frame;

typedef struct {
    int64_t frame;
    int32_t body;
    int32_t status;
    double ra, dec;          /* radians, equatorial J2000 */
    double margin;           /* min over edges of asin(n.u/|n||u|), radians */
    double tau;              /* light time, days */
} ko_hit;

typedef struct {
    double batch_span;       /* <= 3 days by default (Sec. 2) */
    double twobody_max;      /* maximum two-body interval (0 = pure n-body) */
    double prefilter_deg;    /* 0: brute force over all frames of a batch */
} ko_survey_opts;

typedef struct {
    int64_t steps, rejected, force_evals, iterations;
} ko_stats;

/* one astrometric observation of one body (48 bytes) */
typedef struct {
    double epoch;            /* TDB JD */
    double ra, dec;          /* observed, radians (equatorial J2000) */
    double obs[3];           /* observer position, barycentric ecliptic AU */
} ko_obs;

void ko_force_model_default(ko_force_model *fm);
int  ko_ephem_load(ko_ephem *e, const void *buf, size_t n);
void ko_ephem_free(ko_ephem *e);
int  ko_ephem_eval(const ko_ephem *e, int body, double t, double pos[3], double vel[3]);

void ko_radau_nodes(double h[8]);
int  ko_accel(const ko_ephem *e, const ko_force_model *fm, double t,
              const double x[3], const double v[3], double a[3]);
int  ko_propagate(const ko_ephem *e, const ko_force_model *fm, double st[6], double *t,
                  double t_target, double *dt, ko_stats *stats);
int  ko_propagate_stops(const ko_ephem *e, const ko_force_model *fm, const double st0[6],
                        double epoch, const double *stops, int64_t n_stops,
                        double *out /* [n_stops][6] */, ko_stats *stats);
/* ng_bodies (may be NULL): per-body non-gravitational terms replacing fm->ng */
int  ko_propagate_many(const ko_ephem *e, const ko_force_model *fm, double *states /*6xN SoA*/,
                       double *epochs, int64_t n, double t_target, int32_t *status,
                       int n_threads, ko_stats *stats, const ko_nongrav *ng_bodies);

/* Close encounters (R12): p(t0 + off) - p(t0) of table body `body` from the
 * segment holding t0, by the recurrence on Chebyshev differences; and the
 * nearest active planet within 0.1 AU of x at t (*m = -1: none), x - p_m(t)
 * in d0, and the end of the step range toward t_target in *t_stop (the next
 * table segment boundary during an encounter). */
int  ko_ephem_delta(const ko_ephem *e, int body, double t0, double off, double dp[3]);
int  ko_find_close(const ko_ephem *e, const ko_force_model *fm, double t, const double x[3],
                   double t_target, int *m, double d0[3], double *t_stop);

void ko_stumpff(double z, double *c2, double *c3);
int  ko_kepler(double mu, const double r0[3], const double v0[3], double dt,
               double r[3], double v[3]);
int  ko_apparent(const ko_ephem *e, const double st_ref[6], double t_ref, double t_obs,
                 const double obs[3], double u[3], double *tau);
void ko_radec(const double u[3], double *ra, double *dec);
/* FoV membership (Sec. 3.1).  n_edges 3..4: spherical polygon, inside iff
 * normals[k].u > 0 for every edge; margin = min over edges of the angle of u
 * above the edge's plane.  n_edges 0: cone of centre normals[0] and angular
 * radius normals[1][0] (radians), inside iff angle(u, centre) < radius;
 * margin = radius - angle.  Points on the boundary are outside. */
int  ko_in_polygon(const ko_frame *f, const double u[3], double *margin);

int64_t ko_make_batches(const double *epochs_sorted, int64_t n, double batch_span,
                        double twobody_max, int64_t *batch_start, double *t_ref);
int  ko_fov_check(const ko_ephem *e, const ko_force_model *fm, const double *states,
                  const double *epochs, int64_t n, const ko_frame *frames, int64_t n_frames,
                  const double *observers, int64_t n_obs, const ko_survey_opts *opt,
                  const int32_t *body_subset, int64_t n_subset, ko_hit *hits,
                  int64_t capacity, int64_t *n_hits, int32_t *status, int n_threads,
                  ko_stats *stats, const ko_nongrav *ng_bodies);

/* Magnitude model of one body (Sec. 3.3 flux estimation; comet magnitudes of
 * the appendix): kind 1 = asteroid V by the H-G system (p1 = H, p2 = G);
 * kind 2 = comet total T_mag (p1 = M1, p2 = K1); kind 3 = comet nucleus
 * N_mag (p1 = M2, p2 = K2).  kind 0: no magnitude. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double p1, p2;
} ko_mag;

/* Apparent magnitude of a body seen at t_obs from obs, its state st_ref at
 * t_ref propagated by two-body + light time (ko_apparent): r_h = |body - Sun|
 * at t_obs - tau, delta = |u|, alpha = Sun-body-observer angle (degrees).
 *   H-G:    V = H + 5 log10(r_h delta) - 2.5 log10((1-G) Phi1 + G Phi2),
 *           Phi_i = exp(-A_i tan(alpha/2)^B_i), A = (3.33, 1.87), B = (0.63, 1.22)
 *   comet:  M + 5 log10(delta) + K log10(r_h) (+ 0.035 alpha for N_mag)
 * mag, r_h, delta, alpha_deg: outputs (each may be NULL). */
int  ko_magnitude(const ko_ephem *e, const double st_ref[6], double t_ref, double t_obs,
                  const double obs[3], const ko_mag *p, double *mag, double *r_h,
                  double *delta, double *alpha_deg);

/* Orbit-fit loss of one body and its gradient w.r.t. the initial state.
 * Forward model: the body's observation epochs (sorted) are batched by the
 * <= batch_span rule, the n-body chain visits the union of the batch midpoints
 * and the checkpoint grid epoch0 + ckpt_days * k, then two-body + light time +
 * RA/Dec per observation (Sec. 2).  loss = sum (wrap(RA-RA_obs) cos Dec_obs)^2
 * + (Dec-Dec_obs)^2.  pred (may be NULL): [m][2] model RA, Dec.
 * grad_var (may be NULL): dL/d(x0, v0) by the variational equations (6x6
 * state-transition matrix integrated with the body, Jacobians of Eq. A.1 by
 * central differences) chained with central-difference partials of the
 * observation operator. */
int  ko_body_loss(const ko_ephem *e, const ko_force_model *fm, const double st0[6], double epoch0,
                  const ko_obs *obs, int m, double batch_span, double twobody_max,
                  double ckpt_days, double *loss, double *pred, double grad_var[6]);
/* Per-observation sky partials: jac [m][2][6] = d(RA_j, Dec_j)/d(x0, v0) of
 * the forward model of ko_body_loss (state-transition matrix at each batch
 * midpoint chained with central-difference observation partials); pred (may
 * be NULL) [m][2]. */
int  ko_body_sky_jacobian(const ko_ephem *e, const ko_force_model *fm, const double st0[6],
                          double epoch0, const ko_obs *obs, int m, double batch_span,
                          double twobody_max, double ckpt_days, double *pred, double *jac);
/* the state-transition matrix Phi (6x6, row-major, Phi[r*6+c] = dy_r/dy0_c)
 * propagated with the body along exactly the body's own step sequence */
int  ko_propagate_stm(const ko_ephem *e, const ko_force_model *fm, double st[6], double phi[36],
                      double *t, double t_target, double *dt, ko_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
