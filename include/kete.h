/*
 * kete.h -- C ABI of the GB300 survey-prediction library (libkete_gpu.so).
 *
 * The library answers the question of Sec. 2 of the Kete paper: given a list
 * of telescope fields of view (FoVs, each with an epoch and an observer
 * position, Sec. 3.1) and the Cartesian states of many minor bodies, which
 * bodies fall inside which FoV.  The path it runs on the GPU:
 *
 *   1. planetary positions from a device-resident Chebyshev table (the
 *      stand-in for the SPICE kernels of Sec. 3.2 / App. A);
 *   2. n-body propagation of massless bodies under Sun + planets with the
 *      force model of Eq. A.1 (Newton + GR of Eq. A.3 + J2 of Eq. A.4, and
 *      optionally per-body radiation pressure, Eq. A.6, and the JPL comet
 *      model, Eq. A.7) by a Gauss-Radau integrator with IAS15 convergence
 *      and step control and the predictor removed (Sec. 3.2, App. A.6), in
 *      FP64 or with FP32 planetary terms;
 *   3. FoVs sorted and grouped into <= 3-day batches, bodies integrated to each
 *      batch midpoint, then two-body propagation with light-delay correction
 *      to each FoV epoch (Sec. 2);
 *   4. the membership test of spherical polygons by inward great-circle
 *      normals and of cones (Sec. 3.1), RA/Dec of every hit (App. A.1), and
 *      optionally its apparent magnitude (Sec. 3.3);
 *   5. the gradient of an orbit-fit loss through steps 2-4 with respect to
 *      the initial states (kete_adjoint).
 *
 * Units and frames (App. A.1): AU, AU/day, TDB Julian dates; states are
 * barycentric ecliptic J2000; RA/Dec are equatorial J2000 (obliquity
 * 84381.448 arcsec).
 *
 * Conventions for every call:
 *   - Pointers marked (device) must be device memory of the context's GPU;
 *     pointers marked (host) are host memory.  The caller owns every buffer
 *     it passes; the library owns only its ephemeris copy and its scratch.
 *   - All work is ordered on the context's CUDA stream.  Calls that return a
 *     count to the host (kete_fov_check) synchronize that stream.
 *   - Return value: KETE_OK (0) or a negative KETE_ERR_*; nothing is thrown.
 *     kete_last_error() gives a one-line message for the last failure.
 *   - A body whose integration fails gets a per-body status code; the other
 *     bodies' results stay valid.
 */
#ifndef KETE_H
#define KETE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KETE_MAX_BODIES 16   /* massive bodies a table may hold */
#define KETE_MAX_EDGES 4     /* edges of one spherical polygon */

/* return codes */
#define KETE_OK 0
#define KETE_ERR_BAD_ARG -1      /* invalid size, pointer, frame layout or option */
#define KETE_ERR_EPHEM_SPAN -2   /* an epoch lies outside the loaded table */
#define KETE_ERR_CAPACITY -3     /* hit buffer too small: *n_hits holds the count needed */
#define KETE_ERR_NO_EPHEM -4     /* no ephemeris loaded */
#define KETE_ERR_CUDA -5         /* a CUDA call failed (message in kete_last_error) */
#define KETE_ERR_NOMEM -6        /* device allocation of library scratch failed */

/* per-body status (int32, written to the caller's status array) */
#define KETE_BODY_OK 0
#define KETE_BODY_STEP_CAP 1      /* more than max_steps step attempts in one leg */
#define KETE_BODY_OUT_OF_SPAN 2   /* the integrator needed planets outside the table */
#define KETE_BODY_NONFINITE 3     /* state or acceleration became NaN/Inf */
#define KETE_BODY_KEPLER_CAP 4    /* two-body solve did not converge (no hits emitted) */

/* precision modes */
#define KETE_FP64 0    /* everything in FP64 */
#define KETE_MIXED 1   /* planetary perturbation terms in FP32, the rest FP64 */

/* Non-gravitational terms of one body (App. A.4-A.5; 80 bytes).  All zero:
 * none.  Forces act in the heliocentric frame (position and velocity
 * relative to table body 0, the Sun, whose GM is mu below).
 *   beta > 0: radiation pressure with Poynting-Robertson drag (Eq. A.6),
 *     beta mu / r^2 [(1 - rdot/c) rhat - v/c], rdot = rhat . v.
 *   a1, a2, a3 (AU/day^2, radial, transverse, normal; Eq. A.7):
 *     g(r) (a1 rhat + a2 that + a3 nhat), g(r) = alpha (r/r0)^-m
 *     (1 + (r/r0)^n)^-k, nhat = r x v / |r x v|, that = nhat x rhat, all
 *     from the two-body state dt days earlier (thermal lag; dt = 0: now).
 *     JPL comet defaults: alpha 0.1112620426, r0 2.808 AU, m 2.15,
 *     n 5.093, k 4.6142; asteroid defaults alpha 1, r0 1, m 2, n 1, k 0
 *     (g = 1/r^2).
 * A failed thermal-lag two-body solve ends the body with
 * KETE_BODY_KEPLER_CAP. */
typedef struct kete_nongrav {
    double a1, a2, a3;
    double alpha, r0, m, n, k;
    double dt;
    double beta;
} kete_nongrav;

/* Force model and integrator controls (Eq. A.1, App. A.2-A.3, App. A.6).
 * Bit b of a mask refers to body b of the loaded table (0 = Sun, 1..8 =
 * Mercury, Venus, Earth-Moon, Mars, Jupiter, Saturn, Uranus, Neptune).
 * Fill with kete_force_model_default() and change what you need. */
typedef struct kete_force_model {
    uint32_t body_mask;          /* bodies whose gravity acts (default 0x1FF) */
    uint32_t gr_mask;            /* GR term of Eq. A.3 (default Sun, Earth, Jupiter) */
    uint32_t j2_mask;            /* J2 term of Eq. A.4 (default Sun, Jupiter) */
    int32_t precision;           /* KETE_FP64 or KETE_MIXED */
    double j2[KETE_MAX_BODIES];  /* J2 coefficient per body */
    double radius[KETE_MAX_BODIES];   /* equatorial radius, AU */
    double pole_ra[KETE_MAX_BODIES];  /* pole right ascension, rad (equatorial J2000) */
    double pole_dec[KETE_MAX_BODIES]; /* pole declination, rad */
    double eps;                  /* IAS15 step-size control parameter (1e-9) */
    double eps_pc;               /* corrector convergence threshold on max|db6|/max|a| (1e-10) */
    double safety;               /* IAS15 safety factor (0.25) */
    double dt_init;              /* first step of each propagation chain, days (4) */
    int32_t max_iter;            /* corrector iteration cap (12) */
    int32_t reserved;
    int64_t max_steps;           /* step attempts per leg before KETE_BODY_STEP_CAP */
    /* Per-body non-gravitational terms: device array of one kete_nongrav per
     * body of the call, indexed like its states (8-byte aligned), or NULL
     * (default).  Read by kete_propagate, kete_propagate_stops,
     * kete_propagate_noalloc, kete_fov_check(_mag), kete_adjoint and
     * kete_sky_jacobian (whose derivatives then take the terms' partials);
     * kete_autotune times its sample without it. */
    const kete_nongrav *nongrav;
} kete_force_model;

/* One FoV patch (Sec. 3.1): a spherical polygon or a cone.  Patches with the
 * same exposure_id must be contiguous and share epoch and observer_idx:
 * together they form the union-of-detectors FoV of one exposure.  Frames
 * must be sorted by epoch (non-decreasing).
 *   n_edges 3..4, polygon: normals[k] is the inward normal of edge k (any
 *   length); a direction u is inside iff normals[k].u > 0 for every k.
 *   n_edges 0 (KETE_FRAME_CONE), cone: normals[0] is the centre direction
 *   (any length), normals[1][0] the angular radius in radians (0 < r < pi);
 *   u is inside iff its angle to the centre is below r.
 * Boundary points are outside.  An extended exposure is approximated by
 * several instantaneous frames along it (kete_fov_check_extended). */
#define KETE_FRAME_CONE 0
typedef struct kete_frame {
    double epoch;                /* TDB JD of the (instantaneous) observation */
    int64_t observer_idx;        /* row of the observers array */
    int64_t exposure_id;         /* groups the sub-fields of one exposure */
    int32_t n_edges;             /* 3 or 4 (polygon), 0 (cone) */
    int32_t reserved;
    double normals[KETE_MAX_EDGES][3];
} kete_frame;                    /* 128 bytes */

/* Options of the survey driver (Sec. 2). */
typedef struct kete_survey_opts {
    double batch_span;           /* a batch holds epochs t with t - t_first < span (3 days) */
    double twobody_max;          /* longest two-body interval (1.5 days); 0 = n-body to every epoch */
    double cell_deg;             /* sky-cell size for candidate search; 0 = automatic */
    double mem_budget_gb;        /* device scratch budget for batch states (0 = 8 GB) */
} kete_survey_opts;

/* One body inside one polygon.  Hits come back sorted by (frame, body). */
typedef struct kete_hit {
    int64_t frame;               /* index into the frames array */
    int32_t body;                /* index into the states arrays */
    float mag;                   /* apparent magnitude (kete_fov_check_mag), else NaN */
    double ra;                   /* rad in [0, 2 pi), equatorial J2000, light-time corrected */
    double dec;                  /* rad */
} kete_hit;                      /* 32 bytes */

/* Counters and device timings of the last call (CUDA events on the context
 * stream around the named kernels). */
typedef struct kete_stats {
    double prop_ms;              /* propagation kernels */
    double fov_ms;               /* everything after propagation in kete_fov_check */
    double total_ms;             /* whole call on the stream */
    int64_t steps;               /* accepted integrator steps */
    int64_t rejected;            /* rejected step attempts */
    int64_t force_evals;         /* acceleration evaluations */
    int64_t iterations;          /* corrector iterations */
    int64_t n_batches;
    int64_t n_exposures;
    int64_t n_candidates;        /* (exposure, body) pairs given the exact test */
    int64_t n_hits;
    int64_t prop_launches;       /* propagation kernel launches */
    int64_t launches;            /* all kernel launches of the call */
    double prep_ms;              /* frame/exposure preparation, batching, sky cells */
    double cand_ms;              /* candidate search */
    double exact_ms;             /* two-body + light-time + polygon test */
    double order_ms;             /* hit ordering */
    int64_t node_evals;          /* force evaluations served by batch node rows (steps that
                                    span a whole leg between consecutive stops) */
    int64_t prop_kind;           /* propagation launch used: KETE_PROP_STATIC or _WORK_STEALING */
    int64_t prop_block;          /* its threads per block */
    int64_t prop_split;          /* lanes per set-aside long body (0: no second phase) */
    int64_t prop_budget;         /* step attempts per stop before a body is set aside */
    int64_t deferred;            /* bodies set aside and finished by the split phase */
    int64_t prop_order;          /* 1: bodies were taken most expensive first */
    int64_t n_exact;             /* candidates the FP32 prefilter passed on to the FP64
                                    two-body solve (the rest cannot be hits) */
} kete_stats;

/* propagation launch variants (kete_set_propagation, kete_autotune) */
#define KETE_PROP_STATIC 0         /* one body per thread, one launch per chunk of stops */
#define KETE_PROP_WORK_STEALING 1  /* persistent: lanes take bodies from an atomic counter and
                                      advance one step attempt per iteration */

typedef struct kete_ctx kete_ctx;

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Errors: KETE_ERR_BAD_ARG (null out), KETE_ERR_CUDA. */
int kete_create(kete_ctx **out, int device, void *cuda_stream);
/* Free the context, its ephemeris and its scratch.  NULL is a no-op. */
void kete_destroy(kete_ctx *ctx);
/* Change the stream later calls are ordered on. */
int kete_set_stream(kete_ctx *ctx, void *cuda_stream);
/* Message of the last failure on this context ("" if none). */
const char *kete_last_error(const kete_ctx *ctx);

/* Defaults: Sun + 8 planets, GR for Sun/Earth/Jupiter (App. A.2), J2 for
 * Sun/Jupiter (App. A.3), IAS15 step control eps 1e-9 and safety 0.25, at most
 * 12 corrector iterations, corrector threshold tuned to 1e-10 (App. A.6), FP64. */
void kete_force_model_default(kete_force_model *fm);
/* Defaults: 3-day batches and 1.5-day two-body interval (Sec. 2). */
void kete_survey_opts_default(kete_survey_opts *opt);

/* Load a planetary Chebyshev table (host buffer, `nbytes` bytes) into device
 * memory owned by the context (App. A: SPICE-like segments).  Layout:
 * 256-byte header {char magic[8] = "KETECHB1"; int32 version = 1; int32
 * n_bodies; int32 n_coef; int32 n_seg; double t_start; double seg_len;
 * double gm[16] at byte 48}, then double coef[n_bodies][n_seg][3][n_coef]
 * (ecliptic x, y, z of each body, AU; segment s covers [t_start + s L,
 * t_start + (s+1) L) with tau = 2 (t - t_mid)/L).  2 <= n_coef <= 64; tables of
 * at most 16 coefficients per segment are evaluated per thread from one
 * shared Chebyshev basis per force evaluation, longer ones with the basis
 * made per body (the same sums, more FP64 work).  Replaces any earlier table.
 * Errors: KETE_ERR_BAD_ARG (malformed header/size), KETE_ERR_CUDA. */
int kete_load_ephem(kete_ctx *ctx, const void *buf, size_t nbytes);

/* Evaluate the loaded table for body `body` at n epochs t (device, n) into
 * pos (device, [n][3]) and, if vel != NULL, vel (device, [n][3], AU/day).
 * An epoch outside the table gives NaN.  Errors: BAD_ARG, NO_EPHEM, CUDA. */
int kete_ephem_eval(kete_ctx *ctx, const double *t, int64_t n, int body, double *pos,
                    double *vel);

/* Propagate n bodies in place to t_target (Sec. 3.2, App. A).
 * states (device, SoA [6][n]: x[n], y[n], z[n], vx[n], vy[n], vz[n]);
 * epochs (device, [n]) give each body's epoch and are set to t_target on
 * success; status (device, [n] int32, may be NULL) receives KETE_BODY_*.
 * A failed body keeps its input state and epoch.
 * Errors: BAD_ARG, NO_EPHEM, CUDA.  Per-body failures are not call errors. */
int kete_propagate(kete_ctx *ctx, double *states, double *epochs, int64_t n, double t_target,
                   const kete_force_model *fm, int32_t *status);

/* kete_propagate through a chain of stops every leg_days days (the survey's
 * batch-midpoint chain, Sec. 2, applied to a single target): the stops are
 * epochs[0] + k leg_days toward t_target (which ends the chain), so that
 * the bodies stay together in time and a step spanning a whole leg reads the
 * planets from rows shared by all bodies instead of evaluating the table.
 * The price is more steps wherever the natural step exceeds leg_days (with
 * 8-day legs, main-belt bodies and comet clones take about twice as many
 * steps, which outweighed the cheaper evaluations on GB300: 1.2-1.3x slower
 * than kete_propagate).  Results agree
 * with a chain of stops on the same grid (kete_propagate_stops), not
 * bit for bit with kete_propagate (another step sequence; the difference is
 * at the integrator's truncation level).  Bodies at other epochs than
 * epochs[0] join the chain at its first stop.  leg_days > 0; at most
 * 10,000,000 legs.  Arguments, results and status otherwise as
 * kete_propagate.  Errors: BAD_ARG, NO_EPHEM, NOMEM, CUDA. */
int kete_propagate_legs(kete_ctx *ctx, double *states, double *epochs, int64_t n,
                        double t_target, double leg_days, const kete_force_model *fm,
                        int32_t *status);

/* Propagate n bodies (not modified) along the chain epoch -> stops[0] ->
 * stops[1] -> ... (host, [n_stops], ascending), carrying the step size along
 * the chain: the schedule kete_fov_check uses for the batch midpoints (Sec. 2,
 * "between the median observation times of consecutive batches").
 * out (device, [n_stops][6][n]) receives the states; a failed body gets NaN
 * from its failing stop on.  Errors: BAD_ARG, NO_EPHEM, CUDA. */
int kete_propagate_stops(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                         const double *stops, int64_t n_stops, const kete_force_model *fm,
                         double *out, int32_t *status);

/* Which bodies fall inside which FoV (Sec. 2, Sec. 3.1).
 * states/epochs: as kete_propagate (device, not modified).
 * frames (device, [n_frames]): see kete_frame; sorted by epoch.
 * observers (device, [n_obs][3]): observer positions, AU, barycentric ecliptic.
 * hits (device, [capacity]): receives the hits sorted by (frame, body).
 * n_hits (host): number of hits.  If it exceeds capacity the call returns
 * KETE_ERR_CAPACITY, writes nothing to hits and leaves the count needed in
 * *n_hits (retry with a larger buffer).  status (device, [n], may be NULL).
 * Errors: BAD_ARG (sizes, unsorted epochs, inconsistent exposures, bad
 * observer index, n_edges not 0, 3 or 4), NO_EPHEM, EPHEM_SPAN (a batch epoch
 * outside the table), CAPACITY, NOMEM, CUDA. */
int kete_fov_check(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                   const kete_frame *frames, int64_t n_frames, const double *observers,
                   int64_t n_obs, const kete_force_model *fm, const kete_survey_opts *opt,
                   kete_hit *hits, int64_t capacity, int64_t *n_hits, int32_t *status);

/* Magnitude model of one body (Sec. 3.3 flux estimation; the comet
 * magnitudes of the appendix), 24 bytes:
 *   KETE_MAG_HG           asteroid V by the H-G system (Bowell et al. 1989,
 *                         two-exponential form): p1 = H, p2 = G
 *   KETE_MAG_COMET_TOTAL  T_mag = M1 + 5 log10(delta) + K1 log10(r_h): p1 = M1, p2 = K1
 *   KETE_MAG_COMET_NUCLEUS N_mag = M2 + 5 log10(delta) + K2 log10(r_h)
 *                         + 0.035 (phase angle in degrees): p1 = M2, p2 = K2
 *   KETE_MAG_NONE         no magnitude (NaN)
 * r_h = heliocentric distance of the body at the light-emission epoch, delta =
 * observer distance, phase = Sun-body-observer angle. */
#define KETE_MAG_NONE 0
#define KETE_MAG_HG 1
#define KETE_MAG_COMET_TOTAL 2
#define KETE_MAG_COMET_NUCLEUS 3
typedef struct kete_mag_params {
    int32_t kind;
    int32_t reserved;
    double p1, p2;
} kete_mag_params;

/* kete_fov_check that also gives every hit its apparent magnitude, computed
 * in the exact FoV test from the same light-time corrected geometry (FP32
 * magnitude arithmetic, ~1e-5 mag).  mag_params: device, [n], one model per
 * body (may be NULL: magnitudes NaN).  Everything else, errors included, as
 * kete_fov_check. */
int kete_fov_check_mag(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                       const kete_frame *frames, int64_t n_frames, const double *observers,
                       int64_t n_obs, const kete_force_model *fm, const kete_survey_opts *opt,
                       const kete_mag_params *mag_params, kete_hit *hits, int64_t capacity,
                       int64_t *n_hits, int32_t *status);

/* Largest n_sub kete_fov_check_extended accepts. */
#define KETE_EXT_MAX_SUB 64

/* kete_fov_check for extended exposures (Sec. 3.1: an exposure of finite
 * length is approximated by several instantaneous observations along it).
 * Frame f (device, [n_frames], sorted by epoch, exposures contiguous, as in
 * kete_fov_check) starts at frames[f].epoch and lasts durations[f] days
 * (device, [n_frames], finite, >= 0, equal within an exposure).  It is split
 * into n_sub (1..KETE_EXT_MAX_SUB) equal sub-intervals; sub-frame k is the
 * same patch at epoch frames[f].epoch + ((k + 0.5) durations[f]) / n_sub seen
 * from observers row frames[f].observer_idx + k (so each exposure owns n_sub
 * consecutive observer rows, one per sub-epoch; rows up to observer_idx +
 * n_sub - 1 must exist).  The sub-frames of one sub-interval of one exposure
 * form one instantaneous exposure of the survey path; the sub-frame epochs
 * must be non-decreasing across exposures (exposures that overlap in time
 * are rejected with KETE_ERR_BAD_ARG).
 * A body is in frame f if it is in any of its sub-frames: hits (device,
 * [capacity]) receive one hit per (frame, body), frame = f, with the RA/Dec
 * (and magnitude, if mag_params is not NULL; see kete_fov_check_mag) of the
 * earliest sub-frame that holds it, sorted by (frame, body).  *n_hits, the
 * CAPACITY retry and status as kete_fov_check; kete_get_stats counts the
 * merged hits and the sub-frame exposures.  Library scratch grows with
 * n_frames * n_sub.  Errors: as kete_fov_check, and BAD_ARG for n_sub,
 * durations or observer rows out of range. */
int kete_fov_check_extended(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                            const kete_frame *frames, int64_t n_frames, const double *durations,
                            int32_t n_sub, const double *observers, int64_t n_obs,
                            const kete_force_model *fm, const kete_survey_opts *opt,
                            const kete_mag_params *mag_params, kete_hit *hits, int64_t capacity,
                            int64_t *n_hits, int32_t *status);

/* Copy the counters of the last call into *out (host). */
int kete_get_stats(const kete_ctx *ctx, kete_stats *out);

/* Choose how the propagation kernel of `precision` (KETE_FP64 / KETE_MIXED)
 * is launched by later calls: kind KETE_PROP_STATIC or
 * KETE_PROP_WORK_STEALING, block 32..128 threads (multiple of 32).  Both
 * produce identical results; they differ in load balance when bodies need
 * very different numbers of steps.  split_lanes 4, 8 or 16 (0 or 1: off) with
 * defer_steps > 0 adds a second phase: a body that has made more than
 * defer_steps step attempts per stop reached is set aside at a step boundary
 * and finished by a persistent launch in which split_lanes lanes share each
 * body's force evaluations (the masses split over the lanes, partial sums
 * combined by shuffles).  Which bodies are set aside depends on each body
 * alone, so the static and work-stealing schedules still agree bit for bit;
 * a set-aside body's force sums are added in another order than in one lane
 * (differences at the rounding level).  cost_order != 0: lanes take the bodies
 * most expensive first (cost estimated from each body's heliocentric conic:
 * steps ~ integral dt / r^1.5), so a warp holds bodies of similar cost; this
 * changes only the schedule, not any result.  Default: work stealing, 128, no
 * split, cost order.
 * Errors: BAD_ARG. */
int kete_set_propagation(kete_ctx *ctx, int precision, int kind, int block, int split_lanes,
                         int defer_steps, int cost_order);

/* Autotuner: time every launch variant (static 128, work stealing 64 and 128,
 * each in index and in cost order; work stealing 128 in cost order with long
 * bodies set aside after 64 attempts per stop for 8 or 4 lanes each, or after
 * 24 for 8 lanes) on an evenly spread sample of min(max_sample, n) of the n
 * bodies (device states [6][n] / epochs [n], not modified), run on persistent
 * grids scaled down by sample / n so that each lane works through as many
 * bodies as in the whole run, propagated along
 * the chain of stops (host, ascending) with force model fm, keep the fastest
 * for fm's precision -- the variant already set stays unless another beats it
 * by more than 5 % on the sample and then by more than 2 % on all n bodies
 * (checked when n_stops x n x 48 bytes of output fit in 2 GB; a sample ranks
 * close variants unreliably) -- and report it in *kind, *block,
 * *split_lanes, *defer_steps,
 * *cost_order (host, each may be NULL).
 * Errors: BAD_ARG, NO_EPHEM, NOMEM, CUDA. */
int kete_autotune(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                  const double *stops, int64_t n_stops, const kete_force_model *fm,
                  int64_t max_sample, int32_t *kind, int32_t *block, int32_t *split_lanes,
                  int32_t *defer_steps, int32_t *cost_order);

/* One astrometric observation of one body (48 bytes). */
typedef struct kete_obs {
    double epoch;                /* TDB JD; NaN marks an unused slot (at the end of a row) */
    double ra, dec;              /* observed, rad, equatorial J2000 */
    double obs[3];               /* observer position, AU, barycentric ecliptic */
} kete_obs;

#define KETE_ADJ_MAX_OBS 32      /* observations per body (m) */
#define KETE_ADJ_MAX_STEPS 256   /* integrator steps per body kept for the backward pass */
#define KETE_BODY_ADJ_CAP 5      /* status: more steps than KETE_ADJ_MAX_STEPS (no gradient) */

/* Orbit-fit loss and its gradient by the adjoint of the propagation and sky
 * projection (differentiation of the path of Sec. 2 / App. A).
 * Forward model of body i: its observations obs[i][0..m) (device, [n][m],
 * sorted by epoch) are batched by the <= batch_span rule (opt, Sec. 2); the
 * n-body chain visits the batch midpoints and the checkpoint grid
 * epochs[i] + ckpt_days * k (k >= 1, before the last midpoint); two-body +
 * light time + RA/Dec give each observation's prediction.
 *   loss[i] = sum_j (wrap(RA_j - RA_obs_j) cos Dec_obs_j)^2 + (Dec_j - Dec_obs_j)^2
 * (device, [n]); grad (device, [6][n], may be NULL) = d loss[i] / d(x0, v0)
 * from the adjoint equations integrated backward over every stored forward
 * step, plus the partials of the two-body, light-time and RA/Dec map by
 * forward-mode differentiation.  fm->nongrav NULL: the Newtonian da/dx alone
 * (the GR and J2 parts of da/dx and GR's da/dv, below 1e-8 relative, are
 * omitted).  fm->nongrav set (per-body terms, as kete_propagate): the forward
 * model includes them and, for every body whose terms are not all zero, the
 * adjoint takes the full model's da/dx and da/dv -- Newtonian, GR, J2 and
 * the body's non-gravitational terms with their thermal lag -- by
 * forward-mode dual numbers at every node of every step (about 300 KB more
 * scratch per body, and a slower forward pass for those bodies; bodies with
 * and without terms are scheduled apart); a body whose terms are all zero is
 * differentiated as without fm->nongrav; pred (device,
 * [n][m][2], may be NULL) = predicted RA, Dec.  FP64 only (fm->precision is
 * ignored).  status (device, [n], may be NULL).
 * ckpt_days: 0 (no grid) or >= 1e-3; a body whose grid would exceed 65536
 * checkpoints gets KETE_BODY_STEP_CAP.  A body with more than
 * KETE_ADJ_MAX_STEPS steps keeps its loss and predictions, gets
 * KETE_BODY_ADJ_CAP and a NaN gradient; any other failing body gets NaN loss
 * and gradient and its KETE_BODY_* code.  Scratch: about 100 KB per body,
 * processed in chunks within opt->mem_budget_gb (0 = 8 GB).
 * Errors: BAD_ARG (m outside 1..KETE_ADJ_MAX_OBS, unsorted observations, bad
 * ckpt_days), NO_EPHEM, NOMEM, CUDA. */
int kete_adjoint(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                 const kete_obs *obs, int32_t m, const kete_force_model *fm,
                 const kete_survey_opts *opt, double ckpt_days, double *loss, double *grad,
                 double *pred, int32_t *status);

/* Per-observation sky partials of an orbit fit: the rows of its Jacobian,
 * d(RA_j, Dec_j)/d(x0, v0) for every observation j of every body, whose
 * J^T J (weighted by the observation errors) gives the covariance of the
 * fitted initial state (the differentiation of the path of Sec. 2 / App. A,
 * for orbit fitting and uncertainty).  The forward model, arguments, batching,
 * checkpoint grid, FP64 and the status codes are kete_adjoint's; the observed
 * ra/dec of obs are not used.  jac (device, [n][m][2][6]): jac[i][j][0][c] =
 * d RA_ij / d y0_c and jac[i][j][1][c] = d Dec_ij / d y0_c, y0 = (x0, v0) of
 * body i (rad per AU, rad per AU/day); rows of unused observation slots and
 * of failed bodies (status not KETE_BODY_OK) are NaN.  Each row is the state-
 * transition matrix at the observation's batch midpoint -- the variational
 * equations dx'' = (da/dx) dx + (da/dv) dx' (the Jacobians of kete_adjoint)
 * integrated forward over every stored step -- multiplied by the partials of the
 * two-body, light-time and RA/Dec map there.  pred (device, [n][m][2], may be
 * NULL): predicted RA, Dec.  Scratch: about 100 KB + 290 m bytes per body, in
 * chunks within opt->mem_budget_gb.  Errors: as kete_adjoint. */
int kete_sky_jacobian(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                      const kete_obs *obs, int32_t m, const kete_force_model *fm,
                      const kete_survey_opts *opt, double ckpt_days, double *jac, double *pred,
                      int32_t *status);

/* Largest n kete_propagate_noalloc accepts. */
#define KETE_NOALLOC_MAX_BODIES 65536

/* kete_propagate without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run -- an application that gives all GPU memory to
 * its own pool at start-up, a real-time host thread that must not block in
 * the driver's allocator, a framework that forbids allocation outside its
 * set-up phase.  kete_propagate allocates its per-body chain scratch on first
 * use; this variant uses a fixed array in the library's device data instead
 * (about 4.5 MB, held on every GPU that loads the library until exit).
 *
 * Arguments, layouts and per-body status are those of kete_propagate; the
 * context must already exist and hold an ephemeris (kete_create and
 * kete_load_ephem allocate; call them during set-up).  It always runs one
 * launch variant: the static schedule, one lane per body, bodies in index
 * order, the planets summed per thread (no shared node rows), whatever
 * kete_set_propagation chose -- so it is slower than kete_propagate on
 * uneven populations, and its results agree with kete_propagate's to the
 * integrator's truncation level, not bit for bit.
 * n above KETE_NOALLOC_MAX_BODIES is rejected with KETE_ERR_BAD_ARG and a
 * message in kete_last_error; split larger populations into several calls.
 * The call calls no cudaMalloc or cudaFree and does not update
 * kete_get_stats.  The first call on a device resolves the array's device
 * address (which may load the library's device data): make that first call
 * before any stream capture.  The address is kept for the life of the
 * process; a cudaDeviceReset of that device invalidates it, so do not call
 * this entry point on a device after resetting it.  All calls on a device
 * share the one array: calls whose work overlaps on the GPU race, so order
 * them on one stream. */
int kete_propagate_noalloc(kete_ctx *ctx, double *states, double *epochs, int64_t n,
                           double t_target, const kete_force_model *fm, int32_t *status);

#ifdef __cplusplus
}
#endif
#endif
