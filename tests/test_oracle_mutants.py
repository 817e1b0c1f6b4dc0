"""Planted mistakes: the oracle's pins are not vacuous.

Each case plants one plausible mistake (a dropped term, a wrong sign or
index, a transposed operand) in a copy of oracle/kete_oracle.c, builds the
copy in a temporary directory with the oracle's own flags, and runs the pin
that should catch it against that library (the oracle module loads the
library named by KETE_ORACLE_LIB).  The pin must fail.  The committed oracle
is never modified; the mutants run on the CPU only."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "kete_oracle.c")
HDR = os.path.join(ROOT, "oracle", "kete_oracle.h")

ORA_I = "tests/test_oracle_integrator.py::"
ORA_G = "tests/test_oracle_geometry.py::"
ORA_K = "tests/test_oracle_kepler.py::"
ORA_E = "tests/test_oracle_encounter.py::"
ORA_N = "tests/test_oracle_nongrav.py::"
ORA_M = "tests/test_oracle_magnitude.py::"

# (name, text in kete_oracle.c (exactly once), mistake, pins that must fail)
MUTANTS = [
    # force model (Eq. A.1, A.3, A.4)
    ("gr_sign", "a[i] += k * ((4.0 * mu / rn - w2) * r[i] + 4.0 * rw * w[i]);",
     "a[i] -= k * ((4.0 * mu / rn - w2) * r[i] + 4.0 * rw * w[i]);",
     [ORA_I + "test_gr_perihelion_advance_mercury"]),
    ("gr_velocity_term", "(4.0 * mu / rn - w2) * r[i] + 4.0 * rw * w[i]",
     "(4.0 * mu / rn - w2) * r[i] + 4.0 * rw * r[i]",
     [ORA_I + "test_gr_perihelion_advance_mercury"]),
    ("j2_sign", "double ab[3] = {-psi * (1.0 - q) * xb, -psi * (1.0 - q) * yb, -psi * (3.0 - q) * zb};",
     "double ab[3] = {psi * (1.0 - q) * xb, psi * (1.0 - q) * yb, psi * (3.0 - q) * zb};",
     [ORA_I + "test_j2_nodal_regression_rate"]),
    ("planet_gm_index", "double mu = e->gm[m];", "double mu = e->gm[m > 0 ? m - 1 : 0];",
     [ORA_I + "test_planet_terms_conserve_jacobi_integral"]),
    ("planet_position_component", "double r[3] = {x[0] - pm[0], x[1] - pm[1], x[2] - pm[2]};",
     "double r[3] = {x[0] - pm[0], x[1] - pm[1], x[2] - pm[1]};",
     [ORA_I + "test_planet_terms_conserve_jacobi_integral"]),
    # ephemeris (App. A: Chebyshev segments)
    ("ephem_velocity_scale", "if (vel) vel[c] = sv * 2.0 / e->seg_len;",
     "if (vel) vel[c] = sv / e->seg_len;", [ORA_I + "test_chebyshev_eval_against_numpy"]),
    ("ephem_recurrence", "T[k] = 2.0 * tau * T[k - 1] - T[k - 2];",
     "T[k] = 2.0 * tau * T[k - 1] + T[k - 2];", [ORA_I + "test_chebyshev_eval_against_numpy"]),
    # Gauss-Radau / IAS15 (App. A.6)
    ("divided_difference_index",
     "g_{n-1} */\n            for (int i = 0; i < 3; i++) {\n                double d = (F[n][i] - F[0][i]) / (R->h[n] - R->h[0]);\n                for (int k = 1; k < n; k++) d = (d - g[k][i]) / (R->h[n] - R->h[k]);",
     "g_{n-1} */\n            for (int i = 0; i < 3; i++) {\n                double d = (F[n][i] - F[0][i]) / (R->h[n] - R->h[0]);\n                for (int k = 1; k < n; k++) d = (d - g[k][i]) / (R->h[n] - R->h[k - 1]);",
     [ORA_I + "test_integrator_reproduces_kepler_orbit"]),
    ("predictor_coefficient",
     "/* s^(k+2) */\n                for (int k = 0; k < 7; k++) {\n                    acc += b[k][i] * sp * s / ((k + 2.0) * (k + 3.0));",
     "/* s^(k+2) */\n                for (int k = 0; k < 7; k++) {\n                    acc += b[k][i] * sp * s / ((k + 2.0) * (k + 2.0));",
     [ORA_I + "test_integrator_reproduces_kepler_orbit"]),
    # close encounters (R12)
    ("delta_recurrence_term", "D[k + 1] = 2.0 * tau1 * D[k] - D[k - 1] + 2.0 * dtau * T[k];",
     "D[k + 1] = 2.0 * tau1 * D[k] - D[k - 1];",
     [ORA_E + "test_ephem_delta_matches_exact_rational_difference"]),
    ("delta_recurrence_argument", "D[k + 1] = 2.0 * tau1 * D[k] - D[k - 1] + 2.0 * dtau * T[k];",
     "D[k + 1] = 2.0 * tau0 * D[k] - D[k - 1] + 2.0 * dtau * T[k];",
     [ORA_E + "test_ephem_delta_matches_exact_rational_difference"]),
    ("encounter_vector_sign", "for (int i = 0; i < 3; i++) r[i] = cl->d0[i] + (cl->dx[i] - dp[i]);",
     "for (int i = 0; i < 3; i++) r[i] = cl->d0[i] + (cl->dx[i] + dp[i]);",
     [ORA_E + "test_flyby_of_uniformly_moving_mass_is_the_closed_form_hyperbola"]),
    ("encounter_displacement_stale",
     "if (cl) cl->dx[i] = dxn;\n            }\n            int st = accel_off_cl",
     "if (cl) cl->dx[i] = 0.0;\n            }\n            int st = accel_off_cl",
     [ORA_E + "test_flyby_of_uniformly_moving_mass_is_the_closed_form_hyperbola"]),
    ("encounter_boundary", "double b = (dir > 0) ? e->t_start + (k + 1.0) * e->seg_len",
     "double b = (dir > 0) ? e->t_start + (k + 2.0) * e->seg_len",
     [ORA_E + "test_find_close_picks_the_nearest_planet_and_the_segment_boundary"]),
    ("encounter_farthest", "        if (d < best) {\n            best = d;\n            cl->m = m;",
     "        if (d < KO_CLOSE_AU) {\n            best = d;\n            cl->m = m;",
     [ORA_E + "test_find_close_picks_the_nearest_planet_and_the_segment_boundary"]),
    # two-body, light time, sky projection, FoV, batches (Sec. 2, Sec. 3.1)
    ("stumpff_series", "t3 *= -z / ((2.0 * k + 4.0) * (2.0 * k + 5.0));",
     "t3 *= -z / ((2.0 * k + 3.0) * (2.0 * k + 5.0));", [ORA_K + "test_stumpff_against_mpmath"]),
    ("kepler_derivative", "double dF = A * chi * (1.0 - z * c3) + B * chi * chi * c2 + r0;",
     "double dF = A * chi * (1.0 - z * c2) + B * chi * chi * c2 + r0;",
     [ORA_K + "test_kepler_elliptic_closed_form", ORA_K + "test_kepler_hyperbolic_closed_form"]),
    ("light_time_iterations", "    for (int it = 0; it < 3; it++) {\n        s = twobody_pos(e, helio, t_ref, dt_obs - tau, pos);",
     "    for (int it = 0; it < 0; it++) {\n        s = twobody_pos(e, helio, t_ref, dt_obs - tau, pos);",
     [ORA_G + "test_light_time_uniform_motion_closed_form"]),
    ("obliquity_sign", "double y = ce * u[1] - se * u[2];", "double y = ce * u[1] + se * u[2];",
     [ORA_G + "test_radec_known_directions"]),
    ("polygon_not_strict", "if (!(d > 0.0)) inside = 0;", "if (!(d >= 0.0)) inside = 0;",
     [ORA_G + "test_fov_boundary_is_outside"]),
    ("batch_span", "while (j + 1 < n && (ep[j + 1] == ep[i] || ep[j + 1] - ep[i] < span)) j++;",
     "while (j + 1 < n && (ep[j + 1] == ep[i] || ep[j + 1] - ep[i] <= span)) j++;",
     [ORA_G + "test_batches_greedy_three_day_rule"]),
    ("batch_twobody_cap", "if (2.0 * twobody_max < span) span = 2.0 * twobody_max;",
     "if (twobody_max < span) span = twobody_max;",
     [ORA_G + "test_batches_greedy_three_day_rule", ORA_G + "test_batches_zero_twobody_interval_is_per_epoch"]),
    # non-gravitational terms (Eq. A.6, A.7)
    ("pr_drag_sign", "a[i] += f * ((1.0 - rdot / c) * r[i] / rn - w[i] / c);",
     "a[i] += f * ((1.0 - rdot / c) * r[i] / rn + w[i] / c);",
     [ORA_N + "test_poynting_robertson_decays_angular_momentum"]),
    ("pr_radial_factor", "a[i] += f * ((1.0 - rdot / c) * r[i] / rn - w[i] / c);",
     "a[i] += f * ((1.0 + rdot / c) * r[i] / rn - w[i] / c);",
     [ORA_N + "test_poynting_robertson_secular_decay_of_a"]),
    ("comet_g_exponent", "double g = p->alpha * pow(q, -p->m) * pow(1.0 + pow(q, p->n), -p->k);",
     "double g = p->alpha * pow(q, p->m) * pow(1.0 + pow(q, p->n), -p->k);",
     [ORA_N + "test_comet_g_is_normalised_at_one_au_and_at_r0"]),
    ("transverse_direction", "double th[3] = {nh[1] * rh[2] - nh[2] * rh[1], nh[2] * rh[0] - nh[0] * rh[2],",
     "double th[3] = {nh[2] * rh[1] - nh[1] * rh[2], nh[0] * rh[2] - nh[2] * rh[0],",
     [ORA_N + "test_transverse_force_changes_a_at_gauss_rate"]),
    ("thermal_lag_sign", "int s = ko_kepler(mu, r, w, -p->dt, rl, wl);",
     "int s = ko_kepler(mu, r, w, p->dt, rl, wl);",
     [ORA_N + "test_thermal_lag_turns_the_radial_force_backwards"]),
    ("normal_direction", "p->a2 * th[i] + p->a3 * nh[i]);", "p->a2 * th[i] + p->a3 * rh[i]);",
     [ORA_N + "test_normal_force_tilts_the_plane_only"]),
    ("nongrav_barycentric", "double r[3] = {x[0] - ps[0], x[1] - ps[1], x[2] - ps[2]};",
     "double r[3] = {x[0], x[1], x[2]};", [ORA_N + "test_nongrav_terms_follow_the_sun"]),
    # per-observation sky partials (the orbit-fit Jacobian)
    ("sky_jacobian_transposed_stm", "for (int c = 0; c < 6; c++) acc += dr[a][c] * phi[c * 6 + c0];",
     "for (int c = 0; c < 6; c++) acc += dr[a][c] * phi[c0 * 6 + c];",
     ["tests/test_oracle_adjoint.py::test_sky_jacobian_matches_finite_differences_of_the_predictions"]),
    # magnitudes (Sec. 3.3)
    ("hg_phase_constant", "const double phi1 = exp(-3.33 * pow(t, 0.63));",
     "const double phi1 = exp(-3.33 * pow(t, 1.22));", [ORA_M + "test_hg_phase_function_exponents"]),
    ("nucleus_phase_coefficient", "+ 0.035 * (alpha * 180.0 / M_PI);", "+ 0.035 * alpha;",
     [ORA_M + "test_comet_magnitudes"]),
]


def _source():
    with open(SRC) as f:
        return f.read()


def test_every_mutant_names_text_that_occurs_once():
    src = _source()
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for name, old, new, pins in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new and pins, name


def _run_mutant(tmp, name, old, new, pins):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    with open(os.path.join(d, "kete_oracle.c"), "w") as f:
        f.write(_source().replace(old, new))
    with open(HDR) as f, open(os.path.join(d, "kete_oracle.h"), "w") as g:
        g.write(f.read())
    lib = os.path.join(d, "libkete_oracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-pthread", os.path.join(d, "kete_oracle.c"),
                           "-o", lib, "-lm"])
    env = dict(os.environ, KETE_ORACLE_LIB=lib, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-2000:]


def test_each_planted_mistake_fails_its_pin():
    """Exit code 1 of pytest = tests ran and at least one failed (2-5 would be
    an interrupted run, a usage error or nothing collected)."""
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
            res = list(ex.map(lambda m: _run_mutant(tmp, *m), MUTANTS))
    survived = [(name, rc, out) for name, rc, out in res if rc != 1]
    assert not survived, "\n\n".join(f"{n}: rc {rc}\n{out}" for n, rc, out in survived)


@pytest.mark.parametrize("name", ["gr_sign"])
def test_the_unmutated_oracle_passes_the_same_pins(name):
    """Control: the committed oracle passes the pins the mutants fail (the
    suite runs them anyway; this keeps the harness honest if pins move)."""
    pins = [p for m in MUTANTS if m[0] == name for p in m[3]]
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("KETE_ORACLE_LIB", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
