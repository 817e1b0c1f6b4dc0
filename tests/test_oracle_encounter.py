"""Pins of the oracle's close-encounter formulation (reading R12; App. A /
Sec. 3.2 integration near planets).

With a planet within 0.1 AU at a step start the oracle forms the body-planet
vector at a substep as (x0 - p(t0)) + (dx - dp), dp = p(t0 + off) - p(t0)
from a recurrence on Chebyshev differences (ephem_delta), and ends the step
at the next table segment boundary (find_close).  Independent references:

  * the displacement against exact rational arithmetic over the table's own
    coefficients (Python fractions: no rounding at all), for every planet and
    offsets from 1e-6 day to a whole segment;
  * a flyby of a point mass in uniform straight-line motion, whose frame is
    inertial, so the body's relative orbit is the closed-form hyperbola
    (e sinh H - H = M, solved here) -- deflections of 1 to 141 degrees at
    0.002-0.05 AU;
  * the encounter set-up against its definition (nearest active planet within
    0.1 AU, the segment boundary in the direction of motion)."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W


def _cheb_exact(c, tau):
    """sum_k c_k T_k(tau) in exact rational arithmetic (three-term recurrence)."""
    Tm, T = Fr(1), tau
    s = c[0] + c[1] * tau
    for k in range(2, len(c)):
        Tm, T = T, 2 * tau * T - Tm
        s += c[k] * T
    return s


def test_ephem_delta_matches_exact_rational_difference(mb1k):
    """dp = p(t0 + off) - p(t0), both read from the polynomial of the segment
    holding t0, agrees with the exact value to 5e-17 AU per day of offset for
    every planet and offsets of 1e-6 to 16 days in both directions (the
    difference of two rounded positions would carry ~1e-16 AU whatever the
    offset: 1e-10 AU per day at off = 1e-6)."""
    e = mb1k.ephem
    orc = O.Oracle(e.to_bytes())
    rng = np.random.default_rng(5)
    L = Fr(e.seg_len)
    worst = 0.0
    for b in range(1, e.n_bodies):
        for t0 in rng.uniform(e.t_start, e.t_end - 1e-3, 4):
            s = min(int((t0 - e.t_start) // e.seg_len), e.n_seg - 1)
            t_mid = Fr(e.t_start) + (Fr(s) + Fr(1, 2)) * L
            tau0 = 2 * (Fr(t0) - t_mid) / L
            for off in (1e-6, -1e-6, 3.7e-5, 1e-3, -0.02, 0.5, -2.0, 7.9, -15.9, 16.0):
                rc, dp = orc.ephem_delta(b, t0, off)
                assert rc == O.OK
                tau1 = tau0 + 2 * Fr(off) / L
                for c in range(3):
                    cf = [Fr(x) for x in e.coef[b, s, c]]
                    exact = _cheb_exact(cf, tau1) - _cheb_exact(cf, tau0)
                    worst = max(worst, abs(dp[c] - float(exact)) / abs(off))
    assert worst < 5e-17, worst
    # zero offset: exactly zero; outside the table: an error
    assert np.array_equal(orc.ephem_delta(3, e.t_start + 5.0, 0.0)[1], np.zeros(3))
    assert orc.ephem_delta(3, e.t_start - 1.0, 0.5)[0] == O.OUT_OF_SPAN


def _hyperbola(q, ecc, mu, t_peri, t, P, Q):
    """Relative state on the hyperbola of periapsis q (AU), eccentricity ecc,
    periapsis epoch t_peri and orbital axes P (to periapsis), Q, at t."""
    a = q / (1.0 - ecc)
    n = math.sqrt(mu / (-a) ** 3)
    M = n * (t - t_peri)
    H = math.asinh(M / ecc)
    for _ in range(200):
        dH = (ecc * math.sinh(H) - H - M) / (ecc * math.cosh(H) - 1.0)
        H -= dH
        if abs(dH) < 1e-16 * max(1.0, abs(H)):
            break
    r = a * (1.0 - ecc * math.cosh(H))
    xp = a * (math.cosh(H) - ecc)
    yp = -a * math.sqrt(ecc * ecc - 1.0) * math.sinh(H)
    vf = math.sqrt(-mu * a) / r
    vx, vy = -vf * math.sinh(H), vf * math.sqrt(ecc * ecc - 1.0) * math.cosh(H)
    return P * xp + Q * yp, P * vx + Q * vy


def _uniform_mass_table(p0, u, mu, t0, n_seg=6, seg_len=16.0, n_coef=12, extra=None):
    """Table of a massless-by-mask Sun at the origin and one point mass (body 1)
    on p(t) = p0 + u (t - t0): per segment c_0 = p(t_mid), c_1 = u L / 2.
    extra: (p0, u, mu) of a second mass (body 2)."""
    masses = [(p0, u, mu)] + ([extra] if extra else [])
    t_start = t0 - 2 * seg_len
    coef = np.zeros((1 + len(masses), n_seg, 3, n_coef))
    for b, (pb, ub, _) in enumerate(masses, start=1):
        for s in range(n_seg):
            tm = t_start + (s + 0.5) * seg_len
            coef[b, s, :, 0] = pb + ub * (tm - t0)
            coef[b, s, :, 1] = ub * seg_len / 2
    gm = np.array([W.GM_SUN] + [m for _, _, m in masses])
    return W.EphemTable(t_start, seg_len, n_seg, n_coef, gm, coef)


FLYBYS = [  # periapsis AU, GM AU^3/day^2, v_inf km/s
    (0.002, 2.8e-7, 10.0),       # Jupiter-mass point, 108 deg deflection
    (0.002, 2.8e-7, 5.0),        # 141 deg
    (0.002, 8.997e-10, 10.0),    # Earth-mass point, 1.5 deg
    (0.01, 8.997e-10, 5.0),
    (0.02, 2.8e-7, 3.0),
    (0.05, 2.8e-7, 20.0),
]


@pytest.mark.parametrize("q,mu,vinf", FLYBYS)
def test_flyby_of_uniformly_moving_mass_is_the_closed_form_hyperbola(q, mu, vinf):
    """A body passes a point mass moving uniformly at ~1 AU from the origin
    (Sun masked off, no GR or J2): after 20 days through periapsis its
    position is the closed-form hyperbola carried along with the mass, to
    1e-12 AU, and the pass takes a bounded number of steps."""
    v = vinf * 86400.0 / W.AU_KM
    ecc = 1.0 + q * v * v / mu
    p0 = np.array([0.9, 0.35, 0.05])
    u = np.array([-0.006, 0.015, 0.0004])
    rng = np.random.default_rng(4)
    P = rng.normal(size=3); P /= np.linalg.norm(P)
    Q = np.cross(P, rng.normal(size=3)); Q /= np.linalg.norm(Q)
    t0, t_peri, t1 = W.T0, W.T0 + 10.0, W.T0 + 20.0
    orc = O.Oracle(_uniform_mass_table(p0, u, mu, t0).to_bytes())
    fm = orc.force_model(body_mask=0b10, gr_mask=0, j2_mask=0, max_steps=100000)
    r0, w0 = _hyperbola(q, ecc, mu, t_peri, t0, P, Q)
    rc, st, t, _, stats = orc.propagate(fm, np.concatenate([r0 + p0, w0 + u]), t0, t1)
    assert rc == O.OK and t == t1
    r1, w1 = _hyperbola(q, ecc, mu, t_peri, t1, P, Q)
    assert np.abs(st[:3] - (r1 + p0 + u * (t1 - t0))).max() < 1e-12
    assert np.abs(st[3:] - (w1 + u)).max() < 1e-12
    assert stats.steps < 400


def test_find_close_picks_the_nearest_planet_and_the_segment_boundary():
    """Encounter set-up at a step start: the nearest active mass within
    0.1 AU (an inactive or more distant one is ignored), x - p_m(t), and the
    step range cut at the next segment boundary in the direction of motion
    (the previous boundary backward; the target if it comes first)."""
    p1, u1 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.017, 0.0])
    p2, u2 = np.array([1.03, 0.0, 0.0]), np.array([0.0, 0.017, 0.0])
    tab = _uniform_mass_table(p1, u1, 1e-9, W.T0, extra=(p2, u2, 2e-9))
    orc = O.Oracle(tab.to_bytes())
    fm = orc.force_model(body_mask=0b110, gr_mask=0, j2_mask=0)
    t = W.T0 + 3.25                        # segment [T0, T0 + 16)
    pm1, pm2 = p1 + u1 * 3.25, p2 + u2 * 3.25
    x = pm1 + np.array([0.02, 0.001, 0.0])   # 0.02 from mass 1, 0.01 from mass 2
    rc, m, d0, t_stop = orc.find_close(fm, t, x, W.T0 + 40.0)
    assert rc == O.OK and m == 2
    np.testing.assert_allclose(d0, x - pm2, rtol=0, atol=1e-15)
    assert t_stop == W.T0 + 16.0
    rc, m, _, t_stop = orc.find_close(fm, t, x, W.T0 - 40.0)
    assert m == 2 and t_stop == W.T0
    rc, m, _, t_stop = orc.find_close(fm, t, x, W.T0 + 5.0)
    assert m == 2 and t_stop == W.T0 + 5.0
    # mass 2 switched off: mass 1 is the nearest active one
    rc, m, d0, _ = orc.find_close(orc.force_model(body_mask=0b010), t, x, W.T0 + 40.0)
    assert m == 1
    np.testing.assert_allclose(d0, x - pm1, rtol=0, atol=1e-15)
    # beyond 0.1 AU of both: no encounter, the step range is the target
    far = pm1 + np.array([0.0, 0.0, 0.15])
    rc, m, _, t_stop = orc.find_close(fm, t, far, W.T0 + 40.0)
    assert m == -1 and t_stop == W.T0 + 40.0
    # at a boundary, moving backward: the boundary before it
    rc, m, _, t_stop = orc.find_close(fm, W.T0 + 16.0, p1 + u1 * 16.0 + 0.01, W.T0 - 40.0)
    assert m == 1 and t_stop == W.T0
