"""Pins of the oracle's non-gravitational terms (App. A.4: radiation pressure
with Poynting-Robertson drag, Eq. A.6; App. A.5: the JPL comet model with its
thermal lag, Eq. A.7), each against mechanics that does not restate the force:

- a radial 1/r^2 force is a weaker Sun: Kepler's closed form with mu - A1;
- the comet g(r) is normalised to 1 at 1 AU and equals alpha 2^-k at r0
  (circular orbits stay circular at the matching speed);
- a transverse force changes the semi-major axis at Gauss's rate 2 T / n;
- a normal force leaves energy and |h| alone and lifts the orbit by A t^2/2;
- the thermal lag turns the radial force backwards by the angle the body
  moved: the same motion as A1 cos(n dt) radial, -A1 sin(n dt) transverse;
- the terms follow the Sun: a Sun in uniform motion changes nothing
  heliocentric (Galilean invariance; the force takes heliocentric r and v);
- radiation pressure weakens the Sun by (1 - beta), drag decays the angular
  momentum as dh/dt = -beta mu h / (c r^2), and the secular decay of a over
  one orbit follows Wyatt & Whipple's (2 + 3e^2) / (a (1-e^2)^1.5) rate.
"""
import math

import numpy as np
import pytest
from scipy.integrate import simpson

import oracle as O
from paper_2509_04666_gb300 import workloads as W

MU = W.GM_SUN
C_AU_D = 299792.458 * 86400.0 / 149597870.7


def _orc(days=800):
    orc = O.Oracle(W.static_sun_table(W.T0 - 40, W.T0 + days).to_bytes())
    return orc


def _fm(orc, ng):
    fm = orc.force_model(body_mask=1, gr_mask=0, j2_mask=0)
    fm.ng = ng
    return fm


def _elements(a, e, inc, node, peri, M, mu):
    r, v = W.elements_to_state(np.array([a]), np.array([e]), inc, node, peri, M, mu)
    return np.concatenate([r[:, 0], v[:, 0]])


def _circular(r, v):
    return np.array([r, 0.0, 0.0, 0.0, v, 0.0])


def _run(orc, ng, x0, days):
    rc, st, t, _, _ = orc.propagate(_fm(orc, ng), x0, W.T0, W.T0 + days)
    assert rc == 0 and t == W.T0 + days
    return st


def _a_osc(st, mu):
    r = np.linalg.norm(st[:3])
    return 1.0 / (2.0 / r - st[3:] @ st[3:] / mu)


@pytest.mark.parametrize("A", [2e-6, -1e-6])
def test_radial_inverse_square_force_is_a_weaker_sun(A):
    orc = _orc()
    mu = MU - A
    x0 = _elements(1.8, 0.4, 0.3, 1.2, 2.1, 0.4, mu)
    st = _run(orc, O.asteroid_ng(a1=A), x0, 365.0)
    ref = _elements(1.8, 0.4, 0.3, 1.2, 2.1, 0.4 + math.sqrt(mu / 1.8 ** 3) * 365.0, mu)
    assert np.abs(st[:3] - ref[:3]).max() < 1e-12


def test_comet_g_is_normalised_at_one_au_and_at_r0():
    orc = _orc()
    A = 1e-6
    # alpha makes g(1 AU) = 1 to 2.4e-9, which leaves a radial oscillation of
    # 2 A 2.4e-9 / mu ~ 1.6e-11 AU; a wrong exponent would give ~A / mu ~ 3e-3
    for r, g, tol in ((1.0, 1.0, 5e-11), (2.808, 0.1112620426 * 2.0 ** -4.6142, 1e-11)):
        v = math.sqrt(MU / r - A * g * r)
        st = _run(orc, O.comet_ng(a1=A), _circular(r, v), 200.0)
        assert abs(np.linalg.norm(st[:3]) - r) < tol * r
        n = v / r
        ang = math.atan2(st[1], st[0]) % (2 * math.pi)
        assert abs(ang - (n * 200.0) % (2 * math.pi)) < 1e-10


@pytest.mark.parametrize("A", [1e-9, -1e-9])
def test_transverse_force_changes_a_at_gauss_rate(A):
    orc = _orc()
    days = 100.0
    st = _run(orc, O.asteroid_ng(a2=A), _circular(1.0, math.sqrt(MU)), days)
    da = _a_osc(st, MU) - 1.0
    ref = 2.0 * A / math.sqrt(MU) * days          # da/dt = 2 T a^1.5 / sqrt(mu), T = A
    assert abs(da - ref) < 2e-3 * abs(ref)


def test_normal_force_tilts_the_plane_only():
    orc = _orc()
    A = 1e-8
    x0 = _circular(1.0, math.sqrt(MU))
    E0 = 0.5 * x0[3:] @ x0[3:] - MU
    h0 = np.linalg.norm(np.cross(x0[:3], x0[3:]))
    st = _run(orc, O.asteroid_ng(a3=A), x0, 5.0)
    assert abs(st[2] - 0.5 * A * 25.0) < 1e-2 * 0.5 * A * 25.0
    for days in (5.0, 200.0):
        st = _run(orc, O.asteroid_ng(a3=A), x0, days)
        E = 0.5 * st[3:] @ st[3:] - MU / np.linalg.norm(st[:3])
        assert abs(E - E0) < 1e-14
        assert abs(np.linalg.norm(np.cross(st[:3], st[3:])) - h0) < 1e-14


def test_thermal_lag_turns_the_radial_force_backwards():
    orc = _orc()
    A, D, days = 1e-9, 30.0, 100.0
    x0 = _circular(1.0, math.sqrt(MU))
    n = math.sqrt(MU)
    lag = _run(orc, O.asteroid_ng(a1=A, dt=D), x0, days)
    rot = _run(orc, O.asteroid_ng(a1=A * math.cos(n * D), a2=-A * math.sin(n * D)), x0, days)
    nolag = _run(orc, O.asteroid_ng(a1=A), x0, days)
    free = _run(orc, O.NonGrav(), x0, days)
    effect = np.linalg.norm(lag[:3] - free[:3])
    assert effect > 1e-6
    assert np.linalg.norm(lag[:3] - rot[:3]) < 1e-3 * effect
    assert np.linalg.norm(lag[:3] - nolag[:3]) > 0.2 * effect


def test_radiation_pressure_weakens_the_sun_by_beta():
    orc = _orc()
    beta = 0.01
    mu = MU * (1.0 - beta)
    x0 = _elements(1.5, 0.3, 0.2, 0.7, 1.1, 0.9, mu)
    st = _run(orc, O.dust_ng(beta), x0, 10.0)
    ref = _elements(1.5, 0.3, 0.2, 0.7, 1.1, 0.9 + math.sqrt(mu / 1.5 ** 3) * 10.0, mu)
    # the drag terms (v/c ~ 1e-4 of the radial one) move it by ~1e-8 AU here
    assert np.abs(st[:3] - ref[:3]).max() < 1e-7
    plain = _elements(1.5, 0.3, 0.2, 0.7, 1.1, 0.9 + math.sqrt(MU / 1.5 ** 3) * 10.0, MU)
    assert np.abs(st[:3] - plain[:3]).max() > 1e-5


def test_poynting_robertson_decays_angular_momentum():
    orc = _orc()
    beta = 0.02
    mu = MU * (1.0 - beta)
    x0 = _elements(1.3, 0.35, 0.4, 0.2, 0.5, 0.0, mu)
    stops = W.T0 + np.arange(1.0, 366.0)
    rc, out, _ = orc.propagate_stops(_fm(orc, O.dust_ng(beta)), x0, W.T0, stops)
    assert rc == 0
    traj = np.vstack([x0, out])
    h = np.cross(traj[:, :3], traj[:, 3:])
    r2 = (traj[:, :3] ** 2).sum(1)
    integ = simpson(1.0 / r2, dx=1.0)          # integral of 1/r^2 over the year
    ref = -beta * MU / C_AU_D * integ
    got = math.log(np.linalg.norm(h[-1]) / np.linalg.norm(h[0]))
    assert abs(got - ref) < 1e-4 * abs(ref)
    # the plane does not move: dh/dt is parallel to h
    cr = np.linalg.norm(np.cross(h[0], h[-1])) / (np.linalg.norm(h[0]) * np.linalg.norm(h[-1]))
    assert cr < 1e-12


def test_poynting_robertson_secular_decay_of_a():
    orc = _orc(days=900)
    beta, a0, e0 = 0.05, 1.0, 0.5
    mu = MU * (1.0 - beta)
    x0 = _elements(a0, e0, 0.1, 0.0, 0.0, 0.0, mu)          # at perihelion
    T = 2 * math.pi / math.sqrt(mu / a0 ** 3)
    st = _run(orc, O.dust_ng(beta), x0, T)
    da = _a_osc(st, mu) - _a_osc(x0, mu)
    # Wyatt & Whipple (1950): <da/dt> = -(beta mu_sun / c) (2 + 3e^2) / (a (1-e^2)^1.5)
    ref = -(beta * MU / C_AU_D) * (2 + 3 * e0 ** 2) / (a0 * (1 - e0 ** 2) ** 1.5) * T
    assert abs(da - ref) < 0.02 * abs(ref)


def _moving_sun_oracle(V, days=200):
    """The Sun in uniform motion p(t) = V (t - T0): Chebyshev c0, c1 per segment."""
    tab = W.static_sun_table(W.T0 - 40, W.T0 + days)
    for s in range(tab.n_seg):
        t_mid = tab.t_start + (s + 0.5) * tab.seg_len
        tab.coef[0, s, :, 0] = V * (t_mid - W.T0)
        tab.coef[0, s, :, 1] = V * 0.5 * tab.seg_len
    return O.Oracle(tab.to_bytes())


@pytest.mark.parametrize("ng", [O.dust_ng(0.02), O.comet_ng(1e-7, -3e-8, 2e-8, dt=10.0),
                                O.asteroid_ng(a2=5e-8, a3=-5e-8)])
def test_nongrav_terms_follow_the_sun(ng):
    V = np.array([0.004, -0.007, 0.002])          # AU/day, comparable to orbital speeds
    still, moving = _orc(), _moving_sun_oracle(V)
    x0 = _elements(1.4, 0.3, 0.4, 0.3, 1.0, 0.5, MU)
    days = 60.0
    a = _run(still, ng, x0, days)
    b = _run(moving, ng, x0 + np.concatenate([np.zeros(3), V]), days)
    b_helio = b - np.concatenate([V * days, V])
    assert np.abs(a[:3] - b_helio[:3]).max() < 1e-12
    assert np.abs(a[3:] - b_helio[3:]).max() < 1e-14
    free = _run(still, O.NonGrav(), x0, days)
    assert np.abs(a[:3] - free[:3]).max() > 1e-6        # the terms act
