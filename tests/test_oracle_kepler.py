"""Pins of the oracle's two-body (universal-variable) propagation (Sec. 2).

Independent references: mpmath's Stumpff functions at 40 digits, the
elliptic/hyperbolic anomaly solution of Kepler's equation (a different
formulation from the universal variable), and round trips."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300.workloads import GM_SUN, elements_to_state

pytestmark = pytest.mark.filterwarnings("ignore")


def test_stumpff_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for z in [-50.0, -3.0, -1.0, -0.999, -0.2, -0.1, -1e-6, 0.0, 1e-8, 0.05, 0.1, 0.5,
              0.999, 1.0, 2.0, 9.0, 35.0]:
        c2, c3 = O.stumpff(z)
        if z == 0:
            e2, e3 = mp.mpf(1) / 2, mp.mpf(1) / 6
        elif z > 0:
            s = mp.sqrt(z)
            e2, e3 = (1 - mp.cos(s)) / z, (s - mp.sin(s)) / s ** 3
        else:
            s = mp.sqrt(-z)
            e2, e3 = (mp.cosh(s) - 1) / (-z), (mp.sinh(s) - s) / s ** 3
        assert abs(c2 - float(e2)) <= 1e-15 * abs(float(e2)) + 1e-300, z
        assert abs(c3 - float(e3)) <= 1e-15 * abs(float(e3)) + 1e-300, z


def _hyperbolic_state(a, e, inc, node, peri, M, mu):
    """Hyperbolic elements (a<0) -> state via e sinh H - H = M (test-local)."""
    H = math.asinh(M / e)
    for _ in range(100):
        dH = (e * math.sinh(H) - H - M) / (e * math.cosh(H) - 1)
        H -= dH
        if abs(dH) < 1e-16:
            break
    r = a * (1 - e * math.cosh(H))
    xp = a * (math.cosh(H) - e)
    yp = -a * math.sqrt(e * e - 1) * math.sinh(H)
    vf = math.sqrt(-mu * a) / r
    vxp = -vf * math.sinh(H)
    vyp = vf * math.sqrt(e * e - 1) * math.cosh(H)
    cO, sO, ci, si, cw, sw = (math.cos(node), math.sin(node), math.cos(inc), math.sin(inc),
                              math.cos(peri), math.sin(peri))
    P = np.array([cO * cw - sO * sw * ci, sO * cw + cO * sw * ci, sw * si])
    Q = np.array([-cO * sw - sO * cw * ci, -sO * sw + cO * cw * ci, cw * si])
    return P * xp + Q * yp, P * vxp + Q * vyp


@pytest.mark.parametrize("a,e", [(2.7, 0.1), (1.2, 0.6), (30.0, 0.99), (5.2, 0.0),
                                 (0.4, 0.2)])
@pytest.mark.parametrize("dt", [0.013, -1.5, 1.5, 40.0, -400.0])
def test_kepler_elliptic_closed_form(a, e, dt):
    rng = np.random.default_rng(7)
    inc, node, peri, M0 = rng.uniform(0, 1), rng.uniform(0, 6), rng.uniform(0, 6), rng.uniform(0, 6)
    n = math.sqrt(GM_SUN / a ** 3)
    r0, v0 = elements_to_state(np.array([a]), np.array([e]), inc, node, peri, M0, GM_SUN)
    r1, v1 = elements_to_state(np.array([a]), np.array([e]), inc, node, peri, M0 + n * dt, GM_SUN)
    rc, r, v = O.kepler(GM_SUN, r0[:, 0], v0[:, 0], dt)
    assert rc == 0
    scale = max(1.0, a)
    assert np.abs(r - r1[:, 0]).max() < 2e-13 * scale * max(1.0, abs(dt) / 100)
    assert np.abs(v - v1[:, 0]).max() < 2e-14 * max(1.0, abs(dt) / 100) / math.sqrt(scale) + 1e-16


@pytest.mark.parametrize("e", [1.2, 3.0])
def test_kepler_hyperbolic_closed_form(e):
    a = -1.5
    n = math.sqrt(GM_SUN / (-a) ** 3)
    M0, dt = 0.3, 60.0
    r0, v0 = _hyperbolic_state(a, e, 0.4, 1.1, 2.0, M0, GM_SUN)
    r1, v1 = _hyperbolic_state(a, e, 0.4, 1.1, 2.0, M0 + n * dt, GM_SUN)
    rc, r, v = O.kepler(GM_SUN, r0, v0, dt)
    assert rc == 0
    assert np.abs(r - r1).max() < 1e-12
    assert np.abs(v - v1).max() < 1e-14


def test_kepler_round_trip():
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, e = rng.uniform(0.8, 40), rng.uniform(0, 0.98)
        r0, v0 = elements_to_state(np.array([a]), np.array([e]), rng.uniform(0, 3),
                                   rng.uniform(0, 6), rng.uniform(0, 6), rng.uniform(0, 6), GM_SUN)
        dt = rng.uniform(-5, 5)
        _, r, v = O.kepler(GM_SUN, r0[:, 0], v0[:, 0], dt)
        _, rb, vb = O.kepler(GM_SUN, r, v, -dt)
        assert np.abs(rb - r0[:, 0]).max() < 1e-13 * max(1, a)


def test_kepler_zero_dt_identity():
    r0 = np.array([1.0, 2.0, 0.1]); v0 = np.array([0.001, -0.01, 0.0])
    rc, r, v = O.kepler(GM_SUN, r0, v0, 0.0)
    assert rc == 0 and np.array_equal(r, r0) and np.array_equal(v, v0)
