"""Pins of the oracle's apparent magnitudes (Sec. 3.3: asteroid V by the H-G
system; appendix: comet total and nucleus magnitudes): the viewing geometry
against a stationary body seen across a massless Sun, and the magnitude laws
against their special cases (zero phase, a right-angle phase, the log-log
slope of each phase function, distance and phase slopes of the comet laws)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

LN10 = math.log(10.0)


def _orc():
    # a Sun of negligible mass at rest at the origin: bodies stand still
    return O.Oracle(W.static_sun_table(W.T0 - 40, W.T0 + 40, gm_scale=1e-20).to_bytes())


def _body(r):
    return np.concatenate([np.asarray(r, float), np.zeros(3)])


def test_geometry_of_a_stationary_body():
    orc = _orc()
    rng = np.random.default_rng(3)
    for _ in range(5):
        r0 = rng.normal(0, 2, 3); o = rng.normal(0, 1, 3)
        rc, m, rh, dl, al = orc.magnitude(_body(r0), W.T0, W.T0 + 0.7, o, 1, 15.0, 0.15)
        assert rc == 0
        assert abs(rh - np.linalg.norm(r0)) < 1e-14
        assert abs(dl - np.linalg.norm(r0 - o)) < 1e-14
        # angle at the body between the Sun (origin) and the observer
        a = -r0; b = o - r0
        ref = math.degrees(math.atan2(np.linalg.norm(np.cross(a, b)), a @ b))
        assert abs(al - ref) < 1e-9


def test_hg_at_zero_phase_is_the_distance_law():
    orc = _orc()
    # Sun, observer and body on one line, observer between: phase angle 0
    for H, G in ((15.0, 0.15), (8.2, -0.1), (21.0, 0.6)):
        rc, m, rh, dl, al = orc.magnitude(_body([3.0, 0, 0]), W.T0, W.T0, [1.0, 0, 0], 1, H, G)
        assert rc == 0 and al < 1e-6
        assert abs(m - (H + 5 * math.log10(3.0 * 2.0))) < 1e-12


@pytest.mark.parametrize("G,A", [(0.0, 3.33), (1.0, 1.87)])
def test_hg_at_right_angle_phase(G, A):
    """At 90 deg phase tan(alpha/2) = 1, so the phase term is A_i 2.5/ln 10."""
    orc = _orc()
    r0 = np.array([0.0, 2.0, 0.0]); o = np.array([0.0, 2.0, 1.5])   # Sun-body-observer 90 deg
    rc, m, rh, dl, al = orc.magnitude(_body(r0), W.T0, W.T0, o, 1, 12.0, G)
    assert rc == 0 and abs(al - 90.0) < 1e-9
    assert abs(m - (12.0 + 5 * math.log10(2.0 * 1.5) + 2.5 * A / LN10)) < 1e-12


@pytest.mark.parametrize("G,B", [(0.0, 0.63), (1.0, 1.22)])
def test_hg_phase_function_exponents(G, B):
    """ln(-ln Phi) is linear in ln tan(alpha/2) with slope B_i."""
    orc = _orc()
    vals = []
    for deg in (20.0, 70.0):
        a = math.radians(deg)
        r0 = np.array([2.0, 0.0, 0.0])
        o = r0 + 1.3 * np.array([-math.cos(a), math.sin(a), 0.0])
        rc, m, rh, dl, al = orc.magnitude(_body(r0), W.T0, W.T0, o, 1, 10.0, G)
        assert rc == 0 and abs(al - deg) < 1e-9
        phase_term = m - (10.0 + 5 * math.log10(rh * dl))        # = -2.5 log10 Phi
        vals.append((math.log(math.tan(a / 2)), math.log(phase_term * LN10 / 2.5)))
    slope = (vals[1][1] - vals[0][1]) / (vals[1][0] - vals[0][0])
    assert abs(slope - B) < 1e-9


def test_comet_magnitudes():
    orc = _orc()
    M, K = 9.0, 12.5
    # r_h = 10 AU, delta = 1 AU, zero phase: T = M + K, N = M + K
    rc, t1, rh, dl, al = orc.magnitude(_body([10.0, 0, 0]), W.T0, W.T0, [9.0, 0, 0], 2, M, K)
    rc2, n1, *_ = orc.magnitude(_body([10.0, 0, 0]), W.T0, W.T0, [9.0, 0, 0], 3, M, K)
    assert rc == rc2 == 0 and abs(t1 - (M + K)) < 1e-12 and abs(n1 - (M + K)) < 1e-9
    # nucleus: 0.035 mag per degree of phase beyond the distance terms
    r0 = np.array([0.0, 2.0, 0.0]); o = np.array([0.0, 2.0, 1.5])
    rc, n90, rh, dl, al = orc.magnitude(_body(r0), W.T0, W.T0, o, 3, M, K)
    rc, t90, *_ = orc.magnitude(_body(r0), W.T0, W.T0, o, 2, M, K)
    assert abs((n90 - t90) - 0.035 * 90.0) < 1e-9
    assert abs(t90 - (M + 5 * math.log10(1.5) + K * math.log10(2.0))) < 1e-12


def test_no_model_gives_nan():
    rc, m, *_ = _orc().magnitude(_body([2.0, 0, 0]), W.T0, W.T0, [1.0, 0, 0], 0, 0.0, 0.0)
    assert rc == 0 and math.isnan(m)
