"""Pins of the oracle's light-delay correction (Sec. 2), spherical-polygon FoV
test (Sec. 3.1), RA/Dec projection (App. A.1) and batching rule (Sec. 2)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C_AU_D = 299792.458 * 86400.0 / 149597870.7


# ---- light time ----------------------------------------------------------
def _near_massless_oracle():
    # a Sun of negligible mass: two-body motion is a straight line
    return O.Oracle(W.static_sun_table(W.T0 - 40, W.T0 + 40, gm_scale=1e-20).to_bytes())


@pytest.mark.parametrize("seed", range(5))
def test_light_time_uniform_motion_closed_form(seed):
    orc = _near_massless_oracle()
    rng = np.random.default_rng(seed)
    r0 = rng.normal(0, 3, 3)
    v = rng.normal(0, 0.02, 3)
    o = rng.normal(0, 1, 3)
    t_ref, t_obs = W.T0, W.T0 + rng.uniform(-1.5, 1.5)
    rc, u, tau = orc.apparent(np.concatenate([r0, v]), t_ref, t_obs, o)
    assert rc == 0
    d = r0 + v * (t_obs - t_ref) - o
    # |d - v tau| = c tau  ->  (c^2 - v^2) tau^2 + 2 (d.v) tau - |d|^2 = 0
    A = C_AU_D ** 2 - v @ v
    B = 2 * (d @ v)
    tau_ref = (-B + math.sqrt(B * B + 4 * A * (d @ d))) / (2 * A)
    assert abs(tau - tau_ref) < 1e-15
    np.testing.assert_allclose(u, d - v * tau_ref, atol=2e-14)


def test_light_time_stationary_body():
    orc = _near_massless_oracle()
    r0 = np.array([2.0, -1.0, 0.5]); o = np.array([0.3, 0.9, -0.1])
    rc, u, tau = orc.apparent(np.concatenate([r0, np.zeros(3)]), W.T0, W.T0 + 1.0, o)
    assert rc == 0
    assert abs(tau - np.linalg.norm(r0 - o) / C_AU_D) < 1e-17
    np.testing.assert_allclose(u, r0 - o, atol=1e-14)


def test_light_time_is_self_consistent(mb1k):
    orc = O.Oracle(mb1k.ephem.to_bytes())
    for i in range(0, 1000, 111):
        st = mb1k.states[:, i]
        rc, u, tau = orc.apparent(st, W.T0, W.T0 + 1.2, mb1k.observers[0])
        assert rc == 0
        assert abs(np.linalg.norm(u) / C_AU_D - tau) < 1e-15 * tau + 1e-18


# ---- FoV geometry --------------------------------------------------------
def _frame_from_case(lon, lat, h, psi):
    lon, lat, h, psi = map(math.radians, (lon, lat, h, psi))
    p = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.cross(p, east)
    e = math.cos(psi) * east + math.sin(psi) * north
    n = np.cross(p, e)
    fr = np.zeros(1, W.FRAME_DTYPE)
    fr["n_edges"] = 4
    fr["normals"][0] = W.square_normals(p[None], e[None], h)[0]
    return fr[0], p, e, n, h


def test_fov_golden_cases():
    rows = [l.split() for l in open(os.path.join(GOLD, "fov_cases.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for r in rows:
        lon, lat, h, psi, xi, eta, exp = map(float, r)
        fr, p, e, n, hr = _frame_from_case(lon, lat, h, psi)
        u = p + xi * math.tan(hr) * e + eta * math.tan(hr) * n
        u = 2.7 * u / np.linalg.norm(u)
        inside, margin = O.in_polygon(fr, u)
        assert inside == bool(exp), r


def test_fov_matches_gnomonic_test():
    rng = np.random.default_rng(11)
    n_checked = 0
    for _ in range(200):
        lon, lat = rng.uniform(0, 360), math.degrees(math.asin(rng.uniform(-1, 1)))
        fr, p, e, n, h = _frame_from_case(lon, lat, rng.uniform(0.1, 5), rng.uniform(0, 180))
        for _ in range(20):
            xi, eta = rng.uniform(-1.6, 1.6, 2) * math.tan(h)
            u = p + xi * e + eta * n
            u *= rng.uniform(0.1, 30) / np.linalg.norm(u)
            inside, margin = O.in_polygon(fr, u)
            x, y = (u @ e) / (u @ p), (u @ n) / (u @ p)
            g = abs(x) < math.tan(h) and abs(y) < math.tan(h)
            if min(abs(abs(x) - math.tan(h)), abs(abs(y) - math.tan(h))) > 1e-12:
                assert inside == g
                n_checked += 1
        # the antipode is never inside
        assert not O.in_polygon(fr, -p)[0]
    assert n_checked > 3000


def test_fov_boundary_is_outside():
    fr = np.zeros(1, W.FRAME_DTYPE)[0]
    fr["n_edges"] = 4
    fr["normals"] = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]
    assert O.in_polygon(fr, np.array([1.0, 1.0, 1.0]))[0]
    assert not O.in_polygon(fr, np.array([0.0, 1.0, 1.0]))[0]      # on n_0's plane
    inside, margin = O.in_polygon(fr, np.array([0.0, 1.0, 1.0]))
    assert margin == 0.0


def _cone(c, rho):
    fr = np.zeros(1, W.FRAME_DTYPE)[0]
    fr["n_edges"] = 0
    fr["normals"][0] = c
    fr["normals"][1][0] = rho
    return fr


def test_cone_matches_angular_distance():
    """Cone FoVs (Sec. 3.1): inside iff the angle to the centre, taken here
    as atan2(|c x u|, c.u), is below the radius."""
    rng = np.random.default_rng(12)
    n_checked = 0
    for _ in range(200):
        c = rng.normal(size=3) * rng.uniform(0.1, 10)
        rho = rng.uniform(0.001, 1.5)
        fr = _cone(c, rho)
        for _ in range(20):
            # directions spread around the boundary
            u = c / np.linalg.norm(c) + rng.normal(size=3) * rng.uniform(0.0, 2.0 * rho)
            u *= rng.uniform(0.1, 30) / np.linalg.norm(u)
            ang = math.atan2(np.linalg.norm(np.cross(c, u)), c @ u)
            inside, margin = O.in_polygon(fr, u)
            assert abs(margin - (rho - ang)) < 1e-7
            if abs(ang - rho) > 1e-12:
                assert inside == (ang < rho)
                n_checked += 1
        assert not O.in_polygon(fr, -c)[0] and O.in_polygon(fr, c)[0]
    assert n_checked > 3000
    # a hemisphere: the boundary (c.u = 0) is outside
    assert not O.in_polygon(_cone([0, 0, 1.0], math.pi / 2), np.array([1.0, 0, 0]))[0]
    assert O.in_polygon(_cone([0, 0, 1.0], math.pi / 2), np.array([1.0, 0, 1e-9]))[0]


def test_cone_frames_prefilter_equals_brute_force(mb1k_dense):
    w = mb1k_dense
    fr = W.cone_frames(w.frames, slice(0, None, 2), math.radians(0.6))
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    brute, _, _ = orc.fov_check(fm, w.states, w.epochs, fr, w.observers)
    fast, _, _ = orc.fov_check(fm, w.states, w.epochs, fr, w.observers, prefilter_deg=0.5)
    cones = fr["n_edges"][brute["frame"]] == 0
    assert cones.sum() > 50 and (~cones).sum() > 50
    np.testing.assert_array_equal(brute[["frame", "body"]], fast[["frame", "body"]])


def test_radec_known_directions():
    eps = math.radians(84381.448 / 3600)
    ra, dec = O.radec(np.array([2.0, 0, 0]))
    assert ra == 0.0 and dec == 0.0
    ra, dec = O.radec(np.array([0, 0, 1.0]))                 # ecliptic north pole
    assert abs(ra - 1.5 * math.pi) < 1e-15 and abs(dec - (math.pi / 2 - eps)) < 1e-15
    ra, dec = O.radec(np.array([0, math.sin(eps), math.cos(eps)]))   # celestial pole
    assert abs(dec - math.pi / 2) < 1e-15
    ra, dec = O.radec(np.array([0, 1.0, 0]))                 # ecliptic y axis
    assert abs(ra - math.pi / 2) < 1e-15 and abs(dec - eps) < 1e-15
    ra, dec = O.radec(np.array([-1.0, -1e-30, 0]))
    assert 0 <= ra < 2 * math.pi


# ---- batching ------------------------------------------------------------
def test_batches_greedy_three_day_rule():
    rng = np.random.default_rng(5)
    ep = np.sort(W.T0 + rng.uniform(0, 40, 500))
    bs, tr = O.make_batches(ep, 3.0, 1.5)
    ends = list(bs[1:]) + [len(ep)]
    for k, (s, e) in enumerate(zip(bs, ends)):
        seg = ep[s:e]
        assert seg[-1] - seg[0] < 3.0
        assert tr[k] == 0.5 * (seg[0] + seg[-1])
        assert np.abs(seg - tr[k]).max() <= 1.5
        if e < len(ep):
            assert ep[e] - seg[0] >= 3.0          # greedy: the next epoch does not fit
    assert bs[0] == 0 and np.all(np.diff(bs) > 0)
    # an epoch exactly one span after the batch start opens the next batch
    # (R6: t - t_first < span, strict); equal epochs always share a batch
    ep = W.T0 + np.array([0.0, 1.0, 3.0, 3.0, 5.5, 6.0, 6.0])
    bs, tr = O.make_batches(ep, 3.0, 1.5)
    assert list(bs) == [0, 2, 5]
    np.testing.assert_array_equal(tr, [W.T0 + 0.5, W.T0 + 4.25, W.T0 + 6.0])


def test_batches_zero_twobody_interval_is_per_epoch():
    ep = np.array([1.0, 1.0, 1.5, 2.0, 2.0, 2.0, 7.0]) + W.T0
    bs, tr = O.make_batches(ep, 3.0, 0.0)
    assert list(bs) == [0, 2, 3, 6]
    np.testing.assert_array_equal(tr, ep[[0, 2, 3, 6]])
    bs, tr = O.make_batches(ep, 3.0, 0.2)        # span shrinks to 0.4 days
    assert list(bs) == [0, 2, 3, 6]


# ---- survey driver --------------------------------------------------------
def test_prefilter_equals_brute_force(mb1k_dense):
    w = mb1k_dense
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    brute, st1, _ = orc.fov_check(fm, w.states, w.epochs, w.frames, w.observers)
    fast, st2, _ = orc.fov_check(fm, w.states, w.epochs, w.frames, w.observers,
                                 prefilter_deg=0.5)
    assert len(brute) > 100
    np.testing.assert_array_equal(brute[["frame", "body"]], fast[["frame", "body"]])
    np.testing.assert_array_equal(brute["ra"], fast["ra"])


def test_twobody_batches_approximate_pure_nbody(mb1k_dense):
    """Interval 0 (n-body to every FoV epoch) vs the <= 1.5 d two-body interval:
    the hit lists differ only next to an edge; the approximation error is small."""
    w = mb1k_dense
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    a, _, _ = orc.fov_check(fm, w.states, w.epochs, w.frames, w.observers)
    b, _, _ = orc.fov_check(fm, w.states, w.epochs, w.frames, w.observers, twobody_max=0.0)
    ka = {(int(x["frame"]), int(x["body"])): x for x in a}
    kb = {(int(x["frame"]), int(x["body"])): x for x in b}
    for k in set(ka) ^ set(kb):
        x = ka.get(k, kb.get(k))
        assert abs(x["margin"]) < 1e-6
    common = set(ka) & set(kb)
    assert len(common) > 100
    err = max(math.hypot((ka[k]["ra"] - kb[k]["ra"]) * math.cos(ka[k]["dec"]),
                         ka[k]["dec"] - kb[k]["dec"]) for k in common)
    assert err < 5e-7     # < 0.1 arcsec for main-belt bodies over 1.5 days
