"""The seeded synthetic inputs follow their stated recipes: population
elements, the WISE-like scan, the ZTF-like night-time exposures from a
rotating site, the ragged population's counts, and seed determinism."""
import math

import numpy as np
import pytest

from paper_2509_04666_gb300 import workloads as W

DEG = math.pi / 180.0


def _helio_elements(ps, states):
    r = states[:3] - ps.pos0[0][:, None]
    v = states[3:] - ps.vel0[0][:, None]
    return W.state_to_elements(r, v, W.GM_SUN)


def test_population_elements_follow_the_recipe():
    seed = W.SEED_BASE + 1
    ps = W.make_planets(seed)
    st, lab = W.population(seed, ps, 2000, 500, 300, 300)
    assert st.shape == (6, 3100)
    assert list(np.bincount(lab)) == [2000, 500, 300, 300]
    a, e, inc, node, peri, M = _helio_elements(ps, st)
    mb, neo, tro, com = (lab == k for k in range(4))
    assert a[mb].min() >= 2.1 - 1e-9 and a[mb].max() <= 3.3 + 1e-9
    assert e[mb].max() < 0.3 and abs(np.median(inc[mb]) / DEG - 8 * math.sqrt(2 * math.log(2))) < 1.0
    assert a[neo].min() >= 0.8 - 1e-9 and a[neo].max() <= 2.0 + 1e-9 and e[neo].max() <= 0.7
    assert np.allclose(a[tro], 5.2, atol=1e-9)
    jp = ps.pos0[5] - ps.pos0[0]
    lam = (node + peri + M)[tro]
    dl = (lam - math.atan2(jp[1], jp[0]) + math.pi) % (2 * math.pi) - math.pi
    assert (np.abs(np.abs(dl) - 60 * DEG) <= 10 * DEG + 1e-9).all()
    q = a[com] * (1 - e[com])
    assert e[com].min() >= 0.7 - 1e-9 and e[com].max() <= 0.99 + 1e-9
    assert q.min() >= 0.5 - 1e-9 and q.max() <= 3.0 + 1e-9


def test_wise_like_scan():
    ps = W.make_planets(W.SEED_BASE + 1)
    n = 3288 * 2 + 50
    fr, obs, centre, h = W.wise_frames(ps, n)
    ep = fr["epoch"]
    assert len(fr) == n and np.all(np.diff(ep) >= 0)
    # one block of 3,288 frames a day, 11 s apart, from 0.1 d
    assert np.allclose(ep[:3288] - W.T0 - 0.1, np.arange(3288) * 11.0 / 86400.0, atol=1e-9)
    assert math.isclose(ep[3288] - W.T0, 1.1, abs_tol=1e-9)
    # squares of 0.78 deg: every inward normal leans 0.39 deg into the centre
    m = fr["normals"] / np.linalg.norm(fr["normals"], axis=-1, keepdims=True)
    ang = np.arcsin(np.einsum("fkc,fc->fk", m, centre))
    assert np.allclose(ang, 0.39 * DEG, atol=1e-12) and math.isclose(h, 0.39 * DEG)
    # observer on a 1-AU circle around the Sun; pointing at 90 deg elongation
    sun = W.integrate_planets(ps, ep[::500])[:, 0, :3]
    r = obs[::500] - sun
    assert np.allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-6)
    assert np.abs(np.einsum("fc,fc->f", centre[::500], r)).max() < 1e-6
    # 0.7 deg between consecutive pointings
    step = np.arccos(np.clip(np.einsum("fc,fc->f", centre[1:100], centre[:99]), -1, 1))
    assert np.allclose(step, 0.7 * DEG, atol=2e-5)


def test_ztf_like_exposures():
    seed = W.SEED_BASE + 2
    ps = W.make_planets(seed)
    fr, obs, sub_c, h = W.ztf_frames(ps, 300, days=30, seed_rng=W._rng(seed, 3))
    assert len(fr) == 300 * 64 and math.isclose(h, 0.435 * DEG)
    ex = fr["exposure_id"]
    assert np.array_equal(ex, np.repeat(np.arange(300), 64))
    ep = fr["epoch"][::64]
    assert np.all(np.diff(ep) >= 0) and np.all(fr["epoch"] == np.repeat(ep, 64))
    # night at the site: the Sun below -12 deg
    st = W.integrate_planets(ps, ep)
    sdir = W.ecl_to_eq(st[:, 0, :3] - st[:, 3, :3])
    sdir /= np.linalg.norm(sdir, axis=1, keepdims=True)
    zen = W._site_zenith_eq(ep)
    assert ((zen * sdir).sum(1) < math.sin(-12 * DEG)).all()
    # exposure centres: Dec >= -30 deg and altitude > 30 deg
    cen = W.ecl_to_eq(sub_c.reshape(300, 64, 3).mean(axis=1))
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    assert (np.arcsin(cen[:, 2]) >= -30 * DEG - 1e-3).all()
    assert ((cen * zen).sum(1) > math.sin(30 * DEG) - 1e-3).all()
    # the observer is the site: 6,378 km from the Earth
    assert np.allclose(np.linalg.norm(obs - st[:, 3, :3], axis=1), W.EARTH_RADIUS_AU, rtol=1e-9)


def test_ragged_population_counts():
    from conftest import cached_workload
    w = cached_workload("ragged1y", n_bodies=2000)
    assert list(np.bincount(w.labels)) == [1200, 380, 200, 200, 20]
    assert ((w.meta["t_enc"] > 30) & (w.meta["t_enc"] < 335)).all()
    assert ((w.meta["miss"] >= 0.001) & (w.meta["miss"] <= 0.01)).all()
    assert (w.epochs == W.T0).all() and w.t_end == W.T0 + 365.0


def test_inputs_are_seeded():
    a = W.population(7, W.make_planets(7), 50, 10)[0]
    b = W.population(7, W.make_planets(7), 50, 10)[0]
    c = W.population(8, W.make_planets(8), 50, 10)[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    m1, m2 = W.mag_params(np.zeros(100)), W.mag_params(np.zeros(100))
    n1, n2 = W.nongrav_params(np.full(100, 3)), W.nongrav_params(np.full(100, 3))
    assert np.array_equal(m1, m2) and np.array_equal(n1, n2)


@pytest.mark.parametrize("labels", [np.array([3, 0, 0, 3, 1, 2, 0, 0, 0, 0, 0, 0])])
def test_nongrav_and_magnitude_recipes(labels):
    ng = W.nongrav_params(labels, dust_frac=1.0, yarkovsky_every=3)
    com = labels == 3
    assert (ng["alpha"][com] == 0.1112620426).all() and (ng["k"][com] == 4.6142).all()
    assert ((ng["a1"][com] >= 1e-9) & (ng["a1"][com] <= 1e-7)).all()
    rest = np.nonzero(~com)[0]
    yk = rest[::3]
    assert (ng["m"][yk] == 2.0).all() and (ng["k"][yk] == 0.0).all()
    others = np.setdiff1d(rest, yk)
    assert ((ng["beta"][others] >= 1e-3) & (ng["beta"][others] <= 0.1)).all()
    mp = W.mag_params(labels)
    assert mp["kind"][0] == 0                       # every 50th body has none
    assert set(mp["kind"][com][1:].tolist()) <= {2, 3}
    assert ((mp["p1"][~com][1:] >= 10) & (mp["p1"][~com][1:] <= 20)).all()
