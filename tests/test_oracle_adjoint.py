"""Pins of the oracle's orbit-fit gradient: the state-transition matrix from
the variational equations (symplectic for conservative forces; equal to
finite differences of the pinned two-body solution) and the gradient of the
loss (equal to central finite differences of the loss)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

OMEGA = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])


def test_stm_is_symplectic_without_gr(mb1k):
    orc = O.Oracle(mb1k.ephem.to_bytes())
    fm = orc.force_model(gr_mask=0)
    for i in (3, 400, 777):
        rc, st, phi, t, dt, _ = orc.propagate_stm(fm, mb1k.states[:, i], W.T0, W.T0 + 30.0)
        assert rc == 0
        assert np.abs(phi.T @ OMEGA @ phi - OMEGA).max() < 1e-7 * np.abs(phi).max() ** 2
        assert abs(np.linalg.det(phi) - 1.0) < 1e-7


def test_stm_matches_finite_differences_of_kepler():
    """Sun only: Phi equals central differences of the universal-variable
    two-body solution (pinned against the anomaly solution)."""
    orc = O.Oracle(W.static_sun_table(W.T0 - 10, W.T0 + 120).to_bytes())
    fm = orc.force_model(body_mask=1, gr_mask=0, j2_mask=0)
    r0, v0 = W.elements_to_state(np.array([1.4]), np.array([0.4]), 0.3, 1.0, 2.0, 0.7, W.GM_SUN)
    y0 = np.concatenate([r0[:, 0], v0[:, 0]])
    rc, st, phi, *_ = orc.propagate_stm(fm, y0, W.T0, W.T0 + 100.0)
    assert rc == 0
    fd = np.zeros((6, 6))
    for c in range(6):
        h = 1e-6 if c < 3 else 1e-8
        yp, ym = y0.copy(), y0.copy()
        yp[c] += h; ym[c] -= h
        _, rp, vp = O.kepler(W.GM_SUN, yp[:3], yp[3:], 100.0)
        _, rm, vm = O.kepler(W.GM_SUN, ym[:3], ym[3:], 100.0)
        fd[:, c] = (np.concatenate([rp, vp]) - np.concatenate([rm, vm])) / (2 * h)
    assert np.abs(phi - fd).max() < 1e-6 * np.abs(fd).max()


@pytest.fixture(scope="module")
def adj_small():
    from conftest import cached_workload
    return cached_workload("adjoint90", n_bodies=40, n_obs=20)


def _observations(orc, fm, w, i, truth_offset=True):
    """Observed RA/Dec = oracle prediction from the truth state + the noise draws."""
    obs = w.meta["obs"][i].copy()
    rc, loss, pred, _ = orc.body_loss(fm, w.states[:, i], W.T0, obs, grad=False)
    assert rc == 0
    obs["ra"] = pred[:, 0] + w.meta["noise"][i, :, 0] / np.cos(pred[:, 1])
    obs["dec"] = pred[:, 1] + w.meta["noise"][i, :, 1]
    return obs


def test_loss_vanishes_on_its_own_predictions(adj_small):
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = w.meta["obs"][0].copy()
    _, _, pred, _ = orc.body_loss(fm, w.states[:, 0], W.T0, obs, grad=False)
    obs["ra"], obs["dec"] = pred[:, 0], pred[:, 1]
    rc, loss, _, g = orc.body_loss(fm, w.states[:, 0], W.T0, obs)
    assert rc == 0 and loss == 0.0
    assert np.abs(g).max() == 0.0


@pytest.mark.parametrize("i", [0, 7, 19, 33])
def test_variational_gradient_matches_finite_differences(adj_small, i):
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = _observations(orc, fm, w, i)
    y = w.states[:, i] + w.meta["offsets"][:, i]
    rc, loss, _, g = orc.body_loss(fm, y, W.T0, obs)
    assert rc == 0 and loss > 0
    for hx, hv in ((1e-7, 1e-9), (1e-8, 1e-10)):
        fd = np.zeros(6)
        for c in range(6):
            h = hx if c < 3 else hv
            yp, ym = y.copy(), y.copy()
            yp[c] += h; ym[c] -= h
            _, lp, _, _ = orc.body_loss(fm, yp, W.T0, obs, grad=False)
            _, lm, _, _ = orc.body_loss(fm, ym, W.T0, obs, grad=False)
            fd[c] = (lp - lm) / (2 * h)
        scale = np.abs(g[:3]).max(), np.abs(g[3:]).max()
        assert np.abs(g[:3] - fd[:3]).max() < 1e-6 * scale[0], (g, fd)
        assert np.abs(g[3:] - fd[3:]).max() < 1e-6 * scale[1], (g, fd)


@pytest.mark.parametrize("i,k", [(13, 1), (5, 2), (21, 1)])
def test_gradient_of_few_observations_matches_finite_differences(adj_small, i, k):
    """Rows of one or two observations soon after the initial epoch, where the
    velocity part of the gradient rests on the observation partials alone."""
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = _observations(orc, fm, w, i)[:k]
    y = w.states[:, i] + w.meta["offsets"][:, i]
    rc, loss, _, g = orc.body_loss(fm, y, W.T0, obs)
    assert rc == 0 and loss > 0
    def cd(c, h):
        yp, ym = y.copy(), y.copy()
        yp[c] += h; ym[c] -= h
        return (orc.body_loss(fm, yp, W.T0, obs, grad=False)[1]
                - orc.body_loss(fm, ym, W.T0, obs, grad=False)[1]) / (2 * h)
    # Richardson-extrapolated central differences (error O(h^4)), steps large
    # enough that the rounding of the loss stays below 1e-9 of the gradient
    fd = np.zeros(6)
    for c in range(6):
        h = 1e-6 if c < 3 else 1e-7
        fd[c] = (4.0 * cd(c, h / 2) - cd(c, h)) / 3.0
    assert np.abs(g[:3] - fd[:3]).max() < 1e-7 * np.abs(g[:3]).max(), (g, fd)
    assert np.abs(g[3:] - fd[3:]).max() < 1e-7 * np.abs(g[3:]).max(), (g, fd)


@pytest.mark.parametrize("i", [0, 19, 33])
def test_sky_jacobian_matches_finite_differences_of_the_predictions(adj_small, i):
    """The per-observation sky partials (rows of the orbit-fit Jacobian) equal
    central differences of the whole forward model's RA/Dec predictions --
    n-body chain, two-body, light time -- with respect to the initial state,
    Richardson-extrapolated (error O(h^4))."""
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = w.meta["obs"][i].copy()
    y = w.states[:, i] + w.meta["offsets"][:, i]
    rc, jac, pred = orc.sky_jacobian(fm, y, W.T0, obs)
    assert rc == 0 and jac.shape == (len(obs), 2, 6)
    _, _, pred_loss, _ = orc.body_loss(fm, y, W.T0, obs, grad=False)
    assert np.array_equal(pred, pred_loss)

    def cd(c, h):
        yp, ym = y.copy(), y.copy()
        yp[c] += h; ym[c] -= h
        _, _, pp, _ = orc.body_loss(fm, yp, W.T0, obs, grad=False)
        _, _, pm, _ = orc.body_loss(fm, ym, W.T0, obs, grad=False)
        d = pp - pm
        d[:, 0] = (d[:, 0] + math.pi) % (2 * math.pi) - math.pi
        return d / (2 * h)
    fd = np.zeros_like(jac)
    for c in range(6):
        h = 1e-6 if c < 3 else 1e-8
        fd[:, :, c] = (4.0 * cd(c, h / 2) - cd(c, h)) / 3.0
    for part in (slice(0, 3), slice(3, 6)):
        scale = np.abs(fd[:, :, part]).max()
        assert np.abs(jac[:, :, part] - fd[:, :, part]).max() < 1e-6 * scale


def test_sky_jacobian_gives_the_loss_gradient(adj_small):
    """Chain rule: dL/dy0 = sum_j 2 (wrap(RA_j - RA_obs) cos^2 Dec_obs dRA_j/dy0
    + (Dec_j - Dec_obs) dDec_j/dy0) equals the loss gradient."""
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = _observations(orc, fm, w, 7)
    y = w.states[:, 7] + w.meta["offsets"][:, 7]
    rc, _, _, g = orc.body_loss(fm, y, W.T0, obs)
    rc2, jac, pred = orc.sky_jacobian(fm, y, W.T0, obs)
    assert rc == rc2 == 0
    cd2 = np.cos(obs["dec"]) ** 2
    dra = (pred[:, 0] - obs["ra"] + math.pi) % (2 * math.pi) - math.pi
    g2 = (2 * (dra * cd2)[:, None] * jac[:, 0, :] + 2 * (pred[:, 1] - obs["dec"])[:, None] * jac[:, 1, :]).sum(0)
    assert np.abs(g2 - g).max() < 1e-9 * np.abs(g).max()


@pytest.mark.parametrize("kind", ["dust", "lagged", "comet"])
def test_variational_gradient_with_nongrav_matches_finite_differences(adj_small, kind):
    """With non-gravitational terms the variational equations take the full
    model's da/dx and da/dv (radiation pressure with drag; the comet model,
    its thermal lag through the two-body map): the gradient still equals
    central differences of the loss."""
    w = adj_small
    orc = O.Oracle(w.ephem.to_bytes())
    ng = {"dust": O.dust_ng(0.03),
          "lagged": O.asteroid_ng(2e-8, -1e-8, 5e-9, dt=20.0),
          "comet": O.comet_ng(5e-8, 1e-8, -2e-9, dt=15.0)}[kind]
    fm = orc.force_model(ng=ng)
    i = {"dust": 3, "lagged": 11, "comet": 27}[kind]
    obs = _observations(orc, fm, w, i)
    y = w.states[:, i] + w.meta["offsets"][:, i]
    rc, loss, _, g = orc.body_loss(fm, y, W.T0, obs)
    assert rc == 0 and loss > 0
    fd = np.zeros(6)
    for c in range(6):
        h = 1e-7 if c < 3 else 1e-9
        yp, ym = y.copy(), y.copy()
        yp[c] += h; ym[c] -= h
        _, lp, _, _ = orc.body_loss(fm, yp, W.T0, obs, grad=False)
        _, lm, _, _ = orc.body_loss(fm, ym, W.T0, obs, grad=False)
        fd[c] = (lp - lm) / (2 * h)
    assert np.abs(g[:3] - fd[:3]).max() < 1e-6 * np.abs(g[:3]).max(), (g, fd)
    assert np.abs(g[3:] - fd[3:]).max() < 1e-6 * np.abs(g[3:]).max(), (g, fd)
    # the terms change the gradient by far more than that
    rc, _, _, g0 = orc.body_loss(orc.force_model(), y, W.T0, obs)
    assert np.abs(g0 - g).max() > 1e-4 * np.abs(g).max()
