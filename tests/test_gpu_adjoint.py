"""GPU adjoint (kete_adjoint) against the FP64 oracle's variational-equation
gradient and against central finite differences of the GPU's own loss.

Tolerances: gradient within a relative 1e-6 of the reference (position and
velocity parts each against their own largest component); loss within a
relative 1e-6; predicted RA/Dec within 1 mas of the oracle's.  Observed
RA/Dec are the oracle's truth predictions plus the workload's N(0, 0.1")
noise draws; the gradient is taken at truth + the workload's offsets.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-6
MAS = math.radians(1.0 / 3.6e6)


@pytest.fixture(scope="module")
def K():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_04666_gb300 import build as B, kete
    B.build()
    k = kete.Kete(0)
    yield k
    k.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _obs_dev(obs):
    n, m = obs.shape
    return _dev(np.ascontiguousarray(obs).view(np.float64).reshape(n, m, 6))


def _oracle_observations(orc, fm, w, obs, idx=None, **kw):
    """Observed RA/Dec = oracle prediction at the truth state + noise."""
    obs = obs.copy()
    idx = range(obs.shape[0]) if idx is None else idx
    for i in idx:
        k = int(np.isfinite(obs["epoch"][i]).sum())
        if k == 0:
            continue
        rc, _, pred, _ = orc.body_loss(fm, w.states[:, i], W.T0, obs[i, :k], grad=False, **kw)
        assert rc == 0
        obs["ra"][i, :k] = pred[:, 0] + w.meta["noise"][i, :k, 0] / np.cos(pred[:, 1])
        obs["dec"][i, :k] = pred[:, 1] + w.meta["noise"][i, :k, 1]
    return obs


def _oracle_refs(orc, fm, y, obs, grad=True, **kw):
    n = obs.shape[0]
    loss, g, pred, rcs = np.zeros(n), np.zeros((6, n)), np.full(obs.shape + (2,), np.nan), []
    for i in range(n):
        k = int(np.isfinite(obs["epoch"][i]).sum())
        if k == 0:
            rcs.append(0)
            continue
        rc, L, p, gi = orc.body_loss(fm, y[:, i], W.T0, obs[i, :k], grad=grad, **kw)
        rcs.append(rc)
        loss[i] = L
        pred[i, :k] = p
        if grad:
            g[:, i] = gi
    return np.array(rcs), loss, g, pred


def _gpu(K, w, y, obs, **kw):
    K.load_ephem(w.ephem.to_bytes())
    loss, g, pred, status = K.adjoint(_dev(y), _dev(np.full(y.shape[1], W.T0)), _obs_dev(obs),
                                      pred=True, **kw)
    return (loss.cpu().numpy(), None if g is None else g.cpu().numpy(), pred.cpu().numpy(),
            status.cpu().numpy())


def _assert_grad_close(g, ref, rel=REL, mask=None):
    n = g.shape[1]
    for i in range(n):
        if mask is not None and not mask[i]:
            continue
        for sl in (slice(0, 3), slice(3, 6)):
            scale = np.abs(ref[sl, i]).max()
            err = np.abs(g[sl, i] - ref[sl, i]).max()
            assert err <= rel * scale, (i, g[:, i], ref[:, i])


@pytest.fixture(scope="module")
def adj():
    from conftest import cached_workload
    w = cached_workload("adjoint90", n_bodies=256, n_obs=20, neo_frac=0.1)
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    obs = _oracle_observations(orc, fm, w, w.meta["obs"])
    y = w.states + w.meta["offsets"]
    rcs, loss, g, pred = _oracle_refs(orc, fm, y, obs)
    assert (rcs == 0).all()
    return w, obs, y, loss, g, pred


def test_adjoint_matches_oracle_variational_gradient(K, adj):
    w, obs, y, loss_r, g_r, pred_r = adj
    loss, g, pred, status = _gpu(K, w, y, obs)
    assert (status == 0).all()
    dra = (pred[..., 0] - pred_r[..., 0] + math.pi) % (2 * math.pi) - math.pi
    sky = np.hypot(dra * np.cos(pred_r[..., 1]), pred[..., 1] - pred_r[..., 1])
    assert sky.max() < MAS, sky.max()
    assert (loss > 0).all()
    assert np.abs(loss - loss_r).max() <= REL * loss_r.max()
    assert (np.abs(loss - loss_r) <= REL * loss_r).all()
    _assert_grad_close(g, g_r)
    # the NEOs of the sample (label 1) are covered too
    assert (w.labels == 1).sum() >= 10


def test_adjoint_gradient_matches_finite_differences(K, adj):
    """Central differences of the GPU loss itself, every body at once."""
    w, obs, y, *_ = adj
    loss, g, _, status = _gpu(K, w, y, obs)
    assert (status == 0).all()
    for hx, hv in ((1e-7, 1e-9), (1e-8, 1e-10)):
        fd = np.zeros_like(g)
        for c in range(6):
            h = hx if c < 3 else hv
            yp, ym = y.copy(), y.copy()
            yp[c] += h
            ym[c] -= h
            lp, *_ = _gpu(K, w, yp, obs, grad=False)
            lm, *_ = _gpu(K, w, ym, obs, grad=False)
            fd[c] = (lp - lm) / (2 * h)
        _assert_grad_close(g, fd)


def test_autograd_function_returns_the_adjoint_gradient(K, adj):
    import torch
    from paper_2509_04666_gb300 import kete
    w, obs, y, *_ = adj
    n = y.shape[1]
    K.load_ephem(w.ephem.to_bytes())
    ep, ob = _dev(np.full(n, W.T0)), _obs_dev(obs)
    _, g, _, _ = K.adjoint(_dev(y), ep, ob)
    states = _dev(y).requires_grad_(True)
    loss, status = kete.orbit_fit_loss(K, states, ep, ob)
    assert loss.requires_grad and (status == 0).all()
    wts = torch.linspace(0.5, 2.0, n, dtype=torch.float64, device="cuda")
    (loss * wts).sum().backward()
    assert torch.equal(states.grad, g * wts.unsqueeze(0))


def test_loss_only_equals_loss_with_gradient(K, adj):
    w, obs, y, *_ = adj
    l1, g1, p1, s1 = _gpu(K, w, y, obs)
    l0, g0, p0, s0 = _gpu(K, w, y, obs, grad=False)
    assert g0 is None
    assert np.array_equal(l0, l1) and np.array_equal(p0, p1, equal_nan=True)
    assert np.array_equal(s0, s1)


def test_ragged_rows_and_single_observations(K, adj):
    """NaN epochs pad a row: the body uses the observations before them;
    a body without observations has loss 0 and gradient 0."""
    w, obs, y, *_ = adj
    n = 48
    obs = obs[:n].copy()
    keep = np.array([0, 1, 2, 5, 19, 20] * 8)
    for i in range(n):
        obs["epoch"][i, keep[i]:] = np.nan
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    rcs, loss_r, g_r, pred_r = _oracle_refs(orc, fm, y[:, :n], obs)
    assert (rcs == 0).all()
    loss, g, pred, status = _gpu(K, w, y[:, :n], obs)
    assert (status == 0).all()
    none = keep == 0
    assert (loss[none] == 0).all() and (g[:, none] == 0).all()
    assert np.isnan(pred[none]).all()
    assert np.isnan(pred[1, 1:]).all() and np.isfinite(pred[1, 0]).all()
    assert (np.abs(loss - loss_r) <= REL * loss_r).all()
    _assert_grad_close(g, g_r, mask=~none)


def test_observations_around_the_initial_epoch(K, adj):
    """Batches before the initial epoch (the chain runs backward first), one
    batch whose midpoint is the initial epoch itself, and no checkpoint grid."""
    w, obs, y, *_ = adj
    n = 24
    obs = w.meta["obs"][:n].copy()
    rng = np.random.default_rng(7)
    m = obs.shape[1]
    for i in range(n):
        if i % 3 == 0:   # a batch of its own centred on T0: the rest 4 days before
            u = rng.uniform(-12.0, 14.0, m - 2)      # or 2 days after
            u = np.where(u >= -4.0, u + 6.0, u)
            e = np.concatenate([W.T0 + u, [W.T0 - 1.0, W.T0 + 1.0]])
        else:
            e = W.T0 + rng.uniform(-12.0, 20.0, m)
        obs["epoch"][i] = np.sort(e)
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    for ck in (8.0, 0.0):
        ob = _oracle_observations(orc, fm, w, obs, ckpt_days=ck)
        rcs, loss_r, g_r, _ = _oracle_refs(orc, fm, y[:, :n], ob, ckpt_days=ck)
        assert (rcs == 0).all()
        loss, g, _, status = _gpu(K, w, y[:, :n], ob, ckpt_days=ck)
        assert (status == 0).all()
        assert (np.abs(loss - loss_r) <= REL * loss_r).all()
        _assert_grad_close(g, g_r)


def test_step_record_capacity_keeps_the_loss(K, adj):
    """A body needing more steps than the record holds (a checkpoint every 6
    hours: 360 stops in 90 days) keeps its loss and predictions and reports
    KETE_BODY_ADJ_CAP with a NaN gradient."""
    from paper_2509_04666_gb300 import kete
    w, obs, y, *_ = adj
    n = 8
    orc = O.Oracle(w.ephem.to_bytes())
    rcs, loss_r, _, pred_r = _oracle_refs(orc, orc.force_model(), y[:, :n], obs[:n], grad=False,
                                          ckpt_days=0.25)
    assert (rcs == 0).all()
    loss, g, pred, status = _gpu(K, w, y[:, :n], obs[:n], ckpt_days=0.25)
    assert (status == kete.BODY_ADJ_CAP).all()
    assert np.isnan(g).all()
    assert (np.abs(loss - loss_r) <= REL * loss_r).all()
    assert np.isfinite(pred).all()


def test_epoch_outside_table_and_bad_arguments(K, adj):
    from paper_2509_04666_gb300 import kete
    w, obs, y, *_ = adj
    n = 16
    ob = obs[:n].copy()
    ob["epoch"][3, -1] = W.T0 + 400.0        # beyond the table: that body alone fails
    loss, g, _, status = _gpu(K, w, y[:, :n], ob)
    assert status[3] == kete.BODY_OUT_OF_SPAN and np.isnan(loss[3]) and np.isnan(g[:, 3]).all()
    others = np.arange(n) != 3
    assert (status[others] == 0).all() and np.isfinite(loss[others]).all()
    bad = obs[:n].copy()
    bad["epoch"][5, [2, 3]] = bad["epoch"][5, [3, 2]]
    with pytest.raises(kete.KeteError) as e:
        _gpu(K, w, y[:, :n], bad)
    assert e.value.code == kete.ERR_BAD_ARG
    wide = np.zeros((n, kete.ADJ_MAX_OBS + 1), W.OBS_DTYPE)
    wide["epoch"] = W.T0 + np.arange(kete.ADJ_MAX_OBS + 1)
    with pytest.raises(kete.KeteError) as e:
        _gpu(K, w, y[:, :n], wide)
    assert e.value.code == kete.ERR_BAD_ARG
    loss, g, pred, status = _gpu(K, w, y[:, :0], obs[:0])
    assert loss.shape == (0,) and g.shape == (6, 0)
