"""GPU adjoint and sky partials with non-gravitational terms (App. A.4-A.5)
against the FP64 oracle, whose variational equations take the full force
model's Jacobian (position and velocity) by central differences.

The bodies of the adjoint workload get, in turn: radiation pressure with
Poynting-Robertson drag (beta ~ logU[1e-3, 0.05]); the comet model with the
asteroid g(r) = 1/r^2 and A1..A3 ~ N(0, 1e-8) AU/day^2, every other one with
a thermal lag of 10-30 days; the comet g(r) with A1 ~ logU[1e-9, 1e-7]; and
none.  Observed RA/Dec are the oracle's truth predictions with the body's
terms plus the workload's noise.  Tolerances as for gravity alone: relative
1e-6 on loss, gradient and each sky-partial row, 1 mas on the predictions."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-6
MAS = math.radians(1.0 / 3.6e6)
N = 64


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


def _ng_params(n, seed=2509046690):
    rng = np.random.default_rng(seed)
    ng = np.zeros(n, W.NONGRAV_DTYPE)
    for i in range(n):
        kind = i % 4
        if kind == 0:
            ng["beta"][i] = 10.0 ** rng.uniform(-3.0, math.log10(0.05))
        elif kind == 1:
            ng["alpha"][i], ng["r0"][i], ng["m"][i], ng["n"][i] = 1.0, 1.0, 2.0, 1.0
            for f in ("a1", "a2", "a3"):
                ng[f][i] = rng.normal(0.0, 1e-8)
            ng["dt"][i] = rng.uniform(10.0, 30.0) if (i // 4) % 2 == 0 else 0.0
        elif kind == 2:
            ng["alpha"][i], ng["r0"][i], ng["m"][i] = 0.1112620426, 2.808, 2.15
            ng["n"][i], ng["k"][i] = 5.093, 4.6142
            ng["a1"][i] = 10.0 ** rng.uniform(-9.0, -7.0)
            ng["a2"][i] = rng.normal(0.0, 1e-9)
            ng["dt"][i] = rng.uniform(10.0, 30.0)
    return ng


def _fm_o(orc, rec):
    fm = orc.force_model()
    fm.ng = O.NonGrav(*[float(rec[f]) for f in O.NG_FIELDS])
    return fm


@pytest.fixture(scope="module")
def prob():
    from conftest import cached_workload
    w = cached_workload("adjoint90", n_bodies=256, n_obs=20, neo_frac=0.1)
    orc = O.Oracle(w.ephem.to_bytes())
    ng = _ng_params(N)
    obs = w.meta["obs"][:N].copy()
    y = (w.states + w.meta["offsets"])[:, :N]
    loss, g, pred = np.zeros(N), np.zeros((6, N)), np.zeros((N, obs.shape[1], 2))
    for i in range(N):
        fm = _fm_o(orc, ng[i])
        rc, _, p, _ = orc.body_loss(fm, w.states[:, i], W.T0, obs[i], grad=False)
        assert rc == 0
        obs["ra"][i] = p[:, 0] + w.meta["noise"][i, :, 0] / np.cos(p[:, 1])
        obs["dec"][i] = p[:, 1] + w.meta["noise"][i, :, 1]
        rc, loss[i], pred[i], g[:, i] = orc.body_loss(fm, y[:, i], W.T0, obs[i])
        assert rc == 0
    return w, ng, obs, y, loss, g, pred


def _adjoint(K, w, ng, y, obs, with_ng=True, **kw):
    from paper_2509_04666_gb300 import kete
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model(nongrav=kete.nongrav_to_device(ng, "cuda")) if with_ng else None
    loss, g, pred, status = K.adjoint(_dev(y), _dev(np.full(y.shape[1], W.T0)), _obs_dev(obs),
                                      fm=fm, pred=True, **kw)
    return (loss.cpu().numpy(), None if g is None else g.cpu().numpy(), pred.cpu().numpy(),
            status.cpu().numpy())


def _assert_rows_close(g, ref, rel=REL):
    for i in range(g.shape[1]):
        for sl in (slice(0, 3), slice(3, 6)):
            scale = np.abs(ref[sl, i]).max()
            assert np.abs(g[sl, i] - ref[sl, i]).max() <= rel * scale, (i, g[:, i], ref[:, i])


def test_adjoint_with_nongrav_matches_oracle(K, prob):
    w, ng, obs, y, loss_r, g_r, pred_r = prob
    loss, g, pred, status = _adjoint(K, w, ng, y, obs)
    assert (status == 0).all()
    dra = (pred[..., 0] - pred_r[..., 0] + math.pi) % (2 * math.pi) - math.pi
    sky = np.hypot(dra * np.cos(pred_r[..., 1]), pred[..., 1] - pred_r[..., 1])
    assert sky.max() < MAS, sky.max()
    assert (np.abs(loss - loss_r) <= REL * loss_r).all()
    _assert_rows_close(g, g_r)
    # the terms act: without them the dust grains' gradients change by far more
    # than the tolerance
    _, g0, _, _ = _adjoint(K, w, ng, y, obs, with_ng=False)
    dust = np.nonzero(ng["beta"] > 0.01)[0]
    assert dust.size >= 4
    off = np.abs(g0[:3, dust] - g_r[:3, dust]).max(axis=0) / np.abs(g_r[:3, dust]).max(axis=0)
    assert (off > 1e-3).all(), off


def test_adjoint_with_nongrav_matches_finite_differences(K, prob):
    """Central differences of the GPU's own loss with the terms."""
    w, ng, obs, y, *_ = prob
    _, g, _, status = _adjoint(K, w, ng, y, obs)
    assert (status == 0).all()
    fd = np.zeros_like(g)
    for c in range(6):
        h = 1e-7 if c < 3 else 1e-9
        yp, ym = y.copy(), y.copy()
        yp[c] += h
        ym[c] -= h
        lp, *_ = _adjoint(K, w, ng, yp, obs, grad=False)
        lm, *_ = _adjoint(K, w, ng, ym, obs, grad=False)
        fd[c] = (lp - lm) / (2 * h)
    _assert_rows_close(g, fd)


def test_sky_jacobian_with_nongrav_matches_oracle(K, prob):
    from paper_2509_04666_gb300 import kete
    w, ng, obs, y, *_ = prob
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model(nongrav=kete.nongrav_to_device(ng, "cuda"))
    jac, _, status = K.sky_jacobian(_dev(y), _dev(np.full(N, W.T0)), _obs_dev(obs), fm=fm)
    jac, status = jac.cpu().numpy(), status.cpu().numpy()
    assert (status == 0).all()
    orc = O.Oracle(w.ephem.to_bytes())
    for i in range(0, N, 3):
        rc, jr, _ = orc.sky_jacobian(_fm_o(orc, ng[i]), y[:, i], W.T0, obs[i])
        assert rc == 0
        for a in range(2):
            for part in (slice(0, 3), slice(3, 6)):
                ref = jr[:, a, part]
                err = np.abs(jac[i, :, a, part] - ref).max()
                assert err < REL * np.abs(ref).max(), (i, a, part, err, np.abs(ref).max())
