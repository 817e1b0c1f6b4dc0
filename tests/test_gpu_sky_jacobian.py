"""GPU per-observation sky partials (kete_sky_jacobian): the rows of the
orbit-fit Jacobian d(RA_j, Dec_j)/d(x0, v0), against the FP64 oracle's rows
(state-transition matrix from the variational equations chained with
central-difference observation partials; pinned against finite differences
of the oracle's whole forward model) and against the GPU's own adjoint
gradient by the chain rule.

Tolerances: each row within a relative 1e-6 of the oracle's (position and
velocity parts each against their own largest component, per body and row
kind), the chain-rule gradient within 1e-8 of the adjoint's."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import cached_workload
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-6


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


@pytest.fixture(scope="module")
def adj():
    return cached_workload("adjoint90", n_bodies=256, n_obs=20)


def test_sky_jacobian_matches_oracle(K, adj):
    w = adj
    y = w.states + w.meta["offsets"]
    obs = w.meta["obs"].copy()
    obs["epoch"][5, 12:] = np.nan            # a ragged row: 12 observations
    K.load_ephem(w.ephem.to_bytes())
    jac, pred, status = K.sky_jacobian(_dev(y), _dev(np.full(w.n_bodies, W.T0)), _obs_dev(obs),
                                       pred=True)
    jac, pred, status = jac.cpu().numpy(), pred.cpu().numpy(), status.cpu().numpy()
    assert (status == 0).all()
    assert np.isnan(jac[5, 12:]).all() and np.isfinite(jac[5, :12]).all()
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    for i in list(range(0, w.n_bodies, 16)) + [5]:
        k = int(np.isfinite(obs["epoch"][i]).sum())
        rc, jr, pr = orc.sky_jacobian(fm, y[:, i], W.T0, obs[i, :k])
        assert rc == 0
        assert np.abs(pred[i, :k] - pr).max() < 1e-12
        for a in range(2):
            for part in (slice(0, 3), slice(3, 6)):
                ref = jr[:, a, part]
                err = np.abs(jac[i, :k, a, part] - ref).max()
                assert err < REL * np.abs(ref).max(), (i, a, part, err, np.abs(ref).max())


def test_sky_jacobian_chain_rule_gives_the_adjoint_gradient(K, adj):
    """dL/dy0 = sum_j 2 (wrap(RA_j - RA_obs) cos^2 Dec_obs dRA_j/dy0
    + (Dec_j - Dec_obs) dDec_j/dy0): the forward state-transition pass and the
    backward adjoint pass give the same gradient."""
    w = adj
    y = w.states + w.meta["offsets"]
    obs = w.meta["obs"].copy()
    # observed = prediction at the truth + noise (any data will do here)
    K.load_ephem(w.ephem.to_bytes())
    ep = _dev(np.full(w.n_bodies, W.T0))
    _, _, p0, _ = K.adjoint(_dev(w.states), ep, _obs_dev(obs), grad=False, pred=True)
    p0 = p0.cpu().numpy()
    obs["ra"] = p0[..., 0] + w.meta["noise"][..., 0] / np.cos(p0[..., 1])
    obs["dec"] = p0[..., 1] + w.meta["noise"][..., 1]
    loss, g, pred, st1 = K.adjoint(_dev(y), ep, _obs_dev(obs), pred=True)
    jac, pred2, st2 = K.sky_jacobian(_dev(y), ep, _obs_dev(obs), pred=True)
    g, pred, jac, pred2 = (t.cpu().numpy() for t in (g, pred, jac, pred2))
    assert (st1.cpu().numpy() == 0).all() and (st2.cpu().numpy() == 0).all()
    assert np.array_equal(pred, pred2)
    cd2 = np.cos(obs["dec"]) ** 2
    dra = (pred[..., 0] - obs["ra"] + math.pi) % (2 * math.pi) - math.pi
    g2 = (2 * (dra * cd2)[..., None] * jac[:, :, 0, :]
          + 2 * (pred[..., 1] - obs["dec"])[..., None] * jac[:, :, 1, :]).sum(1).T
    for part in (slice(0, 3), slice(3, 6)):
        scale = np.abs(g[part]).max(axis=0)
        assert (np.abs(g2[part] - g[part]).max(axis=0) < 1e-8 * scale).all()
