"""Long spans and backward steps on the GPU against the FP64 oracle: a body
population carried back 50 years (the pre-discovery use) and Monte-Carlo
clones of a Jupiter-family comet with non-gravitational terms carried back
170 years (the orbital-evolution use).

Over decades two correct FP64 integrations drift apart as the dynamics
amplifies their different rounding; the tolerance of each body is therefore
1,000 times the oracle's own response to a one-ulp change of the body's
initial x (measured per body), and never below 1e-9 AU.  A wrong force term
or a wrong step rule moves a body by many orders of magnitude more.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _ng_o(rec):
    return O.NonGrav(*[float(rec[f]) for f in O.NG_FIELDS])


def _tolerances(orc, w, idx, ng=None):
    """(oracle state at t_end, tolerance) per body of idx."""
    refs, tols = [], []
    for i in idx:
        fm = orc.force_model()
        if ng is not None:
            fm.ng = _ng_o(ng[i])
        x0 = w.states[:, i]
        rc, a, *_ = orc.propagate(fm, x0, W.T0, w.t_end)
        assert rc == 0
        x1 = x0.copy()
        x1[0] *= 1.0 + 2.0 ** -52
        rc, b, *_ = orc.propagate(fm, x1, W.T0, w.t_end)
        assert rc == 0
        refs.append(a)
        tols.append(max(1e-9, 1e3 * np.abs(a[:3] - b[:3]).max()))
    return np.array(refs), np.array(tols)


def _gpu(K, w, ng=None, precision=0):
    from paper_2509_04666_gb300 import kete
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model(precision=precision)
    keep = None
    if ng is not None:
        keep = kete.nongrav_to_device(ng, "cuda")
        fm.nongrav = keep.data_ptr()
    s = _dev(w.states.copy()); e = _dev(w.epochs.copy())
    status = K.propagate(s, e, w.t_end, fm=fm)
    assert (e.cpu().numpy() == w.t_end).all()
    return s.cpu().numpy(), status.cpu().numpy()


def test_population_fifty_years_back(K):
    from conftest import cached_workload
    w = cached_workload("backward_catalogue", n_bodies=2000, years=50.0)
    got, status = _gpu(K, w)
    assert (status == 0).all()
    idx = np.unique(np.concatenate([np.arange(0, w.n_bodies, 50),
                                    np.nonzero(w.labels == 1)[0][::2]]))
    orc = O.Oracle(w.ephem.to_bytes())
    ref, tol = _tolerances(orc, w, idx)
    err = np.abs(got[:3, idx].T - ref[:, :3]).max(axis=1)
    assert (err < tol).all(), [(int(i), e, t) for i, e, t in zip(idx, err, tol) if e >= tol][:5]
    assert (w.labels[idx] == 1).sum() >= 10


@pytest.mark.parametrize("split", [0, 8])
def test_comet_clones_170_years_back(K, split):
    """256 clones with the JPL comet model; split 8: after 4 step attempts
    per stop every clone finishes with 8 lanes (the few-long-bodies case)."""
    from conftest import cached_workload
    from paper_2509_04666_gb300 import kete
    w = cached_workload("clones", n_clones=256, years=170.0)
    ng = w.meta["nongrav"]
    K.set_propagation(kete.FP64, kete.PROP_WORK_STEALING, 128, split, 4 if split else 0)
    try:
        got, status = _gpu(K, w, ng)
        deferred = K.get_stats()["deferred"]
    finally:
        K.set_propagation(kete.FP64, kete.PROP_WORK_STEALING, 128)
    assert (status == 0).all()
    if split:
        assert deferred > 200
    idx = np.arange(0, 256, 16)
    orc = O.Oracle(w.ephem.to_bytes())
    ref, tol = _tolerances(orc, w, idx, ng)
    err = np.abs(got[:3, idx].T - ref[:, :3]).max(axis=1)
    assert (err < tol).all(), list(zip(err, tol))
    # the cloud has spread far beyond any of these differences
    spread = got[:3].std(axis=1).min()
    assert spread > 1e-4 and err.max() < 1e-4 * spread
