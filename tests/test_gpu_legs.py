"""kete_propagate_legs (a single-target propagation through stops every
leg_days days, so that the bodies share the planets' node rows) against the
oracle's chain of stops over the same grid: within 1e-9 AU after a year in
FP64 and in mixed precision (5e-9 AU for the forced Earth encounters in
mixed precision), forward and backward."""
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


def _grid(e0, t_target, leg):
    """The library's stops: e0 + k leg toward the target, which ends them."""
    span = t_target - e0
    k_legs = max(1, int(np.ceil(abs(span) / leg)))
    sgn = -1.0 if span < 0 else 1.0
    return np.array([e0 + sgn * leg * (k + 1) for k in range(k_legs - 1)] + [t_target])


@pytest.mark.parametrize("precision", [0, 1])
def test_legs_match_the_oracle_chain(K, precision):
    from conftest import cached_workload
    from paper_2509_04666_gb300 import kete
    w = cached_workload("ragged1y", n_bodies=2000)
    t1 = W.T0 + 365.0
    K.load_ephem(w.ephem.to_bytes())
    s, e = _dev(w.states.copy()), _dev(w.epochs.copy())
    status = K.propagate(s, e, t1, fm=kete.force_model(precision=precision), leg_days=8.0)
    assert (status.cpu().numpy() == 0).all() and (e.cpu().numpy() == t1).all()
    got = s.cpu().numpy()
    stops = _grid(W.T0, t1, 8.0)
    assert len(stops) == 46
    orc = O.Oracle(w.ephem.to_bytes())
    idx = list(np.nonzero(w.labels == 4)[0]) + list(range(0, w.n_bodies, 53))
    worst = {}
    for i in idx:
        rc, out, _ = orc.propagate_stops(orc.force_model(), w.states[:, i], W.T0, stops)
        assert rc == 0
        lab = int(w.labels[i])
        worst[lab] = max(worst.get(lab, 0.0), np.abs(got[:3, i] - out[-1, :3]).max())
    enc = worst.pop(4)
    assert max(worst.values()) < 1e-9, worst
    assert enc < (1e-9 if precision == 0 else 5e-9), enc


def test_legs_backward_single_leg_and_bad_arguments(K, mb1k):
    from paper_2509_04666_gb300 import kete
    w = mb1k
    K.load_ephem(w.ephem.to_bytes())
    orc = O.Oracle(w.ephem.to_bytes())
    t1 = W.T0 - 20.0
    s, e = _dev(w.states.copy()), _dev(w.epochs.copy())
    status = K.propagate(s, e, t1, leg_days=3.0)
    assert (status.cpu().numpy() == 0).all()
    got = s.cpu().numpy()
    stops = _grid(W.T0, t1, 3.0)
    assert len(stops) == 7 and stops[0] == W.T0 - 3.0
    for i in range(0, w.n_bodies, 97):
        rc, out, _ = orc.propagate_stops(orc.force_model(), w.states[:, i], W.T0, stops)
        assert rc == 0
        assert np.abs(got[:3, i] - out[-1, :3]).max() < 1e-9
    # one leg longer than the whole span: the same as kete_propagate
    s1, e1 = _dev(w.states.copy()), _dev(w.epochs.copy())
    s2, e2 = _dev(w.states.copy()), _dev(w.epochs.copy())
    K.propagate(s1, e1, W.T0 + 10.0, leg_days=50.0)
    K.propagate(s2, e2, W.T0 + 10.0)
    assert np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())
    for leg in (0.0, -1.0, float("nan")):
        with pytest.raises(kete.KeteError) as ei:
            K.propagate(_dev(w.states.copy()), _dev(w.epochs.copy()), t1, leg_days=leg)
        assert ei.value.code == kete.ERR_BAD_ARG
