"""Non-gravitational terms on the GPU (App. A.4: radiation pressure with
Poynting-Robertson drag; App. A.5: the JPL comet model with thermal lag)
against the FP64 oracle.

Workload: the mixed population of the ragged year (2,000 bodies) with
per-body terms from workloads.nongrav_params: comets with the comet g(r)
(half of them lagged 5-40 days), a transverse drift on every tenth asteroid,
radiation pressure on 5 % of the rest.  Tolerances as for gravity alone:
1e-9 AU after 365 days in FP64 (5e-9 AU for the forced Earth encounters in
mixed precision), 1 mas on the sky.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAS = math.radians(1.0 / 3.6e6)
EDGE = 1e-9


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


@pytest.fixture(scope="module")
def pop():
    from conftest import cached_workload
    w = cached_workload("ragged1y", n_bodies=2000)
    return w, W.nongrav_params(w.labels, dust_frac=0.05)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _ng_o(rec):
    return O.NonGrav(*[float(rec[f]) for f in O.NG_FIELDS])


def _gpu_propagate(K, w, ng, precision=0, days=365.0):
    from paper_2509_04666_gb300 import kete
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model(precision=precision,
                          nongrav=None if ng is None else kete.nongrav_to_device(ng, "cuda"))
    s = _dev(w.states.copy()); e = _dev(w.epochs.copy())
    status = K.propagate(s, e, W.T0 + days, fm=fm)
    return s.cpu().numpy(), status.cpu().numpy()


def _sample(w, ng):
    kinds = {"comet": np.nonzero(w.labels == 3)[0][::4],
             "lagged": np.nonzero((w.labels == 3) & (ng["dt"] != 0))[0][::4],
             "drift": np.nonzero(ng["a2"] != 0)[0][::6],
             "dust": np.nonzero(ng["beta"] != 0)[0][::2],
             "encounter": np.nonzero(w.labels == 4)[0],
             "plain": np.arange(0, w.n_bodies, 53)}
    return kinds


@pytest.mark.parametrize("precision", [0, 1])
def test_propagation_with_nongrav_matches_oracle(K, pop, precision):
    w, ng = pop
    got, status = _gpu_propagate(K, w, ng, precision)
    assert (status == 0).all()
    orc = O.Oracle(w.ephem.to_bytes())
    worst = {}
    for kind, idx in _sample(w, ng).items():
        assert len(idx) >= 3, kind
        for i in idx:
            fm = orc.force_model()
            fm.ng = _ng_o(ng[i])
            rc, ref, *_ = orc.propagate(fm, w.states[:, i], W.T0, W.T0 + 365.0)
            assert rc == 0
            worst[kind] = max(worst.get(kind, 0.0), np.abs(got[:3, i] - ref[:3]).max())
    enc = worst.pop("encounter")
    assert max(worst.values()) < 1e-9, worst
    assert enc < (1e-9 if precision == 0 else 5e-9), enc


def test_nongrav_terms_act_and_zero_terms_change_nothing(K, pop):
    w, ng = pop
    plain, _ = _gpu_propagate(K, w, None)
    withng, _ = _gpu_propagate(K, w, ng)
    zero, _ = _gpu_propagate(K, w, np.zeros_like(ng))
    # all-zero records: bit for bit the gravity-only result
    assert np.array_equal(zero, plain)
    # a terms tensor whose rows do not match the bodies is refused
    from paper_2509_04666_gb300 import kete
    fm = kete.force_model(nongrav=kete.nongrav_to_device(ng[:10], "cuda"))
    with pytest.raises(TypeError):
        K.propagate(_dev(w.states.copy()), _dev(w.epochs.copy()), W.T0 + 1.0, fm=fm)
    moved = np.abs(withng[:3] - plain[:3]).max(axis=0)
    # comets: g(r) falls as r^-(m + n k) ~ r^-26 beyond r0 = 2.8 AU, so only the
    # comets that come in close during the year move by much
    com = moved[w.labels == 3]
    assert com.max() > 1e-5 and (com > 1e-6).sum() >= 10, np.sort(com)[-12:]
    assert (moved[ng["beta"] > 0] > 1e-5).all()                  # dust: a weaker Sun
    untouched = (ng["a1"] == 0) & (ng["a2"] == 0) & (ng["a3"] == 0) & (ng["beta"] == 0)
    assert (moved[untouched] == 0).all()


def test_stops_and_noalloc_with_nongrav(K, pop):
    """The chain of stops and the no-allocation entry point read the terms too."""
    from paper_2509_04666_gb300 import kete
    w, ng = pop
    idx = np.nonzero((w.labels == 3) | (ng["beta"] != 0))[0][:64]
    sub = w.states[:, idx]
    K.load_ephem(w.ephem.to_bytes())
    keep = kete.nongrav_to_device(ng[idx], "cuda")
    fm = kete.force_model()
    fm.nongrav = keep.data_ptr()
    stops = np.array([W.T0 + 30.0, W.T0 + 90.0, W.T0 + 200.0])
    out, status = K.propagate_stops(_dev(sub), _dev(w.epochs[idx]), stops, fm=fm)
    out = out.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    orc = O.Oracle(w.ephem.to_bytes())
    for j, i in enumerate(idx[::4]):
        fmo = orc.force_model()
        fmo.ng = _ng_o(ng[i])
        rc, ref, _ = orc.propagate_stops(fmo, w.states[:, i], W.T0, stops)
        assert rc == 0
        assert np.abs(out[:, :3, 4 * j] - ref[:, :3]).max() < 1e-9
    s1 = _dev(sub); e1 = _dev(w.epochs[idx])
    s2 = _dev(sub); e2 = _dev(w.epochs[idx])
    K.propagate(s1, e1, W.T0 + 200.0, fm=fm)
    K.propagate_noalloc(s2, e2, W.T0 + 200.0, fm=fm)
    # the no-allocation entry point runs another launch variant (static, no
    # node rows): equal to the integrator's truncation level, not bit for bit
    a, b = s1.cpu().numpy(), s2.cpu().numpy()
    assert np.abs(a[:3] - b[:3]).max() < 1e-9 and np.abs(a[3:] - b[3:]).max() < 1e-11


def test_fov_check_with_nongrav_matches_oracle(K, mb1k_dense):
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    lab = np.asarray(w.labels).copy()
    lab[::3] = 3                               # comet laws on a third of the bodies
    ng = W.nongrav_params(lab, dust_frac=0.1, yarkovsky_every=4)
    K.load_ephem(w.ephem.to_bytes())
    keep = kete.nongrav_to_device(ng, "cuda")
    fm = kete.force_model()
    fm.nongrav = keep.data_ptr()
    hits, nh, status = K.fov_check(_dev(w.states), _dev(w.epochs),
                                   kete.frames_to_device(w.frames, "cuda"), _dev(w.observers), fm=fm)
    got = kete.decode_hits(hits, nh)
    assert (status.cpu().numpy() == 0).all()
    orc = O.Oracle(w.ephem.to_bytes())
    ref, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, w.frames, w.observers,
                              nongrav=ng)
    plain, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, w.frames, w.observers)
    assert len(ref) > 100
    g = {(int(f), int(b)): (ra, de) for f, b, ra, de in
         zip(got["frame"].tolist(), got["body"].tolist(), got["ra"].tolist(), got["dec"].tolist())}
    r = {(int(h["frame"]), int(h["body"])): h for h in ref}
    bad = [k for k in set(g) ^ set(r) if k not in r or abs(r[k]["margin"]) >= EDGE]
    assert not bad, bad[:5]
    worst = 0.0
    for key in set(g) & set(r):
        ra, de = g[key]
        dra = (ra - r[key]["ra"] + math.pi) % (2 * math.pi) - math.pi
        worst = max(worst, math.hypot(dra * math.cos(de), de - r[key]["dec"]))
    assert worst < MAS, worst
    # the terms matter here: the gravity-only sky positions differ by far more
    p = {(int(h["frame"]), int(h["body"])): h for h in plain}
    shift = max(math.hypot(((r[k]["ra"] - p[k]["ra"] + math.pi) % (2 * math.pi) - math.pi)
                           * math.cos(r[k]["dec"]), r[k]["dec"] - p[k]["dec"])
                for k in set(r) & set(p))
    assert shift > 100 * MAS
