"""The rest of the FoV family on the GPU against the FP64 oracle (Sec. 3.1):
cone FoVs, and extended exposures approximated by instantaneous sub-frames
whose hits are merged per exposure.  Tolerances as for polygons: membership
identical outside a 1e-9 rad band around the boundary, sky positions within
1 mas."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _gpu_hits(K, w, frames, observers):
    from paper_2509_04666_gb300 import kete
    K.load_ephem(w.ephem.to_bytes())
    hits, nh, status = K.fov_check(_dev(w.states), _dev(w.epochs),
                                   kete.frames_to_device(frames, "cuda"), _dev(observers))
    assert (status.cpu().numpy() == 0).all()
    return {k: v.numpy() for k, v in kete.decode_hits(hits, nh).items()}


def _compare(got, ref):
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


def test_cone_fovs_match_oracle(K, mb1k_dense):
    w = mb1k_dense
    fr = W.cone_frames(w.frames, slice(0, None, 3), math.radians(0.6))
    got = _gpu_hits(K, w, fr, w.observers)
    orc = O.Oracle(w.ephem.to_bytes())
    ref, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, fr, w.observers)
    cones = fr["n_edges"][ref["frame"]] == 0
    assert cones.sum() > 50 and (~cones).sum() > 50
    _compare(got, ref)
    # a wide cone (beyond the binning's 1.4 rad) covers its whole hemisphere
    wide = W.cone_frames(w.frames, slice(0, 5), 1.5)
    got = _gpu_hits(K, w, wide, w.observers)
    ref, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, wide, w.observers)
    _compare(got, ref)
    assert (ref["frame"] < 5).sum() > 100


def test_bad_cone_radius_is_refused(K, mb1k_dense):
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    for rho in (0.0, math.pi, float("nan")):
        fr = W.cone_frames(w.frames, [7], rho)
        with pytest.raises(kete.KeteError) as e:
            _gpu_hits(K, w, fr, w.observers)
        assert e.value.code == kete.ERR_BAD_ARG


def test_streak_exposures_match_oracle(K, mb1k_dense):
    """60 one-hour exposures (half of them cones) as 6 sub-frames each, the
    observer (the Earth of the table) moving along; the merged hits agree."""
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    orc = O.Oracle(w.ephem.to_bytes())
    base = W.cone_frames(w.frames, slice(0, None, 2), math.radians(0.5))
    # the 60 frames with the most bodies in them at their own epoch
    plain, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, base, w.observers)
    pick = np.argsort(-np.bincount(plain["frame"], minlength=len(base)), kind="stable")[:60]
    sub, obs, parent = [], [], []
    for j, f in enumerate(pick):
        t0 = float(w.frames["epoch"][f]) - 1.0 / 48
        rows = np.arange(len(obs), len(obs) + 6)
        s = kete.streak_frames(base[f], t0, t0 + 1.0 / 24, rows, 6 * j)
        for t in s["epoch"]:
            rc, p, _ = orc.ephem(3, float(t))
            assert rc == 0
            obs.append(p)
        sub.append(s)
        parent += [j] * 6
    fr = np.concatenate(sub)
    order = np.argsort(fr["epoch"], kind="stable")
    fr = fr[order]
    fr["exposure_id"] = np.arange(len(fr))
    parent = np.asarray(parent)[order]
    obs = np.asarray(obs)
    got = _gpu_hits(K, w, fr, obs)
    ref, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, fr, obs)
    assert len(ref) > 100
    _compare(got, ref)
    mg = kete.merge_streak_hits(got, parent)
    mr = kete.merge_streak_hits({"frame": ref["frame"], "body": ref["body"],
                                 "margin": ref["margin"]}, parent)
    kg = set(zip(mg["exposure"].tolist(), mg["body"].tolist()))
    kr = set(zip(mr["exposure"].tolist(), mr["body"].tolist()))
    # a body seen in some sub-frame on one side only sits at a boundary there
    near = {(int(parent[h["frame"]]), int(h["body"])) for h in ref if abs(h["margin"]) < EDGE}
    assert not ((kg ^ kr) - near)
    assert len(kr) > 60
