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


def _subframes(frames, durations, n_sub):
    """The sub-frames kete_fov_check_extended defines (test-local, from its
    header): sub-frame k of frame f at epoch + ((k + 0.5) d) / n_sub from
    observer row observer_idx + k, sub-interval k of an exposure forming one
    exposure, exposures in order; returns them and each one's parent frame."""
    start = np.ones(len(frames), bool)
    start[1:] = frames["exposure_id"][1:] != frames["exposure_id"][:-1]
    first = np.nonzero(start)[0]
    bounds = list(first) + [len(frames)]
    subs, parent = [], []
    for f0, f1 in zip(bounds[:-1], bounds[1:]):
        for k in range(n_sub):
            for f in range(f0, f1):
                x = frames[f].copy()
                x["epoch"] = frames["epoch"][f] + ((k + 0.5) * durations[f]) / n_sub
                x["observer_idx"] = frames["observer_idx"][f] + k
                x["exposure_id"] = f0 * n_sub + k
                subs.append(x)
                parent.append(f)
    return np.array(subs, dtype=frames.dtype), np.array(parent)


def _union(ref, parent):
    """Per (frame, body): the hit of the earliest sub-frame."""
    out = {}
    for h in ref:
        key = (int(parent[h["frame"]]), int(h["body"]))
        if key not in out or h["frame"] < out[key]["frame"]:
            out[key] = h
    return out


@pytest.mark.parametrize("n_sub", [1, 6])
def test_extended_exposures_match_oracle(K, mb1k_dense, n_sub):
    """60 one-hour exposures (half of them cones, one of them a union of two
    patches) through kete_fov_check_extended, the observer (the Earth of the
    table) at every sub-epoch; one hit per (frame, body) with the earliest
    sub-frame's position, identical to the union of the oracle's sub-frame
    hits outside the edge band."""
    import torch
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    orc = O.Oracle(w.ephem.to_bytes())
    base = W.cone_frames(w.frames, slice(0, None, 2), math.radians(0.5))
    plain, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, base, w.observers)
    # the 60 frames with the most bodies whose hour-long exposures do not overlap
    pick = []
    for f in np.argsort(-np.bincount(plain["frame"], minlength=len(base)), kind="stable"):
        if all(abs(base["epoch"][f] - base["epoch"][g]) > 1.5 / 24 for g in pick):
            pick.append(f)
        if len(pick) == 60:
            break
    fr = base[np.sort(pick)].copy()
    fr["epoch"] -= 1.0 / 48
    fr["exposure_id"] = np.arange(len(fr))
    fr[1]["epoch"] = fr[0]["epoch"]          # frames 0 and 1: one exposure of two patches
    fr[1]["exposure_id"] = 0
    dur = np.full(len(fr), 1.0 / 24)
    # n_sub observer rows per exposure: the Earth at each sub-epoch
    obs = np.zeros((len(fr) * n_sub, 3))
    for f in range(len(fr)):
        fr[f]["observer_idx"] = f * n_sub
        for k in range(n_sub):
            rc, p, _ = orc.ephem(3, fr[f]["epoch"] + ((k + 0.5) * dur[f]) / n_sub)
            assert rc == 0
            obs[f * n_sub + k] = p
    fr[1]["observer_idx"] = fr[0]["observer_idx"]
    sub, parent = _subframes(fr, dur, n_sub)
    ref, _, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, sub, obs)
    want = _union(ref, parent)
    assert len(want) > 60
    K.load_ephem(w.ephem.to_bytes())
    hits, nh, status = K.fov_check_extended(
        torch.from_numpy(w.states).cuda(), torch.from_numpy(w.epochs).cuda(),
        kete.frames_to_device(fr, "cuda"), torch.from_numpy(dur).cuda(), n_sub,
        torch.from_numpy(obs).cuda(), capacity=16)            # too small: the CAPACITY retry
    assert (status.cpu().numpy() == 0).all()
    got = kete.decode_hits(hits, nh)
    g = {(int(f), int(b)): (ra, de) for f, b, ra, de in
         zip(got["frame"].tolist(), got["body"].tolist(), got["ra"].tolist(), got["dec"].tolist())}
    assert len(g) == nh
    keys = list(zip(got["frame"].tolist(), got["body"].tolist()))
    assert keys == sorted(keys)
    # a pair on one side only: seen only in sub-frames where it sits at an edge
    near = {(int(parent[h["frame"]]), int(h["body"])) for h in ref if abs(h["margin"]) < EDGE}
    assert not ((set(g) ^ set(want)) - near)
    worst = 0.0
    for key in set(g) & set(want):
        h = want[key]
        if abs(h["margin"]) < EDGE:
            continue   # the earliest sub-frame may differ at an edge
        ra, de = g[key]
        dra = (ra - h["ra"] + math.pi) % (2 * math.pi) - math.pi
        worst = max(worst, math.hypot(dra * math.cos(de), de - h["dec"]))
    assert worst < MAS, worst
    st = K.get_stats()
    assert st["n_hits"] == nh


def test_extended_exposures_reject_bad_input(K, mb1k_dense):
    import torch
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    K.load_ephem(w.ephem.to_bytes())
    fr = w.frames[:10].copy()
    obs = np.repeat(w.observers[:1], 40, axis=0)
    fr["observer_idx"] = np.arange(10) * 4
    st, ep = torch.from_numpy(w.states).cuda(), torch.from_numpy(w.epochs).cuda()
    ob = torch.from_numpy(obs).cuda()

    def call(frames, dur, n_sub, observers=ob):
        return K.fov_check_extended(st, ep, kete.frames_to_device(frames, "cuda"),
                                    torch.from_numpy(np.asarray(dur, float)).cuda(), n_sub, observers)
    call(fr, np.full(10, 0.001), 4)                       # valid
    bad = [(fr, np.full(10, 0.001), 0), (fr, np.full(10, 0.001), kete.EXT_MAX_SUB + 1),
           (fr, np.full(10, -0.001), 4), (fr, np.r_[np.full(9, 0.001), np.nan], 4),
           (fr, np.full(10, 0.001), 5)]                  # n_sub 5: rows beyond the observers
    long = fr.copy(); long["epoch"] = fr["epoch"][0] + np.arange(10) * 0.01
    bad.append((long, np.full(10, 0.5), 4))              # exposures overlap in time
    for frames, dur, n_sub in bad:
        with pytest.raises(kete.KeteError) as e:
            call(frames, dur, n_sub)
        assert e.value.code == kete.ERR_BAD_ARG
