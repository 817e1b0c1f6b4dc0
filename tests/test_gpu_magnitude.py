"""Per-hit apparent magnitudes (kete_fov_check_mag: Sec. 3.3's H-G V for
asteroids, the comet total and nucleus magnitudes) against the FP64 oracle.

For a hit of body b in frame f the oracle takes b's state at the batch
midpoint of f's epoch (n-body from b's epoch, same force model), then the
light-time corrected two-body geometry to the exposure epoch, as the GPU
does.  Tolerance 1e-4 mag: the GPU evaluates the laws in FP32 (a dozen
operations of relative error ~1e-7 on terms below 30 mag give < 1e-5) from
FP64 geometry; the oracle's own arc cosine of the phase cosine costs it up
to ~3e-5 mag at zero phase.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAG_TOL = 1e-4


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


def _labels(w):
    # every fifth body is given a comet law, so that all three laws occur
    lab = np.asarray(w.labels).copy()
    lab[::5] = 3
    return lab


def _run(K, w, mag=None, fm=None):
    import torch
    from paper_2509_04666_gb300 import kete
    dev = "cuda"
    K.load_ephem(w.ephem.to_bytes())
    mp = None if mag is None else kete.mag_params_to_device(mag, dev)
    hits, nh, status = K.fov_check(torch.from_numpy(w.states).to(dev),
                                   torch.from_numpy(w.epochs).to(dev),
                                   kete.frames_to_device(w.frames, dev),
                                   torch.from_numpy(np.ascontiguousarray(w.observers)).to(dev),
                                   fm=fm, mag_params=mp)
    got = kete.decode_hits(hits, nh)
    return {k: v.numpy() for k, v in got.items()}, status.cpu().numpy(), hits[:nh].cpu().numpy()


def _oracle_mags(w, mag, frames, bodies):
    orc = O.Oracle(w.ephem.to_bytes())
    fm = orc.force_model()
    ep = w.frames["epoch"]
    order = np.argsort(ep, kind="stable")
    bs, tr = O.make_batches(ep[order], 3.0, 1.5)
    t_ref = np.empty(len(ep))
    ends = list(bs[1:]) + [len(ep)]
    for k, (s, e) in enumerate(zip(bs, ends)):
        t_ref[order[s:e]] = tr[k]
    cache, out = {}, np.empty(len(frames))
    for q, (f, b) in enumerate(zip(frames, bodies)):
        key = (int(b), float(t_ref[f]))
        if key not in cache:
            rc, st, _, _, _ = orc.propagate(fm, w.states[:, b], float(w.epochs[b]), key[1])
            assert rc == 0
            cache[key] = st
        obs = w.observers[int(w.frames["observer_idx"][f])]
        p = mag[b]
        rc, m, rh, dl, al = orc.magnitude(cache[key], key[1], float(ep[f]), obs,
                                          int(p["kind"]), float(p["p1"]), float(p["p2"]))
        assert rc == 0
        out[q] = m
    return out


def test_hit_magnitudes_match_oracle(K, mb1k_dense):
    w = mb1k_dense
    mag = W.mag_params(_labels(w))
    got, status, _ = _run(K, w, mag)
    assert (status == 0).all() and len(got["frame"]) > 100
    sel = np.linspace(0, len(got["frame"]) - 1, min(400, len(got["frame"]))).astype(int)
    f, b, m = got["frame"][sel], got["body"][sel], got["mag"][sel].astype(np.float64)
    ref = _oracle_mags(w, mag, f, b)
    kinds = mag["kind"][b]
    assert set(kinds.tolist()) == {0, 1, 2, 3}
    none = kinds == 0
    assert np.isnan(m[none]).all() and np.isnan(ref[none]).all()
    err = np.abs(m[~none] - ref[~none])
    assert np.isfinite(m[~none]).all() and err.max() < MAG_TOL, err.max()
    # plausible values for these laws at main-belt and NEO distances
    assert (m[~none] > 0).all() and (m[~none] < 40).all()


def test_magnitudes_leave_the_hit_list_unchanged(K, mb1k_dense):
    """The epilogue only fills the magnitude word: frame, body, RA/Dec and the
    order are bit-identical to kete_fov_check's, whose magnitudes are NaN."""
    w = mb1k_dense
    mag = W.mag_params(_labels(w))
    got0, st0, raw0 = _run(K, w)
    got1, st1, raw1 = _run(K, w, mag)
    assert np.array_equal(st0, st1)
    assert raw0.shape == raw1.shape
    assert np.array_equal(raw0[:, 0], raw1[:, 0])
    assert np.array_equal(raw0[:, 2:], raw1[:, 2:])
    assert np.array_equal(raw0[:, 1] & 0xFFFFFFFF, raw1[:, 1] & 0xFFFFFFFF)
    assert np.isnan(got0["mag"]).all()


def test_magnitude_kinds_and_bad_arguments(K, mb1k_dense):
    """A kind outside 1..3 gives NaN; a parameter buffer of the wrong size or
    on the host is refused before any launch."""
    import torch
    from paper_2509_04666_gb300 import kete
    w = mb1k_dense
    mag = W.mag_params(w.labels)
    mag["kind"][1::2] = 7
    got, status, _ = _run(K, w, mag)
    odd = got["body"] % 2 == 1
    even_asteroid = (~odd) & (mag["kind"][got["body"]] != 0)
    assert np.isnan(got["mag"][odd]).all()
    assert np.isfinite(got["mag"][even_asteroid]).all()
    K.load_ephem(w.ephem.to_bytes())
    args = (torch.from_numpy(w.states).cuda(), torch.from_numpy(w.epochs).cuda(),
            kete.frames_to_device(w.frames, "cuda"),
            torch.from_numpy(np.ascontiguousarray(w.observers)).cuda())
    short = kete.mag_params_to_device(mag[:-1], "cuda")
    with pytest.raises(TypeError):
        K.fov_check(*args, mag_params=short)
    with pytest.raises(TypeError):
        K.fov_check(*args, mag_params=kete.mag_params_to_device(mag, "cuda").cpu())
