"""Full-size parity on sampled outputs: the two survey years at their full
sizes, the GPU run over every body, compared with the FP64 oracle on an
evenly spaced body sample (the oracle checks each sampled body against every
frame, with its plain conservative prefilter, which the CPU tests pin to
brute force).

- WISE-like year (757,000 bodies x 1.2 M square frames from a 1-AU
  heliocentric observer), FP64, the configuration bench.py times: every
  oracle hit of the sample found, none extra outside a 1e-9 rad edge band,
  sky positions within 1 mas.
- ZTF-like year (757,000 bodies x 150,000 exposures of 8x8 sub-fields from a
  rotating ground site = 9.6 M frames), mixed precision: the same, with the
  edge band widened to twice the largest sky difference measured on the
  sample (mixed-precision positions differ by up to ~0.01 mas).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

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


def _run(K, w, fm):
    import torch
    from paper_2509_04666_gb300 import kete
    dev = "cuda"
    K.load_ephem(w.ephem.to_bytes())
    hits, nh, status = K.fov_check(torch.from_numpy(w.states).to(dev),
                                   torch.from_numpy(w.epochs).to(dev),
                                   kete.frames_to_device(w.frames, dev),
                                   torch.from_numpy(np.ascontiguousarray(w.observers)).to(dev),
                                   fm=fm)
    got = kete.decode_hits(hits, nh)
    return ({k: v.numpy() for k, v in got.items()}, status.cpu().numpy(), nh)


def _compare(got, ref, sub, edge_min):
    keep = np.isin(got["body"], sub)
    g = {(int(f), int(b)): (ra, de) for f, b, ra, de in
         zip(got["frame"][keep], got["body"][keep], got["ra"][keep], got["dec"][keep])}
    r = {(int(h["frame"]), int(h["body"])): h for h in ref}
    worst = 0.0
    for key in set(g) & set(r):
        ra, de = g[key]
        dra = (ra - r[key]["ra"] + math.pi) % (2 * math.pi) - math.pi
        worst = max(worst, math.hypot(dra * math.cos(de), de - r[key]["dec"]))
    band = max(edge_min, 2.0 * worst)
    bad = [k for k in set(g) ^ set(r) if k not in r or abs(r[k]["margin"]) >= band]
    return worst, bad, len(r)


def test_wise_like_year_fp64_full_size(K):
    from paper_2509_04666_gb300 import kete
    w = W.wise1y()
    got, status, nh = _run(K, w, kete.force_model())
    assert (status == 0).all() and nh > 5_000_000
    sub = np.linspace(0, w.n_bodies - 1, 256).astype(np.int32)
    orc = O.Oracle(w.ephem.to_bytes())
    ref, ost, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, w.frames, w.observers,
                                prefilter_deg=1.0, subset=sub)
    worst, bad, n_ref = _compare(got, ref, sub, 1e-9)
    assert n_ref > 1000
    assert not bad, bad[:5]
    assert worst < MAS, worst / MAS


def test_ztf_like_year_mixed_precision_full_size(K):
    from paper_2509_04666_gb300 import kete
    w = W.ztf1y()
    got, status, nh = _run(K, w, kete.force_model(precision=kete.MIXED))
    assert (status == 0).all() and nh > 1_000_000
    sub = np.linspace(0, w.n_bodies - 1, 128).astype(np.int32)
    orc = O.Oracle(w.ephem.to_bytes())
    ref, ost, _ = orc.fov_check(orc.force_model(), w.states, w.epochs, w.frames, w.observers,
                                prefilter_deg=1.0, subset=sub)
    worst, bad, n_ref = _compare(got, ref, sub, 1e-9)
    assert n_ref > 200
    assert not bad, bad[:5]
    assert worst < MAS, worst / MAS
