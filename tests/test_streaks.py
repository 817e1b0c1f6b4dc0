"""Host logic of extended exposures (Sec. 3.1: an exposure of finite length
is approximated by several instantaneous observations): the sub-frames and
the union of their hits."""
import numpy as np

from paper_2509_04666_gb300 import workloads as W


def _kete():
    import pytest
    pytest.importorskip("torch")
    from paper_2509_04666_gb300 import kete
    return kete


def test_streak_frames_split_the_exposure():
    kete = _kete()
    fr = np.zeros(1, W.FRAME_DTYPE)[0]
    fr["n_edges"] = 4
    fr["normals"] = np.eye(4, 3)
    sub = kete.streak_frames(fr, 100.0, 100.5, [3, 4, 5, 6, 7], 40)
    np.testing.assert_allclose(sub["epoch"], 100.0 + (np.arange(5) + 0.5) * 0.1)
    assert list(sub["observer_idx"]) == [3, 4, 5, 6, 7]
    assert list(sub["exposure_id"]) == [40, 41, 42, 43, 44]
    assert (sub["normals"] == fr["normals"]).all() and (sub["n_edges"] == 4).all()
    assert np.all(np.diff(sub["epoch"]) > 0)


def test_merge_streak_hits_is_the_union_per_exposure():
    kete = _kete()
    # frames 0-2 belong to exposure 0, 3-4 to exposure 1, 5 to exposure 2
    parent = np.array([0, 0, 0, 1, 1, 2])
    hits = {"frame": np.array([0, 0, 1, 2, 2, 3, 4, 4, 5]),
            "body": np.array([4, 9, 9, 1, 4, 9, 2, 9, 9]),
            "ra": np.arange(9.0), "dec": -np.arange(9.0)}
    m = kete.merge_streak_hits(hits, parent)
    got = list(zip(m["exposure"].tolist(), m["body"].tolist(), m["frame"].tolist()))
    assert got == [(0, 1, 2), (0, 4, 0), (0, 9, 0), (1, 2, 4), (1, 9, 3), (2, 9, 5)]
    # the earliest sub-frame's sky position is kept
    assert m["ra"][got.index((0, 9, 0))] == 1.0
    empty = kete.merge_streak_hits({k: v[:0] for k, v in hits.items()}, parent)
    assert empty["body"].size == 0
