"""Host-side frame builders of the binding (Sec. 3.1): polygons from RA/Dec
corners in either winding, cones about an RA/Dec centre, checked with the
oracle's membership test against independent constructions."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

torch = pytest.importorskip("torch")
from paper_2509_04666_gb300 import kete  # noqa: E402


def test_frame_layout_matches_the_abi_record():
    assert kete.FRAME_DTYPE == W.FRAME_DTYPE and kete.FRAME_DTYPE.itemsize == 128


def test_radec_to_vec_inverts_the_reported_radec():
    rng = np.random.default_rng(4)
    ra = rng.uniform(0, 2 * math.pi, 200)
    dec = np.arcsin(rng.uniform(-1, 1, 200))
    v = kete.radec_to_vec(ra, dec)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    for k in range(200):
        r2, d2 = O.radec(v[k] * 2.5)
        assert abs((r2 - ra[k] + math.pi) % (2 * math.pi) - math.pi) * math.cos(dec[k]) < 1e-14
        assert abs(d2 - dec[k]) < 1e-14


@pytest.mark.parametrize("winding", [1, -1])
def test_polygon_from_corners_equals_the_gnomonic_square(winding):
    rng = np.random.default_rng(5 + winding)
    n_checked = 0
    for _ in range(40):
        p = rng.normal(size=3); p /= np.linalg.norm(p)
        e = rng.normal(size=3)
        h = math.radians(rng.uniform(0.2, 5.0))
        sq = np.zeros(1, W.FRAME_DTYPE)[0]
        sq["n_edges"] = 4
        sq["normals"] = W.square_normals(p[None], e[None], h)[0]
        e = e - (e @ p) * p; e /= np.linalg.norm(e)
        n = np.cross(p, e)
        t = math.tan(h)
        corners = [p + t * (a * e + b * n) for a, b in ((1, 1), (-1, 1), (-1, -1), (1, -1))]
        corners = corners[::winding]
        radec = [O.radec(c) for c in corners]
        fr = kete.polygon_frame(radec, 2459215.5, 0)
        assert fr["n_edges"] == 4
        for _ in range(50):
            u = p + rng.uniform(-1.5, 1.5) * t * e + rng.uniform(-1.5, 1.5) * t * n
            a, _ = O.in_polygon(sq, u)
            b, margin = O.in_polygon(fr, u)
            if abs(margin) > 1e-12:
                assert a == b
                n_checked += 1
    assert n_checked > 1500


def test_triangle_and_cone_frames():
    # a triangle around the north ecliptic pole's neighbourhood
    fr = kete.polygon_frame([(0.0, 1.2), (2.1, 1.2), (4.2, 1.2)], 0.0, 3, 7)
    assert fr["n_edges"] == 3 and fr["observer_idx"] == 3 and fr["exposure_id"] == 7
    assert O.in_polygon(fr, kete.radec_to_vec(1.0, 1.5))[0]
    assert not O.in_polygon(fr, kete.radec_to_vec(1.0, 1.0))[0]
    c = kete.cone_frame(1.0, 0.3, math.radians(2.0), 1.0, 0)
    rng = np.random.default_rng(6)
    centre = kete.radec_to_vec(1.0, 0.3)
    for _ in range(500):
        u = centre + rng.normal(size=3) * 0.05
        ang = math.atan2(np.linalg.norm(np.cross(centre, u)), centre @ u)
        inside, margin = O.in_polygon(c, u)
        if abs(ang - math.radians(2.0)) > 1e-12:
            assert inside == (ang < math.radians(2.0))
    with pytest.raises(ValueError):
        kete.polygon_frame([(0.0, 0.0), (0.1, 0.0)], 0.0, 0)
    with pytest.raises(ValueError):
        kete.cone_frame(0.0, 0.0, 0.0, 0.0, 0)
