"""Seeded synthetic inputs for the survey-prediction path (Sec. 2, Sec. 3.1, App. A).

This module builds INPUT DATA only: the planetary ephemeris table (the stand-in
for the DE440 SPICE kernel of App. A), the Cartesian states of the minor
bodies, the telescope fields of view and the observer positions.  It holds none
of the method's arithmetic (no force model, no Gauss-Radau integrator, no
universal-variable Kepler solve, no light-time correction, no FoV test); both
the CUDA path and the CPU oracle consume what it writes.

Random numbers come from numpy's counter-based Philox-4x32 generator, one
stream per purpose (planets, bodies, frames), keyed by the workload seed.

Units: AU, TDB days, barycentric ecliptic J2000 frame (App. A.1).

Workloads (sizes, distributions) -- the synthetic stand-ins for the paper's
ZTF / WISE runs of Sec. 2, whose metadata and MPC orbits are not available:

* ``mb1k``     -- 1,000 main-belt bodies, 30-day span, 200 square 1 deg frames
                  seen from the Earth (the small parity case).
* ``wise1y``   -- 757,000 bodies (2 % NEOs), 365 days, 1.2 M square 0.78 deg
                  frames from a circular 1-AU heliocentric observer scanning the
                  90 deg solar-elongation great circle (WISE-like).
* ``ztf1y``    -- same bodies, 150,000 night-time exposures of 8x8 sub-fields of
                  0.87 deg from a rotating ground site (ZTF-like).
* ``adjoint90``-- 100,000 bodies, 90 days, 20 observations per body, noise
                  draws and state offsets for the orbit-fit gradient.
* ``ragged1y`` -- 500,000 mixed population (main belt, NEOs with forced Earth
                  encounters (label 4), Trojans, comets), 365 days.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Constants used to BUILD the data (the table carries the GM values it was
# integrated with, so every consumer reads the same masses from the table).
# ---------------------------------------------------------------------------
T0 = 2459215.5                     # JD TDB of the state epoch of every workload
GAUSS_K = 0.01720209895            # Gaussian gravitational constant, AU^1.5 / day
GM_SUN = GAUSS_K * GAUSS_K         # AU^3 / day^2
# Sun-to-body mass ratios (IAU nominal values); "Earth" is the Earth-Moon system.
MASS_RATIO = [1.0, 6023597.400017, 408523.718655, 328900.559709, 3098703.59,
              1047.348644, 3497.901768, 22902.981613, 19412.237346]
GM = [GM_SUN / r for r in MASS_RATIO]
BODY_NAMES = ["sun", "mercury", "venus", "earth", "mars",
              "jupiter", "saturn", "uranus", "neptune"]
PLANET_A = [0.0, 0.387098, 0.723332, 1.000000, 1.523679,
            5.2044, 9.5826, 19.2184, 30.110]
AU_KM = 149597870.7
OBLIQUITY = math.radians(84381.448 / 3600.0)   # ecliptic J2000 obliquity
EARTH_RADIUS_AU = 6378.0 / AU_KM
SIDEREAL_DAY = 0.99726957
SITE_LAT = math.radians(33.36)

SEED_BASE = 2509046660

FRAME_DTYPE = np.dtype([
    ("epoch", "<f8"), ("observer_idx", "<i8"), ("exposure_id", "<i8"),
    ("n_edges", "<i4"), ("reserved", "<i4"), ("normals", "<f8", (4, 3)),
])
assert FRAME_DTYPE.itemsize == 128

EPHEM_MAGIC = b"KETECHB1"
EPHEM_HEADER_BYTES = 256
MAX_TABLE_BODIES = 16


def _rng(seed: int, stream: int) -> np.random.Generator:
    """Philox-4x32 counter-based stream ``stream`` of workload seed ``seed``."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, stream])))


# ---------------------------------------------------------------------------
# Orbital elements -> Cartesian (input construction, C21)
# ---------------------------------------------------------------------------
def _rot_matrix(inc, node, peri):
    """Rows of R_z(node) R_x(inc) R_z(peri) applied to perifocal vectors."""
    cO, sO = np.cos(node), np.sin(node)
    ci, si = np.cos(inc), np.sin(inc)
    cw, sw = np.cos(peri), np.sin(peri)
    px = cO * cw - sO * sw * ci
    py = sO * cw + cO * sw * ci
    pz = sw * si
    qx = -cO * sw - sO * cw * ci
    qy = -sO * sw + cO * cw * ci
    qz = cw * si
    return (px, py, pz), (qx, qy, qz)


def elements_to_state(a, e, inc, node, peri, mean_anom, mu):
    """Elliptic osculating elements -> (pos[3,n], vel[3,n]) relative to the focus."""
    a = np.asarray(a, float); e = np.asarray(e, float)
    M = np.mod(np.asarray(mean_anom, float), 2 * np.pi)
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(100):
        f = E - e * np.sin(E) - M
        dE = f / (1.0 - e * np.cos(E))
        E = E - dE
        if np.all(np.abs(dE) < 1e-15):
            break
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = a * b * sE
    r = a * (1.0 - e * cE)
    vfac = np.sqrt(mu * a) / r
    vxp = -vfac * sE
    vyp = vfac * b * cE
    (px, py, pz), (qx, qy, qz) = _rot_matrix(inc, node, peri)
    pos = np.stack([px * xp + qx * yp, py * xp + qy * yp, pz * xp + qz * yp])
    vel = np.stack([px * vxp + qx * vyp, py * vxp + qy * vyp, pz * vxp + qz * vyp])
    return pos, vel


def _rayleigh_capped(rng, scale, cap, n):
    out = rng.rayleigh(scale, n)
    bad = out > cap
    while np.any(bad):
        out[bad] = rng.rayleigh(scale, int(bad.sum()))
        bad = out > cap
    return out


# ---------------------------------------------------------------------------
# Planetary ephemeris: mutual FP64 integration of Sun + 8 planets, then a
# Chebyshev fit per body per segment (the project's own stand-in for DE440).
# ---------------------------------------------------------------------------
@dataclass
class PlanetSystem:
    t0: float
    pos0: np.ndarray      # (9, 3) barycentric at t0
    vel0: np.ndarray      # (9, 3)
    gm: np.ndarray        # (9,)


def make_planets(seed: int, planets: bool = True) -> PlanetSystem:
    """Seeded near-circular planets (e ~ U[0,0.01], i ~ U[0,2 deg]), barycentric."""
    rng = _rng(seed, 1)
    gm = np.array(GM)
    helio_p = np.zeros((9, 3)); helio_v = np.zeros((9, 3))
    e = rng.uniform(0.0, 0.01, 8)
    inc = np.radians(rng.uniform(0.0, 2.0, 8))
    node, peri, M = (rng.uniform(0, 2 * np.pi, 8) for _ in range(3))
    if planets:
        p, v = elements_to_state(np.array(PLANET_A[1:]), e, inc, node, peri, M,
                                 GM_SUN + gm[1:])
        helio_p[1:] = p.T; helio_v[1:] = v.T
    else:
        gm[1:] = 0.0
    mtot = gm.sum()
    sun_p = -(gm[:, None] * helio_p).sum(0) / mtot
    sun_v = -(gm[:, None] * helio_v).sum(0) / mtot
    return PlanetSystem(T0, helio_p + sun_p, helio_v + sun_v, gm)


def _nbody_rhs(gm):
    def rhs(t, y):
        p = y[:27].reshape(9, 3); v = y[27:].reshape(9, 3)
        d = p[None, :, :] - p[:, None, :]            # d[i,j] = p_j - p_i
        r2 = (d * d).sum(-1)
        np.fill_diagonal(r2, 1.0)
        inv3 = r2 ** -1.5
        np.fill_diagonal(inv3, 0.0)
        a = (d * (gm[None, :] * inv3)[:, :, None]).sum(1)
        return np.concatenate([v.ravel(), a.ravel()])
    return rhs


def integrate_planets(ps: PlanetSystem, t_eval: np.ndarray) -> np.ndarray:
    """Barycentric planet positions/velocities at t_eval: returns (len, 9, 6).

    scipy's DOP853 with rtol 3e-14 and steps of at most 2 days (a library integrator, not the method's)."""
    from scipy.integrate import solve_ivp
    t_eval = np.asarray(t_eval, float)
    out = np.empty((t_eval.size, 9, 6))
    y0 = np.concatenate([ps.pos0.ravel(), ps.vel0.ravel()])
    rhs = _nbody_rhs(ps.gm)
    for sel, t_end in ((t_eval >= ps.t0, None), (t_eval < ps.t0, None)):
        if not np.any(sel):
            continue
        ts = t_eval[sel]
        t_far = ts.max() if ts[0] >= ps.t0 else ts.min()
        if t_far == ps.t0:
            y = np.repeat(y0[:, None], ts.size, 1)
        else:
            sol = solve_ivp(rhs, (ps.t0, t_far), y0, method="DOP853", rtol=3e-14,
                            atol=1e-16, max_step=2.0, dense_output=True)
            y = sol.sol(ts)
        out[sel, :, :3] = y[:27].T.reshape(-1, 9, 3)
        out[sel, :, 3:] = y[27:].T.reshape(-1, 9, 3)
    return out


@dataclass
class EphemTable:
    t_start: float
    seg_len: float
    n_seg: int
    n_coef: int
    gm: np.ndarray                 # (n_bodies,)
    coef: np.ndarray               # (n_bodies, n_seg, 3, n_coef)

    @property
    def n_bodies(self):
        return self.coef.shape[0]

    @property
    def t_end(self):
        return self.t_start + self.n_seg * self.seg_len

    def to_bytes(self) -> bytes:
        hdr = bytearray(EPHEM_HEADER_BYTES)
        gm = np.zeros(MAX_TABLE_BODIES); gm[: self.n_bodies] = self.gm
        struct.pack_into("<8s4i2d", hdr, 0, EPHEM_MAGIC, 1, self.n_bodies,
                         self.n_coef, self.n_seg, self.t_start, self.seg_len)
        struct.pack_into("<16d", hdr, 48, *gm)
        return bytes(hdr) + np.ascontiguousarray(self.coef, "<f8").tobytes()

    @staticmethod
    def from_bytes(buf: bytes) -> "EphemTable":
        magic, ver, nb, nc, ns, t_start, seg = struct.unpack_from("<8s4i2d", buf, 0)
        assert magic == EPHEM_MAGIC and ver == 1
        gm = np.array(struct.unpack_from("<16d", buf, 48))[:nb]
        coef = np.frombuffer(buf, "<f8", nb * ns * 3 * nc, EPHEM_HEADER_BYTES)
        return EphemTable(t_start, seg, ns, nc, gm, coef.reshape(nb, ns, 3, nc).copy())


def cheb_nodes(n):
    return np.cos(np.pi * (np.arange(n) + 0.5) / n)


def build_ephemeris(ps: PlanetSystem, t_lo: float, t_hi: float,
                    seg_len: float = 16.0, n_coef: int = 12) -> EphemTable:
    """Chebyshev interpolation of the integrated planets over [t_lo, t_hi]."""
    t_start = math.floor(t_lo)
    n_seg = int(math.ceil((t_hi - t_start) / seg_len))
    x = cheb_nodes(n_coef)
    mids = t_start + (np.arange(n_seg) + 0.5) * seg_len
    t_nodes = (mids[:, None] + x[None, :] * 0.5 * seg_len).ravel()
    st = integrate_planets(ps, t_nodes)[:, :, :3].reshape(n_seg, n_coef, 9, 3)
    k = np.arange(n_coef)
    dct = np.cos(np.pi * k[:, None] * (np.arange(n_coef)[None, :] + 0.5) / n_coef)
    dct *= 2.0 / n_coef
    dct[0] *= 0.5
    coef = np.einsum("kj,sjbc->bsck", dct, st)
    return EphemTable(float(t_start), float(seg_len), n_seg, n_coef, ps.gm.copy(), coef)


def circular_pair_table(body: int, a: float, t_lo: float, t_hi: float, seg_len: float = 16.0,
                        n_coef: int = 12) -> EphemTable:
    """Sun and one table body on exact circular orbits about their barycentre in
    the ecliptic plane (the circular restricted three-body setting); the other
    bodies are massless.  Used to pin the planet terms by the Jacobi integral."""
    t_start = math.floor(t_lo)
    n_seg = int(math.ceil((t_hi - t_start) / seg_len))
    gm = np.zeros(9); gm[0] = GM_SUN; gm[body] = GM[body]
    mt = gm[0] + gm[body]
    n = math.sqrt(mt / a ** 3)
    x = cheb_nodes(n_coef)
    mids = t_start + (np.arange(n_seg) + 0.5) * seg_len
    t_nodes = mids[:, None] + x[None, :] * 0.5 * seg_len          # (n_seg, n_coef)
    ang = n * (t_nodes - T0)
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], -1)
    st = np.zeros((n_seg, n_coef, 9, 3))
    st[:, :, 0] = -(gm[body] / mt) * a * ring
    st[:, :, body] = (gm[0] / mt) * a * ring
    k = np.arange(n_coef)
    dct = np.cos(np.pi * k[:, None] * (np.arange(n_coef)[None, :] + 0.5) / n_coef) * 2.0 / n_coef
    dct[0] *= 0.5
    coef = np.einsum("kj,sjbc->bsck", dct, st)
    return EphemTable(float(t_start), float(seg_len), n_seg, n_coef, gm, coef)


def static_sun_table(t_lo: float, t_hi: float, seg_len: float = 16.0, n_coef: int = 12,
                     gm_scale: float = 1.0) -> EphemTable:
    """A table with the Sun at rest at the origin and massless planets (pins)."""
    t_start = math.floor(t_lo)
    n_seg = int(math.ceil((t_hi - t_start) / seg_len))
    gm = np.zeros(9); gm[0] = GM_SUN * gm_scale
    return EphemTable(float(t_start), float(seg_len), n_seg, n_coef, gm,
                      np.zeros((9, n_seg, 3, n_coef)))


# ---------------------------------------------------------------------------
# Minor-body populations (heliocentric elements at T0 -> barycentric states)
# ---------------------------------------------------------------------------
def _main_belt(rng, n):
    a = rng.uniform(2.1, 3.3, n)
    e = _rayleigh_capped(rng, 0.08, 0.3, n)
    inc = np.radians(_rayleigh_capped(rng, 8.0, 90.0, n))
    return a, e, inc


def _neo(rng, n):
    a = rng.uniform(0.8, 2.0, n)
    e = rng.uniform(0.0, 0.7, n)
    inc = np.radians(_rayleigh_capped(rng, 15.0, 90.0, n))
    return a, e, inc


def _angles(rng, n):
    return rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)


def bodies_from_elements(ps: PlanetSystem, a, e, inc, node, peri, M):
    pos, vel = elements_to_state(a, e, inc, node, peri, M, GM_SUN)
    st = np.empty((6, pos.shape[1]))
    st[:3] = pos + ps.pos0[0][:, None]
    st[3:] = vel + ps.vel0[0][:, None]
    return st


def population(seed: int, ps: PlanetSystem, n_mb: int, n_neo: int = 0, n_trojan: int = 0,
               n_comet: int = 0, return_elements: bool = False):
    """Barycentric states (6, n) and population labels (0 MB, 1 NEO, 2 Trojan, 3 comet)."""
    rng = _rng(seed, 2)
    parts, labels = [], []
    if n_mb:
        a, e, i = _main_belt(rng, n_mb); parts.append((a, e, i) + _angles(rng, n_mb))
        labels.append(np.zeros(n_mb, np.int8))
    if n_neo:
        a, e, i = _neo(rng, n_neo); parts.append((a, e, i) + _angles(rng, n_neo))
        labels.append(np.ones(n_neo, np.int8))
    if n_trojan:
        a = np.full(n_trojan, 5.2)
        e = _rayleigh_capped(rng, 0.05, 0.3, n_trojan)
        i = np.radians(_rayleigh_capped(rng, 10.0, 60.0, n_trojan))
        node, peri, _ = _angles(rng, n_trojan)
        # mean longitude of Jupiter at T0 from its barycentric-minus-Sun position
        jp = ps.pos0[5] - ps.pos0[0]
        lam_j = math.atan2(jp[1], jp[0])
        side = np.where(rng.uniform(0, 1, n_trojan) < 0.5, 1.0, -1.0)
        lam = lam_j + side * np.radians(60.0) + np.radians(rng.uniform(-10, 10, n_trojan))
        M = lam - node - peri
        parts.append((a, e, i, node, peri, M)); labels.append(np.full(n_trojan, 2, np.int8))
    if n_comet:
        e = rng.uniform(0.7, 0.99, n_comet)
        q = rng.uniform(0.5, 3.0, n_comet)
        a = q / (1.0 - e)
        i = np.radians(_rayleigh_capped(rng, 20.0, 180.0, n_comet))
        parts.append((a, e, i) + _angles(rng, n_comet)); labels.append(np.full(n_comet, 3, np.int8))
    cols = [np.concatenate([p[j] for p in parts]) for j in range(6)]
    if return_elements:
        return bodies_from_elements(ps, *cols), np.concatenate(labels), np.stack(cols)
    return bodies_from_elements(ps, *cols), np.concatenate(labels)


# ---------------------------------------------------------------------------
# Fields of view: square spherical polygons with inward great-circle normals
# ---------------------------------------------------------------------------
def cone_frames(frames, which, radius):
    """Turn frames[which] into cones (n_edges 0, Sec. 3.1): centre = the
    frame's own centre direction (sum of its inward normals' axis, i.e. the
    normalised sum of the normals), angular radius `radius` (radians) in
    normals[1][0]; the rest of the record is zero."""
    out = frames.copy()
    idx = np.arange(len(frames))[which]
    c = frames["normals"][idx].sum(axis=1)
    c /= np.linalg.norm(c, axis=-1, keepdims=True)
    out["n_edges"][idx] = 0
    out["normals"][idx] = 0.0
    out["normals"][idx, 0, :] = c
    out["normals"][idx, 1, 0] = radius
    return out


def square_normals(centre, e_axis, half_width):
    """Inward normals m = p sin h - t cos h of the edges t = +e, +n, -e, -n, in
    that (cyclic) order around the square (Sec. 3.1)."""
    p = centre / np.linalg.norm(centre, axis=-1, keepdims=True)
    e = e_axis - (e_axis * p).sum(-1, keepdims=True) * p
    e /= np.linalg.norm(e, axis=-1, keepdims=True)
    n = np.cross(p, e)
    sh, ch = math.sin(half_width), math.cos(half_width)
    out = np.empty(p.shape[:-1] + (4, 3))
    out[..., 0, :] = p * sh - e * ch
    out[..., 1, :] = p * sh - n * ch
    out[..., 2, :] = p * sh + e * ch
    out[..., 3, :] = p * sh + n * ch
    return out


def eq_to_ecl(v):
    """Equatorial J2000 -> ecliptic J2000 (rotation about x by -obliquity)."""
    c, s = math.cos(OBLIQUITY), math.sin(OBLIQUITY)
    v = np.asarray(v, float)
    out = np.empty_like(v)
    out[..., 0] = v[..., 0]
    out[..., 1] = c * v[..., 1] + s * v[..., 2]
    out[..., 2] = -s * v[..., 1] + c * v[..., 2]
    return out


def ecl_to_eq(v):
    c, s = math.cos(OBLIQUITY), math.sin(OBLIQUITY)
    v = np.asarray(v, float)
    out = np.empty_like(v)
    out[..., 0] = v[..., 0]
    out[..., 1] = c * v[..., 1] - s * v[..., 2]
    out[..., 2] = s * v[..., 1] + c * v[..., 2]
    return out


def _frames_array(epochs, obs_idx, exp_id, normals):
    f = np.zeros(len(epochs), FRAME_DTYPE)
    f["epoch"] = epochs; f["observer_idx"] = obs_idx; f["exposure_id"] = exp_id
    f["n_edges"] = 4; f["normals"] = normals
    return f


# ---------------------------------------------------------------------------
# Workload container
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    seed: int
    ephem: EphemTable
    states: np.ndarray            # (6, N) barycentric ecliptic, AU and AU/day
    epochs: np.ndarray            # (N,) TDB JD
    frames: np.ndarray            # FRAME_DTYPE, sorted by epoch, exposures contiguous
    observers: np.ndarray         # (n_obs, 3)
    t_end: float                  # propagation target / end of survey
    labels: np.ndarray = None
    frame_centres: np.ndarray = None    # (F, 3) unit centres (tests only)
    frame_half_width: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_bodies(self):
        return self.states.shape[1]


def _earth_positions(ps, t):
    return integrate_planets(ps, t)[:, 3, :3]


def mb1k(n_bodies=1000, n_frames=200, span=30.0, dense_frac=0.0, seed=None):
    """The small parity case: main-belt bodies, 1 deg squares seen from the Earth.

    ``dense_frac`` of the frames are pointed near bodies (test-only option that
    raises the hit count; the standard case uses 0)."""
    seed = SEED_BASE + 0 if seed is None else seed
    ps = make_planets(seed)
    states, labels, elem = population(seed, ps, n_bodies, return_elements=True)
    rng = _rng(seed, 3)
    ep = np.sort(rng.uniform(T0, T0 + span, n_frames))
    earth_sun = integrate_planets(ps, ep)
    obs = earth_sun[:, 3, :3]
    sinb = rng.uniform(-0.5, 0.5, n_frames)
    lon = rng.uniform(0, 2 * np.pi, n_frames)
    cb = np.sqrt(1 - sinb ** 2)
    centre = np.stack([cb * np.cos(lon), cb * np.sin(lon), sinb], -1)
    n_dense = int(round(dense_frac * n_frames))
    if n_dense:
        # aim near where a body is at the frame epoch: advance its mean anomaly
        # on the heliocentric ellipse it was drawn from (a pointing aid only)
        pick = rng.integers(0, n_bodies, n_dense)
        a, e, inc, node, peri, M = elem[:, pick]
        dt = ep[:n_dense] - T0
        hp, _ = elements_to_state(a, e, inc, node, peri, M + np.sqrt(GM_SUN / a ** 3) * dt, GM_SUN)
        d = hp.T + earth_sun[:n_dense, 0, :3] - obs[:n_dense]
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        jitter = rng.normal(0, np.radians(0.2), (n_dense, 3))
        c = d + jitter
        centre[:n_dense] = c / np.linalg.norm(c, axis=1, keepdims=True)
    psi = rng.uniform(0, np.pi, n_frames)
    pole = np.array([0.0, 0.0, 1.0])
    east = np.cross(pole, centre); east /= np.linalg.norm(east, axis=1, keepdims=True)
    north = np.cross(centre, east)
    e_axis = np.cos(psi)[:, None] * east + np.sin(psi)[:, None] * north
    h = np.radians(0.5)
    normals = square_normals(centre, e_axis, h)
    frames = _frames_array(ep, np.arange(n_frames), np.arange(n_frames), normals)
    eph = build_ephemeris(ps, T0 - 32.0, T0 + span + 64.0)
    return Workload("mb1k", seed, eph, states, np.full(n_bodies, T0), frames, obs,
                    T0 + span, labels, centre, h)


def wise_frames(ps, n_frames=1_200_000, days=365, per_day=3288, cadence_s=11.0,
                step_deg=0.7, width_deg=0.78, block_start=0.1):
    """WISE-like scan from a circular 1-AU heliocentric orbit (see module doc)."""
    n_days = int(math.ceil(n_frames / per_day))
    n_days = min(n_days, days)
    j = np.arange(n_frames)
    day = j // per_day
    within = j % per_day
    ep = T0 + day + block_start + within * cadence_s / 86400.0
    # observer: Sun + unit circle in the ecliptic, mean motion of a 1-AU orbit
    theta = 0.3 + GAUSS_K * (ep - T0)
    rhat = np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], -1)
    uniq = np.unique(np.floor((ep - T0) * 24.0))   # hourly Sun samples, interpolated
    t_s = T0 + np.concatenate([uniq, [uniq[-1] + 1]]) / 24.0
    sun = integrate_planets(ps, t_s)[:, 0, :3]
    sun_at = np.stack([np.interp(ep, t_s, sun[:, c]) for c in range(3)], -1)
    obs = sun_at + rhat
    zhat = np.array([0.0, 0.0, 1.0])
    that = np.cross(zhat, rhat)
    phi = np.radians(step_deg) * j
    centre = np.cos(phi)[:, None] * zhat + np.sin(phi)[:, None] * that
    e_axis = -np.sin(phi)[:, None] * zhat + np.cos(phi)[:, None] * that
    h = np.radians(width_deg / 2)
    normals = square_normals(centre, e_axis, h)
    frames = _frames_array(ep, j, j, normals)
    return frames, obs, centre, h


def wise1y(n_bodies=757_000, n_frames=1_200_000, seed=None, neo_frac=0.02):
    seed = SEED_BASE + 1 if seed is None else seed
    ps = make_planets(seed)
    n_neo = int(round(neo_frac * n_bodies))
    states, labels = population(seed, ps, n_bodies - n_neo, n_neo)
    frames, obs, centre, h = wise_frames(ps, n_frames)
    eph = build_ephemeris(ps, T0 - 64.0, T0 + 365.0 + 80.0)
    return Workload("wise1y", seed, eph, states, np.full(n_bodies, T0), frames, obs,
                    T0 + 365.0, labels, centre, h)


def _site_zenith_eq(t):
    theta = 1.2 + 2 * np.pi * (t - T0) / SIDEREAL_DAY
    c = math.cos(SITE_LAT)
    return np.stack([c * np.cos(theta), c * np.sin(theta), np.full_like(theta, math.sin(SITE_LAT))], -1)


def ztf_frames(ps, n_exposures=150_000, days=365, grid=8, sub_deg=0.87, seed_rng=None):
    """ZTF-like exposures: 8x8 sub-fields of 0.87 deg from a rotating ground site."""
    rng = seed_rng
    # night-time samples every 30 s (an exposure + readout cadence); Sun
    # altitude < -12 deg at the site: ~370,000 night samples in a year
    ts = T0 + np.arange(0, days * 2880) / 2880.0
    st = integrate_planets(ps, np.linspace(T0, T0 + days, days * 4 + 1))
    tt = np.linspace(T0, T0 + days, days * 4 + 1)
    sun = np.stack([np.interp(ts, tt, st[:, 0, c]) for c in range(3)], -1)
    earth = np.stack([np.interp(ts, tt, st[:, 3, c]) for c in range(3)], -1)
    sdir = ecl_to_eq(sun - earth)
    sdir /= np.linalg.norm(sdir, axis=1, keepdims=True)
    zen = _site_zenith_eq(ts)
    night = (zen * sdir).sum(1) < math.sin(math.radians(-12.0))
    tn = ts[night]
    if n_exposures > tn.size:
        raise ValueError(f"{n_exposures} exposures do not fit {tn.size} night-time slots")
    ep = np.sort(rng.choice(tn, n_exposures, replace=False)
                 + rng.uniform(0, 1.0 / 2880.0, n_exposures))
    # pointings: Dec in [-30, 90], altitude > 30 deg at the exposure epoch
    zen_e = _site_zenith_eq(ep)
    cen = np.empty((n_exposures, 3))
    todo = np.arange(n_exposures)
    while todo.size:
        sd = rng.uniform(math.sin(math.radians(-30.0)), 1.0, todo.size)
        ra = rng.uniform(0, 2 * np.pi, todo.size)
        cd = np.sqrt(1 - sd * sd)
        v = np.stack([cd * np.cos(ra), cd * np.sin(ra), sd], -1)
        ok = (v * zen_e[todo]).sum(1) > math.sin(math.radians(30.0))
        cen[todo[ok]] = v[ok]
        todo = todo[~ok]
    # tangent axes aligned with RA/Dec at the exposure centre (equatorial)
    pole = np.array([0.0, 0.0, 1.0])
    east = np.cross(pole, cen)
    nrm = np.linalg.norm(east, axis=1, keepdims=True)
    east = np.where(nrm > 1e-12, east / np.maximum(nrm, 1e-300), np.array([1.0, 0, 0]))
    north = np.cross(cen, east)
    w = math.tan(math.radians(sub_deg))
    off = (np.arange(grid) - (grid - 1) / 2.0) * w
    oi, oj = np.meshgrid(off, off, indexing="ij")
    oi = oi.ravel(); oj = oj.ravel()
    sub_c = cen[:, None, :] + oi[None, :, None] * east[:, None, :] + oj[None, :, None] * north[:, None, :]
    sub_c /= np.linalg.norm(sub_c, axis=-1, keepdims=True)
    sub_c = eq_to_ecl(sub_c.reshape(-1, 3))
    e_ax = eq_to_ecl(np.repeat(east, grid * grid, 0))
    h = math.radians(sub_deg / 2)
    normals = square_normals(sub_c, e_ax, h)
    n_sub = grid * grid
    frames = _frames_array(np.repeat(ep, n_sub), np.repeat(np.arange(n_exposures), n_sub),
                           np.repeat(np.arange(n_exposures), n_sub), normals)
    earth_e = integrate_planets(ps, ep)[:, 3, :3]
    obs = earth_e + EARTH_RADIUS_AU * eq_to_ecl(zen_e)
    return frames, obs, sub_c, h


def ztf1y(n_bodies=757_000, n_exposures=150_000, seed=None, days=365, neo_frac=0.02):
    seed = SEED_BASE + 2 if seed is None else seed
    ps = make_planets(seed)
    n_neo = int(round(neo_frac * n_bodies))
    states, labels = population(seed, ps, n_bodies - n_neo, n_neo)
    frames, obs, centre, h = ztf_frames(ps, n_exposures, days, seed_rng=_rng(seed, 3))
    eph = build_ephemeris(ps, T0 - 64.0, T0 + days + 80.0)
    return Workload("ztf1y", seed, eph, states, np.full(n_bodies, T0), frames, obs,
                    T0 + days, labels, centre, h)


def state_to_elements(r, v, mu):
    """Heliocentric state (3, n) -> elliptic elements (a, e, i, node, peri, M)."""
    r = np.asarray(r, float); v = np.asarray(v, float)
    rn = np.linalg.norm(r, axis=0)
    h = np.cross(r.T, v.T).T
    hn = np.linalg.norm(h, axis=0)
    inc = np.arccos(np.clip(h[2] / hn, -1, 1))
    node = np.arctan2(h[0], -h[1])
    ev = (np.cross(v.T, h.T).T / mu) - r / rn
    e = np.linalg.norm(ev, axis=0)
    a = 1.0 / (2.0 / rn - (v * v).sum(0) / mu)
    # argument of perihelion and true anomaly in the orbital plane
    nvec = np.stack([np.cos(node), np.sin(node), np.zeros_like(node)])
    w_dir = np.cross(h.T, nvec.T).T / hn
    peri = np.arctan2((ev * w_dir).sum(0), (ev * nvec).sum(0))
    nu = np.arctan2((r * np.cross(h.T, ev.T).T / hn).sum(0), (r * ev).sum(0))
    E = 2.0 * np.arctan2(np.sqrt(1 - e) * np.sin(nu / 2), np.sqrt(1 + e) * np.cos(nu / 2))
    M = E - e * np.sin(E)
    return a, e, inc, node, peri, M


def ragged1y(n_bodies=500_000, seed=None, days=365.0):
    """Mixed population with very uneven step counts (see module doc):
    60 % main belt, 20 % NEOs of which 5 % pass 0.001-0.01 AU from the Earth,
    10 % Jupiter Trojans, 10 % comets (e ~ U[0.7, 0.99], q ~ U[0.5, 3] AU).

    An encounter is placed at t_enc ~ U(30, 335) d at the chosen miss distance
    from the generator's Earth with a 5-20 km/s relative velocity, and carried
    back to T0 along the heliocentric conic through that state (a construction
    aid: planetary perturbations move the actual closest approach a little)."""
    seed = SEED_BASE + 4 if seed is None else seed
    ps = make_planets(seed)
    n_neo = n_bodies // 5
    n_troj = n_bodies // 10
    n_com = n_bodies // 10
    n_mb = n_bodies - n_neo - n_troj - n_com
    states, labels = population(seed, ps, n_mb, n_neo, n_troj, n_com)
    n_force = n_neo // 20
    rng = _rng(seed, 5)
    t_enc = rng.uniform(30.0, 335.0, n_force)
    miss = rng.uniform(0.001, 0.01, n_force)
    vrel = rng.uniform(5.0, 20.0, n_force) * 86400.0 / AU_KM
    st_enc = integrate_planets(ps, t_enc + T0)
    sun_p, sun_v = st_enc[:, 0, :3], st_enc[:, 0, 3:]
    ear_p, ear_v = st_enc[:, 3, :3], st_enc[:, 3, 3:]
    forced = np.zeros((6, n_force))
    todo = np.arange(n_force)
    while todo.size:
        d = rng.normal(size=(todo.size, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        u = rng.normal(size=(todo.size, 3))
        u -= (u * d).sum(1, keepdims=True) * d
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        r = ear_p[todo] + miss[todo, None] * d - sun_p[todo]
        v = ear_v[todo] + vrel[todo, None] * u - sun_v[todo]
        with np.errstate(invalid="ignore"):
            a, e, inc, node, peri, M = state_to_elements(r.T, v.T, GM_SUN)
        ok = (e < 0.95) & (a > 0) & (a * (1 - e) > 0.2)
        idx = todo[ok]
        n_mean = np.sqrt(GM_SUN / a[ok] ** 3)
        r0, v0 = elements_to_state(a[ok], e[ok], inc[ok], node[ok], peri[ok],
                                   M[ok] - n_mean * t_enc[idx], GM_SUN)
        forced[:3, idx] = r0 + ps.pos0[0][:, None]
        forced[3:, idx] = v0 + ps.vel0[0][:, None]
        todo = todo[~ok]
    first_neo = n_mb
    states[:, first_neo:first_neo + n_force] = forced
    labels = labels.copy()
    labels[first_neo:first_neo + n_force] = 4
    eph = build_ephemeris(ps, T0 - 64.0, T0 + days + 80.0)
    w = Workload("ragged1y", seed, eph, states, np.full(n_bodies, T0),
                 np.zeros(0, FRAME_DTYPE), np.zeros((0, 3)), T0 + days, labels)
    w.meta["t_enc"] = t_enc
    w.meta["miss"] = miss
    return w


def fov_edge(n_bodies=2000, seed=None):
    """FoV-stage edge cases (test workload): ragged1y's population (main belt,
    NEOs with forced 0.001-0.01 AU Earth encounters, Trojans, comets) plus one
    sungrazing comet (q 0.01 AU, e 0.995, perihelion at T0 + 100 d), seen
    from the Earth by frames aimed where the two-body + light-time step is
    stressed: comets within 6 days of a perihelion inside the year, the forced
    encounters within 2 days of closest approach, Trojans, the sungrazer
    within 3 days of perihelion, and a few main-belt bodies and NEOs.  Frames
    alternate squares and cones, one per exposure, offset from the aim point
    by up to 0.3 of their radius; frames at encounters are 0.1-0.3 rad wide
    (the body crosses the sky at up to ~3 rad/day), at the sungrazer 0.01-
    0.02 rad.  Each frame is aimed along the body's heliocentric conic from
    T0 (a construction aid: the n-body motion differs a little, so some
    frames miss); the observer is the Earth at the frame's epoch."""
    seed = SEED_BASE + 11 if seed is None else seed
    w = ragged1y(n_bodies=n_bodies, seed=seed)
    ps = make_planets(seed)
    rng = _rng(seed, 12)
    # the sungrazer, appended as a comet
    q, ecc, t_peri = 0.01, 0.995, T0 + 100.0
    a_sg = q / (1.0 - ecc)
    inc, node, peri = math.radians(rng.uniform(10, 80)), rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi)
    M0 = -math.sqrt(GM_SUN / a_sg ** 3) * (t_peri - T0)
    sg = bodies_from_elements(ps, np.array([a_sg]), np.array([ecc]), inc, node, peri, np.array([M0]))
    states = np.concatenate([w.states, sg], axis=1)
    labels = np.concatenate([w.labels, np.array([3], np.int8)])
    n = states.shape[1]
    a, e, i, om, w_, M = state_to_elements(states[:3] - ps.pos0[0][:, None],
                                           states[3:] - ps.vel0[0][:, None], GM_SUN)
    mm = np.sqrt(GM_SUN / a ** 3)
    aims, kinds = [], []          # (body, epoch), frame size class
    for b in np.nonzero(labels == 3)[0][:-1]:
        tp = T0 + np.mod(-M[b], 2 * np.pi) / mm[b]
        if T0 + 8.0 <= tp <= T0 + 357.0:
            aims += [(b, tp + d) for d in (-6.0, -1.5, 0.0, 0.7, 6.0)]; kinds += [0] * 5
    for b, te in zip(np.nonzero(labels == 4)[0], w.meta["t_enc"]):
        aims += [(b, T0 + te + d) for d in (-2.0, -0.4, -0.05, 0.0, 0.03, 0.3, 1.5)]; kinds += [1] * 7
    for b in np.nonzero(labels == 2)[0]:
        aims += [(b, t) for t in rng.uniform(T0 + 5.0, T0 + 360.0, 2)]; kinds += [0] * 2
    aims += [(n - 1, t_peri + d) for d in (-3.0, -0.5, -0.1, -0.02, 0.0, 0.02, 0.1, 0.6, 3.0)]
    kinds += [2] * 9
    other = np.nonzero(labels <= 1)[0]
    for b in rng.choice(other, 60, replace=False):
        aims += [(b, rng.uniform(T0 + 5.0, T0 + 360.0))]; kinds += [0]
    body = np.array([x[0] for x in aims]); ep = np.array([x[1] for x in aims]); kinds = np.array(kinds)
    order = np.argsort(ep, kind="stable")
    body, ep, kinds = body[order], ep[order], kinds[order]
    pl = integrate_planets(ps, ep)
    hp, _ = elements_to_state(a[body], e[body], i[body], om[body], w_[body],
                              M[body] + mm[body] * (ep - T0), GM_SUN)
    d = hp.T + pl[:, 0, :3] - pl[:, 3, :3]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    size = np.where(kinds == 1, rng.uniform(0.1, 0.3, len(ep)),
                    np.where(kinds == 2, rng.uniform(0.01, 0.02, len(ep)),
                             rng.uniform(0.005, 0.012, len(ep))))
    # offset the centre from the aim point by up to 0.3 of the size
    t1 = np.cross(d, rng.normal(size=d.shape)); t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    off = size * rng.uniform(0.0, 0.3, len(ep))
    cen = d * np.cos(off)[:, None] + t1 * np.sin(off)[:, None]
    e_ax = np.cross(cen, rng.normal(size=d.shape))
    normals = square_normals(cen, e_ax, 0.0)
    for k in range(len(ep)):
        normals[k] = square_normals(cen[k], e_ax[k], size[k])
    fr = _frames_array(ep, np.arange(len(ep)), np.arange(len(ep)), normals)
    cone = np.arange(len(ep)) % 2 == 1
    fr["n_edges"][cone] = 0
    fr["normals"][cone] = 0.0
    fr["normals"][cone, 0, :] = cen[cone]
    fr["normals"][cone, 1, 0] = size[cone]
    out = Workload("fov_edge", seed, w.ephem, states, np.full(n, T0), fr, pl[:, 3, :3].copy(),
                   T0 + 365.0, labels)
    out.meta.update(aim_body=body, sungrazer=n - 1, t_enc=w.meta["t_enc"])
    return out


OBS_DTYPE = np.dtype([("epoch", "<f8"), ("ra", "<f8"), ("dec", "<f8"), ("obs", "<f8", (3,))])
assert OBS_DTYPE.itemsize == 48


def backward_catalogue(n_bodies=20_000, years=50.0, seed=None, neo_frac=0.02):
    """Whole-catalogue backward propagation (the pre-discovery use: every
    numbered body carried back decades to an old plate epoch): wise1y's
    population at T0 propagated to T0 - years (365.25-day years); the table
    spans [T0 - years - 64 d, T0 + 64 d]."""
    seed = SEED_BASE + 1 if seed is None else seed
    ps = make_planets(seed)
    n_neo = int(round(neo_frac * n_bodies))
    states, labels = population(seed, ps, n_bodies - n_neo, n_neo)
    t_end = T0 - 365.25 * years
    eph = build_ephemeris(ps, t_end - 64.0, T0 + 64.0)
    return Workload("backward", seed, eph, states, np.full(n_bodies, T0),
                    np.zeros(0, FRAME_DTYPE), np.zeros((0, 3)), t_end, labels)


# elements of the nominal Jupiter-family comet of the clone workload (a
# 103P-like orbit: q ~ 1.06 AU, aphelion near Jupiter's orbit)
CLONE_ELEMENTS = dict(a=3.47, e=0.694, inc=13.6, node=219.8, peri=181.3, M=0.0)


def clones(n_clones=1000, years=170.0, seed=None):
    """Monte-Carlo clones of one Jupiter-family comet propagated back over
    centuries (the orbital-evolution use): the nominal orbit CLONE_ELEMENTS
    (at perihelion at T0) plus Gaussian state offsets, sigma 1e-6 AU and
    1e-8 AU/day per axis (a stand-in for a fit covariance); every clone
    carries the JPL comet model with comet g(r), A1 = 1e-8 and A2 = 5e-10
    AU/day^2 scattered by 5 % (meta['nongrav']).  Propagated to
    T0 - years."""
    seed = SEED_BASE + 11 if seed is None else seed
    ps = make_planets(seed)
    el = CLONE_ELEMENTS
    r, v = elements_to_state(np.array([el["a"]]), np.array([el["e"]]), math.radians(el["inc"]),
                             math.radians(el["node"]), math.radians(el["peri"]), el["M"],
                             GM_SUN)
    nominal = np.concatenate([r[:, 0] + ps.pos0[0], v[:, 0] + ps.vel0[0]])
    rng = _rng(seed, 12)
    states = nominal[:, None] + np.concatenate(
        [rng.normal(0.0, 1e-6, (3, n_clones)), rng.normal(0.0, 1e-8, (3, n_clones))])
    ng = np.zeros(n_clones, NONGRAV_DTYPE)
    ng["alpha"], ng["r0"], ng["m"], ng["n"], ng["k"] = 0.1112620426, 2.808, 2.15, 5.093, 4.6142
    ng["a1"] = 1e-8 * (1.0 + 0.05 * rng.normal(size=n_clones))
    ng["a2"] = 5e-10 * (1.0 + 0.05 * rng.normal(size=n_clones))
    t_end = T0 - 365.25 * years
    eph = build_ephemeris(ps, t_end - 64.0, T0 + 64.0)
    w = Workload("clones", seed, eph, states, np.full(n_clones, T0), np.zeros(0, FRAME_DTYPE),
                 np.zeros((0, 3)), t_end, np.full(n_clones, 3, np.int8))
    w.meta["nongrav"] = ng
    w.meta["nominal"] = nominal
    return w


MAG_DTYPE = np.dtype([("kind", "<i4"), ("reserved", "<i4"), ("p1", "<f8"), ("p2", "<f8")])
assert MAG_DTYPE.itemsize == 24


def mag_params(labels, seed=SEED_BASE + 7):
    """Magnitude models per body: asteroids H ~ U[10, 20], G ~ U[0.05, 0.35]
    (H-G); comets (label 3) alternately total (M1 ~ U[5, 15], K1 ~ U[5, 15])
    and nucleus (M2, K2 alike) magnitudes; every 50th body none."""
    labels = np.asarray(labels)
    rng = _rng(seed, 8)
    n = labels.size
    out = np.zeros(n, MAG_DTYPE)
    out["kind"] = 1
    out["p1"] = rng.uniform(10.0, 20.0, n)
    out["p2"] = rng.uniform(0.05, 0.35, n)
    com = np.nonzero(labels == 3)[0]
    out["kind"][com] = np.where(np.arange(com.size) % 2 == 0, 2, 3)
    out["p1"][com] = rng.uniform(5.0, 15.0, com.size)
    out["p2"][com] = rng.uniform(5.0, 15.0, com.size)
    out["kind"][::50] = 0
    return out


NONGRAV_DTYPE = np.dtype([(f, "<f8") for f in ("a1", "a2", "a3", "alpha", "r0", "m", "n", "k",
                                                "dt", "beta")])
assert NONGRAV_DTYPE.itemsize == 80


def nongrav_params(labels, seed=SEED_BASE + 9, dust_frac=0.0, yarkovsky_every=10):
    """Non-gravitational terms per body (kete_nongrav records).
    Comets (label 3): JPL comet model with the comet g(r) (alpha 0.1112620426,
    r0 2.808 AU, m 2.15, n 5.093, k 4.6142), A1 ~ logU[1e-9, 1e-7] AU/d^2,
    A2 = +-logU[1e-10, 1e-8], A3 ~ N(0, 1e-9); half of them with a thermal
    lag dt ~ U[5, 40] d.  Every `yarkovsky_every`-th other body: a transverse
    A2 ~ N(0, 1e-13) with g = 1/r^2 (asteroid defaults).  A `dust_frac` share
    of the rest: radiation pressure beta ~ logU[1e-3, 0.1]."""
    labels = np.asarray(labels)
    n = labels.size
    rng = _rng(seed, 9)
    out = np.zeros(n, NONGRAV_DTYPE)
    com = np.nonzero(labels == 3)[0]
    out["alpha"][com], out["r0"][com], out["m"][com] = 0.1112620426, 2.808, 2.15
    out["n"][com], out["k"][com] = 5.093, 4.6142
    out["a1"][com] = 10.0 ** rng.uniform(-9.0, -7.0, com.size)
    out["a2"][com] = np.where(rng.uniform(size=com.size) < 0.5, -1.0, 1.0) \
        * 10.0 ** rng.uniform(-10.0, -8.0, com.size)
    out["a3"][com] = rng.normal(0.0, 1e-9, com.size)
    lag = rng.uniform(5.0, 40.0, com.size)
    out["dt"][com] = np.where(np.arange(com.size) % 2 == 0, lag, 0.0)
    rest = np.nonzero(labels != 3)[0]
    yk = rest[::yarkovsky_every] if yarkovsky_every else rest[:0]
    out["alpha"][yk], out["r0"][yk], out["m"][yk], out["n"][yk] = 1.0, 1.0, 2.0, 1.0
    out["a2"][yk] = rng.normal(0.0, 1e-13, yk.size)
    others = np.setdiff1d(rest, yk)
    dust = others[rng.uniform(size=others.size) < dust_frac]
    out["beta"][dust] = 10.0 ** rng.uniform(-3.0, -1.0, dust.size)
    return out


def adjoint90(n_bodies=100_000, n_obs=20, days=90.0, seed=None, neo_frac=0.02):
    """Orbit-fit inputs: bodies drawn as in wise1y, n_obs observation epochs per
    body ~ U[T0, T0 + days] (sorted) seen from the circular 1-AU observer of
    wise1y, N(0, 0.1 arcsec) noise draws for each (RA cos Dec, Dec), and
    Gaussian offsets (1e-6 AU, 1e-8 AU/day per component) giving the states at
    which the gradient is evaluated.  The observed RA/Dec are left at zero: a
    forward model fills them (truth prediction + noise)."""
    seed = SEED_BASE + 3 if seed is None else seed
    ps = make_planets(seed)
    n_neo = int(round(neo_frac * n_bodies))
    states, labels = population(seed, ps, n_bodies - n_neo, n_neo)
    rng = _rng(seed, 6)
    ep = np.sort(rng.uniform(T0, T0 + days, (n_bodies, n_obs)), axis=1)
    # observer: Sun + unit circle in the ecliptic (Sun interpolated from hourly samples)
    t_s = T0 + np.arange(0, days * 24 + 25) / 24.0
    sun = integrate_planets(ps, t_s)[:, 0, :3]
    flat = ep.ravel()
    sun_at = np.stack([np.interp(flat, t_s, sun[:, c]) for c in range(3)], -1)
    theta = 0.3 + GAUSS_K * (flat - T0)
    obs_pos = sun_at + np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], -1)
    obs = np.zeros((n_bodies, n_obs), OBS_DTYPE)
    obs["epoch"] = ep
    obs["obs"] = obs_pos.reshape(n_bodies, n_obs, 3)
    noise = rng.normal(0.0, math.radians(0.1 / 3600.0), (n_bodies, n_obs, 2))
    off = np.concatenate([rng.normal(0, 1e-6, (3, n_bodies)), rng.normal(0, 1e-8, (3, n_bodies))])
    eph = build_ephemeris(ps, T0 - 64.0, T0 + days + 80.0)
    w = Workload("adjoint90", seed, eph, states, np.full(n_bodies, T0), np.zeros(0, FRAME_DTYPE),
                 np.zeros((0, 3)), T0 + days, labels)
    w.meta.update(obs=obs, noise=noise, offsets=off)
    return w


def propagation_only(name, n_bodies, days, seed_offset, n_neo=0, n_trojan=0, n_comet=0,
                     seed=None):
    seed = SEED_BASE + seed_offset if seed is None else seed
    ps = make_planets(seed)
    n_mb = n_bodies - n_neo - n_trojan - n_comet
    states, labels = population(seed, ps, n_mb, n_neo, n_trojan, n_comet)
    eph = build_ephemeris(ps, T0 - 64.0, T0 + days + 80.0)
    return Workload(name, seed, eph, states, np.full(n_bodies, T0),
                    np.zeros(0, FRAME_DTYPE), np.zeros((0, 3)), T0 + days, labels)
