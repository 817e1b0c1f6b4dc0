"""Thin Python binding of libkete_gpu.so (include/kete.h).

Argument marshalling only: every step of the survey path runs in the CUDA
library.  Tensors are torch CUDA tensors passed by ``data_ptr()``; work is
ordered on the current torch stream of the context's device.  If the library
is missing the binding raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkete_gpu.so")

OK, ERR_BAD_ARG, ERR_EPHEM_SPAN, ERR_CAPACITY, ERR_NO_EPHEM, ERR_CUDA, ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
BODY_OK, BODY_STEP_CAP, BODY_OUT_OF_SPAN, BODY_NONFINITE, BODY_KEPLER_CAP = 0, 1, 2, 3, 4
BODY_ADJ_CAP = 5
ADJ_MAX_OBS, ADJ_MAX_STEPS = 32, 256
FP64, MIXED = 0, 1
PROP_STATIC, PROP_WORK_STEALING = 0, 1
NOALLOC_MAX_BODIES = 65536

EXPORTS = ["kete_create", "kete_destroy", "kete_set_stream", "kete_last_error",
           "kete_force_model_default", "kete_survey_opts_default", "kete_load_ephem",
           "kete_ephem_eval", "kete_propagate", "kete_propagate_stops", "kete_fov_check",
           "kete_get_stats", "kete_propagate_noalloc", "kete_set_propagation", "kete_autotune",
           "kete_adjoint", "kete_fov_check_mag", "kete_propagate_legs",
           "kete_fov_check_extended", "kete_sky_jacobian"]
EXT_MAX_SUB = 64
MAG_NONE, MAG_HG, MAG_COMET_TOTAL, MAG_COMET_NUCLEUS = 0, 1, 2, 3


class KeteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kete error {code}: {msg}")
        self.code = code


class ForceModel(C.Structure):
    _fields_ = [("body_mask", C.c_uint32), ("gr_mask", C.c_uint32), ("j2_mask", C.c_uint32),
                ("precision", C.c_int32), ("j2", C.c_double * 16), ("radius", C.c_double * 16),
                ("pole_ra", C.c_double * 16), ("pole_dec", C.c_double * 16),
                ("eps", C.c_double), ("eps_pc", C.c_double), ("safety", C.c_double),
                ("dt_init", C.c_double), ("max_iter", C.c_int32), ("reserved", C.c_int32),
                ("max_steps", C.c_int64), ("nongrav", C.c_void_p)]


class SurveyOpts(C.Structure):
    _fields_ = [("batch_span", C.c_double), ("twobody_max", C.c_double),
                ("cell_deg", C.c_double), ("mem_budget_gb", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("prop_ms", C.c_double), ("fov_ms", C.c_double), ("total_ms", C.c_double),
                ("steps", C.c_int64), ("rejected", C.c_int64), ("force_evals", C.c_int64),
                ("iterations", C.c_int64), ("n_batches", C.c_int64), ("n_exposures", C.c_int64),
                ("n_candidates", C.c_int64), ("n_hits", C.c_int64), ("prop_launches", C.c_int64),
                ("launches", C.c_int64), ("prep_ms", C.c_double), ("cand_ms", C.c_double),
                ("exact_ms", C.c_double), ("order_ms", C.c_double), ("node_evals", C.c_int64),
                ("prop_kind", C.c_int64), ("prop_block", C.c_int64), ("prop_split", C.c_int64),
                ("prop_budget", C.c_int64), ("deferred", C.c_int64), ("prop_order", C.c_int64),
                ("n_exact", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libkete_gpu.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
        L.kete_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        L.kete_destroy.argtypes = [vp]
        L.kete_destroy.restype = None
        L.kete_set_stream.argtypes = [vp, vp]
        L.kete_last_error.argtypes = [vp]
        L.kete_last_error.restype = C.c_char_p
        L.kete_force_model_default.argtypes = [C.POINTER(ForceModel)]
        L.kete_force_model_default.restype = None
        L.kete_survey_opts_default.argtypes = [C.POINTER(SurveyOpts)]
        L.kete_survey_opts_default.restype = None
        L.kete_load_ephem.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.kete_ephem_eval.argtypes = [vp, vp, i64, C.c_int, vp, vp]
        L.kete_propagate.argtypes = [vp, vp, vp, i64, dbl, C.POINTER(ForceModel), vp]
        L.kete_propagate_stops.argtypes = [vp, vp, vp, i64, C.POINTER(C.c_double), i64,
                                           C.POINTER(ForceModel), vp, vp]
        L.kete_fov_check.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, C.POINTER(ForceModel),
                                     C.POINTER(SurveyOpts), vp, i64, C.POINTER(i64), vp]
        L.kete_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.kete_fov_check_mag.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, C.POINTER(ForceModel),
                                         C.POINTER(SurveyOpts), vp, vp, i64, C.POINTER(i64), vp]
        L.kete_fov_check_extended.argtypes = [vp, vp, vp, i64, vp, i64, vp, C.c_int32, vp, i64,
                                              C.POINTER(ForceModel), C.POINTER(SurveyOpts), vp,
                                              vp, i64, C.POINTER(i64), vp]
        L.kete_propagate_noalloc.argtypes = [vp, vp, vp, i64, dbl, C.POINTER(ForceModel), vp]
        L.kete_propagate_legs.argtypes = [vp, vp, vp, i64, dbl, dbl, C.POINTER(ForceModel), vp]
        L.kete_set_propagation.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                           C.c_int]
        L.kete_autotune.argtypes = [vp, vp, vp, i64, C.POINTER(C.c_double), i64,
                                    C.POINTER(ForceModel), i64, C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.kete_adjoint.argtypes = [vp, vp, vp, i64, vp, C.c_int32, C.POINTER(ForceModel),
                                   C.POINTER(SurveyOpts), dbl, vp, vp, vp, vp]
        L.kete_sky_jacobian.argtypes = [vp, vp, vp, i64, vp, C.c_int32, C.POINTER(ForceModel),
                                        C.POINTER(SurveyOpts), dbl, vp, vp, vp]
        _lib = L
    return _lib


def force_model(**kw) -> ForceModel:
    """Default force model (App. A defaults) with keyword overrides; per-body
    arrays (j2, radius, pole_ra, pole_dec) take {body_index: value} dicts;
    nongrav takes the CUDA tensor of nongrav_to_device (kept alive with the
    model) or None."""
    fm = ForceModel()
    lib().kete_force_model_default(C.byref(fm))
    for k, v in kw.items():
        if k in ("j2", "radius", "pole_ra", "pole_dec"):
            arr = getattr(fm, k)
            for i, x in v.items():
                arr[i] = x
        elif k == "nongrav":
            set_nongrav(fm, v)
        else:
            setattr(fm, k, v)
    return fm


def set_nongrav(fm: ForceModel, t) -> None:
    """Attach per-body non-gravitational terms (nongrav_to_device) to fm."""
    if t is None:
        fm.nongrav = None
        fm._nongrav = None
        return
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.dim() == 2 and t.shape[1] == 10 and t.is_contiguous()):
        raise TypeError("nongrav must be a contiguous CUDA float64 tensor [n, 10] "
                        "(see nongrav_to_device)")
    fm.nongrav = t.data_ptr()
    fm._nongrav = t


def _check_nongrav(fm: ForceModel, n: int) -> None:
    t = getattr(fm, "_nongrav", None)
    if t is not None and (t.shape[0] != n or fm.nongrav != t.data_ptr()):
        raise TypeError(f"the force model's nongrav tensor has {t.shape[0]} rows for {n} bodies")


NONGRAV_FIELDS = ("a1", "a2", "a3", "alpha", "r0", "m", "n", "k", "dt", "beta")


def nongrav_to_device(params, device) -> torch.Tensor:
    """Per-body non-gravitational records (a structured array with the
    kete_nongrav fields) -> CUDA float64 [n, 10].  Set the force model's
    nongrav to its data_ptr() and keep the tensor alive for the call."""
    a = np.stack([np.asarray(params[f], np.float64) for f in NONGRAV_FIELDS], axis=-1)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def survey_opts(**kw) -> SurveyOpts:
    o = SurveyOpts()
    lib().kete_survey_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dev_f64(t, name, shape=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def frames_to_device(frames: np.ndarray, device) -> torch.Tensor:
    """kete_frame records (128 bytes each, numpy structured array) -> CUDA bytes."""
    raw = np.ascontiguousarray(frames).view(np.uint8).reshape(-1)
    return torch.from_numpy(raw.copy()).to(device)


def mag_params_to_device(params: np.ndarray, device) -> torch.Tensor:
    """kete_mag_params records (24 bytes: kind, reserved, p1, p2) -> CUDA bytes."""
    a = np.ascontiguousarray(params)
    if a.dtype.itemsize != 24:
        raise TypeError("magnitude parameters must be 24-byte kete_mag_params records")
    return torch.from_numpy(a.view(np.uint8).reshape(-1).copy()).to(device)


FRAME_CONE = 0
# kete_frame records (128 bytes)
FRAME_DTYPE = np.dtype([
    ("epoch", "<f8"), ("observer_idx", "<i8"), ("exposure_id", "<i8"),
    ("n_edges", "<i4"), ("reserved", "<i4"), ("normals", "<f8", (4, 3)),
])
_OBLIQUITY = math.radians(84381.448 / 3600.0)


def radec_to_vec(ra, dec):
    """Unit vectors (ecliptic J2000, [..., 3]) of equatorial J2000 RA/Dec
    (radians): the inverse of the RA/Dec the library reports."""
    ra, dec = np.asarray(ra, float), np.asarray(dec, float)
    x = np.cos(dec) * np.cos(ra)
    y = np.cos(dec) * np.sin(ra)
    z = np.sin(dec)
    c, s_ = math.cos(_OBLIQUITY), math.sin(_OBLIQUITY)
    return np.stack([x, c * y + s_ * z, -s_ * y + c * z], axis=-1)


def polygon_frame(corners_radec, epoch: float, observer_idx: int, exposure_id: int = 0):
    """A kete_frame record of the spherical polygon (Sec. 3.1) with 3 or 4
    corners given as (RA, Dec) pairs in radians, in either winding order:
    edge k's inward normal is c_k x c_(k+1), turned to face the corners'
    mean direction.  The polygon must be convex and smaller than a
    hemisphere."""
    cr = np.asarray(corners_radec, float).reshape(-1, 2)
    if not 3 <= len(cr) <= 4:
        raise ValueError("a polygon frame has 3 or 4 corners")
    v = radec_to_vec(cr[:, 0], cr[:, 1])
    mean = v.sum(axis=0)
    out = np.zeros(1, FRAME_DTYPE)[0]
    out["epoch"], out["observer_idx"], out["exposure_id"] = epoch, observer_idx, exposure_id
    out["n_edges"] = len(v)
    for k in range(len(v)):
        nk = np.cross(v[k], v[(k + 1) % len(v)])
        out["normals"][k] = nk if nk @ mean > 0 else -nk
    return out


def cone_frame(ra: float, dec: float, radius: float, epoch: float, observer_idx: int,
               exposure_id: int = 0):
    """A kete_frame record of a cone (Sec. 3.1) about (RA, Dec) with angular
    radius `radius` (all radians, 0 < radius < pi)."""
    if not 0.0 < radius < math.pi:
        raise ValueError("the cone's radius must lie in (0, pi)")
    out = np.zeros(1, FRAME_DTYPE)[0]
    out["epoch"], out["observer_idx"], out["exposure_id"] = epoch, observer_idx, exposure_id
    out["n_edges"] = FRAME_CONE
    out["normals"][0] = radec_to_vec(ra, dec)
    out["normals"][1][0] = radius
    return out


def decode_hits(h: torch.Tensor, n: int):
    """kete_hit rows (int64 [n, 4] view) -> dict of CPU tensors."""
    h = h[:n].cpu()
    return {"frame": h[:, 0].clone(),
            "body": (h[:, 1] & 0xFFFFFFFF).to(torch.int32),
            "mag": (h[:, 1] >> 32).to(torch.int32).view(torch.float32),
            "ra": h[:, 2].clone().view(torch.float64),
            "dec": h[:, 3].clone().view(torch.float64)}


class Kete:
    """One library context (device-resident ephemeris + scratch) on one GPU."""

    def __init__(self, device: int = 0):
        self.device = torch.device("cuda", device)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            rc = lib().kete_create(C.byref(self._h), device, C.c_void_p(stream))
        if rc != OK:
            raise KeteError(rc, "kete_create failed")

    def close(self):
        if self._h:
            lib().kete_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        lib().kete_set_stream(self._h, C.c_void_p(s))

    def _check(self, rc):
        if rc != OK:
            raise KeteError(rc, lib().kete_last_error(self._h).decode())

    # -- calls with the ABI's names ------------------------------------------
    def load_ephem(self, table: bytes):
        self._sync_stream()
        self._check(lib().kete_load_ephem(self._h, table, len(table)))

    def ephem_eval(self, t: torch.Tensor, body: int):
        n = t.numel()
        _dev_f64(t, "t")
        pos = torch.empty((n, 3), dtype=torch.float64, device=t.device)
        vel = torch.empty((n, 3), dtype=torch.float64, device=t.device)
        self._sync_stream()
        self._check(lib().kete_ephem_eval(self._h, t.data_ptr(), n, body, pos.data_ptr(),
                                          vel.data_ptr()))
        return pos, vel

    def propagate(self, states, epochs, t_target, fm=None, status=None, leg_days=None):
        """In-place propagation of states [6, n] / epochs [n] to t_target.
        leg_days: go through stops every leg_days days from epochs[0]
        (kete_propagate_legs), so that the bodies share the planets' rows."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        if status is None:
            status = torch.zeros(n, dtype=torch.int32, device=states.device)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        self._sync_stream()
        if leg_days is None:
            self._check(lib().kete_propagate(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                             float(t_target), C.byref(fm), status.data_ptr()))
        else:
            self._check(lib().kete_propagate_legs(self._h, states.data_ptr(), epochs.data_ptr(),
                                                  n, float(t_target), float(leg_days),
                                                  C.byref(fm), status.data_ptr()))
        return status

    def propagate_noalloc(self, states, epochs, t_target, fm=None, status=None):
        """kete_propagate without device allocation (n <= NOALLOC_MAX_BODIES)."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        if status is None:
            status = torch.zeros(n, dtype=torch.int32, device=states.device)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        self._sync_stream()
        self._check(lib().kete_propagate_noalloc(self._h, states.data_ptr(), epochs.data_ptr(),
                                                 n, float(t_target), C.byref(fm),
                                                 status.data_ptr()))
        return status

    def propagate_stops(self, states, epochs, stops, fm=None):
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        st = np.ascontiguousarray(stops, dtype=np.float64)
        out = torch.empty((len(st), 6, n), dtype=torch.float64, device=states.device)
        status = torch.zeros(n, dtype=torch.int32, device=states.device)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        self._sync_stream()
        self._check(lib().kete_propagate_stops(
            self._h, states.data_ptr(), epochs.data_ptr(), n,
            st.ctypes.data_as(C.POINTER(C.c_double)), len(st), C.byref(fm), out.data_ptr(),
            status.data_ptr()))
        return out, status

    def fov_check(self, states, epochs, frames_dev, observers, fm=None, opts=None,
                  capacity=None, hits=None, mag_params=None):
        """Which bodies fall inside which FoV.  Returns (hits int64 [cap, 4],
        n_hits, status).  Grows the hit buffer once if it was too small.
        mag_params (CUDA bytes of n kete_mag_params, see mag_params_to_device):
        also give every hit its apparent magnitude (kete_fov_check_mag)."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        _dev_f64(observers, "observers")
        if not (frames_dev.is_cuda and frames_dev.dtype == torch.uint8 and frames_dev.numel() % 128 == 0):
            raise TypeError("frames must be a CUDA uint8 tensor of 128-byte kete_frame records")
        nf = frames_dev.numel() // 128
        n_obs = observers.numel() // 3
        fm = fm or force_model()
        _check_nongrav(fm, n)
        opts = opts or survey_opts()
        status = torch.zeros(n, dtype=torch.int32, device=states.device)
        if hits is None:
            cap = capacity if capacity is not None else max(1024, 4 * nf)
            hits = torch.empty((cap, 4), dtype=torch.int64, device=states.device)
        nh = C.c_int64(0)
        self._sync_stream()
        for attempt in range(2):
            if mag_params is None:
                rc = lib().kete_fov_check(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                          frames_dev.data_ptr(), nf, observers.data_ptr(), n_obs,
                                          C.byref(fm), C.byref(opts), hits.data_ptr(),
                                          hits.shape[0], C.byref(nh), status.data_ptr())
            else:
                if not (mag_params.is_cuda and mag_params.numel() == 24 * n):
                    raise TypeError("mag_params must hold n kete_mag_params records on the GPU")
                rc = lib().kete_fov_check_mag(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                              frames_dev.data_ptr(), nf, observers.data_ptr(),
                                              n_obs, C.byref(fm), C.byref(opts),
                                              mag_params.data_ptr(), hits.data_ptr(),
                                              hits.shape[0], C.byref(nh), status.data_ptr())
            if rc == ERR_CAPACITY and attempt == 0:
                hits = torch.empty((nh.value + 1024, 4), dtype=torch.int64, device=states.device)
                continue
            self._check(rc)
            break
        return hits, nh.value, status

    def fov_check_extended(self, states, epochs, frames_dev, durations, n_sub, observers,
                           fm=None, opts=None, capacity=None, hits=None, mag_params=None):
        """kete_fov_check_extended: frames are exposures starting at their
        epoch and lasting durations[f] days (CUDA float64 [n_frames]), each
        split into n_sub sub-frames seen from observer rows observer_idx + k.
        Returns (hits int64 [cap, 4], n_hits, status) with one hit per
        (frame, body), as fov_check."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        _dev_f64(observers, "observers")
        if not (frames_dev.is_cuda and frames_dev.dtype == torch.uint8 and frames_dev.numel() % 128 == 0):
            raise TypeError("frames must be a CUDA uint8 tensor of 128-byte kete_frame records")
        nf = frames_dev.numel() // 128
        _dev_f64(durations, "durations", (nf,))
        if mag_params is not None and not (mag_params.is_cuda and mag_params.numel() == 24 * n):
            raise TypeError("mag_params must hold n kete_mag_params records on the GPU")
        fm = fm or force_model()
        _check_nongrav(fm, n)
        opts = opts or survey_opts()
        status = torch.zeros(n, dtype=torch.int32, device=states.device)
        if hits is None:
            cap = capacity if capacity is not None else max(1024, 4 * nf)
            hits = torch.empty((cap, 4), dtype=torch.int64, device=states.device)
        nh = C.c_int64(0)
        self._sync_stream()
        for attempt in range(2):
            rc = lib().kete_fov_check_extended(
                self._h, states.data_ptr(), epochs.data_ptr(), n, frames_dev.data_ptr(), nf,
                durations.data_ptr(), int(n_sub), observers.data_ptr(), observers.numel() // 3,
                C.byref(fm), C.byref(opts), None if mag_params is None else mag_params.data_ptr(),
                hits.data_ptr(), hits.shape[0], C.byref(nh), status.data_ptr())
            if rc == ERR_CAPACITY and attempt == 0:
                hits = torch.empty((nh.value + 1024, 4), dtype=torch.int64, device=states.device)
                continue
            self._check(rc)
            break
        return hits, nh.value, status

    def adjoint(self, states, epochs, obs, fm=None, opts=None, ckpt_days=8.0, grad=True,
                pred=False):
        """Orbit-fit loss per body and, with grad, dL/d(x0, v0) [6, n].

        obs: float64 CUDA tensor [n, m, 6] of kete_obs records (epoch, ra, dec,
        observer x, y, z), sorted by epoch per body, NaN epochs padding the
        end of a row.  Returns (loss [n], grad [6, n] or None, pred [n, m, 2]
        or None, status [n])."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        if obs.dim() != 3 or obs.shape[0] != n or obs.shape[2] != 6:
            raise ValueError("obs must have shape [n, m, 6]")
        m = obs.shape[1]
        _dev_f64(obs, "obs")
        dev = states.device
        loss = torch.empty(n, dtype=torch.float64, device=dev)
        g = torch.empty((6, n), dtype=torch.float64, device=dev) if grad else None
        pr = torch.empty((n, m, 2), dtype=torch.float64, device=dev) if pred else None
        status = torch.zeros(n, dtype=torch.int32, device=dev)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        opts = opts or survey_opts()
        self._sync_stream()
        self._check(lib().kete_adjoint(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                       obs.data_ptr(), m, C.byref(fm), C.byref(opts),
                                       float(ckpt_days), loss.data_ptr(),
                                       g.data_ptr() if g is not None else None,
                                       pr.data_ptr() if pr is not None else None,
                                       status.data_ptr()))
        return loss, g, pr, status

    def sky_jacobian(self, states, epochs, obs, fm=None, opts=None, ckpt_days=8.0, pred=False):
        """Per-observation sky partials (kete_sky_jacobian): jac [n, m, 2, 6] =
        d(RA, Dec)/d(x0, v0) of every observation, obs as for adjoint (its
        observed RA/Dec are not used).  Returns (jac, pred [n, m, 2] or None,
        status [n])."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        if obs.dim() != 3 or obs.shape[0] != n or obs.shape[2] != 6:
            raise ValueError("obs must have shape [n, m, 6]")
        m = obs.shape[1]
        _dev_f64(obs, "obs")
        dev = states.device
        jac = torch.empty((n, m, 2, 6), dtype=torch.float64, device=dev)
        pr = torch.empty((n, m, 2), dtype=torch.float64, device=dev) if pred else None
        status = torch.zeros(n, dtype=torch.int32, device=dev)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        opts = opts or survey_opts()
        self._sync_stream()
        self._check(lib().kete_sky_jacobian(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                            obs.data_ptr(), m, C.byref(fm), C.byref(opts),
                                            float(ckpt_days), jac.data_ptr(),
                                            pr.data_ptr() if pr is not None else None,
                                            status.data_ptr()))
        return jac, pr, status

    def set_propagation(self, precision: int, kind: int, block: int = 128, split: int = 0,
                        defer_steps: int = 0, cost_order: bool = True):
        self._check(lib().kete_set_propagation(self._h, precision, kind, block, split,
                                               defer_steps, 1 if cost_order else 0))

    def autotune(self, states, epochs, stops, fm=None, max_sample=32768):
        """Time the propagation launch variants on a body sample; keep the fastest."""
        n = epochs.numel()
        _dev_f64(states, "states", (6, n)); _dev_f64(epochs, "epochs", (n,))
        st = np.ascontiguousarray(stops, dtype=np.float64)
        fm = fm or force_model()
        _check_nongrav(fm, n)
        kind, block, split, defer, order = (C.c_int32() for _ in range(5))
        self._sync_stream()
        self._check(lib().kete_autotune(self._h, states.data_ptr(), epochs.data_ptr(), n,
                                        st.ctypes.data_as(C.POINTER(C.c_double)), len(st),
                                        C.byref(fm), max_sample, C.byref(kind), C.byref(block),
                                        C.byref(split), C.byref(defer), C.byref(order)))
        return kind.value, block.value, split.value, defer.value, order.value

    def get_stats(self) -> dict:
        s = Stats()
        self._check(lib().kete_get_stats(self._h, C.byref(s)))
        return s.as_dict()


class OrbitFitLoss(torch.autograd.Function):
    """Per-body orbit-fit loss as a differentiable function of the initial
    states [6, n]; the backward pass returns the adjoint gradient computed by
    kete_adjoint in the same call as the loss."""

    @staticmethod
    def forward(ctx, states, engine, epochs, obs, fm=None, opts=None, ckpt_days=8.0):
        loss, g, _, status = engine.adjoint(states.detach().contiguous(), epochs, obs, fm=fm,
                                            opts=opts, ckpt_days=ckpt_days, grad=True)
        ctx.save_for_backward(g)
        ctx.mark_non_differentiable(status)
        return loss, status

    @staticmethod
    def backward(ctx, grad_loss, grad_status):
        (g,) = ctx.saved_tensors
        return g * grad_loss.unsqueeze(0), None, None, None, None, None, None


def orbit_fit_loss(engine, states, epochs, obs, fm=None, opts=None, ckpt_days=8.0):
    """Differentiable per-body loss [n] (and status) of initial states [6, n]."""
    return OrbitFitLoss.apply(states, engine, epochs, obs, fm, opts, ckpt_days)
