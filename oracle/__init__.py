"""ctypes loader for the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and
its binding) never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kete_oracle.c")
LIB = os.path.join(HERE, "libkete_oracle.so")

OK, STEP_CAP, OUT_OF_SPAN, NONFINITE, KEPLER_FAIL = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "kete_oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Ephem(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("n_coef", C.c_int), ("n_seg", C.c_int),
                ("t_start", C.c_double), ("seg_len", C.c_double),
                ("gm", C.c_double * 16), ("coef", C.POINTER(C.c_double))]


class NonGrav(C.Structure):
    """ko_nongrav: beta (Eq. A.6); a1..a3, alpha, r0, m, n, k, dt (Eq. A.7)."""
    _fields_ = [(f, C.c_double) for f in ("a1", "a2", "a3", "alpha", "r0", "m", "n", "k",
                                          "dt", "beta")]


NG_FIELDS = ("a1", "a2", "a3", "alpha", "r0", "m", "n", "k", "dt", "beta")
NG_DTYPE = np.dtype([(f, "<f8") for f in NG_FIELDS])


def comet_ng(a1=0.0, a2=0.0, a3=0.0, dt=0.0):
    """JPL comet model with its default g(r) (App. A.5)."""
    return NonGrav(a1, a2, a3, 0.1112620426, 2.808, 2.15, 5.093, 4.6142, dt, 0.0)


def asteroid_ng(a1=0.0, a2=0.0, a3=0.0, dt=0.0):
    """The same model with the asteroid defaults, g(r) = 1/r^2 (App. A.5)."""
    return NonGrav(a1, a2, a3, 1.0, 1.0, 2.0, 1.0, 0.0, dt, 0.0)


def dust_ng(beta):
    """Radiation pressure with Poynting-Robertson drag (Eq. A.6)."""
    return NonGrav(0, 0, 0, 0, 1.0, 0, 0, 0, 0, beta)


def _ng_array(ng, n):
    """Per-body non-gravitational records (any array with NG_FIELDS) -> ko_nongrav[n]."""
    if ng is None:
        return None
    out = np.zeros(n, NG_DTYPE)
    for f in NG_FIELDS:
        out[f] = ng[f]
    return out


class ForceModel(C.Structure):
    _fields_ = [("body_mask", C.c_uint32), ("gr_mask", C.c_uint32), ("j2_mask", C.c_uint32),
                ("max_iter", C.c_int32), ("j2", C.c_double * 16), ("radius", C.c_double * 16),
                ("pole_ra", C.c_double * 16), ("pole_dec", C.c_double * 16),
                ("eps", C.c_double), ("eps_pc", C.c_double), ("safety", C.c_double),
                ("dt_init", C.c_double), ("max_steps", C.c_int64), ("ng", NonGrav)]


class SurveyOpts(C.Structure):
    _fields_ = [("batch_span", C.c_double), ("twobody_max", C.c_double),
                ("prefilter_deg", C.c_double)]


class Mag(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("p1", C.c_double), ("p2", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rejected", C.c_int64), ("force_evals", C.c_int64),
                ("iterations", C.c_int64)]


OBS_DTYPE = np.dtype([("epoch", "<f8"), ("ra", "<f8"), ("dec", "<f8"), ("obs", "<f8", (3,))])
assert OBS_DTYPE.itemsize == 48

HIT_DTYPE = np.dtype([("frame", "<i8"), ("body", "<i4"), ("status", "<i4"), ("ra", "<f8"),
                      ("dec", "<f8"), ("margin", "<f8"), ("tau", "<f8")])

_lib = None


def lib():
    """The oracle library: built from kete_oracle.c, or the prebuilt library
    named by the environment variable KETE_ORACLE_LIB (the planted-mistake
    tests point it at mutated copies built elsewhere)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("KETE_ORACLE_LIB") or build())
        d = C.POINTER(C.c_double)
        L.ko_ephem_load.argtypes = [C.POINTER(Ephem), C.c_void_p, C.c_size_t]
        L.ko_ephem_eval.argtypes = [C.POINTER(Ephem), C.c_int, C.c_double, d, d]
        L.ko_force_model_default.argtypes = [C.POINTER(ForceModel)]
        L.ko_radau_nodes.argtypes = [d]
        L.ko_accel.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), C.c_double, d, d, d]
        L.ko_propagate.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, d, C.c_double, d,
                                   C.POINTER(Stats)]
        L.ko_propagate_stops.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, C.c_double,
                                         d, C.c_int64, d, C.POINTER(Stats)]
        L.ko_propagate_many.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, d, C.c_int64,
                                        C.c_double, C.c_void_p, C.c_int, C.POINTER(Stats),
                                        C.c_void_p]
        L.ko_ephem_delta.argtypes = [C.POINTER(Ephem), C.c_int, C.c_double, C.c_double, d]
        L.ko_find_close.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), C.c_double, d,
                                    C.c_double, C.POINTER(C.c_int), d, d]
        L.ko_stumpff.argtypes = [C.c_double, d, d]
        L.ko_kepler.argtypes = [C.c_double, d, d, C.c_double, d, d]
        L.ko_apparent.argtypes = [C.POINTER(Ephem), d, C.c_double, C.c_double, d, d, d]
        L.ko_radec.argtypes = [d, d, d]
        L.ko_magnitude.argtypes = [C.POINTER(Ephem), d, C.c_double, C.c_double, d,
                                   C.POINTER(Mag), d, d, d, d]
        L.ko_in_polygon.argtypes = [C.c_void_p, d, d]
        L.ko_make_batches.argtypes = [d, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.ko_make_batches.restype = C.c_int64
        L.ko_body_loss.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, C.c_double,
                                   C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, d,
                                   C.c_void_p, C.c_void_p]
        L.ko_body_sky_jacobian.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, C.c_double,
                                           C.c_void_p, C.c_int, C.c_double, C.c_double,
                                           C.c_double, d, d]
        L.ko_propagate_stm.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, d, d,
                                       C.c_double, d, C.POINTER(Stats)]
        L.ko_fov_check.argtypes = [C.POINTER(Ephem), C.POINTER(ForceModel), d, d, C.c_int64,
                                   C.c_void_p, C.c_int64, d, C.c_int64, C.POINTER(SurveyOpts),
                                   C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_int64), C.c_void_p, C.c_int, C.POINTER(Stats),
                                   C.c_void_p]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """Convenience wrapper holding one loaded ephemeris table."""

    def __init__(self, ephem_bytes: bytes):
        self._buf = bytes(ephem_bytes)
        self.eph = Ephem()
        rc = lib().ko_ephem_load(C.byref(self.eph), self._buf, len(self._buf))
        if rc != 0:
            raise ValueError("oracle: bad ephemeris table")

    def __del__(self):
        try:
            if _lib is not None and self.eph.coef:
                _lib.ko_ephem_free(C.byref(self.eph))
        except Exception:
            pass

    # -- force model ---------------------------------------------------------
    @staticmethod
    def force_model(**kw) -> ForceModel:
        fm = ForceModel()
        lib().ko_force_model_default(C.byref(fm))
        for k, v in kw.items():
            if k in ("j2", "radius", "pole_ra", "pole_dec"):
                arr = getattr(fm, k)
                for i, x in v.items():
                    arr[i] = x
            else:
                setattr(fm, k, v)
        return fm

    def ephem(self, body, t):
        p = np.zeros(3); v = np.zeros(3)
        rc = lib().ko_ephem_eval(C.byref(self.eph), body, t, _dp(p), _dp(v))
        return rc, p, v

    def ephem_delta(self, body, t0, off):
        """p(t0 + off) - p(t0) of table body `body` from the segment holding t0
        (the close-encounter displacement, reading R12)."""
        dp = np.zeros(3)
        rc = lib().ko_ephem_delta(C.byref(self.eph), body, t0, off, _dp(dp))
        return rc, dp

    def find_close(self, fm, t, x, t_target):
        """Encounter set-up at a step start (R12): (rc, planet index or -1,
        x - p_m(t), end of the step range)."""
        m = C.c_int(-2); d0 = np.zeros(3); ts = C.c_double(0.0)
        x = np.ascontiguousarray(x, float)
        rc = lib().ko_find_close(C.byref(self.eph), C.byref(fm), t, _dp(x), t_target, C.byref(m),
                                 _dp(d0), C.byref(ts))
        return rc, m.value, d0, ts.value

    def accel(self, fm, t, x, v):
        a = np.zeros(3)
        x = np.ascontiguousarray(x, float); v = np.ascontiguousarray(v, float)
        rc = lib().ko_accel(C.byref(self.eph), C.byref(fm), t, _dp(x), _dp(v), _dp(a))
        return rc, a

    def propagate(self, fm, state, t, t_target, dt=0.0):
        st = np.ascontiguousarray(state, float).copy()
        tt = C.c_double(t); dd = C.c_double(dt); stats = Stats()
        rc = lib().ko_propagate(C.byref(self.eph), C.byref(fm), _dp(st), C.byref(tt), t_target,
                                C.byref(dd), C.byref(stats))
        return rc, st, tt.value, dd.value, stats

    def propagate_stops(self, fm, state, epoch, stops):
        st = np.ascontiguousarray(state, float)
        stops = np.ascontiguousarray(stops, float)
        out = np.zeros((len(stops), 6)); stats = Stats()
        rc = lib().ko_propagate_stops(C.byref(self.eph), C.byref(fm), _dp(st), epoch,
                                      _dp(stops), len(stops), _dp(out), C.byref(stats))
        return rc, out, stats

    def propagate_many(self, fm, states, epochs, t_target, n_threads=None, nongrav=None):
        st = np.ascontiguousarray(states, float).copy()
        ep = np.ascontiguousarray(epochs, float).copy()
        n = ep.size
        status = np.zeros(n, np.int32); stats = Stats()
        ng = _ng_array(nongrav, n)
        lib().ko_propagate_many(C.byref(self.eph), C.byref(fm), _dp(st), _dp(ep), n, t_target,
                                status.ctypes.data, n_threads or os.cpu_count(), C.byref(stats),
                                None if ng is None else ng.ctypes.data)
        return st, ep, status, stats

    def apparent(self, st_ref, t_ref, t_obs, obs):
        st = np.ascontiguousarray(st_ref, float); o = np.ascontiguousarray(obs, float)
        u = np.zeros(3); tau = C.c_double()
        rc = lib().ko_apparent(C.byref(self.eph), _dp(st), t_ref, t_obs, _dp(o), _dp(u),
                               C.byref(tau))
        return rc, u, tau.value

    def magnitude(self, st_ref, t_ref, t_obs, obs, kind, p1, p2):
        """(rc, mag, r_h, delta, alpha_deg) of a body seen at t_obs from obs."""
        st = np.ascontiguousarray(st_ref, float); o = np.ascontiguousarray(obs, float)
        out = [C.c_double() for _ in range(4)]
        rc = lib().ko_magnitude(C.byref(self.eph), _dp(st), t_ref, t_obs, _dp(o),
                                C.byref(Mag(kind, 0, p1, p2)), *[C.byref(x) for x in out])
        return (rc,) + tuple(x.value for x in out)

    def propagate_stm(self, fm, state, t, t_target, dt=0.0):
        st = np.ascontiguousarray(state, float).copy()
        phi = np.eye(6).ravel().copy()
        tt = C.c_double(t); dd = C.c_double(dt); stats = Stats()
        rc = lib().ko_propagate_stm(C.byref(self.eph), C.byref(fm), _dp(st), _dp(phi), C.byref(tt),
                                    t_target, C.byref(dd), C.byref(stats))
        return rc, st, phi.reshape(6, 6), tt.value, dd.value, stats

    def body_loss(self, fm, state, epoch, obs, batch_span=3.0, twobody_max=1.5, ckpt_days=8.0,
                  grad=True):
        """Loss of one body's observations; (rc, loss, pred [m,2], grad [6] or None)."""
        st = np.ascontiguousarray(state, float)
        ob = np.ascontiguousarray(obs, OBS_DTYPE)
        loss = C.c_double()
        pred = np.zeros((len(ob), 2))
        g = np.zeros(6)
        rc = lib().ko_body_loss(C.byref(self.eph), C.byref(fm), _dp(st), epoch, ob.ctypes.data,
                                len(ob), batch_span, twobody_max, ckpt_days, C.byref(loss),
                                pred.ctypes.data, g.ctypes.data if grad else None)
        return rc, loss.value, pred, (g if grad else None)

    def sky_jacobian(self, fm, state, epoch, obs, batch_span=3.0, twobody_max=1.5,
                     ckpt_days=8.0):
        """Per-observation sky partials of one body: (rc, jac [m, 2, 6] =
        d(RA, Dec)/d(x0, v0), pred [m, 2])."""
        st = np.ascontiguousarray(state, float)
        ob = np.ascontiguousarray(obs, OBS_DTYPE)
        pred = np.zeros((len(ob), 2))
        jac = np.zeros((len(ob), 2, 6))
        rc = lib().ko_body_sky_jacobian(C.byref(self.eph), C.byref(fm), _dp(st), epoch,
                                        ob.ctypes.data, len(ob), batch_span, twobody_max,
                                        ckpt_days, pred.ctypes.data_as(C.POINTER(C.c_double)),
                                        jac.ctypes.data_as(C.POINTER(C.c_double)))
        return rc, jac, pred

    def fov_check(self, fm, states, epochs, frames, observers, batch_span=3.0, twobody_max=1.5,
                  prefilter_deg=0.0, subset=None, n_threads=None, nongrav=None):
        st = np.ascontiguousarray(states, float)
        ep = np.ascontiguousarray(epochs, float)
        fr = np.ascontiguousarray(frames)
        ob = np.ascontiguousarray(observers, float).reshape(-1, 3)
        n = ep.size
        opts = SurveyOpts(batch_span, twobody_max, prefilter_deg)
        sub = None if subset is None else np.ascontiguousarray(subset, np.int32)
        status = np.zeros(n, np.int32)
        nh = C.c_int64(0); stats = Stats()
        args = [C.byref(self.eph), C.byref(fm), _dp(st), _dp(ep), n, fr.ctypes.data, len(fr),
                _dp(ob), len(ob), C.byref(opts), None if sub is None else sub.ctypes.data,
                0 if sub is None else len(sub)]
        nt = n_threads or os.cpu_count()
        ng = _ng_array(nongrav, n)
        cap = 0
        hits = np.zeros(1, HIT_DTYPE)
        for _ in range(2):
            rc = lib().ko_fov_check(*args, hits.ctypes.data, cap, C.byref(nh), status.ctypes.data,
                                    nt, C.byref(stats), None if ng is None else ng.ctypes.data)
            if rc == 0:
                return hits[: nh.value].copy(), status, stats
            cap = nh.value
            hits = np.zeros(max(cap, 1), HIT_DTYPE)
            stats = Stats()
        raise RuntimeError("oracle fov_check failed")


def stumpff(z):
    c2 = C.c_double(); c3 = C.c_double()
    lib().ko_stumpff(z, C.byref(c2), C.byref(c3))
    return c2.value, c3.value


def kepler(mu, r0, v0, dt):
    r0 = np.ascontiguousarray(r0, float); v0 = np.ascontiguousarray(v0, float)
    r = np.zeros(3); v = np.zeros(3)
    rc = lib().ko_kepler(mu, _dp(r0), _dp(v0), dt, _dp(r), _dp(v))
    return rc, r, v


def radau_nodes():
    h = np.zeros(8)
    lib().ko_radau_nodes(_dp(h))
    return h


def radec(u):
    u = np.ascontiguousarray(u, float)
    ra = C.c_double(); dec = C.c_double()
    lib().ko_radec(_dp(u), C.byref(ra), C.byref(dec))
    return ra.value, dec.value


def in_polygon(frame, u):
    fr = np.ascontiguousarray(np.asarray(frame).reshape(1))
    u = np.ascontiguousarray(u, float)
    m = C.c_double()
    inside = lib().ko_in_polygon(fr.ctypes.data, _dp(u), C.byref(m))
    return bool(inside), m.value


def make_batches(epochs_sorted, batch_span=3.0, twobody_max=1.5):
    ep = np.ascontiguousarray(epochs_sorted, float)
    bs = np.zeros(max(ep.size, 1), np.int64); tr = np.zeros(max(ep.size, 1))
    nb = lib().ko_make_batches(_dp(ep), ep.size, batch_span, twobody_max, bs.ctypes.data,
                               tr.ctypes.data)
    return bs[:nb].copy(), tr[:nb].copy()
