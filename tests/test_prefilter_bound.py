"""The error bound of k_exact's FP32 prefilter, restated: the distance between
the prefilter's prediction -- a second-order Taylor step of the body's
heliocentric batch state to the exposure epoch, retarded by the light time in
FP32 -- and the exact position the exact path uses (the oracle's universal-
variable two-body solution at t - tau, tau iterated to convergence) stays
below E = 1.001 (J s^3/6 + a_max tau_max^2/2 + 2e-6 (|r| + |sun - o| + |u| +
|v| |dt|)) + 1e-9 AU, with r_min = |r|/2, a_max = mu / r_min^2, v_max = |v| +
a_max s, J = 4 mu v_max / r_min^3, s = |dt| + tau_max.  Checked on the mixed
ragged population (main belt, NEOs with forced Earth encounters, Trojans,
comets) with random observers near 1 AU and |dt| up to the two-body limit."""
import numpy as np

import oracle as O
from paper_2509_04666_gb300 import workloads as W

F = np.float32
C_AU_DAY = 173.1446326742403


def _predict(hr, hv, dt, so, sun_v):
    r, v = hr.astype(F), hv.astype(F)
    rr = F(r @ r); rn = np.sqrt(rr); vn = np.sqrt(F(v @ v)); adt = F(abs(dt))
    son = np.sqrt(F(so @ so))
    tmax = (rn + son + vn * adt + F(1)) * F(1 / C_AU_DAY) * F(1.01)
    s = adt + tmax
    rmin = F(0.5) * rn
    amax = F(W.GM_SUN) / (rmin * rmin)
    if not (vn * s + F(0.5) * amax * s * s <= rmin):
        return None, None                    # no cheap bound: the exact path runs
    vmax = vn + amax * s
    J = F(4) * F(W.GM_SUN) * vmax / rmin ** 3
    dtf = F(dt)
    k = -F(W.GM_SUN) / (rr * rn)
    p = v * dtf + (F(0.5) * dtf * dtf * k * r + r)
    vt = (k * dtf) * r + v + sun_v.astype(F)
    u = so + p
    tau = np.sqrt(F(u @ u)) * F(1 / C_AU_DAY)
    for _ in range(2):
        w = u - tau * vt
        tau = np.sqrt(F(w @ w)) * F(1 / C_AU_DAY)
    u = u - tau * vt
    un = np.sqrt(F(u @ u))
    E = F(1.001) * (J * s ** 3 / F(6) + F(0.5) * amax * tmax * tmax
                    + F(2e-6) * (rn + son + un + vn * adt)) + F(1e-9)
    return u.astype(np.float64), float(E)


def test_prefilter_bound_covers_the_exact_retarded_position():
    w = W.ragged1y(n_bodies=1000)
    rng = np.random.default_rng(11)
    n, worst = 0, 0.0
    for i in range(w.n_bodies):
        hr, hv = w.states[:3, i], w.states[3:, i]      # the Sun at rest at the origin
        for _ in range(3):
            dt = rng.uniform(-1.6, 1.6)
            o = rng.normal(size=3)
            o *= rng.uniform(0.9, 1.1) / np.linalg.norm(o)
            sun_v = rng.normal(size=3) * 1e-5
            so = (-o).astype(F)
            tau = 0.0
            for _ in range(8):
                rc, rk, _ = O.kepler(W.GM_SUN, hr, hv, dt - tau)
                assert rc == 0
                u = -tau * sun_v + rk - o
                tau = np.linalg.norm(u) / C_AU_DAY
            up, E = _predict(hr, hv, dt, so, sun_v)
            if up is None:
                continue
            err = np.linalg.norm(up - u)
            assert err <= E, (i, dt, err, E)
            worst = max(worst, err / E)
            n += 1
    assert n > 2500          # the bound applies to nearly every case
    assert worst > 1e-4      # and is not vacuous
