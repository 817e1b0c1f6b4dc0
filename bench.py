#!/usr/bin/env python
"""Benchmark of the survey-prediction path on GB300.

One step = one full survey prediction (Sec. 2): 757,000 synthetic bodies
(2 % NEOs) propagated over 365 days under Sun + 8 planets with GR and J2,
batched at <= 3-day midpoints, light-time-corrected two-body to every epoch of
a WISE-like stream of 1.2 M square 0.78 deg frames, polygon test, hits sorted.

value = body-days propagated per second for the whole job (N GPUs x bodies x
365 days / step time); the same line carries the body x frame checks per
second.  Inputs are resident in HBM when a timed step starts; e2e repeats the
step through the host-buffer path (host -> device copies and the hit list
back inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("body-days propagated/s and body×frame FoV checks/s at ≤1 mas vs FP64 oracle, "
          "1 GB300")
MAS = math.radians(1.0 / 3.6e6)

# DRAM traffic of one k_propagate launch from an ncu capture of a smaller case
# of the same workload (100k bodies x 21 stops), per body-stop, scaled to the
# full launch by its body-stops; valid only while the kernel source is
# unchanged (the source hash below).
PROFILED_TRAFFIC = {"src_sha": "6c043addf4c24b22", "bytes_per_body_stop": 65.7}


# FP64 work of the exact FoV test per candidate it solves as ncu counts it (2 x
# DFMA + DMUL + DADD thread instructions of the timed k_exact launch of the
# same small case, divided by the candidates the prefilter passed to it); valid
# only while the FoV kernels' source is unchanged.  The modelled count below leaves out the divisions, square roots
# and convergence tests that the executed count includes.
PROFILED_EXACT = {"src_sha": "78dc3d3396ef0f3c", "fp64_flops_per_candidate": 834.6}

# FP64 arithmetic thread instructions (DFMA + DMUL + DADD) the FP64 survey's
# propagation kernel executes per accepted step, from the same ncu capture as
# the traffic (100k bodies x 21 stops: 16.46 G over 2,119,119 steps); with the
# step count of a run it gives the FP64 pipe's issue rate, which the FLOP
# roofline understates (a DMUL or DADD takes an FMA's issue slot).
PROFILED_ISSUE = {"src_sha": "6c043addf4c24b22", "fp64_inst_per_step": 7765.8}


def kernel_source_sha(files=("kete_prop.cu", "kete_device.cuh", "kete_step.cuh", "kete_order.cu")):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2509_04666_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fov_source_sha():
    return kernel_source_sha(("kete_fov.cu", "kete_device.cuh"))


def _bits(m):
    return bin(m & 0x1FF).count("1")


# coefficients a table may have for the per-thread path's shared Chebyshev
# basis (longer tables take the series with the basis made on the fly)
BASIS_MAX = 16
# FLOPs of the force terms per mass: Newton (with the relative position and
# velocity), GR (Eq. A.3) and J2 (Eq. A.4) with their per-mass factors formed
# on the host
NEWTON_FLOPS, GR_FLOPS, J2_FLOPS = 25, 23, 20


def series64_flops(n_coef, act, gr):
    """FP64 FLOPs of one per-thread evaluation's planet series: the segment
    lookup (10), then either the shared basis (T_k: 1 + 2 (n_coef - 2); with
    a GR mass also k U_(k-1): 3 (n_coef - 2)) and per mass 6 + 6 (n_coef - 2)
    for the position, 10 + 12 (n_coef - 2) for a GR mass's position and
    velocity; or, beyond BASIS_MAX, the basis made on the fly per mass:
    6 + 8 (n_coef - 2), + 9 (n_coef - 2) + 3 for a velocity."""
    k = n_coef - 2
    if n_coef <= BASIS_MAX:
        basis = 1 + 2 * k + (3 * k if gr else 0)
        return 10 + basis + (act - gr) * (6 + 6 * k) + gr * (10 + 12 * k)
    return 10 + act * (6 + 8 * k) + gr * (9 * k + 3)


def prop_flops(st, fm, n_coef, mixed):
    """Algorithmic FLOPs of k_propagate from its counters (FMA = 2), as the
    kernel computes them for the force model fm:
      per force evaluation from node rows: per active mass NEWTON_FLOPS, per
        GR mass + GR_FLOPS, per J2 mass + J2_FLOPS;
      per-thread evaluation (step not spanning a whole leg): + the planet
        series (series64_flops).  FP32 series (mixed precision) by Clenshaw:
        position 3 (3 (n_coef - 1) + 3), velocity 3 (4 (n_coef - 1) + 1);
      per corrector iteration: 7 substep predictors (x, v) and the g/b
        updates, 1440 (+48 for the FP64-part b6 in mixed precision);
      per step attempt: final x, v and step control, 121.
    In mixed precision the FP64 work of an evaluation is the Sun's monopole
    (19) plus, per-thread, the segment lookup and the Sun's position series
    (on the fly); the planetary terms, the Sun's velocity series (with a
    GR term) and the close-planet test at each step start (5 per planet) are
    FP32.  Returns (fp64_flops, fp32_flops)."""
    act, gr, j2 = _bits(fm.body_mask), _bits(fm.gr_mask), _bits(fm.j2_mask)
    pos32, vel32 = 3 * (3 * (n_coef - 1) + 3), 3 * (4 * (n_coef - 1) + 1)
    evals, node = st["force_evals"], st["node_evals"]
    attempts = st["steps"] + st["rejected"]
    if not mixed:
        per = NEWTON_FLOPS * act + GR_FLOPS * gr + J2_FLOPS * j2
        f64 = evals * per + (evals - node) * series64_flops(n_coef, act, gr)
        f64 += st["iterations"] * 1440 + attempts * 121
        return f64, 0
    pos64 = 6 + 8 * (n_coef - 2)
    f64 = evals * 19 + (evals - node) * (pos64 + 10) + st["iterations"] * 1488 + attempts * 121
    sun_gr, sun_j2 = fm.gr_mask & 1, fm.j2_mask & 1
    per32 = NEWTON_FLOPS * (act - 1) + GR_FLOPS * gr + J2_FLOPS * j2
    f32 = evals * per32 + (evals - node) * ((act - 1) * pos32 + (gr - sun_gr) * vel32
                                            + sun_gr * (pos32 + vel32))
    f32 += st["steps"] * 5 * (act - 1)          # close-planet test at each step start
    return f64, f32


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(args, rank):
    from paper_2509_04666_gb300 import workloads as W
    kw = {}
    if args.n_bodies:
        kw["n_bodies"] = args.n_bodies
    if args.n_frames:
        kw["n_frames"] = args.n_frames
    seed = W.SEED_BASE + 1 + 1000 * rank
    return W.wise1y(seed=seed, **kw)


def workload_name(w, args):
    return (f"wise1y: {w.n_bodies} bodies (2% NEOs) x {len(w.frames)} square 0.78 deg frames "
            f"(WISE-like scan from a 1-AU orbit), 365 d, Sun+8 planets, GR+J2, "
            f"{'FP64' if args.precision == 'fp64' else 'mixed FP32/FP64'}")


def oracle_sample(w, n_sample, n_threads=None):
    """The FP64 CPU oracle, as it stands, on a bounded body sample."""
    import oracle as O
    orc = O.Oracle(w.ephem.to_bytes())
    sub = np.linspace(0, w.n_bodies - 1, n_sample).astype(np.int32)
    nt = n_threads or os.cpu_count()
    t0 = time.perf_counter()
    hits, status, stats = orc.fov_check(orc.force_model(), w.states, w.epochs, w.frames, w.observers,
                                        prefilter_deg=1.0, subset=sub, n_threads=nt)
    dt = time.perf_counter() - t0
    return sub, hits, dt, nt


def cpu_model():
    """The host CPU's model name (lscpu), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def measured_hbm_gbs():
    """Copy bandwidth from MEASURED_PEAKS.json (None if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return None


# Algorithmic FP64 work of the exact FoV test per candidate (k_exact): the
# universal-variable solve at the exposure epoch (setup 25, 4 Newton
# iterations of ~55 with the Stumpff series, final f/g and velocity ~70, the
# acceleration and jerk of the cubic ~30), 5 light-time evaluations of the
# cubic (~33 each) and one polygon test (~20); the FP32 cap tests and the
# per-hit RA/Dec are left out.
EXACT_FLOPS_PER_CANDIDATE = 25 + 4 * 55 + 70 + 30 + 5 * 33 + 20


def fov_stage_roofline(stats, n_bodies, peak_fp64_tflops, hbm_gbs):
    """Rooflines of the FoV stage's two kernels from the call's counters:
    the exact test against the FP64 peak (its FP64 work per candidate that
    the FP32 prefilter passed on to the two-body solve, as ncu counts it while
    the kernel source matches the profile, else the model
    EXACT_FLOPS_PER_CANDIDATE; the prefilter's FP32 work is left out), the
    candidate search against HBM (per body and batch the 48-B stop state
    read, per candidate 8 B written and read back)."""
    cand = statistics.mean(s["n_candidates"] for s in stats)
    tested = statistics.mean(s.get("n_exact", s["n_candidates"]) for s in stats)
    batches = stats[-1]["n_batches"]
    exact_ms = statistics.mean(s["exact_ms"] for s in stats)
    cand_ms = statistics.mean(s["cand_ms"] for s in stats)
    per, basis = EXACT_FLOPS_PER_CANDIDATE, "model"
    if PROFILED_EXACT["src_sha"] == fov_source_sha() and PROFILED_EXACT["fp64_flops_per_candidate"]:
        per, basis = PROFILED_EXACT["fp64_flops_per_candidate"], "ncu-counted"
    ex = per * tested / (exact_ms / 1e3) / 1e12
    cbytes = n_bodies * batches * 48.0 + cand * 16.0
    cgbs = cbytes / (cand_ms / 1e3) / 1e9
    return {"exact": {"bound": "alu", "achieved": ex, "peak": peak_fp64_tflops, "unit": "TFLOP/s",
                      "frac": ex / peak_fp64_tflops, "candidates": cand,
                      "past_prefilter": tested, "ms": exact_ms,
                      "flops_per_candidate": per, "flops_basis": basis},
            "candidates": {"bound": "hbm", "achieved": cgbs, "peak": hbm_gbs, "unit": "GB/s",
                           "frac": cgbs / hbm_gbs if hbm_gbs else None,
                           "bytes": cbytes, "ms": cand_ms}}


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the step time of the slowest
    replica); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: every replica processes units_per_rank in the
    (max-over-ranks) step time ms."""
    return world * units_per_rank / (ms / 1e3)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make_workload(args, 0)
    n_sample = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        sub, hits, dt, nt = oracle_sample(w, n_sample)
        if i >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = n_sample * 365.0 / t
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "body-days/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w, args), "sample_bodies": n_sample},
        "cpu_baseline": {"value": value, "unit": "body-days/s", "cores": nt, "kind": "oracle",
                         "sample": f"{n_sample} evenly spaced bodies x all {len(w.frames)} frames, full year"},
        "e2e": {"value": value, "unit": "body-days/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def compare_sample(kete, hits, nh, sub, ref):
    """GPU hits restricted to the sampled bodies vs the oracle's hits."""
    got = kete.decode_hits(hits, nh)
    keep = np.isin(got["body"].numpy(), sub)
    g = {(int(f), int(b)): (ra, de) for f, b, ra, de in
         zip(got["frame"].numpy()[keep], got["body"].numpy()[keep], got["ra"].numpy()[keep],
             got["dec"].numpy()[keep])}
    r = {(int(h["frame"]), int(h["body"])): h for h in ref}
    worst = 0.0
    for key in set(g) & set(r):
        ra, de = g[key]
        dra = (ra - r[key]["ra"] + math.pi) % (2 * math.pi) - math.pi
        worst = max(worst, math.hypot(dra * math.cos(de), de - r[key]["dec"]))
    band = max(1e-9, 2 * worst)
    mism = [k for k in set(g) ^ set(r) if k not in r or abs(r[k]["margin"]) >= band]
    return {"sampled_bodies": len(sub), "oracle_hits": len(r), "gpu_hits": len(g),
            "edge_band_rad": band, "mismatch_outside_edge_band": len(mism),
            "max_sky_err_mas": worst / MAS}


def peak_fma(fp64: bool):
    import ctypes as C
    from paper_2509_04666_gb300 import build as B
    L = C.CDLL(B.PEAK_LIB)
    L.kete_peak_fma.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    v = C.c_double(0)
    rc = L.kete_peak_fma(1 if fp64 else 0, 4096 if fp64 else 65536, 152 * 8, 256, 3, C.byref(v))
    return v.value if rc == 0 else None


def adj_flops(st, fm, n_coef):
    """Algorithmic FP64 FLOPs of the adjoint's forward kernel: the propagation
    count of prop_flops with every evaluation per-thread (per-body stops share
    no node rows) plus the Newtonian da/dx of each mass at every evaluation
    (26 FLOPs)."""
    s = dict(st)
    s["node_evals"] = 0
    f64, _ = prop_flops(s, fm, n_coef, False)
    return f64 + st["force_evals"] * _bits(fm.body_mask) * 26


def _timed(stream, fn, flush, reps):
    import torch
    out, times = None, []
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times), out


def adjoint_leg(args, K, dev, flush, stream, peak):
    """Orbit-fit loss + gradient of 100,000 bodies (20 observations each over
    90 days, 8-day checkpoints).  Observed RA/Dec for the timed run are the
    GPU's truth predictions plus N(0, 0.1") noise; the sampled parity check
    uses observations the oracle makes itself."""
    import concurrent.futures as cf
    import torch
    import oracle as O
    from paper_2509_04666_gb300 import kete, workloads as W
    w = W.adjoint90(n_bodies=args.adj_bodies)
    n, m = w.n_bodies, w.meta["obs"].shape[1]
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model()
    ep = torch.full((n,), W.T0, dtype=torch.float64, device=dev)
    truth = torch.from_numpy(w.states.copy()).to(dev)
    y = torch.from_numpy(w.states + w.meta["offsets"]).to(dev)
    obs = w.meta["obs"].copy()
    ob = torch.from_numpy(obs.view(np.float64).reshape(n, m, 6).copy()).to(dev)
    _, _, pred, status = K.adjoint(truth, ep, ob, fm=fm, grad=False, pred=True)
    pred = pred.cpu().numpy()
    obs["ra"] = pred[..., 0] + w.meta["noise"][..., 0] / np.cos(pred[..., 1])
    obs["dec"] = pred[..., 1] + w.meta["noise"][..., 1]
    ob = torch.from_numpy(obs.view(np.float64).reshape(n, m, 6).copy()).to(dev)
    opts = kete.survey_opts(mem_budget_gb=24.0)    # one chunk: ~105 KB of step records a body
    call = lambda: K.adjoint(y, ep, ob, fm=fm, opts=opts, ckpt_days=8.0)
    call()
    ms, (loss, g, _, status) = _timed(stream, call, flush, 3)
    st = K.get_stats()
    flops = adj_flops(st, fm, w.ephem.n_coef)
    fwd_tf = flops / (st["prop_ms"] / 1e3) / 1e12
    ok = int((status == 0).sum().item())
    # the same fit with non-gravitational terms: the bodies with terms on the
    # full-model path (da/dx and da/dv of GR, J2 and the terms at every node)
    ng = W.nongrav_params(w.labels, dust_frac=0.05)
    ng_dev = kete.nongrav_to_device(ng, dev)
    fm_ng = kete.force_model(nongrav=ng_dev)
    opts_ng = kete.survey_opts(mem_budget_gb=48.0)  # ~400 KB of records a body
    call_ng = lambda: K.adjoint(y, ep, ob, fm=fm_ng, opts=opts_ng, ckpt_days=8.0)
    call_ng()
    ms_ng, (_, _, _, status_ng) = _timed(stream, call_ng, flush, 2)
    st_ng = K.get_stats()
    nongrav = {"ms_per_step": ms_ng, "forward_ms": st_ng["prop_ms"],
               "cost_vs_gravity": ms_ng / ms, "bodies_ok": int((status_ng == 0).sum().item()),
               "terms": "every 10th body a transverse 1/r^2 drift, 5 % of the rest radiation "
                        "pressure with beta logU[1e-3, 0.1]; those bodies on the full-model path"}
    # sampled parity: observations and reference gradient from the oracle alone
    orc = O.Oracle(w.ephem.to_bytes())
    fmo = orc.force_model()
    sub = np.linspace(0, n - 1, args.adj_sample).astype(np.int64)
    y_np = w.states + w.meta["offsets"]

    def one(i):
        o = w.meta["obs"][i].copy()
        _, _, p, _ = orc.body_loss(fmo, w.states[:, i], W.T0, o, grad=False)
        o["ra"] = p[:, 0] + w.meta["noise"][i, :, 0] / np.cos(p[:, 1])
        o["dec"] = p[:, 1] + w.meta["noise"][i, :, 1]
        t0 = time.perf_counter()
        rc, L, _, gi = orc.body_loss(fmo, y_np[:, i], W.T0, o)
        return o, rc, L, gi, time.perf_counter() - t0

    nt = os.cpu_count()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(nt) as ex:
        res = list(ex.map(one, sub))
    wall = time.perf_counter() - t0
    so = np.stack([r[0] for r in res])
    loss_r = np.array([r[2] for r in res]); g_r = np.stack([r[3] for r in res], 1)
    ls, gs, _, ss = K.adjoint(torch.from_numpy(y_np[:, sub].copy()).to(dev),
                              ep[:len(sub)].contiguous(),
                              torch.from_numpy(so.view(np.float64).reshape(len(sub), m, 6).copy()).to(dev),
                              fm=fm, ckpt_days=8.0)
    ls, gs = ls.cpu().numpy(), gs.cpu().numpy()
    rel_x = np.abs(gs[:3] - g_r[:3]).max(0) / np.abs(g_r[:3]).max(0)
    rel_v = np.abs(gs[3:] - g_r[3:]).max(0) / np.abs(g_r[3:]).max(0)
    cpu_rate = len(sub) * 90.0 / wall
    return {
        "workload": f"adjoint90: {n} bodies (2% NEOs), {m} observations each over 90 d from a "
                    f"1-AU circular observer, 8-day checkpoints, loss + dL/d(x0,v0), FP64",
        "value": n * 90.0 / (ms / 1e3), "unit": "body-days/s (loss + gradient)",
        "bodies_per_s": n / (ms / 1e3), "ms_per_step": ms, "forward_ms": st["prop_ms"],
        "bodies_ok": ok, "steps": st["steps"], "force_evals": st["force_evals"],
        "roofline": {"bound": "alu", "kernel": "k_adj_forward", "achieved": fwd_tf, "peak": peak,
                     "unit": "TFLOP/s", "frac": fwd_tf / peak, "traffic": None},
        "nongrav": nongrav,
        "parity": {"sampled_bodies": len(sub), "max_rel_grad_x": float(rel_x.max()),
                   "max_rel_grad_v": float(rel_v.max()),
                   "max_rel_loss": float((np.abs(ls - loss_r) / loss_r).max()),
                   "oracle": "variational equations + central-difference partials"},
        "cpu_baseline": {"value": cpu_rate, "unit": "body-days/s (loss + gradient)", "cores": nt,
                         "kind": "oracle", "sample": f"{len(sub)} evenly spaced bodies, "
                         f"{wall:.1f} s wall incl. making their observations"},
    }


def ztf_leg(args, K, dev, flush, stream, peak_fp64, hbm_gbs):
    """The ZTF-like survey year: 757,000 bodies (2 % NEOs) against 150,000
    night-time exposures of 8 x 8 sub-fields of 0.87 deg (9.6 M FoVs) seen
    from a site on the rotating Earth.  The mixed-precision form (FP32
    planetary terms) against the plain FP64 form on the same workload, each
    with its FoV-stage rooflines and its sky accuracy against the oracle on a
    bounded body sample."""
    import torch
    from paper_2509_04666_gb300 import kete, workloads as W
    kw = {}
    if args.ztf_bodies:
        kw["n_bodies"] = args.ztf_bodies
    if args.ztf_exposures:
        kw["n_exposures"] = args.ztf_exposures
    w = W.ztf1y(**kw)
    n, nf = w.n_bodies, len(w.frames)
    K.load_ephem(w.ephem.to_bytes())
    st = torch.from_numpy(w.states.copy()).to(dev)
    ep = torch.from_numpy(w.epochs.copy()).to(dev)
    fr = kete.frames_to_device(w.frames, dev)
    ob = torch.from_numpy(np.ascontiguousarray(w.observers)).to(dev)
    out = {"workload": f"ztf1y: {n} bodies (2% NEOs) x {len(np.unique(w.frames['exposure_id']))} "
                       f"exposures of 8x8 0.87 deg sub-fields ({nf} FoVs) from a rotating ground "
                       f"site, 365 d"}
    hits = {}
    for name, prec in (("mixed", kete.MIXED), ("fp64", kete.FP64)):
        fm = kete.force_model(precision=prec)
        h, nh, _ = K.fov_check(st, ep, fr, ob, fm=fm)          # sizes the hit buffer
        h = torch.empty((int(nh * 1.1) + 4096, 4), dtype=torch.int64, device=dev)
        ms, (h, nh, status) = _timed(stream, lambda: K.fov_check(st, ep, fr, ob, fm=fm, hits=h),
                                     flush, 2)
        s = K.get_stats()
        hits[name] = (h, nh)
        f64, f32 = prop_flops(s, fm, w.ephem.n_coef, prec == kete.MIXED)
        out[name] = {"value": n * 365.0 / (ms / 1e3), "unit": "body-days/s", "ms_per_step": ms,
                     "fov_checks_per_s": n * nf / (ms / 1e3), "prop_ms": s["prop_ms"],
                     "exact_ms": s["exact_ms"], "cand_ms": s["cand_ms"], "n_hits": int(nh),
                     "candidates": s["n_candidates"], "batches": s["n_batches"],
                     "bodies_ok": int((status == 0).sum().item()),
                     "prop_fp64_tflops": f64 / (s["prop_ms"] / 1e3) / 1e12,
                     "prop_fp32_tflops": f32 / (s["prop_ms"] / 1e3) / 1e12,
                     "fov_stage": fov_stage_roofline([s], n, peak_fp64, hbm_gbs)}
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    if not args.no_cpu_baseline:
        sub, ref, dt, nt = oracle_sample(w, args.ztf_sample)
        for name in ("mixed", "fp64"):
            out[name]["accuracy"] = compare_sample(kete, *hits[name], sub, ref)
        out["cpu_baseline"] = {"value": len(sub) * 365.0 / dt, "unit": "body-days/s",
                               "kind": "oracle", "cores": nt,
                               "sample": f"{len(sub)} evenly spaced bodies x all {nf} FoVs, "
                                         f"{dt:.1f} s"}
    return out


POPULATIONS = ((0, "main_belt"), (1, "neo"), (2, "trojan"), (3, "comet"), (4, "encounter"))


def truncation_by_population(orc, w, sub, t_end, ref, ref_status):
    """The method's own truncation error on the sample: the oracle with the
    step control at eps / 100 and the corrector threshold at eps_pc / 100
    against the oracle at the tuned controls (ref), max |dr| in AU per
    population, over the bodies both runs finish."""
    tight, _, st, _ = orc.propagate_many(orc.force_model(eps=1e-11, eps_pc=1e-12),
                                         w.states[:, sub], w.epochs[sub], t_end)
    ok = (st == 0) & (np.asarray(ref_status) == 0)
    d = np.linalg.norm(tight[:3] - ref[:3], axis=0)
    out = {}
    for lab, nm in POPULATIONS:
        k = (w.labels[sub] == lab) & ok
        if k.any():
            out[nm] = float(d[k].max())
    out["bodies"] = int(ok.sum())
    return out


def ragged_leg(args, K, dev, flush, stream):
    """500,000 bodies of very uneven step counts (main belt, NEOs with forced
    Earth encounters, Trojans, comets) over 365 d: plain FP64 against the
    mixed-precision form, and work stealing against the static schedule."""
    import torch
    import oracle as O
    from paper_2509_04666_gb300 import kete, workloads as W
    w = W.ragged1y(n_bodies=args.ragged_bodies)
    n = w.n_bodies
    K.load_ephem(w.ephem.to_bytes())
    st0 = torch.from_numpy(w.states.copy()).to(dev)
    t_end = W.T0 + 365.0
    out = {"workload": f"ragged1y: {n} bodies (60% main belt, 20% NEOs of which 5% pass "
                       f"0.001-0.01 AU from the Earth, 10% Trojans, 10% comets), 365 d"}
    res = {}
    ng = W.nongrav_params(w.labels)
    ng_dev = kete.nongrav_to_device(ng, dev)
    variants = (("fp64", kete.FP64, kete.PROP_WORK_STEALING, 0, False),
                ("mixed", kete.MIXED, kete.PROP_WORK_STEALING, 0, False),
                ("fp64_static", kete.FP64, kete.PROP_STATIC, 0, False),
                ("fp64_split8", kete.FP64, kete.PROP_WORK_STEALING, 8, False),
                ("mixed_split8", kete.MIXED, kete.PROP_WORK_STEALING, 8, False),
                ("fp64_nongrav", kete.FP64, kete.PROP_WORK_STEALING, 0, True))
    if args.ragged_variants:   # a subset alone (profiling): no comparisons, no oracle
        keep = args.ragged_variants.split(",")
        variants = tuple(v for v in variants if v[0] in keep)
    for name, prec, kind, split, with_ng in variants:
        K.set_propagation(prec, kind, 128, split, 64 if split else 0)
        fm = kete.force_model(precision=prec)
        if with_ng:
            fm.nongrav = ng_dev.data_ptr()
        box = {}

        def call():
            s = st0.clone(); e = torch.full((n,), W.T0, dtype=torch.float64, device=dev)
            box["st"] = s
            return K.propagate(s, e, t_end, fm=fm)
        call()
        ms, status = _timed(stream, call, flush, 2)
        stt = K.get_stats()
        res[name] = (box["st"].cpu().numpy(), status.cpu().numpy())
        out[name] = {"value": n * 365.0 / (ms / 1e3), "unit": "body-days/s", "ms": ms,
                     "prop_ms": stt["prop_ms"], "steps": stt["steps"], "deferred": stt["deferred"]}
    if args.ragged_variants:
        return out
    # the autotuner's pick per precision (kete_autotune on a body sample over
    # the same year), timed on the whole population beside the hand variants;
    # the autotuner starts from the default variant (the loop above left the
    # last hand variant set)
    K.set_propagation(kete.FP64, kete.PROP_WORK_STEALING, 128)
    K.set_propagation(kete.MIXED, kete.PROP_WORK_STEALING, 128)
    for name, prec in (("fp64_autotuned", kete.FP64), ("mixed_autotuned", kete.MIXED)):
        fm = kete.force_model(precision=prec)
        e0 = torch.full((n,), W.T0, dtype=torch.float64, device=dev)
        pick = K.autotune(st0, e0, np.array([t_end]), fm=fm, max_sample=args.tune_sample)
        box = {}

        def call():
            s = st0.clone(); e = torch.full((n,), W.T0, dtype=torch.float64, device=dev)
            box["st"] = s
            return K.propagate(s, e, t_end, fm=fm)
        call()
        ms, status = _timed(stream, call, flush, 2)
        stt = K.get_stats()
        out[name] = {"value": n * 365.0 / (ms / 1e3), "unit": "body-days/s", "ms": ms,
                     "prop_ms": stt["prop_ms"], "steps": stt["steps"], "deferred": stt["deferred"],
                     "variant": dict(zip(("kind", "block", "split_lanes", "defer_steps",
                                          "cost_order"), pick))}
    hand = {k: out[k]["ms"] for k in ("fp64", "fp64_static", "fp64_split8")}
    out["autotune"] = {"fp64_pick_ms": out["fp64_autotuned"]["ms"],
                       "fp64_best_hand_ms": min(hand.values()),
                       "mixed_pick_ms": out["mixed_autotuned"]["ms"],
                       "mixed_best_hand_ms": min(out["mixed"]["ms"], out["mixed_split8"]["ms"]),
                       "sample": f"{min(n, args.tune_sample)} of {n} bodies on grids scaled by "
                                 f"{min(n, args.tune_sample) / n:.3f}"}
    K.set_propagation(kete.FP64, kete.PROP_WORK_STEALING, 128)
    K.set_propagation(kete.MIXED, kete.PROP_WORK_STEALING, 128)
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["work_stealing_speedup_vs_static"] = out["fp64_static"]["ms"] / out["fp64"]["ms"]
    out["nongrav_cost_vs_fp64"] = out["fp64_nongrav"]["ms"] / out["fp64"]["ms"]
    out["nongrav_terms"] = ("comets: JPL comet model, comet g(r), A1 logU[1e-9, 1e-7] AU/d^2, "
                            "half lagged 5-40 d; every 10th other body: transverse 1/r^2 drift")
    # accuracy on a sample (every population, all forced encounters in it)
    orc = O.Oracle(w.ephem.to_bytes())
    enc = np.nonzero(w.labels == 4)[0]
    sub = np.unique(np.concatenate([np.linspace(0, n - 1, args.ref_sample).astype(np.int64),
                                    enc[:: max(1, len(enc) // 64)]]))
    t0 = time.perf_counter()
    ref, _, rst, _ = orc.propagate_many(orc.force_model(), w.states[:, sub], w.epochs[sub], t_end)
    dt = time.perf_counter() - t0
    ref_ng, _, _, _ = orc.propagate_many(orc.force_model(), w.states[:, sub], w.epochs[sub], t_end,
                                         nongrav=ng[sub])
    _, pe, _ = orc.ephem(3, t_end)
    acc = {}
    for name in ("fp64", "mixed", "fp64_nongrav"):
        s, stat = res[name]
        d = np.linalg.norm(s[:3, sub] - (ref_ng if name == "fp64_nongrav" else ref)[:3], axis=0)
        rho = np.linalg.norm(ref[:3] - pe[:, None], axis=0)
        by = {}
        for lab, nm in ((0, "main_belt"), (1, "neo"), (2, "trojan"), (3, "comet"), (4, "encounter")):
            k = w.labels[sub] == lab
            if k.any():
                by[nm] = {"max_au": float(d[k].max()), "max_sky_mas_from_earth": float((d[k] / rho[k]).max() / MAS)}
        acc[name] = {"bodies_ok": int((stat == 0).sum()), "sample": len(sub), "by_population": by}
    out["accuracy"] = acc
    out["truncation_au"] = truncation_by_population(orc, w, sub, t_end, ref, rst)
    out["cpu_baseline"] = {"value": len(sub) * 365.0 / dt, "unit": "body-days/s", "kind": "oracle",
                           "cores": os.cpu_count(), "sample": f"{len(sub)} bodies, {dt:.1f} s"}
    return out


def longspan_leg(args, K, dev, flush, stream):
    """Backward propagation over decades and centuries: 20,000 bodies of the
    survey population carried back 50 years, and 1,000 clones of a
    Jupiter-family comet (JPL comet model) carried back 170 years, one lane
    per body against lane groups of 4, 8 and 16."""
    import torch
    import oracle as O
    from paper_2509_04666_gb300 import kete, workloads as W
    out = {}
    legs = (("catalogue", W.backward_catalogue(n_bodies=args.back_bodies, years=50.0), None,
             (("fp64", kete.FP64, 0), ("mixed", kete.MIXED, 0))),
            ("clones", W.clones(n_clones=1000, years=170.0), "nongrav",
             (("fp64", kete.FP64, 0), ("fp64_split4", kete.FP64, 4),
              ("fp64_split8", kete.FP64, 8), ("fp64_split16", kete.FP64, 16),
              ("mixed", kete.MIXED, 0), ("mixed_split4", kete.MIXED, 4),
              ("mixed_split8", kete.MIXED, 8))))
    for leg, w, ngkey, variants in legs:
        n = w.n_bodies
        days = abs(w.t_end - W.T0)
        K.load_ephem(w.ephem.to_bytes())
        ng = w.meta[ngkey] if ngkey else None
        ng_dev = kete.nongrav_to_device(ng, dev) if ng is not None else None
        st0 = torch.from_numpy(w.states.copy()).to(dev)
        res = {"workload": (f"{n} bodies of the survey population, {days / 365.25:.0f} years back"
                            if leg == "catalogue" else
                            f"{n} clones of a Jupiter-family comet (q 1.06 AU, JPL comet model), "
                            f"{days / 365.25:.0f} years back")}
        got = {}
        for name, prec, split in variants:
            K.set_propagation(prec, kete.PROP_WORK_STEALING, 128, split, 4 if split else 0)
            fm = kete.force_model(precision=prec)
            if ng_dev is not None:
                fm.nongrav = ng_dev.data_ptr()
            box = {}

            def call():
                s = st0.clone(); e = torch.full((n,), W.T0, dtype=torch.float64, device=dev)
                box["st"] = s
                return K.propagate(s, e, w.t_end, fm=fm)
            call()
            ms, status = _timed(stream, call, flush, 2)
            stt = K.get_stats()
            got[name] = box["st"].cpu().numpy()
            res[name] = {"value": n * days / (ms / 1e3), "unit": "body-days/s", "ms": ms,
                         "steps": stt["steps"], "deferred": stt["deferred"],
                         "bodies_ok": int((status.cpu().numpy() == 0).sum())}
        K.set_propagation(kete.FP64, kete.PROP_WORK_STEALING, 128)
        K.set_propagation(kete.MIXED, kete.PROP_WORK_STEALING, 128)
        # the oracle on a bounded sample: accuracy and the CPU rate
        orc = O.Oracle(w.ephem.to_bytes())
        sub = np.linspace(0, n - 1, 16 if leg == "clones" else 48).astype(np.int64)
        t0 = time.perf_counter()
        ref, _, _, _ = orc.propagate_many(orc.force_model(), w.states[:, sub], w.epochs[sub],
                                          w.t_end, nongrav=None if ng is None else ng[sub])
        dt = time.perf_counter() - t0
        res["max_err_au"] = {k: float(np.abs(v[:3, sub] - ref[:3]).max()) for k, v in got.items()}
        res["cpu_baseline"] = {"value": len(sub) * days / dt, "unit": "body-days/s",
                               "kind": "oracle", "cores": min(os.cpu_count(), len(sub)),
                               "sample": f"{len(sub)} bodies, {dt:.1f} s"}
        out[leg] = res
    return out


def run_leg(args):
    """One leg alone (--leg adjoint|ragged), e.g. for a profiler; prints the
    leg's own JSON object, not the benchmark line."""
    import torch
    from paper_2509_04666_gb300 import build as B, kete
    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K = kete.Kete(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    peak = 152 * 2 * 2 * 2.07e9 / 1e12
    if args.leg == "adjoint":
        out = adjoint_leg(args, K, dev, flush, stream, peak)
    elif args.leg == "longspan":
        out = longspan_leg(args, K, dev, flush, stream)
    elif args.leg == "ztf":
        out = ztf_leg(args, K, dev, flush, stream, peak, measured_hbm_gbs())
    else:
        out = ragged_leg(args, K, dev, flush, stream)
    print(json.dumps({"leg": args.leg, **out}))
    K.close()
    return 0


def fp64_lane_probe():
    """FP64 FMA warp-instructions per second with 32 and with 1 active lane
    per warp (the cost of an FP64 instruction does not shrink with its mask)."""
    import ctypes as C
    from paper_2509_04666_gb300 import build as B
    L = C.CDLL(B.PEAK_LIB)
    L.kete_peak_fma_lanes.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(C.c_double)]
    out = {}
    for lanes in (32, 1):
        v = C.c_double(0)
        rc = L.kete_peak_fma_lanes(1, lanes, 4096, 152 * 8, 256, 2, C.byref(v))
        out[f"active_{lanes}"] = v.value if rc == 0 else None
    return out


def run_gb300(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2509_04666_gb300 import build as B, kete
    B.build()
    dev = torch.device("cuda", local)
    w = make_workload(args, rank)
    K = kete.Kete(local)
    K.load_ephem(w.ephem.to_bytes())
    fm = kete.force_model(precision=kete.MIXED if args.precision == "mixed" else kete.FP64)
    st = torch.from_numpy(w.states.copy()).to(dev)
    ep = torch.from_numpy(w.epochs.copy()).to(dev)
    fr = kete.frames_to_device(w.frames, dev)
    ob = torch.from_numpy(np.ascontiguousarray(w.observers)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # first call sizes the hit buffer
    hits, nh, status = K.fov_check(st, ep, fr, ob, fm=fm)
    hits = torch.empty((int(nh * 1.1) + 4096, 4), dtype=torch.int64, device=dev)

    def step():
        return K.fov_check(st, ep, fr, ob, fm=fm, hits=hits)

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream(dev)
    times, stats = [], []
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)                       # L2 flush between steps (256 MB write)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, nh, status = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(K.get_stats())
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clocks = clk.summary()
    ms = max_over_ranks(statistics.mean(times), dist, dev)
    n, nf = w.n_bodies, len(w.frames)
    value = job_rate(world, n * 365.0, ms)
    checks = job_rate(world, n * nf, ms)
    # ---- roofline of the dominant kernel (k_propagate, FP64 ALU bound) --------
    s0 = stats[-1]
    mixed = args.precision == "mixed"
    flops = statistics.mean(prop_flops(s, fm, w.ephem.n_coef, mixed)[0] for s in stats)
    flops32 = statistics.mean(prop_flops(s, fm, w.ephem.n_coef, mixed)[1] for s in stats)
    prop_ms = statistics.mean(s["prop_ms"] for s in stats)
    achieved = flops / (prop_ms / 1e3) / 1e12
    peak_nominal = 152 * 2 * 2 * 2.07e9 / 1e12      # SMs x FP64 FMA/clk x 2 x max clock
    peak_probe = peak_fma(True)
    lane_probe = fp64_lane_probe()
    src_sha = kernel_source_sha()
    traffic = None
    if PROFILED_TRAFFIC["src_sha"] == src_sha and PROFILED_TRAFFIC["bytes_per_body_stop"]:
        traffic = PROFILED_TRAFFIC["bytes_per_body_stop"] * n * s0["n_batches"] / max(1, s0["prop_launches"])
    issue = None
    if PROFILED_ISSUE["src_sha"] == src_sha and not mixed:
        per = PROFILED_ISSUE["fp64_inst_per_step"]
        rate = per * s0["steps"] / (prop_ms / 1e3)
        issue = {"fp64_thread_inst_per_step": per, "thread_inst_per_s": rate,
                 "frac_nominal": rate / (peak_nominal * 1e12 / 2),
                 "frac_probe": rate / (peak_probe / 2) if peak_probe else None,
                 "basis": "ncu-counted DFMA+DMUL+DADD per accepted step (100k-body case)"}
    # ---- e2e: the public call with host buffers ----------------------------------
    e2e = None
    if not args.no_e2e:
        h_st = torch.from_numpy(w.states.copy()).pin_memory()
        h_ep = torch.from_numpy(w.epochs.copy()).pin_memory()
        h_fr = torch.from_numpy(np.ascontiguousarray(w.frames).view(np.uint8).reshape(-1).copy()).pin_memory()
        h_ob = torch.from_numpy(np.ascontiguousarray(w.observers)).pin_memory()
        e_times, d2h = [], 0
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            d_st = h_st.to(dev, non_blocking=True); d_ep = h_ep.to(dev, non_blocking=True)
            d_fr = h_fr.to(dev, non_blocking=True); d_ob = h_ob.to(dev, non_blocking=True)
            hh, nhh, _ = K.fov_check(d_st, d_ep, d_fr, d_ob, fm=fm, hits=hits)
            out = hh[:nhh].cpu()
            t1 = time.perf_counter()
            if i >= args.warmup:
                e_times.append(t1 - t0)
                d2h = out.numel() * 8
        h2d = sum(t.numel() * t.element_size() for t in (h_st, h_ep, h_fr, h_ob))
        et = statistics.mean(e_times)
        e2e = {"value": world * n * 365.0 / et, "unit": "body-days/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": et * 1e3}
    # ---- CPU baseline (the oracle as it stands) + sampled accuracy ------------------
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sub, ref, dt, nt = oracle_sample(w, args.ref_sample)
        sub1, _, dt1, _ = oracle_sample(w, 64, n_threads=1)
        cpu = {"value": len(sub) * 365.0 / dt, "unit": "body-days/s", "cores": nt, "kind": "oracle",
               "sample": f"{len(sub)} evenly spaced bodies x all {nf} frames, full year, "
                         f"{dt:.1f} s",
               "cpu_model": cpu_model(),
               "one_core": {"value": len(sub1) * 365.0 / dt1, "unit": "body-days/s",
                            "sample": f"{len(sub1)} bodies, 1 thread, {dt1:.1f} s"}}
        accuracy = compare_sample(kete, hits, nh, sub, ref)
    # ---- the mixed-precision form on the same workload (speedup at accuracy) ------
    mixed_leg = None
    if args.precision == "fp64" and not args.no_mixed:
        fm_m = kete.force_model(precision=kete.MIXED)
        hm = torch.empty_like(hits)
        K.fov_check(st, ep, fr, ob, fm=fm_m, hits=hm)
        mt = []
        for _ in range(2):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, nhm, _ = K.fov_check(st, ep, fr, ob, fm=fm_m, hits=hm)
            e1.record(stream)
            e1.synchronize()
            mt.append(e0.elapsed_time(e1))
        mm = statistics.mean(mt)
        sm = K.get_stats()
        f64m, f32m = prop_flops(sm, fm_m, w.ephem.n_coef, True)
        mixed_leg = {"value": world * n * 365.0 / (mm / 1e3), "ms_per_step": mm,
                     "speedup_vs_fp64": ms / mm, "prop_ms": sm["prop_ms"],
                     "prop_fp64_tflops": f64m / (sm["prop_ms"] / 1e3) / 1e12,
                     "prop_fp32_tflops": f32m / (sm["prop_ms"] / 1e3) / 1e12,
                     "accuracy": compare_sample(kete, hm, nhm, sub, ref) if cpu else None}
    # ---- per-hit magnitudes fused into the exact test (kete_fov_check_mag) ----------
    mag_leg = None
    if rank == 0 and world == 1 and not args.no_mag:
        from paper_2509_04666_gb300 import workloads as W
        mp = kete.mag_params_to_device(W.mag_params(w.labels), dev)
        hg = torch.empty_like(hits)
        K.fov_check(st, ep, fr, ob, fm=fm, hits=hg, mag_params=mp)
        gt, ex = [], []
        for _ in range(2):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, nhg, _ = K.fov_check(st, ep, fr, ob, fm=fm, hits=hg, mag_params=mp)
            e1.record(stream)
            e1.synchronize()
            gt.append(e0.elapsed_time(e1))
            ex.append(K.get_stats()["exact_ms"])
        mg = hg[:nhg, 1].cpu().numpy()
        mags = (mg >> 32).astype(np.uint32).view(np.float32)
        same = bool(nhg == nh) and bool(torch.equal(hg[:nhg, 0], hits[:nh, 0]))
        mag_leg = {"ms_per_step": statistics.mean(gt), "exact_ms": statistics.mean(ex),
                   "exact_ms_without": statistics.mean(s["exact_ms"] for s in stats),
                   "n_hits": int(nhg), "finite": int(np.isfinite(mags).sum()),
                   "median_mag": float(np.nanmedian(mags)) if np.isfinite(mags).any() else None,
                   "hit_list_unchanged": same}
    adjoint = ragged = longspan = ztf = None
    if rank == 0 and world == 1 and not args.no_ztf:
        ztf = ztf_leg(args, K, dev, flush, stream, peak_nominal, measured_hbm_gbs())
    if rank == 0 and world == 1 and args.longspan:
        longspan = longspan_leg(args, K, dev, flush, stream)
    if rank == 0 and world == 1 and not args.no_adjoint:
        adjoint = adjoint_leg(args, K, dev, flush, stream, peak_nominal)
    if rank == 0 and world == 1 and not args.no_ragged:
        ragged = ragged_leg(args, K, dev, flush, stream)
    out = {
        "metric": METRIC, "value": value, "unit": "body-days/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": workload_name(w, args), "n_bodies": n, "n_frames": nf, "days": 365,
                   "batches": s0["n_batches"], "precision": args.precision,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "fov_checks_per_s": checks,
        "roofline": {"bound": "alu", "kernel": "k_propagate", "achieved": achieved,
                     "peak": peak_nominal, "unit": "TFLOP/s", "frac": achieved / peak_nominal,
                     "traffic": traffic, "peak_probe_measured": (peak_probe or 0) / 1e12,
                     "flops_per_launch": flops / max(1, s0["prop_launches"]),
                     "fp32_tflops_alongside": flops32 / (prop_ms / 1e3) / 1e12,
                     "prop_ms_per_step": prop_ms, "peak_basis": "152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                     "fp64_warp_inst_per_s": lane_probe, "fp64_issue": issue},
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "e2e": e2e,
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clocks,
        "counters": {k: s0[k] for k in ("steps", "rejected", "force_evals", "node_evals",
                                        "iterations", "n_batches", "n_exposures",
                                        "n_candidates", "n_hits")},
        "phases_ms": {k: s0[k] for k in ("prop_ms", "prep_ms", "cand_ms", "exact_ms", "order_ms")},
        "wall_s_timed": t_wall,
        "magnitudes": mag_leg,
        "longspan": longspan,
        "adjoint": adjoint,
        "ragged": ragged,
        # the survey comparisons last: mixed precision on both survey years
        "ztf1y": ztf,
        "mixed_precision": mixed_leg,
        "fov_stage": fov_stage_roofline(stats, n, peak_nominal, measured_hbm_gbs()),
    }
    if rank == 0:
        print(json.dumps(out))
    K.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--n-bodies", type=int, default=0)
    ap.add_argument("--n-frames", type=int, default=0)
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-mag", action="store_true")
    ap.add_argument("--longspan", action="store_true",
                    help="add the long-span leg (decades back; ~3 min) to the benchmark line")
    ap.add_argument("--back-bodies", type=int, default=20_000)
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-ztf", action="store_true", help="skip the ZTF-like survey year leg")
    ap.add_argument("--ztf-sample", type=int, default=256)
    ap.add_argument("--ztf-bodies", type=int, default=0, help="smaller ZTF-like case (profiling)")
    ap.add_argument("--ztf-exposures", type=int, default=0)
    ap.add_argument("--adj-bodies", type=int, default=100_000)
    ap.add_argument("--adj-sample", type=int, default=512)
    ap.add_argument("--ragged-bodies", type=int, default=500_000)
    ap.add_argument("--tune-sample", type=int, default=131072)
    ap.add_argument("--ragged-variants", default="",
                    help="comma list of ragged-leg variants to run alone (profiling)")
    ap.add_argument("--leg", default="all", choices=["all", "adjoint", "ragged", "longspan", "ztf"],
                    help="run one leg alone (profiling); the default prints the benchmark line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg != "all":
        return run_leg(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
