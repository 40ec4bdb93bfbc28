#!/usr/bin/env python
"""Throughput of the Schwarz-converged MFA encode on GB300.

One step = mfa_encode (setup, projection, iteration 0) + mfa_schwarz_iterate
to the stopping tolerance + mfa_residual (decoded RMS / max error), on one
batch of synthetic data already resident in HBM.  ``value`` is data points
per second over the whole job; ``e2e`` is the same metric through the C ABI
with pinned host buffers (host->device copies of the data and the read-back
of the control points inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload 3d|2d|1d]

With N > 1 (torchrun), every rank fits its own replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2210_06528_gb300 import inputs  # noqa: E402

METRIC = "encode pts/s (Schwarz-converged) + decode pts/s vs plain GPU; serve p50/p99"

WORKLOADS = {
    # 3-D workload: 512^3 FP32 grid of 16 seeded Gaussians + sin(6 pi x) cos(4 pi y) z,
    # p = 3, 8x8x8 subdomains of 24 core spans (192 spans, 195 control points per axis), overlap 2.
    "3d": dict(name="3d_512^3_gauss16_p3_8x8x8sub_24spans_overlap2_mixed", npts=(512, 512, 512), p=3,
               nspans=(192, 192, 192), nsub=(8, 8, 8), delta=2, precision="mixed", tol=1e-7, max_iters=50,
               sample=dict(npts=(128, 128, 128), nspans=(48, 48, 48), nsub=(2, 2, 2))),
    # Profiling-size case of the 3-D workload: 384^3 (226 MB, larger than L2), 6x6x6 subdomains of the
    # same per-subdomain shape; used for ncu captures, not a bench line.
    "3d384": dict(name="3d_384^3_gauss16_p3_6x6x6sub_24spans_overlap2_mixed", npts=(384, 384, 384), p=3,
                  nspans=(144, 144, 144), nsub=(6, 6, 6), delta=2, precision="mixed", tol=1e-7, max_iters=50,
                  sample=dict(npts=(128, 128, 128), nspans=(48, 48, 48), nsub=(2, 2, 2))),
    # 2-D workload: 1024^2 sinc(x) sinc(y) + N(0, 1e-3), p = 3, 4x4 subdomains of 64 core spans,
    # Schwarz to decoded-residual stall |RMS_k - RMS_{k-1}| <= 1e-6 RMS_k.
    "2d": dict(name="2d_1024^2_sinc_noise1e-3_p3_4x4sub_64spans_overlap2_mixed", npts=(1024, 1024), p=3,
               nspans=(256, 256), nsub=(4, 4), delta=2, precision="mixed", tol=0.0, stall=1e-6, max_iters=50,
               sample=dict(npts=(512, 512), nspans=(128, 128), nsub=(2, 2))),
    # 1-D workload: 1024 points of sin(x)/x, p = 3, 4 subdomains of 32 core spans, FP64.
    "1d": dict(name="1d_1024_sinc_p3_4sub_32spans_overlap2_fp64", npts=(1024,), p=3, nspans=(128,), nsub=(4,),
               delta=2, precision="fp64", tol=1e-10, max_iters=200,
               sample=dict(npts=(1024,), nspans=(128,), nsub=(4,))),
}


def make_data(wl, npts, seed=0):
    d = len(npts)
    if d == 3:
        return inputs.gauss_3d(tuple(npts), seed=seed, dtype=np.float32)
    if d == 2:
        return inputs.sinc_2d(npts[0], noise=1e-3, seed=seed, dtype=np.float32)
    return inputs.sinc_1d(npts[0])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_step(wl):
    """One oracle run on the bounded sample of the workload; returns (points, seconds)."""
    from oracle import mfa_oracle as O
    smp = wl["sample"]
    Q = make_data(wl, smp["npts"]).astype(np.float64)
    prob = O.make_problem(wl["p"], list(smp["npts"]), list(smp["nspans"]), list(smp["nsub"]), wl["delta"])
    t0 = time.perf_counter()
    res = O.schwarz_solve(prob, Q, max_iters=wl["max_iters"], tol_dP=wl["tol"], tol_rms_stall=wl.get("stall", 0.0))
    O.residual_stats(prob, Q, res["P"])
    dt = time.perf_counter() - t0
    return int(np.prod(smp["npts"])), dt


def stop_desc(wl):
    if wl.get("stall"):
        return f"|RMS_k - RMS_(k-1)| <= {wl['stall']:g} RMS_k"
    return f"dP_rel <= {wl['tol']:g}"


def sample_desc(wl):
    smp = wl["sample"]
    return (f"{'x'.join(map(str, smp['npts']))} grid, {'x'.join(map(str, smp['nsub']))} subdomains with the "
            f"workload's per-subdomain shape (p={wl['p']}, overlap {wl['delta']}, same points per span), "
            f"oracle Schwarz to {stop_desc(wl)} + residual, FP64 numpy")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def cpu_baseline(wl, budget_s=20.0):
    pts, dt = oracle_sample_step(wl)  # first run includes imports / page-in
    n, tot = 0, 0.0
    while tot < budget_s and n < 50:
        p2, d2 = oracle_sample_step(wl)
        n += 1
        tot += d2
    return {"value": pts * n / tot, "unit": "pts/s", "cores": host_cores(), "kind": "oracle",
            "sample": sample_desc(wl) + f", {n} runs"}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_step(wl)
    times = []
    pts = 0
    for _ in range(args.steps):
        pts, dt = oracle_sample_step(wl)
        times.append(dt)
    t = sum(times) / len(times)
    value = pts / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "sample": sample_desc(wl)},
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample_desc(wl)},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def window_sizes(M, nspans, S, delta, p):
    """(points, L size) of every subdomain window along one axis: cores split
    the spans evenly (the first nspans % S take one more), windows add delta
    spans per interior side, points are those with u_k = k/(M-1) in the
    closed window interval, L = window spans + p."""
    out, a = [], 0
    for i in range(S):
        c = nspans // S + (1 if i < nspans % S else 0)
        b = a + c
        w0, w1 = max(a - delta, 0), min(b + delta, nspans)
        k0 = -((-w0 * (M - 1)) // nspans)
        k1 = (w1 * (M - 1)) // nspans
        out.append((k1 - k0 + 1, (w1 - w0) + p))
        a = b
    return out


# FP32 instructions of one float-float multiply-add: float x float-float
# (exact product + TwoSum accumulate) and float-float x float-float
FF_OPS_F, FF_OPS_V = 11, 12


# DRAM bytes (read + write) of one fused 3-D projection launch, from one ncu
# capture of the current kernel on the 384^3 case (6x6x6 windows of the 512^3
# workload's shape): 290.2 MB read + 55.9 MB written.  The traffic grows with
# the number of windows at a fixed window shape, so a workload of W such
# windows moves W / 216 times that.  Kept for the kernel it was taken on.
PROJECTION_TRAFFIC_384 = {"bytes": (290.206720 + 55.914752) * 1e6, "windows": 216}


def projection_traffic(wl):
    """DRAM bytes per launch scaled from the 384^3 capture, or None when the
    workload's windows differ in shape from the captured ones."""
    npts, nsub, nspans = wl["npts"], wl["nsub"], wl["nspans"]
    same = (len(npts) == 3 and wl["p"] == 3 and wl["delta"] == 2 and wl["precision"] == "mixed"
            and all(n == 64 * k and sp == 24 * k for n, sp, k in zip(npts, nspans, nsub)))
    if not same:
        return None
    windows = nsub[0] * nsub[1] * nsub[2]
    return PROJECTION_TRAFFIC_384["bytes"] * windows / PROJECTION_TRAFFIC_384["windows"]


def projection_ops(wl):
    """Algorithmic FP32 operations of one 3-D float-float projection launch:
    per window point (P+1) float x float-float multiply-adds on the first
    axis, then (P+1) float-float x float-float multiply-adds per element of
    the x-reduced and xy-reduced arrays."""
    W = wl["p"] + 1
    ax = [window_sizes(wl["npts"][a], wl["nspans"][a], wl["nsub"][a], wl["delta"], wl["p"]) for a in range(3)]
    sm = [sum(m for m, _ in ax[a]) for a in range(3)]
    sn = [sum(n for _, n in ax[a]) for a in range(3)]
    return W * (FF_OPS_F * sm[0] * sm[1] * sm[2] + FF_OPS_V * sn[0] * sm[1] * sm[2] + FF_OPS_V * sn[0] * sn[1] * sm[2])


def sm_count(device=0):
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def alu_peak_tops(clock_mhz, sms):
    """FP32 lane instructions per second: SMs x 128 FP32 lanes x SM clock."""
    return sms * 128 * clock_mhz * 1e6 / 1e12


def algorithmic_bytes(cls_name, wl, qbytes, model_info):
    """Algorithmic bytes of one launch of a kernel class (what the method must
    move): the data-reading kernels read every data value once."""
    if cls_name in ("project_data", "residual"):
        return qbytes
    return None


def bench_batch(h, torch, mfa, stream, steps, precision, count=4096, seed=0, decode=True):
    """Batch of independent fits: one full encode (host layout, setup, fit),
    then timed refits of the captured CUDA graph on device data and one
    per-instance residual; with the data-pass kernels timed on their own
    (one traced encode) against the HBM peak."""
    specs, data = inputs.batch_instances(count, seed=seed)
    q = torch.from_numpy(data).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = h.encode_batch(specs, q, precision)
    torch.cuda.synchronize()
    enc_s = time.perf_counter() - t0
    b.refit(q)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(steps, 1)):
        b.refit(q)
    e1.record(stream)
    torch.cuda.synchronize()
    refit_ms = e0.elapsed_time(e1) / max(steps, 1)
    b.residual(q)
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(5):
        rms, mx = b.residual(q)
    r1.record(stream)
    torch.cuda.synchronize()
    res_ms = r0.elapsed_time(r1) / 5
    info = b.info()
    npts = int(info["points"])
    qbytes = 4 * npts
    # data-pass kernels of one fit and one residual, traced (not captured)
    mfa.mfa_trace_enable(h.h, True)
    b2 = h.encode_batch(specs, q, precision)
    b2.residual(q)
    tr = mfa.trace_table(h.h)
    mfa.mfa_trace_enable(h.h, False)
    b2.free()
    peak, peak_kind = load_peaks()
    passes = {}
    # FP32: each pass is one timed region (its launches side by side inside);
    # FP64 / mixed: the groups' launches overlap, so the traced sums are not
    # wall times and get no HBM fraction
    for name in (("project_data", "refine_data", "residual") if precision == mfa.MFA_PREC_FP32 else ()):
        if name in tr and tr[name][0] > 0:
            ms = tr[name][0]
            byts = qbytes
            if name == "refine_data":
                byts = None  # reads only the refined instances' data (reported as time)
            ent = {"ms": ms, "launches": tr[name][1]}
            if byts:
                ach = byts / (ms * 1e-3) / 1e9
                ent.update({"algorithmic_bytes": byts, "achieved_gbs": ach, "hbm_frac": ach / peak})
            passes[name] = ent
    out = {"precision": {mfa.MFA_PREC_FP32: "fp32", mfa.MFA_PREC_MIXED: "mixed", mfa.MFA_PREC_FP64: "fp64"}[precision],
           "points": npts, "instances": count, "refined_instances": info["refined"], "items": info["items"],
           "encode_s_incl_host_layout": enc_s, "refit_ms": refit_ms, "refit_pts_per_s": npts / (refit_ms * 1e-3),
           "residual_ms": res_ms, "residual_pts_per_s": npts / (res_ms * 1e-3),
           "fit_plus_residual_pts_per_s": npts / ((refit_ms + res_ms) * 1e-3),
           "data_passes": passes, "peak_gbs": peak, "peak_source": peak_kind,
           "kernels_ms": {k: round(v[0], 4) for k, v in tr.items()},
           "kernels_ms_note": ("wall time of each pass" if precision == mfa.MFA_PREC_FP32 else
                               "sums of launch durations of groups that run side by side (not wall times)"),
           "rms": rms, "rms_median": float(np.median(rms)), "rms_max": float(rms.max())}
    if decode:
        # scattered decode: 4096 uniform random parameter points per instance,
        # device resident, one query per instance
        per = 4096
        qi = torch.arange(count, dtype=torch.int32, device="cuda")
        poff = torch.arange(count + 1, dtype=torch.int64, device="cuda") * per
        gen = torch.Generator(device="cuda").manual_seed(seed + 7)
        upts = torch.rand((count * per, 3), dtype=torch.float64, device="cuda", generator=gen)
        uout = torch.empty(count * per, dtype=torch.float64, device="cuda")
        b.decode_points(qi, poff, upts, uout)
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = 5
        d0.record(stream)
        for _ in range(nrep):
            b.decode_points(qi, poff, upts, uout)
        d1.record(stream)
        torch.cuda.synchronize()
        dec_ms = d0.elapsed_time(d1) / nrep
        out["scattered_decode"] = {"points": count * per, "ms": dec_ms, "pts_per_s": count * per / (dec_ms * 1e-3),
                                   "inputs": "4096 uniform random parameter points per instance, on the device"}
        del upts, uout
    tun = []
    for g in b.group_tuning():
        cm = g["candidate_ms"]

        def spread(xs):
            xs = [x for x in xs if x > 0]
            return round(max(xs) / min(xs), 3) if xs else None

        ent = {"dim": g["dim"], "degree": g["degree"], "instances": g["instances"], "solve_threads": g["tile_s"],
               "chosen_ms": round(g["chosen_ms"], 4), "candidates_ms": [round(x, 4) for x in cm]}
        if precision == mfa.MFA_PREC_FP32:
            ent.update({"item_pts": g["item_pts"], "solve_spread": spread(cm[0:3]), "item_spread": spread(cm[3:6])})
        else:
            ent.update({"projection_threads": g["tile_c"], "fused": bool(g["fused"]),
                        "tiled_spread": spread(cm[0:9]),
                        "fused_vs_best_tiled": round(cm[9] / min(cm[0:9]), 3) if cm[9] > 0 else None})
        tun.append(ent)
    out["autotune"] = {"groups": tun,
                       "candidates": ("solve threads 32/64/128 per group; projection items of 16K/32K/128K points "
                                      "per batch" if precision == mfa.MFA_PREC_FP32 else
                                      "projection threads 64/128/256 x solve threads 32/64/128, and the fused "
                                      "one-CTA-per-instance path for 3-D groups, per group")}
    b.free()
    return out


def bench_batched(h, torch, mfa, stream, steps, count=4096, seed=0):
    """The batched workload in FP32 data-pass precision (the line's batched
    result) and in mixed precision beside it, with the per-instance decoded
    RMS of the two compared."""
    f32 = bench_batch(h, torch, mfa, stream, steps, mfa.MFA_PREC_FP32, count, seed)
    mix = bench_batch(h, torch, mfa, stream, steps, mfa.MFA_PREC_MIXED, count, seed, decode=False)
    r32, rmx = f32.pop("rms"), mix.pop("rms")
    rel = np.abs(r32 - rmx) / np.maximum(rmx, 1e-300)
    specs, data = inputs.batch_instances(count, seed=seed)
    d2 = sum(1 for sp in specs if sp["dim"] == 2)
    # FP32 data passes meet the 1 % bar where the decoded RMS is at least
    # 100 x 2^-24 x the data range; elsewhere the RMS agrees to that amount
    rng = np.array([float(np.ptp(data[sp["q_offset"]:sp["q_offset"] + int(np.prod(sp["npts"]))])) for sp in specs])
    floor = 100.0 * 2.0 ** -24 * rng
    rule = rmx >= floor
    return {"workload": f"{count} independent fits ({d2} 2-D 32..512^2, {count - d2} 3-D 16..128^3 log-uniform, "
                        "degree 2..5, control points max(p+1, M/4) per axis, sinc / Gaussian sums)",
            "fp32": f32, "mixed": mix,
            "fp32_vs_mixed_rms": {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
                                  "within_1pct": int((rel <= 0.01).sum()), "instances": count,
                                  "rms_at_least_100_fp32_ulps_of_range": int(rule.sum()),
                                  "of_those_within_1pct": int((rule & (rel <= 0.01)).sum()),
                                  "others_within_100_fp32_ulps_of_range":
                                      int((~rule & (np.abs(r32 - rmx) <= floor)).sum()),
                                  "others": int((~rule).sum())},
            "refit": "one CUDA graph per batch (projection, z contraction and solves of every group)"}


def bench_serve(torch, mfa, n_enc=160, mix=4, seed=1, workers=3, budget=48 << 30, precision=None):
    """Serving: a Poisson stream of encode requests (2-D 64..512^2, 3-D
    32..256^3 log-uniform, p = 3, sinc / Gaussian sums, control points M/4 per
    axis) mixed 1:4 with decode queries of 1e3..1e6 uniform random points
    against a resident model chosen uniformly among those already requested.
    Saturation is measured by submitting everything at once; then the same
    stream is offered at 0.5x, 0.8x and 1.0x that rate.  Encodes run in FP32
    data-pass precision."""
    if precision is None:
        precision = mfa.MFA_PREC_FP32
    specs, data = inputs.batch_instances(n_enc, seed=seed, size2=(64, 512), size3=(32, 256), degrees=(3, 3))
    payloads = [torch.from_numpy(data[sp["q_offset"]:sp["q_offset"] + int(np.prod(sp["npts"]))].copy()).pin_memory()
                for sp in specs]
    rng = np.random.default_rng(seed + 1)
    stream = []  # (kind, index): encode k, or decode (model among encodes 0..k, points)
    qpts = []
    for k in range(n_enc):
        stream.append(("enc", k))
        for _ in range(mix):
            m = int(rng.integers(0, k + 1))
            n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e6)))))
            qpts.append(torch.from_numpy(rng.uniform(0, 1, size=(n, 3))).pin_memory())
            stream.append(("dec", m, len(qpts) - 1))
    outs = [torch.empty(len(q), dtype=torch.float64).pin_memory() for q in qpts]
    enc_pts = sum(int(np.prod(sp["npts"])) for sp in specs)
    dec_pts = sum(len(q) for q in qpts)

    def run(rate):
        srv = mfa.Server(0, workers=workers, mem_budget=budget)
        ids, kinds, models = [], [], {}
        t0 = time.perf_counter()
        gaps = rng.exponential(1.0 / rate, size=len(stream)) if rate else np.zeros(len(stream))
        t_next = t0
        for ev, gap in zip(stream, gaps):
            t_next += gap
            while rate and time.perf_counter() < t_next:
                time.sleep(min(1e-4, max(t_next - time.perf_counter(), 0)))
            if ev[0] == "enc":
                rid = srv.encode(specs[ev[1]], payloads[ev[1]], precision)
                models[ev[1]] = rid
            else:
                rid = srv.decode(models[ev[1]], qpts[ev[2]], outs[ev[2]])
            ids.append(rid)
            kinds.append(ev[0])
        lat = {"enc": [], "dec": []}
        t_end = 0.0
        for rid, kd in zip(ids, kinds):
            rc, info = srv.wait(rid, 600.0)
            if rc != mfa.MFA_OK:
                raise RuntimeError(f"serving request failed: {mfa.status_string(rc)}")
            lat[kd].append(info["t_done"] - info["t_submit"])
            t_end = max(t_end, info["t_done"])
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        allv = np.array(lat["enc"] + lat["dec"]) * 1e3
        return {"requests_per_s": len(stream) / wall, "pts_per_s": (enc_pts + dec_pts) / wall, "wall_s": wall,
                "p50_ms": float(np.percentile(allv, 50)), "p99_ms": float(np.percentile(allv, 99)),
                "encode_p50_ms": float(np.percentile(np.array(lat["enc"]) * 1e3, 50)),
                "encode_p99_ms": float(np.percentile(np.array(lat["enc"]) * 1e3, 99)),
                "decode_p50_ms": float(np.percentile(np.array(lat["dec"]) * 1e3, 50)),
                "decode_p99_ms": float(np.percentile(np.array(lat["dec"]) * 1e3, 99)),
                "encode_jobs": st["encode_jobs"], "decode_jobs": st["decode_jobs"],
                "peak_reserved_gb": st["peak_reserved"] / 1e9}

    run(0)  # warm-up (allocations, module loading)
    sat = run(0)
    out = {"workload": f"{n_enc} encodes (2-D 64..512^2 / 3-D 32..256^3, p=3, control points M/4) + "
                       f"{n_enc * mix} decode queries (1e3..1e6 points), Poisson arrivals",
           "encode_points": enc_pts, "decode_points": dec_pts, "workers": workers, "budget_gb": budget / 1e9,
           "encode_precision": "fp32" if precision == mfa.MFA_PREC_FP32 else "mixed",
           "saturation": sat, "offered": {}}
    for f in (0.5, 0.8, 1.0):
        out["offered"][f"{f:.1f}x"] = run(f * sat["requests_per_s"])
    return out


def load_golden():
    """The oracle's Schwarz-converged fits of the 1-D and 2-D workloads
    (written by tests/golden/make_workload_rms.py from the oracle alone)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "workload_rms.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def bench_workload(h, torch, mfa, stream, key, steps):
    """One of the smaller workloads (1-D, 2-D) run like the line's own:
    encode + Schwarz to the workload's stop + residual per step, device data,
    CUDA events; the decoded RMS beside the oracle's, and the HBM fraction of
    its dominant data-reading kernel (these grids fit in L2 and a step is a
    chain of small launches, so the fraction is latency-bound)."""
    wl = WORKLOADS[key]
    npts = wl["npts"]
    q = torch.from_numpy(make_data(wl, npts)).cuda()
    prec = mfa.MFA_PREC_MIXED if wl["precision"] == "mixed" else mfa.MFA_PREC_FP64
    d = len(npts)
    lay = mfa.make_layout(d, wl["p"], npts, wl["nspans"], wl["nsub"], [wl["delta"]] * d, prec)

    def step():
        m = h.encode(q, lay)
        rc, rep = m.iterate(wl["max_iters"], wl["tol"], wl.get("stall", 0.0))
        res = m.residual(q)
        m.free()
        return rep, res

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    mfa.mfa_trace_enable(h.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(steps, 1)
    e0.record(stream)
    for _ in range(n):
        rep, res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    trace = mfa.trace_table(h.h)
    mfa.mfa_trace_enable(h.h, False)
    ms = e0.elapsed_time(e1) / n
    M = q.numel()
    qbytes = M * q.element_size()
    peak, peak_kind = load_peaks()
    data_cls = {k: v for k, v in trace.items() if k in ("project_data", "residual") and v[1] > 0}
    hbm = None
    if data_cls:
        name = max(data_cls.items(), key=lambda kv: kv[1][0])[0]
        ms_per = trace[name][0] / trace[name][1]
        ach = qbytes / (ms_per * 1e-3) / 1e9
        hbm = {"kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
               "peak_source": peak_kind, "algorithmic_bytes_per_launch": qbytes, "ms_per_launch": ms_per,
               "note": f"latency-bound: {qbytes / 1e6:.3g} MB of data per launch, smaller than L2"}
    gold = load_golden().get(key)
    out = {"workload": wl["name"], "points": M, "pts_per_s": M / (ms * 1e-3), "ms_per_step": ms,
           "precision": wl["precision"], "stop": stop_desc(wl), "schwarz_iters": rep.iters,
           "rms_decoded": res.rms_decoded, "maxabs_decoded": res.maxabs_decoded, "hbm": hbm,
           "gpu_launches_per_step": sum(v[1] for v in trace.values()) / n}
    if gold:
        out["oracle"] = {"iters": gold["iters"], "rms": gold["rms"], "max": gold["max"],
                         "source": "tests/golden/workload_rms.json (FP64 oracle)"}
        out["rms_rel_diff_vs_oracle"] = abs(res.rms_decoded - gold["rms"]) / gold["rms"]
        out["iters_equal_oracle"] = rep.iters == gold["iters"]
    return out


# ---------------------------------------------------------------------------
# replicas over ranks (one process per GPU, no collective on the data path)
# ---------------------------------------------------------------------------

def rank_env():
    """(world, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def run_gb300(args, wl):
    import torch
    import torch.distributed as dist

    from paper_2210_06528_gb300 import mfa

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    npts = wl["npts"]
    Qnp = make_data(wl, npts, seed=rank)
    q_dev = torch.from_numpy(Qnp).cuda()
    q_host = torch.from_numpy(Qnp).pin_memory()
    del Qnp
    qbytes = q_dev.numel() * q_dev.element_size()
    M = q_dev.numel()
    prec = mfa.MFA_PREC_MIXED if wl["precision"] == "mixed" else mfa.MFA_PREC_FP64
    d = len(npts)
    lay = mfa.make_layout(d, wl["p"], npts, wl["nspans"], wl["nsub"], [wl["delta"]] * d, prec)
    h = mfa.Handle(local)
    stream = torch.cuda.current_stream()

    iters_seen = []

    def step(q):
        m = h.encode(q, lay)
        rc, rep = m.iterate(wl["max_iters"], wl["tol"], wl.get("stall", 0.0))
        res = m.residual(q)
        iters_seen.append(rep.iters)
        m.free()
        return rep, res

    for _ in range(args.warmup):
        rep, res = step(q_dev)
    torch.cuda.synchronize()

    # ---- timed region: device-resident data
    mfa.mfa_trace_enable(h.h, True)
    iters_seen.clear()
    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rep, res = step(q_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    t_ms = e0.elapsed_time(e1) / args.steps
    trace = mfa.trace_table(h.h)
    mfa.mfa_trace_enable(h.h, False)
    t_ms = max_over_ranks(t_ms, device="cuda")
    value = job_rate(world, M, t_ms * 1e-3)

    # ---- decode throughput (grid decode into a device buffer)
    m = h.encode(q_dev, lay)
    m.iterate(wl["max_iters"], wl["tol"], wl.get("stall", 0.0))
    out = torch.empty_like(q_dev)
    for _ in range(2):
        m.decode_grid(out)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(args.steps):
        m.decode_grid(out)
    d1.record(stream)
    torch.cuda.synchronize()
    dec_ms = max_over_ranks(d0.elapsed_time(d1) / args.steps, device="cuda")
    ncp = mfa.mfa_num_ctrl(m.m)
    m.free()
    del out

    # ---- comparator: the plain per-subdomain FP64 form (one launch per
    # subdomain and stage, window data re-read every iteration), same stop
    lay64 = mfa.make_layout(d, wl["p"], npts, wl["nspans"], wl["nsub"], [wl["delta"]] * d, mfa.MFA_PREC_FP64)
    plain = None
    if not args.no_plain:
        def step_plain():
            m, rc, rep = h.encode_plain(q_dev, lay64, wl["max_iters"], wl["tol"] or 1e-6)
            r = m.residual(q_dev)
            m.free()
            return rep, r
        step_plain()
        torch.cuda.synchronize()
        mfa.mfa_trace_enable(h.h, True)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        prep, pres = step_plain()
        p1.record(stream)
        torch.cuda.synchronize()
        ptrace = mfa.trace_table(h.h)
        mfa.mfa_trace_enable(h.h, False)
        plain_ms = max_over_ranks(p0.elapsed_time(p1), device="cuda")
        plain = {"value": job_rate(world, M, plain_ms * 1e-3), "unit": "pts/s", "ms_per_step": plain_ms,
                 "precision": "fp64", "schwarz_iters": prep.iters, "rms_decoded": pres.rms_decoded,
                 "gpu_launches": sum(n for (_, n) in ptrace.values()),
                 "form": "one launch per subdomain and stage; window data re-read every iteration"}

    # ---- batched independent fits: 4096 uneven 2-D / 3-D grids (sizes
    # log-uniform 32..512 / 16..128, degree 2..5, control points M/4 per axis)
    batched = None if args.no_batch else bench_batched(h, torch, mfa, stream, args.steps)
    serving = None if args.no_serve else bench_serve(torch, mfa)
    # ---- the other workloads of the paper's shapes (1-D FP64, 2-D mixed)
    others = {}
    if not args.no_others:
        for key in ("1d", "2d"):
            if WORKLOADS[key]["name"] != wl["name"]:
                others[key] = bench_workload(h, torch, mfa, stream, key, min(args.steps, 20))

    # ---- end to end through the C ABI with pinned host buffers: the data
    # cross to the device once (encode stages them; the residual reuses that
    # copy) and the fitted control points come back into a pinned buffer
    # each end-to-end handle on its own (non-blocking) stream, so that two
    # handles' work can run side by side
    e2e_streams = [torch.cuda.Stream(device=local) for _ in range(2)]
    handles = tuple(mfa.Handle(local, stream=st.cuda_stream) for st in e2e_streams)
    P_hosts = [torch.empty(ncp, dtype=torch.float64).pin_memory() for _ in handles]

    def step_e2e(hh, P_host):
        m = hh.encode(q_host, lay)  # host -> device copy inside
        m.iterate(wl["max_iters"], wl["tol"], wl.get("stall", 0.0))
        m.ctrl_async(P_host)  # device -> host read of the control points, beside the residual
        m.residual(None)  # against the staged copy
        hh.sync()  # the control points are in P_host
        m.free()

    def timed_e2e(nthreads):
        # nthreads host threads, one handle (stream and copy stream) each, take
        # the steps in turn: one step's copy runs beside another's fit
        import threading
        barrier()
        t0 = time.perf_counter()
        work = [list(range(i, args.steps, nthreads)) for i in range(nthreads)]

        def run(i):
            for _ in work[i]:
                step_e2e(handles[i], P_hosts[i])

        ts = [threading.Thread(target=run, args=(i,)) for i in range(nthreads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        torch.cuda.synchronize()
        return max_over_ranks((time.perf_counter() - t0) / args.steps, device="cuda")

    for hh, Ph in zip(handles, P_hosts):
        step_e2e(hh, Ph)
    torch.cuda.synchronize()
    e2e_serial_s = timed_e2e(1)
    e2e_s = timed_e2e(2)
    e2e = {"value": job_rate(world, M, e2e_s), "unit": "pts/s", "h2d_bytes_per_step": qbytes,
           "d2h_bytes_per_step": ncp * 8,
           "mode": "two host threads with a handle each take the steps in turn (one step's host-to-device copy "
                   "beside another's fit); every step copies its data in and reads its control points back",
           "one_handle": {"value": job_rate(world, M, e2e_serial_s), "unit": "pts/s",
                          "mode": "one handle, steps back to back"}}
    for hh in handles:
        hh.close()

    # ---- roofline of the dominant data-reading kernel: HBM bytes of the
    # method (every data value read once) over its measured time; for the
    # float-float projection the FP32-issue view beside it
    peak, peak_kind = load_peaks()
    launches = sum(n for (_, n) in trace.values())
    dom = max(trace.items(), key=lambda kv: kv[1][0]) if trace else None
    roof = None
    kernels = {k: {"ms_total": v[0], "launches": v[1], "ms_per_launch": v[0] / max(v[1], 1)} for k, v in trace.items()}
    hbm_classes = {k: v for k, v in trace.items() if algorithmic_bytes(k, wl, qbytes, None)}
    if hbm_classes:
        name = max(hbm_classes.items(), key=lambda kv: kv[1][0])[0]
        ms_per = trace[name][0] / trace[name][1]
        ab = algorithmic_bytes(name, wl, qbytes, None)
        achieved = ab / (ms_per * 1e-3) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": projection_traffic(wl) if name == "project_data" else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 384^3 capture of the "
                                  "fused projection, scaled by the number of windows of the same shape",
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": ab, "ms_per_launch": ms_per}
        if name == "project_data" and d == 3 and prec == mfa.MFA_PREC_MIXED:
            mhz = (clocks or {}).get("sm_mhz")
            src = "median SM clock under load" if mhz else "maximum SM clock, no clock samples"
            mhz = mhz or 2070.0
            sms = sm_count(local)
            ops = projection_ops(wl)
            ach = ops / (ms_per * 1e-3) / 1e12
            pk = alu_peak_tops(mhz, sms)
            roof["alu_view"] = {"achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz ({src})",
                                "op_convention": "one FP32 add, mul or fma instruction = 1 op (float-float "
                                                 "multiply-add = 11-12 FP32 instructions)",
                                "algorithmic_ops_per_launch": ops}
    if rank != 0:
        return
    cpu = cpu_baseline(wl, budget_s=args.cpu_budget) if world == 1 and not args.no_cpu else None
    line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "float-float" if prec == mfa.MFA_PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "points": M, "control_points": ncp, "precision": wl["precision"],
                       "stop": stop_desc(wl), "schwarz_iters": sorted(set(iters_seen)),
                       "l2": "inputs larger than L2" if qbytes > 129e6 else "inputs smaller than L2",
                       "parallelism": f"replicas x{world}"},
            "decode_pts_per_s": job_rate(world, M, dec_ms * 1e-3), "decode_ms": dec_ms,
            "plain_gpu": plain, "vs_plain_gpu": (value / plain["value"]) if plain else None,
            "batched_fits": batched, "serving": serving, "workloads": others or None,
            "roofline": roof, "dominant_kernel": dom[0] if dom else None, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "rms_decoded": res.rms_decoded, "maxabs_decoded": res.maxabs_decoded}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="3d", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-subdomain comparator run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched independent fits")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-others", action="store_true", help="skip the 1-D and 2-D workload records")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gb300(args, wl)


if __name__ == "__main__":
    main()
