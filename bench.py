#!/usr/bin/env python3
"""Benchmark: pore-site MLUPS of the color-gradient LBM step on one GB300.

Workload (steady flow at fixed saturation): a seeded 256^3 sphere pack
(radius ~ lognormal mean 10, sd 3 voxels, porosity 0.22, about 3.6 M pore
sites), periodic in z with solid walls in x and y, per-voxel affinity
U[-0.3, 0.3], blob initial phases at Sw = 0.4, tau_a = tau_b = 0.7,
alpha = 0.005, beta = 0.95, body force 1e-5 along z. Synthetic data.

One benchmark step = one bundle of timesteps (default 100: phase pass +
fused collide-stream per timestep) followed by the fp64 basic-analysis
reduction. value = pore sites x timesteps / device time (MLUPS), timed with
CUDA events on the library's stream; the state (0.5 GB in FP32) is larger
than L2, so every step streams from HBM.

e2e = the same metric through the public API with host buffers: per step the
image, the wetting map and the initial phases are copied from pinned host
memory (load_image, set_affinity_map, init_fluids), the bundle runs, and the
measures come back to the host.

--impl reference times the FP64 CPU oracle (the test reference) on the
host cores on a bounded number of timesteps of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the headline metric: pore-site MLUPS of the 256^3 steady-state workload in FP32
# storage, with the HBM fraction, the FP16-storage run and the batched-job
# latencies reported beside it in the same line
METRIC = "pore-site MLUPS + % HBM peak, FP16-store vs FP32; p50/p99 batched-job latency"


def workload_label(w, size: int) -> str:
    return (f"{w.name}: {size}^3 sphere pack, porosity {w.porosity:.3f}, z periodic, x/y walls, "
            f"Sw=0.4 blobs")


# algorithmic bytes per pore site and timestep (FP32 storage)
BYTES_COLLIDE_FP32 = 19 * 4 * 2 + 14 * 4 + 4      # f read+write, A/B write, own phi read = 212
BYTES_PHASE_FP32 = 14 * 4 + 4                     # A/B read, phi write = 60
BYTES_STEP_FP32 = BYTES_COLLIDE_FP32 + BYTES_PHASE_FP32   # 272
BYTES_COLLIDE_FP16 = 19 * 2 * 2 + 14 * 2 + 4      # 108
BYTES_PHASE_FP16 = 14 * 2 + 4                     # 32
BYTES_STEP_FP16 = BYTES_COLLIDE_FP16 + BYTES_PHASE_FP16   # 140


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), \
        int(os.environ.get("WORLD_SIZE", 1))


def shard(n_items: int, rank: int, world: int):
    """Indices of the independent units (jobs) rank `rank` of `world` runs:
    round-robin, every unit on exactly one rank, no data exchange."""
    return list(range(rank, n_items, world))


def reduce_over_ranks(ms: float, units: float, world: int, device="cpu"):
    """(max over ranks of the timed milliseconds, sum over ranks of the units
    processed): the job's time is its slowest rank's."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(precision: str) -> str:
    """Hash of the step kernels' source, comments and whitespace left out, so
    that the recorded DRAM traffic stays tied to the code it was measured on."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_12266_gb300", "csrc")
    for name in ("step_kernels.cuh", "step.cu", "lattice.cuh", "internal.h"):
        with open(os.path.join(csrc, name)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    h.update(precision.encode())
    return h.hexdigest()[:16]


def ncu_traffic(precision: str):
    """DRAM bytes per site of the collide (and, when captured, the phase)
    kernel from the committed ncu summary; None when the kernel source changed
    since the capture."""
    p = os.path.join(ROOT, "profiles", "collide_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(precision)
    if not e or e.get("kernel_hash") != kernel_hash(precision):
        return None
    return e


def traffic_per_launch(precision: str, n_sites: int):
    """DRAM bytes per collide launch, scaled to n_sites (see ncu_traffic)."""
    e = ncu_traffic(precision)
    return None if e is None else float(e["bytes_per_site"]) * n_sites


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout: float = 3.0):
        """Block until the first sample arrived, so the timed region is covered."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[4:8]):
                if flag.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "power_w_max": max(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def build_workload(L: int):
    from synthetic import workload_steady256
    return workload_steady256(L)


def run_cpu_baseline(w, steps: int, threads: int):
    import oracle
    oracle.set_threads(threads)
    ref = oracle.Oracle(w.labels, w.affinity, w.periodic, tau_a=w.tau_a, tau_b=w.tau_b,
                        alpha=w.alpha, beta=w.beta, force=w.force)
    ref.init_fluids(w.phi0)
    ref.step(1)  # warm-up
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ref.step(1)
        times.append(time.perf_counter() - t0)
    n = ref.N
    ref.close()
    return n, times


def bench_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    w = build_workload(args.size)
    threads = os.cpu_count() or 1
    n, times = run_cpu_baseline(w, args.steps + args.warmup, threads)
    timed = times[args.warmup:]
    total = sum(timed)
    value = n * len(timed) / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(w, args.size), "n_sites": n, "storage": "fp64",
                   "timesteps_per_step": 1,
                   "note": "FP64 CPU oracle, one timestep of the full workload per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{len(timed)} timesteps of the {args.size}^3 workload "
                                   f"({n} pore sites), OpenMP={oracle.have_openmp()}"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _spawn_map(fn, items):
    """Generate synthetic inputs in parallel (spawned interpreters, no CUDA)."""
    import multiprocessing as mp
    n = max(1, min(len(items), os.cpu_count() or 1, 16))
    if n == 1:
        return [fn(i) for i in items]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(fn, items, chunksize=1)


def _batched_job(j):
    from synthetic import workload_batched_job
    return workload_batched_job(j)


def _serving_job(args):
    from synthetic import serving_job
    i, choices = args
    return serving_job(i, L_choices=choices)


def _domain(lbm, w, precision, device):
    d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha,
                   beta=w.beta, force=w.force, precision=precision, reservoir_z=w.reservoir_z,
                   rho_in=w.rho_in, rho_out=w.rho_out, device=device)
    d.init_fluids(w.phi0)
    return d


def bench_batched(jobs, precision, steps, device, launch=None):
    """Batched form: all jobs in one launch per pass (or one fused launch per
    bundle), at the shape the autotuner picks, or at `launch` = (threads,
    blocks per SM) when given."""
    import torch

    import paper_2007_12266_gb300 as lbm
    doms = [_domain(lbm, w, precision, device) for w in jobs]
    b = lbm.Batch(device=device)
    for d in doms:
        b.add(d)
    if launch is None:
        shape = b.tune(steps_per_candidate=20)
    else:
        b.set_launch(launch[0], launch[1], launch[1])
        shape = (launch[0], launch[1], launch[1])
    b.advance(20)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    l0 = b.launch_count
    e0.record(stream)
    b.advance(steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1)
    meas = b.measure()
    n = b.n_sites
    out = {"value": n * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_jobs": len(jobs), "n_sites": n,
           "steps": steps, "ms": ms, "launch_shape": {"threads": shape[0], "blocks_per_sm_phase": shape[1],
                                                      "blocks_per_sm_collide": shape[2]},
           "gpu_launches": b.launch_count - l0, "unstable_jobs": sum(1 for m in meas if m["status"])}
    b.close()
    for d in doms:
        d.close()
    return out


def bench_serving(jobs, precision, lam, seed, max_steps, interval, device, flux_tol=1e-4):
    """Continuous-batching server fed by a seeded Poisson arrival stream."""
    import numpy as np

    import paper_2007_12266_gb300 as lbm
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(jobs)))
    srv = lbm.Server(device=device, max_jobs=len(jobs), check_interval=interval)
    tickets = []
    t0 = time.perf_counter()
    nxt = 0
    rounds = 0
    for rounds in range(1, 1_000_000):
        now = time.perf_counter() - t0
        while nxt < len(jobs) and arrivals[nxt] <= now:
            w = jobs[nxt]
            kind = w.meta["kind"]
            tickets.append(srv.submit(w.labels, w.phi0, w.affinity, kind=kind, max_steps=max_steps,
                                      flux_tol=flux_tol, sw_tol=1e-4, force_factor=2.0, force_cap=1.6e-4,
                                      tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force,
                                      precision=precision, periodic=w.periodic, reservoir_z=w.reservoir_z))
            nxt += 1
        running, queued, _ = srv.run()
        if running == 0 and queued == 0:
            if nxt == len(jobs):
                break
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    st = [srv.poll(t) for t in tickets]
    lat = np.array([s["t_done"] - s["t_submit"] for s in st])
    run_t = np.array([s["t_done"] - s["t_admit"] for s in st])
    su = srv.stats()["site_updates"]
    out = {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
           "p50_run_s": float(np.percentile(run_t, 50)), "aggregate_value": su / wall / 1e6,
           "unit": "MLUPS", "n_jobs": len(jobs), "wall_s": wall, "rounds": rounds,
           "arrival_rate_per_s": lam, "check_interval": interval, "max_steps": max_steps,
           "states": {k: sum(1 for s in st if s["state"] == k) for k in ("done", "failed")},
           "converged_early": sum(1 for s in st if s["steps"] < max_steps),
           "site_updates": su, "mean_sites": float(np.mean([s["n_sites"] for s in st])),
           "mean_steps": float(np.mean([s["steps"] for s in st])),
           "kinds": {k: sum(1 for w in jobs if w.meta["kind"] == k) for k in ("steady", "unsteady", "centrifuge")}}
    srv.close()
    return out


def bench_precision(args):
    """1024^3 displacement (reservoirs in z, phi_s = -0.7, F_z = 1e-5) in FP32 and
    FP16 storage, plus per-quantity errors of both against the FP64 oracle on
    the 128^3 crop [448, 576)^3 run as its own domain with the same boundaries."""
    import numpy as np
    import torch

    import oracle
    import paper_2007_12266_gb300 as lbm
    from synthetic import crop, workload_precision1024
    t0 = time.perf_counter()
    w = workload_precision1024(args.size)
    gen_s = time.perf_counter() - t0
    kw = dict(tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force, periodic=w.periodic,
              reservoir_z=1, rho_in=w.rho_in, rho_out=w.rho_out)
    out = {"metric": "pore-site MLUPS, 1024^3 displacement, FP32 vs FP16 storage", "unit": "MLUPS",
           "workload": f"{w.name}: porosity {w.porosity:.3f}, periodic x/y, reservoirs in z, phi_s -0.7",
           "steps": args.precision_steps, "generation_s": gen_s}
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for prec in ("fp32", "fp16"):
        d = lbm.Domain(w.labels, w.affinity, precision=prec, **kw)
        d.init_fluids(w.phi0)
        N = d.n_sites
        d.advance(20)
        d.measure()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps = 0
        trace = []
        while steps < args.precision_steps:
            d.advance(500)
            steps += 500
            m = d.measure()
            trace.append((steps + 20, m["sat_mass"], m["flux"][2]))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        bps = BYTES_STEP_FP32 if prec == "fp32" else BYTES_STEP_FP16
        peak, _ = measured_peaks()
        gbs = bps * N * steps / (ms * 1e-3) / 1e9
        out[prec] = {"value": N * steps / (ms * 1e-3) / 1e6, "n_sites": N, "ms_per_step": ms / steps,
                     "step_achieved_gbs": gbs, "step_frac": gbs / peak, "trace": trace[-3:],
                     "status": m["status"]}
        d.close()
        torch.cuda.empty_cache()
    out["fp16_vs_fp32"] = out["fp16"]["value"] / out["fp32"]["value"]
    # the 128^3 crop: oracle vs both storages
    lo, hi = (448, 448, 448), (576, 576, 576)
    if args.size < 1024:
        c = args.size // 2
        lo, hi = (c - 64, c - 64, c - 64), (c + 64, c + 64, c + 64)
    lab, aff, phi0 = crop(w.labels, lo, hi), crop(w.affinity, lo, hi), crop(w.phi0, lo, hi)
    del w
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.Oracle(lab, aff, kw["periodic"], tau_a=kw["tau_a"], tau_b=kw["tau_b"], alpha=kw["alpha"],
                        beta=kw["beta"], force=kw["force"], reservoir_z=1, rho_in=kw["rho_in"],
                        rho_out=kw["rho_out"])
    ref.init_fluids(phi0)
    t1 = time.perf_counter()
    ref.step(args.crop_steps)
    oracle_s = time.perf_counter() - t1
    mo = ref.measure()
    phi_o, p_o, u_o = ref.fields()
    sv, _ = ref.index()
    crop_out = {"box": [lo, hi], "n_sites": ref.N, "steps": args.crop_steps, "oracle_s": oracle_s,
                "oracle_threads": oracle.get_threads()}
    keys = ("sat_mass", "mass_a", "mass_b", "mass_total", "p_a", "p_b", "ca", "sat_count")
    for prec in ("fp32", "fp16"):
        d = lbm.Domain(lab, aff, precision=prec, **kw)
        d.init_fluids(phi0)
        d.advance(args.crop_steps)
        m = d.measure()
        errs = {k: abs(m[k] - mo[k]) / max(abs(mo[k]), 1e-300) for k in keys}
        for a, ax in enumerate("xyz"):
            for f in ("flux", "flux_a", "flux_b"):
                scale = max(abs(mo[f + "_z"]), 1e-300)
                errs[f"{f}_{ax}"] = abs(m[f][a] - mo[f"{f}_{ax}"]) / scale
        phi_g = d.read_field("phi").ravel()[sv]
        uz_g = d.read_field("uz").ravel()[sv]
        errs["phi_max_abs"] = float(np.abs(phi_g - phi_o).max())
        errs["phi_rms"] = float(np.sqrt(np.mean((phi_g - phi_o) ** 2)))
        errs["uz_rms_rel"] = float(np.sqrt(np.mean((uz_g - u_o[2]) ** 2)) / max(np.sqrt(np.mean(u_o[2] ** 2)), 1e-300))
        crop_out[prec] = {k: float(v) for k, v in errs.items()}
        d.close()
    crop_out["oracle_measures"] = {k: mo[k] for k in ("sat_mass", "flux_z", "ca", "p_a", "p_b")}
    out["crop"] = crop_out
    print(json.dumps(out))
    return 0


def bench_prepare(args):
    """Image preparation calls on a size^3 sphere pack: mixing region (Sec.
    4.2) and mixed-wet relabel at radius 2 (Sec. 3.3). Each call copies the
    image to the device, runs one kernel and copies it back; the line reports
    the wall time per call (median of 5) and the voxel rate. The kernels'
    own device times come from the ncu summary in profiles/."""
    import numpy as np
    import torch

    import paper_2007_12266_gb300 as lbm
    from synthetic import phi0_blob, sphere_pack
    L = args.size
    t0 = time.perf_counter()
    lab = sphere_pack(L, 0.2, 10.0, 3.0, 4).labels
    oil = (phi0_blob(lab, 0.5, 5) < 0) & (lab == 0)
    gen_s = time.perf_counter() - t0
    torch.cuda.init()
    V = lab.size
    out = {"metric": "image preparation, voxels per second through the C ABI (host copies included)",
           "unit": "Gvox/s", "workload": f"{L}^3 sphere pack, porosity 0.2, blob oil phase (Sw 0.5)",
           "voxels": V, "generation_s": gen_s}
    for name, fn in (("mixing_layer", lambda: lbm.mixing_layer(lab, 8, axis=2)),
                     ("mixed_wet_relabel", lambda: lbm.mixed_wet_relabel(lab, oil, radius=2.0, new_label=2))):
        fn()
        ts = []
        for _ in range(5):
            t1 = time.perf_counter()
            r = fn()
            ts.append(time.perf_counter() - t1)
        med = statistics.median(ts)
        out[name] = {"seconds_per_call": med, "value": V / med / 1e9, "changed_voxels": int(np.count_nonzero(r != lab))}
    # shell aggregation step on the 256^3 steady-state workload after 100 steps
    from synthetic import workload_steady256
    w = workload_steady256(256)
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha,
                     beta=w.beta, force=w.force)
    dom.init_fluids(w.phi0)
    dom.advance(100)
    dom.morph(1.0, apply=False)
    ts = []
    for _ in range(5):
        t1 = time.perf_counter()
        b, a = dom.morph(1.0, apply=False)
        ts.append(time.perf_counter() - t1)
    med = statistics.median(ts)
    out["morph_256"] = {"seconds_per_call": med, "sites": dom.n_sites, "value": dom.n_sites / med / 1e9,
                        "unit": "Gsite/s", "a_sites_before": b, "a_sites_after_delta_1": a}
    dom.close()
    print(json.dumps(out))
    return 0


SERVING_L = (64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384)


def serving_trace(jobs, prec, max_steps, device):
    """Serving trace: Poisson arrivals at 20/s of jobs with L in {64, 96, ...,
    384}, each stopping on the flux-change test (1e-4 over 500 steps) or at
    max_steps; then the same jobs again at an arrival rate of 70 % of the
    capacity the first run measured, to show the latency of the continuous
    batcher itself rather than of the queue."""
    r1 = bench_serving(jobs, prec, 20.0, 5, max_steps, 500, device)
    # capacity in jobs per second: aggregate site-update rate over the mean work of a job
    work = r1["mean_sites"] * r1["mean_steps"]
    cap = r1["aggregate_value"] * 1e6 / max(work, 1.0)
    r2 = bench_serving(jobs, prec, 0.7 * cap, 6, max_steps, 500, device)
    r2["capacity_jobs_per_s"] = cap
    return {"workload": (f"{len(jobs)} Poisson arrivals, L uniform on {SERVING_L}, porosity U[0.15, 0.35], "
                         f"50 % steady, 30 % unsteady, 20 % centrifuge; flux-change 1e-4 every 500 steps or "
                         f"{max_steps} steps; {prec} storage"),
            "lambda_20": r1, "lambda_70pct_capacity": r2}


def bench_serving_trace(args):
    """--mode serving: the serving trace alone (see serving_trace)."""
    import torch
    t0 = time.perf_counter()
    jobs = _spawn_map(_serving_job, [(i, SERVING_L) for i in range(args.serving_jobs)])
    gen_s = time.perf_counter() - t0
    torch.cuda.set_device(0)
    out = {"metric": "serving latency p50/p99 and aggregate pore-site MLUPS", "unit": "MLUPS",
           "generation_s": gen_s}
    out.update(serving_trace(jobs, args.precision, args.serving_max_steps, 0))
    print(json.dumps(out))
    return 0


def bench_gpu(args):
    import numpy as np
    import torch

    import paper_2007_12266_gb300 as lbm

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = build_workload(args.size)
    prec = args.precision
    kw = dict(tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force,
              precision=prec, periodic=w.periodic)
    dom = lbm.Domain(w.labels, w.affinity, device=local_rank, **kw)
    dom.init_fluids(w.phi0)
    N = dom.n_sites
    bundle = args.bundle
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(args.warmup):
        dom.advance(bundle)
        dom.measure()
    barrier()

    # device-timed region: step bundles replay as CUDA graphs
    sampler = ClockSampler(local_rank)
    sampler.start()
    sampler.wait_first()
    l0 = dom.launch_count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        dom.advance(bundle)
        m = dom.measure()
    ev1.record(stream)
    barrier()
    launches = dom.launch_count - l0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms, site_updates = reduce_over_ranks(ms, float(N * bundle * args.steps), world, dev)
    value = site_updates / (ms * 1e-3) / 1e6

    # per-kernel durations: a second pass with CUDA events around every launch
    # on the library's stream (plain launches instead of graphs)
    dom.enable_kernel_timing(True)
    dom.kernel_timing()
    for _ in range(max(1, min(args.steps, 4))):
        dom.advance(bundle)
    kt = dom.kernel_timing()
    dom.enable_kernel_timing(False)

    # end to end through the public API, host buffers (pinned)
    lab_h = torch.from_numpy(np.ascontiguousarray(w.labels)).pin_memory()
    aff_h = torch.from_numpy(np.ascontiguousarray(w.affinity)).pin_memory()
    phi_h = torch.from_numpy(np.ascontiguousarray(w.phi0)).pin_memory()
    lab_np, aff_np, phi_np = lab_h.numpy(), aff_h.numpy(), phi_h.numpy()
    e2e_dom = lbm.Domain(lab_np, None, device=local_rank, **kw)
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_dom.load_image(lab_np)
        e2e_dom.set_affinity_map(aff_np)
        e2e_dom.init_fluids(phi_np)
        e2e_dom.advance(bundle)
        me = e2e_dom.measure()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = N * bundle * e2e_steps * world / e2e_s / 1e6
    h2d = w.labels.nbytes + w.affinity.nbytes + w.phi0.nbytes
    e2e_dom.close()

    # the same workload with FP16 storage
    fp16 = None
    if prec == "fp32" and not args.no_fp16:
        d16 = lbm.Domain(w.labels, w.affinity, device=local_rank, **dict(kw, precision="fp16"))
        d16.init_fluids(w.phi0)
        for _ in range(args.warmup):
            d16.advance(bundle)
            d16.measure()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            d16.advance(bundle)
            m16 = d16.measure()
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms16 = f0.elapsed_time(f1)
        d16.enable_kernel_timing(True)
        d16.kernel_timing()
        d16.advance(bundle * 2)
        kt16 = d16.kernel_timing()
        d16.close()
        v16 = N * bundle * args.steps / (ms16 * 1e-3) / 1e6
        fp16 = {"value": v16, "unit": "MLUPS", "ms_per_step": ms16 / args.steps, "ratio_vs_fp32": v16 / value,
                "step_achieved_gbs": BYTES_STEP_FP16 * N * bundle * args.steps / (ms16 * 1e-3) / 1e9,
                "collide_avg_launch_ms": kt16["collide_ms"] / max(kt16["collide_launches"], 1),
                "phase_avg_launch_ms": kt16["phase_ms"] / max(kt16["phase_launches"], 1),
                "sat_mass": m16["sat_mass"], "flux_z": m16["flux"][2]}

    batched = None
    batched_launch = None
    if args.batched_launch:
        batched_launch = tuple(int(x) for x in args.batched_launch.split(":"))
        if len(batched_launch) != 2:
            raise SystemExit("--batched-launch takes THREADS:BLOCKS_PER_SM")
    if not args.no_batched:
        try:
            # the jobs are independent: each rank runs its round-robin share
            mine = shard(args.batched_jobs, rank, world)
            jobs = _spawn_map(_batched_job, mine)
            batched = {"workload": f"{args.batched_jobs} sphere-pack jobs, L in {{64..192}}, porosity U[0.15,0.35]"
                                   + (f", {world} ranks, round-robin shards" if world > 1 else "")}
            for bprec in ("fp32", "fp16"):
                r = bench_batched(jobs, bprec, args.batched_steps, local_rank, batched_launch)
                ms_all, su_all = reduce_over_ranks(r["ms"], float(r["n_sites"] * r["steps"]), world, dev)
                r["value"] = su_all / (ms_all * 1e-3) / 1e6
                r["ms"] = ms_all
                batched[bprec] = r
            batched["fp16_vs_fp32"] = batched["fp16"]["value"] / batched["fp32"]["value"]
            batched["fp16_vs_plain_fp32"] = batched["fp16"]["value"] / value
            del jobs
        except Exception as exc:
            batched = {"error": repr(exc)}

    serving = None
    if not args.no_serving and world == 1:
        try:
            sj = _spawn_map(_serving_job, [(i, SERVING_L) for i in range(args.serving_jobs)])
            serving = serving_trace(sj, "fp16", args.serving_max_steps, local_rank)
            for r in (serving["lambda_20"], serving["lambda_70pct_capacity"]):
                r["vs_plain_fp32"] = r["aggregate_value"] / value
            del sj
        except Exception as exc:
            serving = {"error": repr(exc)}

    peak, peak_kind = measured_peaks()
    bytes_c = BYTES_COLLIDE_FP32 if prec == "fp32" else BYTES_COLLIDE_FP16
    bytes_s = BYTES_STEP_FP32 if prec == "fp32" else BYTES_STEP_FP16
    c_ms = kt["collide_ms"] / max(kt["collide_launches"], 1)
    p_ms = kt["phase_ms"] / max(kt["phase_launches"], 1)
    achieved = bytes_c * N / (c_ms * 1e-3) / 1e9
    traffic = traffic_per_launch(prec, N)

    # HBM fraction the second way: DRAM bytes the ncu capture measured per
    # site for the collide and phase kernels, over the device-timed step
    nt = ncu_traffic(prec)
    step_dram = None
    if nt is not None and "phase_bytes_per_site" in nt:
        gbs = (nt["bytes_per_site"] + nt["phase_bytes_per_site"]) * N * bundle * args.steps / (ms * 1e-3) / 1e9
        step_dram = {"gbs": gbs, "frac": gbs / peak if peak else None, "frac_of_8tbs": gbs / 8000.0,
                     "bytes_per_site": nt["bytes_per_site"] + nt["phase_bytes_per_site"]}

    out = None
    if rank == 0:
        step_gbs = bytes_s * N * bundle * args.steps / (ms * 1e-3) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_label(w, args.size),
                       "n_sites": N, "storage": prec, "timesteps_per_step": bundle,
                       "step_form": ("components carried as per-site fixed-point sums inside each "
                                     f"{bundle}-timestep call (populations at its first and last step)"),
                       "analysis_per_step": "fp64 basic analysis (saturation, fluxes, Ca)",
                       "l2": "state larger than L2 (no flush needed)",
                       "kernel_timing": "second pass, CUDA events around each launch",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "collide_stream", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_site": bytes_c,
                         "dram_bytes_per_site": None if nt is None else nt["bytes_per_site"],
                         "avg_launch_ms": c_ms, "launches": kt["collide_launches"],
                         "phase_avg_launch_ms": p_ms,
                         "step_achieved_gbs": step_gbs, "step_frac": step_gbs / peak,
                         "step_frac_of_8tbs": step_gbs / 8000.0, "step_dram_ncu": step_dram},
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 27 * 8, "steps": e2e_steps},
            "fp16": fp16,
            "batched": batched,
            "serving": serving,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "measures_last": {"sat_mass": m["sat_mass"], "flux_z": m["flux"][2], "ca": m["ca"],
                              "status": m["status"]},
        }
        if not args.no_cpu_baseline:
            try:
                import oracle
                threads = os.cpu_count() or 1
                n, times = run_cpu_baseline(w, args.cpu_steps, threads)
                cv = n * len(times) / sum(times) / 1e6
                out["cpu_baseline"] = {"value": cv, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                                       "sample": f"{len(times)} timesteps of the same workload "
                                                 f"({n} sites), OpenMP={oracle.have_openmp()}"}
                n1, t1 = run_cpu_baseline(w, 3, 1)
                out["cpu_baseline"]["single_thread"] = {
                    "value": n1 * len(t1) / sum(t1) / 1e6, "unit": "MLUPS", "cores": 1,
                    "sample": f"{len(t1)} timesteps of the same workload, one thread"}
            except Exception as exc:  # the baseline is informative only
                out["cpu_baseline"] = {"value": None, "unit": "MLUPS", "cores": None,
                                       "kind": "oracle", "sample": f"failed: {exc}"}
    dom.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser(description="Pore-site MLUPS of the color-gradient LBM step on GB300 "
                                             "(one JSON line on stdout)")
    ap.add_argument("--gpus", type=int, default=1, help="GPUs (launch under torchrun for more than one)")
    ap.add_argument("--steps", type=int, default=10, help="timed bench steps (one step = --bundle timesteps "
                                                          "+ the fp64 analysis)")
    ap.add_argument("--warmup", type=int, default=3, help="untimed warm-up steps")
    ap.add_argument("--impl", default="native", choices=["native", "reference"],
                    help="native: the CUDA library; reference: the FP64 oracle on the host cores")
    ap.add_argument("--mode", default="headline", choices=["headline", "precision", "serving", "prepare"],
                    help="headline line, 1024^3 FP32 vs FP16 with the oracle crop, full serving trace, "
                         "or image preparation")
    ap.add_argument("--precision-steps", type=int, default=5000, help="precision mode: timesteps")
    ap.add_argument("--crop-steps", type=int, default=5000, help="precision mode: timesteps of the oracle crop")
    ap.add_argument("--size", type=int, default=256, help="edge of the headline (or precision) sphere pack")
    ap.add_argument("--bundle", type=int, default=100, help="timesteps per bench step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"], help="storage of the headline run")
    ap.add_argument("--cpu-steps", type=int, default=20, help="timesteps of the oracle's CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle's CPU baseline")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-storage run of the headline workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched job set")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run")
    ap.add_argument("--batched-jobs", type=int, default=64, help="jobs of the batched set")
    ap.add_argument("--batched-steps", type=int, default=2000, help="timesteps of the batched set")
    ap.add_argument("--batched-launch", default=None,
                    help="launch shape of the batched set as THREADS:BLOCKS_PER_SM (-1 one block per tile, "
                         "-2 fused kernel) instead of the autotuner's choice")
    ap.add_argument("--serving-jobs", type=int, default=16, help="arrivals of the serving trace")
    ap.add_argument("--serving-max-steps", type=int, default=10000, help="step ceiling of a serving job")
    args = ap.parse_args()
    if args.impl == "reference":
        return bench_reference(args)
    if args.mode == "precision":
        return bench_precision(args)
    if args.mode == "serving":
        return bench_serving_trace(args)
    if args.mode == "prepare":
        return bench_prepare(args)
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
