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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(precision: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_12266_gb300", "csrc")
    for name in ("step_kernels.cuh", "step.cu", "lattice.cuh", "internal.h"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    h.update(precision.encode())
    return h.hexdigest()[:16]


def traffic_per_launch(precision: str, n_sites: int):
    """DRAM bytes per collide launch from the committed ncu summary, scaled to
    n_sites; None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "collide_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(precision)
    if not e or e.get("kernel_hash") != kernel_hash(precision):
        return None
    return float(e["bytes_per_site"]) * n_sites


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

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
        "impl": "reference", "metric": "pore-site MLUPS", "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_sites": n, "timesteps_per_step": 1,
                   "note": "FP64 CPU oracle, one timestep of the full workload per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{len(timed)} timesteps of the {args.size}^3 workload "
                                   f"({n} pore sites), OpenMP={oracle.have_openmp()}"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
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
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    site_updates = N * bundle * args.steps * world
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

    peak, peak_kind = measured_peaks()
    bytes_c = BYTES_COLLIDE_FP32 if prec == "fp32" else BYTES_COLLIDE_FP16
    bytes_s = BYTES_STEP_FP32 if prec == "fp32" else BYTES_STEP_FP16
    c_ms = kt["collide_ms"] / max(kt["collide_launches"], 1)
    p_ms = kt["phase_ms"] / max(kt["phase_launches"], 1)
    achieved = bytes_c * N / (c_ms * 1e-3) / 1e9
    traffic = traffic_per_launch(prec, N)

    out = None
    if rank == 0:
        step_gbs = bytes_s * N * bundle * args.steps / (ms * 1e-3) / 1e9
        out = {
            "metric": f"pore-site MLUPS ({prec.upper()} store)", "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{w.name}: {args.size}^3 sphere pack, porosity "
                                   f"{w.porosity:.3f}, z periodic, x/y walls, Sw=0.4 blobs",
                       "n_sites": N, "storage": prec, "timesteps_per_step": bundle,
                       "analysis_per_step": "fp64 basic analysis (saturation, fluxes, Ca)",
                       "l2": "state larger than L2 (no flush needed)",
                       "kernel_timing": "second pass, CUDA events around each launch",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "collide_stream", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_site": bytes_c,
                         "avg_launch_ms": c_ms, "launches": kt["collide_launches"],
                         "phase_avg_launch_ms": p_ms,
                         "step_achieved_gbs": step_gbs, "step_frac": step_gbs / peak,
                         "step_frac_of_8tbs": step_gbs / 8000.0},
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 27 * 8, "steps": e2e_steps},
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
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--bundle", type=int, default=100)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return bench_reference(args)
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
