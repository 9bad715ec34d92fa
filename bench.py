#!/usr/bin/env python
"""Benchmark of the SPIDER stencil path on GB300: GStencil/s.

One benchmark "step" is one complete spider_run of the workload: every time
step of it (e.g. 100 steps of a 7x7 box stencil on an 8192^2 grid), with the
input grid resident in HBM.  GStencil/s = grid points x time steps / seconds
/ 1e9.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W]
                  [--workload box2d|heat2d|heat3d|box3d|batched|batched_small|serving|sweep|mma_peak]
                  [--precision tf32|f16x2|bf16x3] [--impl spider|reference] [--no-accuracy] [--no-workloads]

Under torchrun every rank runs the whole workload on its own GPU (independent
replicas, weak scaling); the reported value is the total over ranks divided
by the slowest rank's time.  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import signal
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import stencil_inputs as si  # noqa: E402

WORKLOADS = {
    "box2d": si.BOX2D_R3_8192,
    "heat2d": si.HEAT2D_512,
    "heat3d": si.HEAT3D_512,
    "box3d": si.BOX3D_512,
}
DEFAULT_STEPS = {"box2d": 300, "heat2d": 2000, "heat3d": 60, "box3d": 60, "batched": 10, "batched_small": 10,
                 "serving": 1, "sweep": 10, "mma_peak": 1}
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="spider", choices=["spider", "reference"])
    ap.add_argument("--workload", default="box2d",
                    choices=sorted(WORKLOADS) + ["batched", "batched_small", "serving", "sweep", "mma_peak"])
    ap.add_argument("--precision", default="tf32", choices=["tf32", "f16x2", "bf16x3"])
    ap.add_argument("--engine", default="sparse_tc",
                    choices=["sparse_tc", "dense_tc", "cuda_core", "sparse_tc_copy", "sparse_tc_no_co"])
    ap.add_argument("--steps-per-pass", type=int, default=None,
                    help="time steps fused per HBM pass (default: chosen by spider_plan_autotune)")
    ap.add_argument("--tile-variant", type=int, default=None)
    ap.add_argument("--radius", type=int, default=None,
                    help="override the workload's stencil radius (box2d: 1..7)")
    ap.add_argument("--extents", type=int, nargs="+", default=None,
                    help="override the grid size (same distributions; for profiling runs)")
    ap.add_argument("--jobs", type=int, default=None, help="batched: use the first N of the 64 jobs")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the full-grid relative L2 error against the FP64 oracle (computed by default)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other configurations (Heat-2D, Heat-3D, Box-3D, batched, serving) in the "
                         "default line")
    ap.add_argument("--serving-jobs", type=int, default=None,
                    help="serving: how many of the 2000 Poisson arrivals to run (default 600; 200 in the "
                         "default line's summary)")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = DEFAULT_STEPS[a.workload]

    a.warmup = max(3, a.warmup)
    return a


# ------------------------------------------------------------------ helpers
def reduce_max_seconds(dt: float, device=None) -> float:
    """The slowest rank's time (all ranks receive it); dt itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dt
    t = torch.tensor([dt], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gstencil(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Aggregate throughput: stencil updates of all ranks over the slowest rank's time."""
    return world * units_per_rank / max_seconds / 1e9


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# The files that define the stencil kernels, their geometry and their launch
# configuration: a change to any of them invalidates recorded ncu counters.
KERNEL_SOURCES = ("device_common.cuh", "fused_kernels.cuh", "launch.cu", "launch.h", "launch_impl.cuh",
                  "spider_internal.h", "stencil_kernels.cuh", "stream3d_fused_kernels.cuh", "stream3d_kernels.cuh",
                  "wide_kernels.cuh")


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_22035_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (profiles/traffic.md rows:
    | key | bytes per launch | source sha | ...)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha()
    for line in open(path):
        m = re.match(r"\|\s*([^|]+?)\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]+)\s*\|", line)
        if m and m.group(1) == kernel_key and m.group(3) == sha:
            return float(m.group(2))
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.send_signal(signal.SIGTERM)
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(wl, budget_s: float = 12.0):
    """The FP64 oracle as it stands, timed on the host cores on a bounded
    sample of the workload (a crop of the grid, fewer time steps)."""
    import oracle
    u0, w = si.workload_inputs(wl, extents=wl.extents)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.stencil(u0, w, 1)
    one = max(time.perf_counter() - t0, 1e-4)
    steps = int(max(1, min(wl.steps, budget_s / one)))
    t0 = time.perf_counter()
    oracle.stencil(u0, w, steps)
    dt = time.perf_counter() - t0
    pts = int(np.prod(u0.shape))
    # one core, on a crop of the grid (a bounded sample, about a second)
    side = [min(n, 1024) for n in u0.shape] if u0.ndim < 3 else [min(n, 128) for n in u0.shape]
    crop = np.ascontiguousarray(u0[tuple(slice(0, n) for n in side)])
    t1 = time.perf_counter()
    oracle.stencil(crop, w, 1, threads=1)
    dt1 = max(time.perf_counter() - t1, 1e-6)
    return {"value": pts * steps / dt / 1e9, "unit": "GStencil/s", "cores": cores, "kind": "oracle",
            "cpu": host_cpu_model(),
            "value_1core": crop.size / dt1 / 1e9,
            "sample": f"{wl.name} grid {'x'.join(map(str, u0.shape))}, {steps} of its {wl.steps} time steps, "
                      f"FP64 direct stencil (C, OpenMP, {cores} threads), {dt:.1f} s; 1 core: one step of a "
                      f"{'x'.join(map(str, crop.shape))} crop"}


def host_cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo, or lscpu's fields on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ reference arm
def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = WORKLOADS.get(a.workload, si.BOX2D_R3_8192)
    # each benchmark step is a bounded sample of the workload, sized so the
    # whole run (warm-up + timed) ends within about two minutes
    per_step_budget = 90.0 / (a.steps + a.warmup)
    side = 1024 if wl.ndim == 2 else 96
    u0, w = si.workload_inputs(wl, extents=tuple(min(e, side) for e in wl.extents))
    t0 = time.perf_counter()
    oracle.stencil(u0, w, 1)
    one = max(time.perf_counter() - t0, 1e-5)
    while one > per_step_budget and min(u0.shape) > 16:
        u0 = u0[tuple(slice(0, max(16, s // 2)) for s in u0.shape)].copy()
        t0 = time.perf_counter()
        oracle.stencil(u0, w, 1)
        one = max(time.perf_counter() - t0, 1e-5)
    tsteps = int(max(1, min(wl.steps, per_step_budget / one)))
    for _ in range(a.warmup):
        oracle.stencil(u0, w, tsteps)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.stencil(u0, w, tsteps)
    dt = time.perf_counter() - t0
    pts = int(np.prod(u0.shape))
    value = pts * tsteps * a.steps / dt / 1e9
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": "GStencil/s", "value": value, "unit": "GStencil/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, a, extra={"sample": "x".join(map(str, u0.shape)), "time_steps": tsteps}),
        "cpu_baseline": {"value": value, "unit": "GStencil/s", "cores": cores, "kind": "oracle",
                         "sample": f"{wl.name} cropped to {'x'.join(map(str, u0.shape))}, {tsteps} time steps per "
                                   f"benchmark step"},
        "e2e": {"value": value, "unit": "GStencil/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(wl, a, extra=None):
    cfg = {"workload": f"{wl.name}, {wl.steps} time steps", "stencil": f"{wl.shape} r={wl.r} {wl.ndim}-D",
           "extents": list(wl.extents), "time_steps": wl.steps, "precision": a.precision, "engine": a.engine,
           "steps_per_pass": a.steps_per_pass, "tile_variant": a.tile_variant, "global_batch": 1,
           "l2": "inputs larger than L2" if 4 * int(np.prod(wl.extents)) > L2_BYTES else "L2 flushed between timed runs",
           "parallelism": f"replicas{a.gpus}"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ spider arm
def time_runs(plan, a_in, b_out, steps_per_run, iters, flush_buf, stream):
    """Total device seconds of `iters` runs (CUDA events on `stream`)."""
    import torch
    if flush_buf is None:
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(iters):
            plan.run(a_in, b_out, steps_per_run, stream)
        e.record(stream)
        e.synchronize()
        return s.elapsed_time(e) * 1e-3
    total = 0.0
    for _ in range(iters):
        with torch.cuda.stream(stream):  # ordered before the timed region on the timed stream
            flush_buf.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        plan.run(a_in, b_out, steps_per_run, stream)
        e.record(stream)
        e.synchronize()
        total += s.elapsed_time(e) * 1e-3
    return total


def run_spider(a):
    import torch
    import torch.distributed as dist

    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import build as _b
    _b.build()

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = WORKLOADS[a.workload]
    if a.radius:
        # another radius of the same stencil family (e.g. the wide layout, r = 4..7)
        wl = dataclasses.replace(wl, r=a.radius, name=wl.name.replace(f"-r{wl.r}-", f"-r{a.radius}-"))
    if a.extents:
        wl = dataclasses.replace(wl, extents=tuple(a.extents), name=f"{wl.name.split('-')[0]}-r{wl.r}-"
                                 + "x".join(map(str, a.extents)))
    u0, w = si.workload_inputs(wl, extents=wl.extents)
    pts = int(np.prod(wl.extents))
    grid_bytes = 4 * pts
    plan = spider.Plan(w, wl.extents, wl.shape, a.precision, a.engine)
    a_in = torch.from_numpy(u0).to(dev)
    b_out = torch.empty_like(a_in)

    def configure(p):
        """Steps per pass and tile variant: given on the command line, else
        picked by the library's autotuner (outside the timed region)."""
        if a.steps_per_pass is None and a.tile_variant is None:
            return p.autotune(a_in, b_out, wl.steps, stream)
        t = a.steps_per_pass or 1
        v = a.tile_variant or 0
        if t > 1:
            p.set_steps_per_pass(t)
        p.set_tile_variant(v)
        return t, v

    chosen_T, chosen_v = configure(plan)
    a.steps_per_pass, a.tile_variant = chosen_T, chosen_v
    flush = None if grid_bytes > L2_BYTES else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(a.warmup):
        plan.run(a_in, b_out, wl.steps, stream)
    plan.sync(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    smi_index = visible[local] if local < len(visible) and visible[local].strip().isdigit() else str(local)
    with ClockSampler(smi_index) as clk:
        barrier()
        dt = time_runs(plan, a_in, b_out, wl.steps, a.steps, flush, stream)
        barrier()
    plan.sync(stream)
    dt = reduce_max_seconds(dt, dev)
    T = a.steps_per_pass
    launches_per_run = wl.steps // T + (1 if wl.steps % T else 0)  # one launch per pass
    total_launches = a.steps * launches_per_run
    value = whole_job_gstencil(pts * wl.steps * a.steps, world, dt)
    per_launch_s = dt / total_launches

    result = None
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        alg_bytes = 8.0 * pts  # read every point once and write it once per pass
        achieved = alg_bytes / per_launch_s / 1e9
        if wl.ndim == 3:
            kernel = "stream3d_fused_kernel" if T > 1 else "stream3d_kernel"
        elif wl.ndim == 1 or wl.r > 3:
            kernel = "wide_step_kernel"
        else:
            kernel = "fused_step_kernel" if T > 1 else "stencil_step_kernel"
        # every tile variant of a given T loads the same boxes and writes the
        # same tiles, so DRAM traffic is keyed by T only
        kernel_key = f"{kernel} {wl.name} {a.engine} {a.precision} T{T}"
        traffic = traffic_from_profiles(kernel_key)
        result = {
            "metric": "GStencil/s", "value": value, "unit": "GStencil/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.precision, "data": "synthetic",
            "config": workload_config(wl, a),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]), "traffic": traffic,
                         "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "algorithmic_bytes_per_launch": alg_bytes, "launch_us": per_launch_s * 1e6},
            "gpu_launches": total_launches,
            "clocks": clk.summary(),
        }

    # end-to-end through the host-buffer entry points: pinned host input, H2D,
    # all time steps, D2H, inside the timed region, every step.  The value is
    # a stream of steps through spider_run_host_async (each step's copies
    # overlap the previous step's passes); "sequential" is one blocking
    # spider_run_host call after another (copies and passes in series)
    if not a.no_e2e:
        host_in = torch.from_numpy(u0).pin_memory()
        host_outs = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        hin, houts = host_in.numpy(), [h.numpy() for h in host_outs]
        plan.run_host(hin, wl.steps, houts[0], stream)
        e2e_iters = max(3, min(20, a.steps // 20))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_iters):
            plan.run_host(hin, wl.steps, houts[0], stream)
        seq_dt = time.perf_counter() - t0
        for k in range(6):  # both slots' runs captured as graphs (from the third run of a key)
            plan.run_host_async(hin, wl.steps, houts[k % 2], stream)
        plan.sync(stream)
        async_iters = max(8, e2e_iters)  # the first copy in and the last copy out are not overlapped
        barrier()
        t0 = time.perf_counter()
        for k in range(async_iters):
            plan.run_host_async(hin, wl.steps, houts[k % 2], stream)
        plan.sync(stream)
        e2e_dt = time.perf_counter() - t0
        barrier()
        if rank == 0:
            result["e2e"] = {"value": world * pts * wl.steps * async_iters / e2e_dt / 1e9, "unit": "GStencil/s",
                             "h2d_bytes_per_step": grid_bytes, "d2h_bytes_per_step": grid_bytes,
                             "entry_point": "spider_run_host_async (a stream of steps; each step's copies overlap "
                                            "the previous step's passes)",
                             "sequential": {"value": world * pts * wl.steps * e2e_iters / seq_dt / 1e9,
                                            "entry_point": "spider_run_host (blocking)"},
                             "finite": bool(all(np.isfinite(h).all() for h in houts)),
                             "equal_to_device_run": bool(np.array_equal(houts[0], b_out.cpu().numpy()) and
                                                         np.array_equal(houts[1], houts[0]))}

    # comparators and other precisions on the same GPU and workload
    if rank == 0 and not a.no_comparators:
        comps = {}
        # each comparator at its own autotuned setting; the "/T1" entries run
        # the one-step tile (one step per pass, tile variant 0), the kernel
        # the explicit-copy and no-CO comparators are built on: dense TC ->
        # sparse TC without the Sec. 3.3 optimisations -> SPIDER is the
        # Sec. 4.4 ablation at one step per pass
        variants = [("sparse_tc", "tf32", None), ("sparse_tc", "f16x2", None), ("sparse_tc", "bf16x3", None),
                    ("dense_tc", "tf32", None), ("cuda_core", "tf32", None), ("sparse_tc_copy", "tf32", None),
                    ("sparse_tc_no_co", "tf32", None), ("sparse_tc", "tf32", (1, 0)), ("dense_tc", "tf32", (1, 0))]
        for eng, prec, fixed in variants:
            if (eng, prec) == (a.engine, a.precision) and fixed is None:
                continue
            name = f"{eng}/{prec}" + ("/T1" if fixed else "")
            try:
                p2 = spider.Plan(w, wl.extents, wl.shape, prec, eng)
            except spider.SpiderError as err:  # e.g. radius 4..7 exists for sparse TF32 only
                comps[name] = {"value": None, "unsupported": str(err)}
                continue
            if fixed:
                t2, v2 = fixed
                p2.set_tile_variant(v2)
            else:
                t2, v2 = p2.autotune(a_in, b_out, wl.steps, stream)
            iters = max(3, a.steps // 10)
            for _ in range(2):
                p2.run(a_in, b_out, wl.steps, stream)
            torch.cuda.synchronize(dev)
            d2 = time_runs(p2, a_in, b_out, wl.steps, iters, flush, stream)
            p2.sync(stream)
            comps[name] = {"value": pts * wl.steps * iters / d2 / 1e9, "steps_per_pass": t2, "tile_variant": v2}
            p2.close()
        result["comparators"] = comps

    if rank == 0 and not a.no_accuracy:
        # full-grid relative L2 error of every precision against the FP64
        # oracle (outside the timed region), each at its autotuned setting
        import oracle
        ref_t = torch.from_numpy(oracle.stencil(u0, w, wl.steps)).to(dev)
        errs = {}
        for prec in ("tf32", "f16x2", "bf16x3"):
            p2 = spider.Plan(w, wl.extents, wl.shape, prec, a.engine)
            if prec == a.precision:
                p2.set_steps_per_pass(a.steps_per_pass)
                p2.set_tile_variant(a.tile_variant)
            else:
                p2.autotune(a_in, b_out, wl.steps, stream)
            p2.run(a_in, b_out, wl.steps, stream)
            errs[prec] = {"rel_l2": spider.relative_l2_error(b_out, ref_t, stream),
                          "a_priori_bound": p2.error_bound(wl.steps)}
            p2.close()
        del ref_t
        result["rel_l2_error_vs_fp64"] = errs

    if rank == 0 and a.workload == "box2d" and a.radius in (None, 3) and not a.extents:
        # the tensor-pipe roofline of the fused kernel: sparse MMAs per launch
        # (its tile geometry) over the measured mma.sp peak of this GPU
        peak_mma = spider.measure_mma_rate("sp_tf32" if a.precision == "tf32" else "sp_f16", stream)
        mmas = fused_mmas_per_launch(wl.extents, wl.r, a.steps_per_pass, a.tile_variant)
        if mmas is not None and a.precision == "tf32" and a.engine == "sparse_tc":
            achieved = mmas / per_launch_s
            result["roofline_tensor"] = {
                "bound": "tensor", "achieved": achieved / 1e9, "peak": peak_mma / 1e9, "unit": "G mma.sp/s",
                "frac": achieved / peak_mma, "mmas_per_launch": mmas,
                "peak_source": "measured: spider_measure_mma_rate (mma.sp m16n8k16 TF32, operands in registers)"}

    if rank == 0 and world == 1 and not a.no_workloads and a.workload == "box2d" and not a.extents \
            and a.radius in (None, 3):
        result["workloads"] = other_workloads(a, spider, dev, stream)

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(wl)

    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def fused_mmas_per_launch(extents, r, T, variant):
    """Sparse MMAs one launch of the fused 2-D TF32 kernel issues: every tile
    computes levels 1..T, level t of BY + 2r(T - t) rows and BX + 8(T - t)
    columns in warp units of H rows x 64 columns, each unit (H / 2)(2r + 2)
    MMAs (level 1 is 64 rows, 32 for variant 4; BY = level 1 - 2r(T - 1),
    BX = 8(17 - T); H = 16 for variants 1 and 3, else 8).  Deep tiles (T > 4)
    are 16 x 64 outputs.  None for T = 1 (the one-step kernel)."""
    if T < 2:
        return None
    ny, nx = extents
    if T > 4:
        by, bx, h = 16, 64, 8
    else:
        l1 = 32 if variant == 4 else 64
        by, bx, h = l1 - 2 * r * (T - 1), 8 * (17 - T), 16 if variant in (1, 3) else 8
    units = 0
    for t in range(1, T + 1):
        rows, cols = by + 2 * r * (T - t), bx + 8 * (T - t)
        units += -(-rows // h) * -(-(cols // 8) // 8)
    tiles = -(-nx // bx) * -(-ny // by)
    return tiles * units * (h // 2) * (2 * r + 2)


def timed_workload(spider, wl, dev, stream, runs=5, with_error=True, tune=True):
    """GStencil/s, steps per pass, HBM roofline and error vs FP64 of one
    workload run through spider_run (sparse TF32, autotuned)."""
    import torch
    u0, w = si.workload_inputs(wl)
    pts = int(np.prod(wl.extents))
    plan = spider.Plan(w, wl.extents, wl.shape, "tf32")
    x = torch.from_numpy(u0).to(dev)
    y = torch.empty_like(x)
    T, v = plan.autotune(x, y, wl.steps, stream) if tune else (1, 0)
    flush = None if 4 * pts > L2_BYTES else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.run(x, y, wl.steps, stream)
    dt = time_runs(plan, x, y, wl.steps, runs, flush, stream)
    plan.sync(stream)
    launches = runs * (wl.steps // T + (1 if wl.steps % T else 0))
    per_launch = dt / launches
    peaks, kind = measured_peaks()
    hbm = 8.0 * pts / per_launch / 1e9
    rec = {"workload": f"{wl.name}, {wl.steps} time steps", "gstencil_s": pts * wl.steps * runs / dt / 1e9,
           "us_per_run": dt / runs * 1e6, "steps_per_pass": T, "tile_variant": v,
           "roofline": {"bound": "hbm", "achieved": hbm, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                        "frac": hbm / float(peaks["hbm_gbs"]), "peak_source": f"{kind} HBM copy bandwidth"}}
    if with_error:
        import oracle
        ref = torch.from_numpy(oracle.stencil(u0, w, wl.steps)).to(dev)
        plan.run(x, y, wl.steps, stream)
        rec["rel_l2_error_vs_fp64"] = spider.relative_l2_error(y, ref, stream)
        rec["a_priori_bound"] = plan.error_bound(wl.steps)
        del ref
    plan.close()
    return rec, (u0, w, T, v)


def other_workloads(a, spider, dev, stream):
    """The configurations besides the headline, measured in the same process:
    Heat-2D 512^2 (latency-bound: its time against the same passes on a
    one-tile grid), Heat-3D and Box-3D 512^3 (HBM roofline), the batched mix
    (one spider_batch call) and a serving summary."""
    import torch
    out = {}
    rec, (u0, w, T, v) = timed_workload(spider, si.HEAT2D_512, dev, stream, runs=50)
    # latency floor: the same passes on a grid of one 16 x 64 tile (the
    # critical path of one tile's levels per pass, plus the launches)
    one = spider.Plan(w, (16, 64), "star", "tf32")
    if T > 1:
        one.set_steps_per_pass(T)
    one.set_tile_variant(v)
    x1 = torch.from_numpy(np.ascontiguousarray(u0[:16, :64])).to(dev)
    y1 = torch.empty_like(x1)
    for _ in range(5):
        one.run(x1, y1, si.HEAT2D_512.steps, stream)
    floor = time_runs(one, x1, y1, si.HEAT2D_512.steps, 50, None, stream) / 50
    one.close()
    rec["roofline"] = {"bound": "latency", "achieved_us": rec["us_per_run"], "floor_us": floor * 1e6,
                       "frac": floor * 1e6 / rec["us_per_run"],
                       "floor": "the same passes (steps per pass, tile variant, graph replay) on a one-tile "
                                "16 x 64 grid: per pass the chain of one tile's levels plus the launch",
                       "l2_gbs": 8.0 * 512 * 512 * (-(-si.HEAT2D_512.steps // T)) / (rec["us_per_run"] * 1e-6) / 1e9}
    out["heat2d"] = rec
    out["heat3d"] = timed_workload(spider, si.HEAT3D_512, dev, stream)[0]
    out["box3d"] = timed_workload(spider, si.BOX3D_512, dev, stream)[0]
    out["batched"] = batched_summary(spider, dev, stream, calls=5)
    out["serving"] = serving_run(spider, n_jobs=a.serving_jobs or 200)
    return out


def batched_summary(spider, dev, stream, calls=5):
    """One spider_batch call over the 64-grid mix: GStencil/s over `calls`
    timed calls after three warm-up calls (graphs captured and replayed)."""
    import torch
    jobs = si.batched_jobs()
    plans, ins, outs, work = [], [], [], 0
    for jb in jobs:
        u0, w = si.job_inputs(jb)
        plans.append(spider.Plan(w, jb.extents, jb.shape, "tf32"))
        ins.append(torch.from_numpy(u0).to(dev))
        outs.append(torch.empty_like(ins[-1]))
        work += int(np.prod(jb.extents)) * jb.steps
    steps = [jb.steps for jb in jobs]

    def timed():
        for _ in range(3):
            spider.batch(plans, ins, outs, steps, stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(calls):
            spider.batch(plans, ins, outs, steps, stream)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0

    dt = timed()
    # the same call with every grid in the persistent queue (one launch)
    spider.batch_configure(1 << 40, 2)
    try:
        dt_queue = timed()
    finally:
        spider.batch_configure(0, 0)
    for p in plans:
        p.close()
    return {"workload": "batched: 64 2-D grids, sides log-uniform [256, 4096], star/box r 1-3, 10-200 steps",
            "gstencil_s": work * calls / dt / 1e9, "ms_per_call": dt / calls * 1e3, "stencil_updates": work,
            "launch": "grids of >= 2^16 points as fused passes on side streams, smaller ones in the persistent queue",
            "queue_only": {"gstencil_s": work * calls / dt_queue / 1e9, "ms_per_call": dt_queue / calls * 1e3,
                           "launch": "every grid in the persistent tile queue: one kernel launch (a CUDA graph)"},
            "timing": "host clock around synchronous spider_batch calls"}


def run_batched(a):
    """64 2-D grids of mixed size, shape, radius and step count advanced by one
    spider_batch call (one persistent launch over a tile queue, issued as a CUDA
    graph); compared with the same jobs run one spider_run after another."""
    import torch
    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import build as _b
    _b.build()
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    small = a.workload == "batched_small"
    all_jobs = si.batched_small_jobs() if small else si.batched_jobs()
    jobs = all_jobs[: a.jobs] if a.jobs else all_jobs
    plans, ins, outs = [], [], []
    work = 0
    for jb in jobs:
        u0, w = si.job_inputs(jb)
        plans.append(spider.Plan(w, jb.extents, jb.shape, "tf32"))
        ins.append(torch.from_numpy(u0).to(dev))
        outs.append(torch.empty_like(ins[-1]))
        work += int(np.prod(jb.extents)) * jb.steps
    steps = [jb.steps for jb in jobs]
    for _ in range(a.warmup):
        spider.batch(plans, ins, outs, steps, stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        spider.batch(plans, ins, outs, steps, stream)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    # the same calls with every grid in the persistent queue (one launch)
    spider.batch_configure(1 << 40, 2)
    try:
        for _ in range(3):
            spider.batch(plans, ins, outs, steps, stream)
        torch.cuda.synchronize(dev)
        tq = time.perf_counter()
        for _ in range(a.steps):
            spider.batch(plans, ins, outs, steps, stream)
        torch.cuda.synchronize(dev)
        dt_queue = time.perf_counter() - tq
    finally:
        spider.batch_configure(0, 0)
    # the same jobs one after another through spider_run (each plan tuned)
    for p, x, y, n in zip(plans, ins, outs, steps):
        p.autotune(x, y, n, stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for _ in range(max(1, a.steps // 2)):
        for p, x, y, n in zip(plans, ins, outs, steps):
            p.run(x, y, n, stream)
    torch.cuda.synchronize(dev)
    dt_seq = (time.perf_counter() - t1) / max(1, a.steps // 2)
    line = {"metric": "GStencil/s", "value": world * work * a.steps / dt / 1e9, "unit": "GStencil/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32",
            "data": "synthetic",
            "config": {"workload": ("batched_small: 256 2-D grids, sides log-uniform [32, 255] (< 2^16 points "
                                    "each), star/box r 1-3, 10-200 steps") if small else
                                   ("batched: 64 2-D grids, sides log-uniform [256, 4096], star/box r 1-3, "
                                    "10-200 steps"),
                       "stencil_updates_per_step": work, "engine": "sparse_tc",
                       "launch": "one spider_batch call: grids of >= 2^16 points as fused passes on side streams, "
                                 "each replayed as a CUDA graph; smaller grids and single steps in the persistent "
                                 "tile queue (one graph launch)"},
            "queue_only": {"value": world * work * a.steps / dt_queue / 1e9, "unit": "GStencil/s",
                           "launch": "every grid in the persistent tile queue: one kernel launch (a CUDA graph)"},
            "sequential_spider_run": {"value": work / dt_seq / 1e9, "unit": "GStencil/s",
                                      "note": "same jobs, one autotuned spider_run after another"}}
    for p in plans:
        p.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


SWEEP_SIDES = (512, 1024, 2048, 4096, 8192, 10240)


def run_sweep(a):
    """Size sweep and engine ablation (the paper's 512^2 ... 10240^2 trend
    study and its TC -> SpTC ablation on Box-2D2R): 2-D box stencils of radius
    2 and 3, 100 time steps per run, every side in SWEEP_SIDES, each engine
    (sparse TC, dense TC on the same banded K, CUDA cores) at the steps per
    pass and tile variant its autotuner picks.  Prints one JSON line whose
    "sweep" list holds one record per (radius, side, engine)."""
    import torch
    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import build as _b
    _b.build()
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    steps_per_run = 100
    sides = [int(x) for x in a.extents] if a.extents else list(SWEEP_SIDES)
    records = []
    for r in (2, 3):
        gen = si.rng(30, r)
        w = si.normalised_coeffs(2, r, "box", gen)
        for n in sides:
            u0 = si.grid((n, n), -1.0, 1.0, gen)
            a_in = torch.from_numpy(u0).to(dev)
            b_out = torch.empty_like(a_in)
            fl = None if 4 * n * n > L2_BYTES else flush
            for engine in ("sparse_tc", "dense_tc", "cuda_core"):
                plan = spider.Plan(w, (n, n), "box", "tf32", engine)
                T, v = plan.autotune(a_in, b_out, steps_per_run, stream)
                for _ in range(max(3, a.warmup)):
                    plan.run(a_in, b_out, steps_per_run, stream)
                iters = max(2, min(a.steps, int(2e11 // (n * n * steps_per_run)) or 2))
                dt = time_runs(plan, a_in, b_out, steps_per_run, iters, fl, stream)
                plan.close()
                records.append({"radius": r, "side": n, "engine": engine, "steps_per_pass": T, "tile_variant": v,
                                "gstencil_s": n * n * steps_per_run * iters / dt / 1e9,
                                "us_per_run": dt / iters * 1e6})
            del a_in, b_out
    sp = {(x["radius"], x["side"]): x["gstencil_s"] for x in records if x["engine"] == "sparse_tc"}
    for x in records:
        x["sparse_tc_speedup"] = sp[(x["radius"], x["side"])] / x["gstencil_s"]
    best = max(x["gstencil_s"] for x in records if x["engine"] == "sparse_tc")
    line = {"metric": "GStencil/s", "value": best, "unit": "GStencil/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32",
            "data": "synthetic",
            "config": {"workload": "sweep: 2-D box r = 2, 3, sides " + ",".join(map(str, sides)) +
                                   ", 100 time steps per run, each engine autotuned",
                       "l2": "flushed between timed runs for grids smaller than L2"},
            "sweep": records}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serving_run(spider, n_jobs=600, budget=120 * 10**9):
    """The serving configuration: the first `n_jobs` of the 2000 Poisson
    arrivals (200 jobs/s; 2-D sides 256-8192, 3-D sides 64-512, r 1-3, 10-500
    steps, error target 1e-3 or 1e-5) submitted at their arrival times to a
    server with a 120 GB HBM budget; jobs are neither capped nor
    time-compressed.  Latency is each job's submit-to-completion time."""
    jobs = si.serving_arrivals()[:n_jobs]
    pool = si.serving_grid_pool(jobs)
    work = [int(np.prod(j.extents)) * j.steps for j in jobs]
    server = spider.Server(budget)
    plans = [spider.Plan(si.serving_job_coeffs(j), j.extents, j.shape, "tf32") for j in jobs]
    pending, lat, done_at = {}, [], []
    t0 = time.perf_counter()
    base = jobs[0].arrival_s

    def drain(timeout):
        # collect finished jobs (spider_server_wait hands each out once)
        t = server.wait(timeout)
        while t is not None:
            out = np.empty(pending.pop(t), np.float32)
            _, l = server.poll(t, out)   # copies the result and releases the ticket
            lat.append(l)
            done_at.append(time.perf_counter() - t0)
            t = server.wait(0.0)

    for j, p in zip(jobs, plans):
        while time.perf_counter() - t0 < j.arrival_s - base:
            drain(max(0.0, min(0.002, j.arrival_s - base - (time.perf_counter() - t0))))
        n = int(np.prod(j.extents))
        pending[server.submit(p, pool[:n].reshape(j.extents), j.steps, j.err_target)] = n
    while pending:
        drain(0.05)
    server.close()
    for p in plans:
        p.close()
    ls = np.sort(np.asarray(lat))
    span = jobs[-1].arrival_s - base
    busy = max(done_at)
    return {"workload": f"serving: first {len(jobs)} of 2000 Poisson arrivals at 200 jobs/s, 2-D side 256-8192 / "
                        "3-D side 64-512, r 1-3, 10-500 steps, error target 1e-3 or 1e-5, 120 GB HBM budget",
            "jobs_completed": len(lat), "stencil_updates": int(sum(work)),
            "latency_s": {"p50": float(np.percentile(ls, 50)), "p99": float(np.percentile(ls, 99)),
                          "max": float(ls[-1])},
            "offered_gstencil_s": sum(work) / max(span, 1e-9) / 1e9,
            "delivered_gstencil_s": sum(work) / busy / 1e9,
            "arrival_span_s": span, "wall_s": busy,
            "note": "arrivals at their Poisson times, jobs uncapped; each job runs in the fastest arithmetic whose "
                    "a priori error bound meets its target (sparse TF32, FP16 hi/lo, FP32 CUDA cores); offered "
                    "above delivered means the GPU is saturated and the queue (and p99) grows with the run"}


def run_serving(a):
    import torch
    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import build as _b
    _b.build()
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    rec = serving_run(spider, a.serving_jobs or 600)
    line = {"metric": "GStencil/s", "value": rec["delivered_gstencil_s"], "unit": "GStencil/s", "n_gpus": 1,
            "steps": rec["jobs_completed"], "warmup": 0, "ms_per_step": rec["wall_s"] / rec["jobs_completed"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32+f16x2+f32",
            "data": "synthetic", "config": {"workload": rec["workload"], "hbm_budget_bytes": 120 * 10**9},
            "serving": rec}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_mma_peak(a):
    """Peak issue rates of the warp-level MMA shapes (spider_measure_mma_rate)."""
    import torch
    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import build as _b
    _b.build()
    torch.cuda.set_device(0)
    rates = {k: spider.measure_mma_rate(k) for k in spider.MMA_KINDS}
    flops = {"sp_tf32": 16 * 8 * 16 * 2, "sp_f16": 16 * 8 * 32 * 2, "sp_bf16": 16 * 8 * 32 * 2,
             "dense_tf32": 16 * 8 * 8 * 2}
    line = {"metric": "mma per second", "value": rates["sp_tf32"], "unit": "mma.sp/s", "n_gpus": 1, "steps": 5,
            "warmup": 1, "higher_is_better": True, "dtype": "tf32", "data": "synthetic",
            "config": {"workload": "mma_peak: warp-level MMAs with operands in registers, 8 chains per warp, "
                                   "16 warps per SM"},
            "rates": {k: {"mma_per_s": v, "dense_equivalent_tflops": v * flops[k] / 1e12} for k, v in rates.items()}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload in ("batched", "batched_small"):
        return run_batched(a)
    if a.workload == "serving":
        return run_serving(a)
    if a.workload == "mma_peak":
        return run_mma_peak(a)
    if a.workload == "sweep":
        return run_sweep(a)
    return run_spider(a)


if __name__ == "__main__":
    sys.exit(main())
