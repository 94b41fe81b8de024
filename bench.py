#!/usr/bin/env python
"""Throughput of the rotating shallow-water step on GB300.

A "step" is one full SSP-RK2 time step of the scheme (both stages with
their reconstruction, fluxes, sources and update, the flow relaxation of the
nested edges, and the CFL reduction that sets the next time step) over the
synthetic coastal domain: 1024 x 1024 cells at 800 m, ~30% land, wet-dry
shelves, M2 tide on three nested edges from hourly frames, 10 m/s wind,
quadratic drag, latitude 58-70 N, north angle 0-0.3 rad; FP32 arithmetic
with Kahan-compensated state update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Under torchrun each rank advances its own replica of
the domain (no data-path collective); rank 0 reports the whole-job rate
over the slowest rank's time. ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample, same metric).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s and % HBM peak (single & batched); p50/p99 forecast latency"
UNIT = "cell-updates/s"
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_stage2_coastal1024.txt")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def workload_config(nx, ny, precision):
    return {
        "workload": f"synthetic coastal {nx}x{ny} (800 m, ~30% land, wet-dry shelves, "
                    "nested M2 tide frames, 10 m/s wind, Cd 0.0025, 58-70N, theta 0-0.3 rad)",
        "nx": nx, "ny": ny, "precision": precision,
        "step": "one SSP-RK2 step incl. flow relaxation and CFL reduction",
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": "replicas (one domain per GPU)",
    }


# ---------------------------------------------------------------------------
# rank / timing helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.proc = None
        self.lines = []
        self.cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    "-i", str(gpu_index), "-lms", str(interval_ms)]

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float) -> float:
    """The maximum of x over the ranks of the default process group (x
    itself without one): the job time is that of the slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, world_size: int) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank advances its own replica of the workload)."""
    return units_per_rank * world_size / max_over_ranks(seconds)


def issue_roofline(kernel: str, avg_launch_ms: float, clocks: dict):
    """The dominant kernel against the GPU's instruction-issue rate (the
    stage kernels are bound by issue, not by HBM): warp instructions per
    launch (ncu) over the measured launch time, against SMs x schedulers x
    the median SM clock sampled during the timed region."""
    inst = committed_counter("warp_instructions", kernel)
    mhz = clocks.get("sm_mhz") if isinstance(clocks, dict) else None
    if inst is None or not mhz:
        return None
    peak = SMS * SCHEDULERS_PER_SM * mhz * 1e6
    achieved = inst / (avg_launch_ms * 1e-3)
    return {"bound": "issue", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_launch": inst,
            "peak_source": f"{SMS} SMs x {SCHEDULERS_PER_SM} schedulers x {mhz:.0f} MHz (sampled)"}


def measured_hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources that define the stage kernels (their per-cell arithmetic, their
# arguments and their launch shape); host-side files do not change them
STAGE_KERNEL_SOURCES = ("swe_device.cuh", "swe_internal.h", "swe_stage_fast.cu")


def _code_only(text):
    """C/CUDA source without comments and blank-space differences (string
    literals in these files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """Hash of the stage-kernel sources' code and of their compile flags: a
    comment edit keeps the committed counters, any code or flag change drops
    them."""
    from paper_1912_02457_gb300 import build
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1912_02457_gb300", "csrc")
    for name in STAGE_KERNEL_SOURCES:
        with open(os.path.join(csrc, name)) as fh:
            h.update(_code_only(fh.read()).encode())
    h.update(" ".join(build.NVCC_FLAGS[:2] + build.FILE_FLAGS.get("swe_stage_fast.cu", [])).encode())
    return h.hexdigest()[:16]


def committed_counter(name: str, kernel: str):
    """A per-launch counter of `kernel` (dram_bytes, warp_instructions) from
    the committed ncu summary, if it was taken on the current kernel sources;
    else None."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256_16") != kernel_source_hash():
            return None
        return float(kv[f"{name}_per_launch_{kernel}"])
    except Exception:
        return None


def committed_traffic(kernel: str):
    return committed_counter("dram_bytes", kernel)


# instruction issue of the whole GPU: 152 SMs x 4 schedulers x one warp
# instruction per cycle at the SM clock
SMS, SCHEDULERS_PER_SM = 152, 4


def algorithmic_bytes(wl, precision):
    """Algorithmic bytes each launch must move: a water cell
    reads its state, its bathymetry corner and the f plane (the FP32 stage
    kernels use the north-vector projection in its reduced form and do not
    read the angle) and writes its result; a land cell only needs its corner
    to know it is land. Halo re-reads and forcing frames are not counted."""
    n = wl.nx * wl.ny
    land = int(wl.land_cells().sum())
    wet = n - land
    statics = 4 + (4 if wl.f is not None else 0)
    s1 = 12 + statics + 12                       # Q^n, statics -> D1
    s2 = 12 + 12 + statics + 12                  # Q^n, D1, statics -> Q^{n+1}
    if precision == "f32_kahan":
        s2 += 24                                 # compensation read + write
    s0 = 12 + statics                            # the speed pass of the face-speed step reads Q^n
    return {"stage1": wet * s1 + land * 4, "stage2": wet * s2 + land * 4, "speed": wet * s0 + land * 4,
            "clock": 0, "per_cell_step_wet": s1 + s2}


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle

def oracle_rate(steps: int, warmup: int, nside: int):
    import oracle
    from paper_1912_02457_gb300 import synth
    wl = synth.coastal(nside, nside, dtype=np.float32)
    o = oracle.Oracle(wl)
    st = (wl.eta, wl.hu, wl.hv)
    e, u, v, t, dt = o.run(max(warmup, 0)) if warmup > 0 else (*st, wl.t0, 0.0)
    t0 = time.perf_counter()
    o.run(steps, state=(e, u, v), t=t, dt=dt, step0=warmup)
    el = time.perf_counter() - t0
    return nside * nside * steps / el, el, oracle.num_threads()


REFERENCE_MAX_STEPS, REFERENCE_MAX_WARMUP = 200, 3


def run_reference(args):
    """The oracle on the benchmark's own workload (the coastal 1024 x 1024
    recipe), each of the requested steps one oracle step, at most
    REFERENCE_MAX_STEPS of them timed so that the run stays within minutes."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    timed = max(1, min(args.steps, REFERENCE_MAX_STEPS))
    warm = max(0, min(args.warmup, REFERENCE_MAX_WARMUP))
    value, el, cores = oracle_rate(timed, warm, 1024)
    sample = (f"oracle (FP64 C, OpenMP) on the same coastal 1024x1024 recipe: {timed} timed steps "
              f"after {warm} warm-up steps (of the {args.steps} requested, at most "
              f"{REFERENCE_MAX_STEPS} are timed)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": timed, "warmup": warm,
        "ms_per_step": 1e3 * el / timed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(1024, 1024, args.precision),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm

def run_ours(args):
    import torch
    from paper_1912_02457_gb300 import build, swe, synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    swe.load()

    wl = synth.coastal(1024, 1024, dtype=np.float32)
    wl.params.cfl_faces = 1 if args.cfl == "faces" else 0
    cells = wl.nx * wl.ny
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dom = swe.Domain(wl, args.precision, stream=stream.cuda_stream)
    parts = dom.launch_names()

    # warm-up (untimed)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        dom.step_profiled(1)
    dom.info()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = dom.info().launches
    barrier()
    # the timed steps: one public step call each, on a flushed L2
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            dom.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier()
    info = dom.info()
    launches = info.launches - launches0
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    device_s = max_over_ranks(float(step_ms.sum()) / 1e3)
    value = whole_job_rate(cells * args.steps, device_s, ws)

    # per-kernel times for the roofline: the same flushed steps, each launch
    # bracketed by events on the domain's stream (not timed as steps: the
    # events between the launches add gaps)
    n_prof = min(args.steps, 400)
    kernel_ms = np.zeros((n_prof, len(parts)))
    for k in range(n_prof):
        with torch.cuda.stream(stream):
            flush.zero_()
        kernel_ms[k] = dom.step_profiled(1)[0]
    torch.cuda.synchronize()

    # back-to-back steps without flushing (how a forecast actually runs)
    torch.cuda.synchronize()
    b2b_n = min(args.steps, 500)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    dom.step(b2b_n)
    s1.record(stream)
    torch.cuda.synchronize()
    b2b_ms = s0.elapsed_time(s1) / b2b_n

    # end to end through the public API with pinned host buffers:
    # upload the initial state, run the steps, download the final state
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (wl.eta, wl.hu, wl.hv)]
    host_out = [torch.empty((wl.ny, wl.nx), dtype=torch.float32).pin_memory() for _ in range(3)]
    fields = (swe.ETA, swe.HU, swe.HV)
    torch.cuda.synchronize()
    e2e_t0 = time.perf_counter()
    for f, hbuf in zip(fields, host_in):
        swe._check(dom._L.swe_write_state(dom.h, f, hbuf.data_ptr(), 0), "swe_write_state")
    dom.set_clock(wl.t0, 0.0, 0)
    dom.step(args.steps)
    for f, hbuf in zip(fields, host_out):
        swe._check(dom._L.swe_read_state(dom.h, f, hbuf.data_ptr(), 0), "swe_read_state")
    e2e_s = max_over_ranks(time.perf_counter() - e2e_t0)
    e2e_info = dom.info()
    bytes_state = 3 * cells * 4

    # roofline of the dominant kernel
    kern_avg = kernel_ms.mean(axis=0)
    kern_tot = kernel_ms.sum(axis=0)
    dom_k = int(np.argmax(kern_tot))
    name = parts[dom_k]
    ab = algorithmic_bytes(wl, args.precision)
    peak, peak_src = measured_hbm_peak()
    achieved = ab.get(name, 0) / (kern_avg[dom_k] * 1e-3) / 1e9
    traffic = committed_traffic(name)

    result = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            # the oracle on a bounded sample of the same workload (~10-30 s)
            import oracle
            o = oracle.Oracle(wl)
            n_cpu = args.cpu_steps
            cores = oracle.num_threads()
            c0 = time.perf_counter()
            o.run(n_cpu)
            cel = time.perf_counter() - c0
            # and on one core, a shorter sample of the same run
            n1 = max(2, n_cpu // 8)
            oracle.set_threads(1)
            c1 = time.perf_counter()
            o.run(n1)
            cel1 = time.perf_counter() - c1
            oracle.set_threads(cores)
            cpu = {"value": cells * n_cpu / cel, "unit": UNIT, "cores": cores,
                   "kind": "oracle",
                   "sample": f"FP64 oracle, first {n_cpu} steps of the same 1024x1024 workload "
                             f"({cel:.1f} s); one core: first {n1} steps ({cel1:.1f} s)",
                   "single_core_value": cells * n1 / cel1}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * device_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(wl.nx, wl.ny, args.precision),
                           **({"cfl": "face speeds (speed pass before each step)"} if args.cfl == "faces" else {})),
            "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": ab.get(name, 0),
                         "avg_launch_ms": float(kern_avg[dom_k])},
            "kernels": {p: {"avg_ms": float(kern_avg[i]), "share": float(kern_tot[i] / kern_tot.sum())}
                        for i, p in enumerate(parts)},
            "issue_roofline": issue_roofline(name, float(kern_avg[dom_k]), clocks.summary()),
            "back_to_back_ms_per_step": b2b_ms,
            "back_to_back_value": cells / (b2b_ms * 1e-3),
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_rate(cells * args.steps, e2e_s, ws), "unit": UNIT,
                    "h2d_bytes_per_step": bytes_state / args.steps,
                    "d2h_bytes_per_step": bytes_state / args.steps,
                    "job": f"upload state from pinned host, {args.steps} steps, download state"},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "wall_s_timed_region": wall,
            "sim_time_s": info.t, "dt_s": info.dt,
        }
        if e2e_info.step != args.steps:
            result["e2e"]["warning"] = "step count mismatch"
        print(json.dumps(result), flush=True)
    dom.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# secondary workloads (one JSON line each; the default line is the step above)

def _timed_steps(torch, dom_or_batch, n, stream, method="step"):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    getattr(dom_or_batch, method)(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_sweep(args):
    """Single domains of the coastal recipe at growing sizes (inputs larger
    than L2 from 2048^2 on): cell-updates/s of back-to-back graph steps."""
    import torch
    from paper_1912_02457_gb300 import build, swe, synth
    build.build()
    swe.load()
    stream = torch.cuda.Stream()
    out = []
    for nx, ny in synth.SWEEP_SIZES:
        wl = synth.coastal(nx, ny, dtype=np.float32)
        with swe.Domain(wl, args.precision, stream=stream.cuda_stream) as d:
            d.step(args.warmup)
            n = max(32, min(args.steps, int(4e10 // (nx * ny))))
            el = _timed_steps(torch, d, n, stream)
            ms = d.step_profiled(8).mean(axis=0)
            ab = algorithmic_bytes(wl, args.precision)
            out.append({"nx": nx, "ny": ny, "steps": n, "cell_updates_per_s": float(nx * ny * n / el),
                        "stage_ms": {"stage1": float(ms[0]), "stage2": float(ms[1])},
                        "stage2_hbm_frac": float(ab["stage2"] / (float(ms[1]) * 1e-3) / 1e9
                                                 / measured_hbm_peak()[0])})
        del wl
    print(json.dumps({"metric": METRIC, "workload": "size sweep (coastal recipe)",
                      "unit": UNIT, "precision": args.precision, "results": out}), flush=True)


def run_rossby(args):
    """The beta-plane Rossby workload (350^2 cells of 20 km, periodic on every
    edge, FP32 + Kahan) for two orientations of north: cell-updates/s of
    back-to-back graph steps, stage times, and the simulated days per second."""
    import torch
    from paper_1912_02457_gb300 import build, swe, synth
    build.build()
    swe.load()
    stream = torch.cuda.Stream()
    out = []
    for theta in (0.0, np.pi / 4):
        wl = synth.rossby(n=350, theta=theta, dtype=np.float32)
        with swe.Domain(wl, args.precision, stream=stream.cuda_stream) as d:
            d.step(args.warmup)
            el = _timed_steps(torch, d, args.steps, stream)
            info = d.info()
            ms = d.step_profiled(8).mean(axis=0)
            out.append({"theta": theta, "steps": args.steps,
                        "cell_updates_per_s": float(wl.nx * wl.ny * args.steps / el),
                        "ms_per_step": el * 1e3 / args.steps, "dt_s": info.dt,
                        "simulated_days_per_s": info.dt * args.steps / el / 86400.0,
                        "stage_ms": {"stage1": float(ms[0]), "stage2": float(ms[1])}})
    print(json.dumps({"metric": METRIC, "workload": "beta-plane Rossby waves, 350x350 periodic",
                      "unit": UNIT, "precision": args.precision, "results": out}), flush=True)


def run_split(args):
    """The coastal 4096^2 domain stepped whole and as 2x2 and 4x4 windows
    exchanging halos on this one GPU (swe_split_step): cell-updates/s of
    the whole domain either way, i.e. the cost of the decomposition's extra
    launches, halo cells and copies on one device (not a scaling figure)."""
    import torch
    from paper_1912_02457_gb300 import build, swe, synth
    from paper_1912_02457_gb300.split import SplitDomain
    build.build()
    swe.load()
    stream = torch.cuda.Stream()
    wl = synth.coastal(4096, 4096, dtype=np.float32)
    out = []
    with swe.Domain(wl, args.precision, stream=stream.cuda_stream) as d:
        d.step(args.warmup)
        el = _timed_steps(torch, d, args.steps, stream)
        out.append({"split": "whole", "steps": args.steps,
                    "cell_updates_per_s": float(wl.nx * wl.ny * args.steps / el)})
    for px, py in ((2, 2), (4, 4)):
        with SplitDomain(wl, px, py, args.precision, stream=stream.cuda_stream) as s:
            s.step(args.warmup)
            el = _timed_steps(torch, s, args.steps, stream)
            out.append({"split": f"{px}x{py}", "steps": args.steps,
                        "cell_updates_per_s": float(wl.nx * wl.ny * args.steps / el)})
    print(json.dumps({"metric": METRIC, "workload": "coastal 4096x4096, whole and split into windows on one GPU",
                      "unit": UNIT, "precision": args.precision, "results": out}), flush=True)


def run_ensemble(args):
    """64 domains of uneven sizes in one batch: one launch per
    stage (graph-captured, autotuned tiles) against launching the same
    kernels domain after domain."""
    import torch
    from paper_1912_02457_gb300 import build, swe, synth
    build.build()
    swe.load()
    stream = torch.cuda.Stream()
    wls = synth.ensemble(args.domains)
    cells = sum(w.nx * w.ny for w in wls)
    doms = [swe.Domain(w, "f32_kahan", stream=stream.cuda_stream) for w in wls]
    b = swe.Batch(stream=stream.cuda_stream)
    for d in doms:
        b.add(d)
    b.step(32)                                   # autotune + warm-up
    b.step_serial(4)
    n = args.steps
    t_batched = _timed_steps(torch, b, n, stream, "step")
    t_serial = _timed_steps(torch, b, n, stream, "step_serial")
    res = {"metric": METRIC, "workload": f"ensemble of {len(wls)} coastal domains "
           "(256^2, 512x384, 1024^2, 2048x1024), FP32 + Kahan",
           "unit": UNIT, "domains": len(wls), "cells": cells, "steps": n,
           "batched_value": cells * n / t_batched, "serial_value": cells * n / t_serial,
           "speedup_vs_one_by_one": t_serial / t_batched, "tile_rows": b.rows(),
           "batched_ms_per_step": 1e3 * t_batched / n, "serial_ms_per_step": 1e3 * t_serial / n}
    # the batched step against the HBM roofline: the algorithmic bytes of
    # both stages of every domain over the time of one batched step
    ab = sum(algorithmic_bytes(w, "f32_kahan")["stage1"] + algorithmic_bytes(w, "f32_kahan")["stage2"]
             for w in wls)
    peak, peak_src = measured_hbm_peak()
    res["batched_hbm"] = {"algorithmic_bytes_per_step": ab,
                          "achieved_gbs": ab / (t_batched / n) / 1e9,
                          "frac": ab / (t_batched / n) / 1e9 / peak, "peak": peak, "peak_source": peak_src}
    b.close()
    for d in doms:
        d.close()
    print(json.dumps(res), flush=True)


def run_serve(args):
    """Poisson forecast requests (20/s, sides log-uniform 128-2048, horizons
    U(1, 24) h) served by continuous batching under a 150 GB budget: the
    first --requests arrivals of the seeded 256-arrival trace, horizons
    scaled by --horizon-scale (1: as drawn). Inputs are generated before the
    clock starts."""
    import torch
    from paper_1912_02457_gb300 import build, serve, swe, synth
    build.build()
    swe.load()
    stream = torch.cuda.Stream()
    trace = synth.serving_trace(256)[:args.requests]
    reqs = []
    for r in trace:
        wl = synth.coastal(r["side"], r["side"], seed_config=5, member=r["member"] + 1,
                           dtype=np.float32, hours=int(np.ceil(r["horizon"] * args.horizon_scale / 3600)) + 1)
        reqs.append(serve.Request(rid=r["member"], arrival=r["arrival"],
                                  make_workload=(lambda w=wl: w),
                                  horizon=r["horizon"] * args.horizon_scale,
                                  nx=r["side"], ny=r["side"]))
    backend = serve.GpuBackend(stream=stream.cuda_stream)
    srv = serve.ForecastServer(backend, budget_bytes=150e9, round_steps=args.round_steps)
    t0 = time.perf_counter()
    srv.run(reqs, time_limit=args.serve_time_limit)
    wall = time.perf_counter() - t0
    backend.shutdown()
    st = serve.ForecastServer.stats(reqs, wall)
    offered = sum(r.nx * r.ny * (r.horizon / 0.93) for r in reqs) / max(trace[-1]["arrival"], 1e-9)
    st.update({"metric": METRIC,
               "workload": (f"serving: the first {len(reqs)} arrivals of the seeded 256-request Poisson "
                            f"trace (20/s, sides 128-2048, horizons 1-24 h"
                            + (")" if args.horizon_scale == 1.0 else f" x{args.horizon_scale})")
                            + f", served under a {args.serve_time_limit:.0f} s limit"),
               "unit": "s (latency), cell-updates/s",
               "offered_cell_updates_per_s_est": offered, "peak_device_bytes": srv.peak_used,
               "rounds": srv.rounds, "round_steps": args.round_steps,
               "admitted_while_running": srv.overlapped,
               "unfinished": sum(1 for r in reqs if r.finished is None)})
    print(json.dumps(st), flush=True)


def run_prep(args):
    """Grid pre-processing kernels (Sections 3.8, 3.9), FP32, on inputs larger
    than L2: corner bathymetry (4096^2 and 8192^2, 10 iterations), land
    erosion (8192^2), refinement 8192^2 -> 16384^2 and coarsening back."""
    import torch
    from paper_1912_02457_gb300 import build, swe, synth
    build.build()
    swe.load()
    st = torch.cuda.current_stream()
    peak, peak_src = measured_hbm_peak()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    res = {}
    rng = np.random.default_rng(1912_02457 + 8000)
    # corner bathymetry: one fused kernel per iteration reads the cell
    # averages and the corners and writes the new corners: 12 B per cell
    it = 10
    for n in ((args.prep_size,) if args.prep_size else (4096, 8192)):
        z = synth.spectral_field(rng, n, n, max_fft=n + 1)
        Hm = torch.from_numpy((5.0 + 2995.0 * ((z - z.min()) / (z.max() - z.min())) ** 2)
                              .astype(np.float32)).cuda()
        Hc = torch.empty((n + 1, n + 1), dtype=torch.float32, device="cuda")
        work = torch.empty(swe.bathymetry_work_bytes(n, n), dtype=torch.uint8, device="cuda")
        t0 = timed(lambda: swe.bathymetry_reconstruct(Hm.data_ptr(), n, n, n, Hc.data_ptr(), n + 1,
                                                      work.data_ptr(), n_iter=0, stats=False,
                                                      stream=st.cuda_stream), 5)
        t10 = timed(lambda: swe.bathymetry_reconstruct(Hm.data_ptr(), n, n, n, Hc.data_ptr(), n + 1,
                                                       work.data_ptr(), n_iter=it, stats=False,
                                                       stream=st.cuda_stream), 5)
        per_it = (t10 - t0) / it
        gbs = 12.0 * n * n / per_it / 1e9
        res[f"bathymetry_{n}"] = {"grid": f"{n}x{n}", "dtype": "f32", "iterations": it,
                                  "ms_total": t10 * 1e3, "ms_per_iteration": per_it * 1e3,
                                  "cell_iterations_per_s": n * n / per_it,
                                  "achieved_gbs": gbs, "frac": gbs / peak, "bytes_per_cell_iteration": 12}
        del Hm, Hc, work
    # land erosion: 1 + 4 + 4 B in, 1 + 4 + 4 B out per cell
    n = args.prep_size or 8192
    land = torch.from_numpy((rng.random((n, n)) < 0.3).astype(np.uint8)).cuda()
    eta = torch.randn((n, n), dtype=torch.float32, device="cuda")
    Hm = torch.rand((n, n), dtype=torch.float32, device="cuda")
    lo, eo, ho = torch.empty_like(land), torch.empty_like(eta), torch.empty_like(Hm)
    t = timed(lambda: swe.land_erode(land.data_ptr(), eta.data_ptr(), Hm.data_ptr(), n, n, n,
                                     lo.data_ptr(), eo.data_ptr(), ho.data_ptr(), stream=st.cuda_stream), 10)
    gbs = 18.0 * n * n / t / 1e9
    res["land_erode"] = {"grid": f"{n}x{n}", "dtype": "f32", "ms": t * 1e3, "achieved_gbs": gbs,
                         "frac": gbs / peak, "bytes_per_cell": 18}
    del land, eta, Hm, lo, eo, ho
    # refinement / coarsening: per coarse cell 3 x 4 B + a corner in, 3 x 16 B + 4 corners out
    wl = synth.coastal(n, n, dtype=np.float32)
    q = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (wl.eta, wl.hu, wl.hv)]
    H = torch.from_numpy(np.ascontiguousarray(wl.H)).cuda()
    qf = [torch.empty((2 * n, 2 * n), dtype=torch.float32, device="cuda") for _ in range(3)]
    Hf = torch.empty((2 * n + 1, 2 * n + 1), dtype=torch.float32, device="cuda")
    qp, qfp = [a.data_ptr() for a in q], [a.data_ptr() for a in qf]
    t = timed(lambda: swe.refine2(qp, n, H.data_ptr(), n + 1, n, n, qfp, 2 * n, Hf.data_ptr(), 2 * n + 1,
                                  stream=st.cuda_stream), 10)
    gbs = 80.0 * n * n / t / 1e9
    res["refine2"] = {"grid": f"{n}x{n} -> {2 * n}x{2 * n}", "dtype": "f32", "ms": t * 1e3,
                      "achieved_gbs": gbs, "frac": gbs / peak, "bytes_per_coarse_cell": 80}
    t = timed(lambda: swe.coarsen2(qfp, 2 * n, Hf.data_ptr(), 2 * n + 1, n, n, qp, n, H.data_ptr(), n + 1,
                                   stream=st.cuda_stream), 10)
    gbs = 80.0 * n * n / t / 1e9
    res["coarsen2"] = {"grid": f"{2 * n}x{2 * n} -> {n}x{n}", "dtype": "f32", "ms": t * 1e3,
                       "achieved_gbs": gbs, "frac": gbs / peak, "bytes_per_coarse_cell": 80}
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import prep
        m = 1024
        zs = synth.spectral_field(np.random.default_rng(1912_02457 + 8001), m, m).astype(np.float64)
        c0 = time.perf_counter()
        prep.reconstruct_bathymetry(zs, n_iter=10)
        cel = time.perf_counter() - c0
        cpu = {"value": m * m * 10 / cel, "unit": "cell-iterations/s", "cores": 1, "kind": "oracle",
               "sample": f"numpy oracle, corner bathymetry {m}x{m}, 10 iterations ({cel:.1f} s)"}
    line = {"metric": METRIC, "workload": "grid pre-processing (Sections 3.8, 3.9)", "unit": "GB/s",
            "peak_gbs": peak, "peak_source": peak_src, "results": res,
            "cpu_baseline": cpu, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("f32", "f32_kahan"), default="f32_kahan")
    ap.add_argument("--cfl", choices=("cells", "faces"), default="cells",
                    help="time step from the cell averages (the scheme's reading) or the faces' speeds")
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("coastal1024", "sweep", "ensemble", "serve", "prep", "rossby",
                                           "split"),
                    default="coastal1024")
    ap.add_argument("--domains", type=int, default=64)
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--horizon-scale", type=float, default=1.0)
    ap.add_argument("--serve-time-limit", type=float, default=900.0)
    ap.add_argument("--round-steps", type=int, default=64)
    ap.add_argument("--prep-size", type=int, default=0,
                    help="prep workload: one grid side for every kernel (default 4096/8192)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "prep":
        return run_prep(args)
    if args.workload == "split":
        return run_split(args)
    if args.workload == "rossby":
        return run_rossby(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
