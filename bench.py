#!/usr/bin/env python
"""Ray-volume steps per second of the MS-GWaM-3D hot path on GB300.

Workload (one "step" = one full gwam_step: RK3 advance of every ray volume, exits, splitting,
re-binning, cap, saturation, flux projection, smoothing, divergence, budget): the global
lat-lon sphere 256 x 128 columns x 90 levels (1 km), two 60 m/s jets, isothermal 240 K
atmosphere, the latitude-dependent background source at 5 km launching 8 azimuths x 4 phase
speeds per column (983 040 ray volumes), dt = 180 s, FP64.  Synthetic inputs, seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The workload runs 200 steps; after the launch, 100 untimed lead-in steps (--lead-in) put the W
warm-up and K timed steps into the run's steady part (waves aloft, saturation, exits through the
top); the line also reports the whole 200-step run's rate (config.run) and the live ray counts.

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own replica of the
workload on its own GPU (the replicas exchange nothing); value = all ranks' ray-volume steps
divided by the slowest rank's time.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-volume steps/s"
UNIT = "ray-volume steps/s"
WORKLOAD = "sphere 256x128x90, background source 983040 ray volumes, dt 180 s, FP64"
# Algorithmic FP64 operations per ray-volume step of the advance kernel (RK3: 3 evaluations of
# the ray equations at the centre and 6 faces, incl. the trilinear gather of 4 fields with
# gradients, plus exits and split decisions), counted from the formulas with every add, multiply,
# divide, square root and trigonometric call as one operation.
FLOPS_PER_RAY_STEP = 1460.0
# Peak rate of FP64-precision operations on GB300 (one operation per add or multiply): the kernel
# runs them as double-float pairs on the FP32 pipes (152 SMs x 128 lanes x 2.07 GHz = 40.3 T FP32
# instructions/s; a double-float add takes 11 FP32 instructions, a multiply 4 (its pair is passed on
# unrenormalised), 7.5 on average -> 5.37 T/s) besides the FP64 pipe (2 per clock per SM ->
# 0.63 T/s); together 6.0 T/s.
FP64_EQ_PEAK_TOPS = 152 * 128 * 2.07e9 / 7.5 / 1e12 + 152 * 2 * 2.07e9 / 1e12
# Precision form: algorithmic bytes of the ray step = the 64-byte ray record read and written once.
BYTES_PER_RAY_STEP_FP32 = 128.0
# FP64 form, HBM view of the ray step: the 112-byte ray state read and written once (224 B) plus the
# background it gathers, <= 4 fields x 8 B per touched cell (about 96 B per ray volume at ~1 M rays).
BYTES_PER_RAY_STEP_FP64 = 224.0 + 96.0
# Whole step, algorithmic bytes: the ray state (224 B per ray volume, 128 B in the precision form) and,
# per grid cell, the background read (4 x 8 B), the two saturation sums written and read (32 B), the
# 8 flux fields and the wave-action diagnostic written once and read once by the stencils (144 B) and
# the two tendencies written (16 B): 224 B per cell.
BYTES_PER_CELL_STEP = 224.0
# Representative window: the workloads run 200 steps; the timed steps follow an untimed lead-in.
RUN_STEPS = 200
HBM_PEAK = None
# The ray-step kernels also clear the nine projected FP64 fields the step's projection accumulates
# into (two interface fields of nz + 1 levels, seven centre fields of nz levels): algorithmic bytes
# of that clearing, per launch.
def clear_bytes(nx, ny, nz, theta=False):
    # (with the potential-temperature flux projected, two more centre fields)
    return 8.0 * nx * ny * (2 * (nz + 1) + (9 if theta else 7) * nz)


# DRAM bytes (read + write) of one launch in the ncu captures in profiles/, as a fraction of that
# launch's algorithmic bytes (ray bytes x 253 952 rays + the clearing of the 128 x 64 x 90 fields):
# k_advance 67.75 MB of 134.48 MB, k_advance32 40.77 MB of 85.72 MB (written field lines still in L2
# when the kernel ends are not counted).  The bench's traffic is that fraction of its own launch's
# algorithmic bytes; None while the kernel has changed since its counters were taken: k_advance has
# (narrow, which its double-float splits call on their out-of-range path, changed after the capture;
# its loads and stores did not), so its traffic is null until the next capture.
ADV_TRAFFIC_FRACTION = None     # was 67.75 / 134.48
ADV32_TRAFFIC_FRACTION = 40.77 / 85.72


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# ------------------------------------------------------------------------------------- clocks

class _Nvml:
    """The driver's NVML library through ctypes (read-only queries): SM clock, its maximum, and the
    active clock-event reasons of one GPU; None where the library is missing."""

    SM = 1   # NVML_CLOCK_SM
    REASONS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
               ("hw_thermal_slowdown", 0x40))

    @classmethod
    def open(cls, index: int):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            dev = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(dev)) != 0:
                return None
            self = cls()
            self.ct, self.lib, self.dev = ctypes, lib, dev
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(dev, cls.SM, ctypes.byref(mx)) == 0 else None
            return self
        except Exception:
            return None

    def sample(self):
        ct = self.ct
        clk = ct.c_uint()
        if self.lib.nvmlDeviceGetClockInfo(self.dev, self.SM, ct.byref(clk)) != 0:
            return None
        mask = ct.c_ulonglong(0)
        if self.reasons_fn is not None:
            self.reasons_fn(self.dev, ct.byref(mask))
        return float(clk.value), int(mask.value)

    def close(self):
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """SM clock and clock-event reasons sampled while the timed region runs: from NVML every
    millisecond (the samples of the region itself: settle() drops those taken before it), else
    from nvidia-smi every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.nvml = None
        self.samples = []
        self.running = False

    def start(self):
        self.nvml = _Nvml.open(self.index)
        if self.nvml is not None:
            self.running = True
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def settle(self):
        """Call right before the timed region."""
        if self.nvml is not None:
            time.sleep(0.05)
            self.samples.clear()
        else:
            time.sleep(0.3)

    def _poll(self):
        while self.running:
            v = self.nvml.sample()
            if v is not None:
                self.samples.append(v)
            time.sleep(0.001)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.running = False
            self.t.join(timeout=2)
            self.nvml.close()
            sm = [c for c, _ in self.samples]
            reasons = sorted({nm for _, m in self.samples for nm, bit in _Nvml.REASONS if m & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.nvml.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "NVML every 1 ms during the timed region"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi every 200 ms"}


# ------------------------------------------------------------------------------------- oracle arm

def host_cpu():
    """Host core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_throughput(steps: int, warmup: int, workload: str = "sphere", threads: int = 0):
    """FP64 CPU oracle on the same workload: launch (untimed), `warmup` untimed steps, then
    `steps` timed steps, its per-ray loops on `threads` host threads (0: all cores); returns
    ray-volume steps/s, the timed sample and the threads used."""
    import oracle
    from paper_2309_11257_gb300 import synth
    w = synth.workload(workload)
    M = oracle.Model(w["grid"], w["params"])
    used = M.set_threads(threads or (os.cpu_count() or 1))
    M.set_background(*w["background"])
    M.launch_background(w["source"])
    for _ in range(warmup):
        M.step(w["dt"])
    ray_steps = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        ray_steps += M.n_rays
        M.step(w["dt"])
    dt = time.perf_counter() - t0
    return ray_steps / dt, dict(steps=steps, warmup=warmup, ray_steps=ray_steps, seconds=dt, threads=used)


def reference_arm(args, rank, world):
    """The FP64 CPU oracle on the GPU arm's workload: the launch, W untimed steps, then exactly K
    timed steps of the whole workload, the oracle's per-ray loops on all host cores."""
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    value, sample = oracle_throughput(steps, warm)
    ncpu, cpu_model = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * sample["seconds"] / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sample["threads"], "kind": "oracle",
                         "cpu_model": cpu_model, "host_cores": ncpu,
                         "sample": "%d timed oracle steps (after the launch and %d untimed) of the full workload, "
                                   "%d threads" % (steps, warm, sample["threads"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------- GPU arm

def whole_job(ms, units, extra_sum, dev, world):
    """Whole-job figures of N replicas (one per rank, exchanging nothing else): the slowest rank's
    time, and the units and `extra_sum` (e.g. an end-to-end rate) summed over the ranks."""
    if world <= 1:
        return ms, units, extra_sum
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units), float(extra_sum)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u[0].item()), float(u[1].item())


def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2309_11257_gb300 import gwam, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.workload(args.workload)
    grid, params = w["grid"], dict(w["params"])
    fp32 = args.workload in ("sphere_fp32", "sphere_half_fp32")
    if fp32:
        params["precision"] = 1
    nz, ny, nx = grid["nz"], grid["ny"], grid["nx"]
    ghost = w.get("ghost", False)
    e2e_steps = 0 if args.no_e2e else max(10, args.e2e_steps)
    # untimed lead-in so that the timed window lies in the steady part of the 200-step run (the ghost
    # workload starts from no rays and grows every step: no lead-in)
    lead_in = 0 if ghost else (RUN_STEPS // 2 if args.lead_in < 0 else args.lead_in)
    # ghost-layer emission adds up to one ray volume per bin and step
    cap_rays = 32 * nx * ny * (args.warmup + args.steps + e2e_steps + 5) if ghost else 2.5 * 32 * nx * ny
    T = gwam.Tracer(grid, params, max_rays=int(cap_rays))
    bg_dev = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in w["background"]]
    T.set_background(*bg_dev)
    if not ghost:
        T.launch_sources(w["source"])
    if params.get("theta_flux"):
        T.set_theta(torch.from_numpy(synth.isothermal_theta(grid)).to(dev))
    du = torch.zeros((nz, ny, nx), dtype=torch.float64, device=dev)
    dv = torch.zeros_like(du)
    coupled = w.get("coupled", False)

    # timed steps replay the step's CUDA graph (gwam_step_graph; --eager: gwam_step); the per-phase
    # times of the roofline are the CUDA events the graphs carry at the phase boundaries (those of
    # the last replays inside the timed region), or, eager, the profiled steps of the timed region
    use_graph = not args.eager

    def one_step(graph=use_graph):
        if ghost:
            T.launch_ghost(w["source"], w["dt"])
        if graph:
            T.step_graph(w["dt"], du, dv)
        else:
            T.step(w["dt"], du, dv)
        if coupled:
            # online coupling: the host model advances u, v by the drag and hands the background back
            bg_dev[0].add_(du, alpha=w["dt"])
            bg_dev[1].add_(dv, alpha=w["dt"])
            T.set_background(*bg_dev)

    # lead-in and warm-up, timed separately for the whole-run figure (not the reported value)
    run_ms = 0.0
    run_rs0 = T.stats()["ray_steps"]
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(torch.cuda.current_stream())
    for _ in range(lead_in + args.warmup):
        one_step()
    eb.record(torch.cuda.current_stream())
    eb.synchronize()
    run_ms += ea.elapsed_time(eb)
    if not use_graph:
        T.profile(True)
    s0 = T.stats()
    sampler = ClockSampler(local_rank)
    sampler.start()
    sampler.settle()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    s1 = T.stats()
    run_ms += ms
    if use_graph:
        phases, ngraphs = T.graph_profile_read()   # already averaged over the graphs' last replays
        assert ngraphs > 0
        nprof = 1
    else:
        phases, nprof = T.profile_read()
        T.profile(False)
    ray_steps = s1["ray_steps"] - s0["ray_steps"]
    rays_per_launch = ray_steps / args.steps
    if use_graph and ghost:
        # the graphs' phase times are those of the last steps; the population grows every step
        rays_per_launch = s1["n_live"]
    ms_max, tot_rs, _ = whole_job(ms, ray_steps, 0.0, dev, world)
    value = tot_rs / (ms_max / 1000.0)
    step_window = [lead_in + args.warmup + 1, lead_in + args.warmup + args.steps]

    # the rest of the 200-step run (not part of the value): whole-run ray-volume steps/s
    rest = RUN_STEPS - (lead_in + args.warmup + args.steps) if not ghost else 0
    if rest > 0:
        ea.record(torch.cuda.current_stream())
        for _ in range(rest):
            one_step()
        eb.record(torch.cuda.current_stream())
        eb.synchronize()
        run_ms += ea.elapsed_time(eb)
    s_run = T.stats()
    whole_run = None
    if not ghost:
        whole_run = {"steps": s_run["n_steps"], "value": (s_run["ray_steps"] - run_rs0) / (run_ms / 1000.0),
                     "unit": UNIT, "rays_live_end": s_run["n_live"],
                     "note": "every step of the run after the launch (first graph captures included), "
                             "CUDA events; not the reported value"}

    # roofline of the dominant kernel (its launches in the profiled eager steps)
    adv_ms = phases["advance"] / max(nprof, 1)
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    ncell = nx * ny * nz
    ray_bytes = BYTES_PER_RAY_STEP_FP32 if fp32 else BYTES_PER_RAY_STEP_FP64
    zero_bytes = clear_bytes(nx, ny, nz, theta=bool(params.get("theta_flux")))
    kernel_bytes = ray_bytes * rays_per_launch + zero_bytes
    step_bytes = (BYTES_PER_RAY_STEP_FP32 if fp32 else 224.0) * rays_per_launch + BYTES_PER_CELL_STEP * ncell
    step_ms = ms_max / args.steps
    hbm_view = {"peak_gbs": hbm_peak, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "kernel_bytes_per_ray_step": ray_bytes, "kernel_clearing_bytes": zero_bytes,
                "kernel_gbs": kernel_bytes / (adv_ms / 1000.0) / 1e9,
                "kernel_frac": kernel_bytes / (adv_ms / 1000.0) / 1e9 / hbm_peak,
                "kernel_frac_rays_only": ray_bytes * rays_per_launch / (adv_ms / 1000.0) / 1e9 / hbm_peak,
                "step_bytes": step_bytes, "step_gbs": step_bytes / (step_ms / 1000.0) / 1e9,
                "step_frac": step_bytes / (step_ms / 1000.0) / 1e9 / hbm_peak}
    if fp32:
        # precision form: the ray step reads and writes the 64-byte record and clears the projected fields
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        achieved = kernel_bytes / (adv_ms / 1000.0) / 1e9
        traffic = ADV32_TRAFFIC_FRACTION * kernel_bytes if ADV32_TRAFFIC_FRACTION is not None else None
        roofline = {"bound": "hbm", "kernel": "k_advance32 (FP32 RK3 ray step + clearing of the projected fields)",
                    "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "bytes_per_launch": {"ray_records": BYTES_PER_RAY_STEP_FP32 * rays_per_launch,
                                         "field_clearing": zero_bytes},
                    "traffic": traffic,
                    "traffic_source": "ncu dram bytes of k_advance32 on the 128x64 sphere (profiles/"
                                      "k_advance32_sphere_half_fp32.md) as a fraction of that launch's algorithmic "
                                      "bytes, times this launch's",
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                    "hbm": hbm_view,
                    "phase_ms_per_step": {k: v / max(nprof, 1) for k, v in phases.items()}}
    else:
        achieved = FLOPS_PER_RAY_STEP * rays_per_launch / (adv_ms / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": "k_advance (FP64 RK3 ray step)", "achieved": achieved,
                    "peak": FP64_EQ_PEAK_TOPS, "unit": "TFLOP/s", "frac": achieved / FP64_EQ_PEAK_TOPS,
                    "traffic": ADV_TRAFFIC_FRACTION * kernel_bytes if ADV_TRAFFIC_FRACTION is not None else None,
                    "traffic_source": ("ncu dram bytes of k_advance on the 128x64 sphere (profiles/"
                                       "k_advance_sphere_half_fp64.md) as a fraction of that launch's algorithmic "
                                       "bytes (ray state, gathers, field clearing), times this launch's")
                    if ADV_TRAFFIC_FRACTION is not None else
                    "null: k_advance changed after its ncu capture (profiles/k_advance_sphere_half_fp64.md: "
                    "DRAM 50 % of the algorithmic bytes then)",
                    "peak_source": "modelled (not measured) from unit counts and the 2.07 GHz clock: "
                                   "FP64-precision operations as double-float on the FP32 pipes (5.37 T/s at 7.5 "
                                   "instructions each) plus the FP64 pipe (0.63 T/s)",
                    "flops_per_ray_step": FLOPS_PER_RAY_STEP,
                    "hbm": hbm_view,
                    "phase_ms_per_step": {k: v / max(nprof, 1) for k, v in phases.items()}}

    # end to end through the public API with host buffers: each step uploads that step's
    # background from pinned host memory and reads du/dt, dv/dt back into pinned host memory, with
    # the asynchronous entry points (host-link copies on the context's copy streams, overlapping the
    # neighbouring steps) and one synchronising call at the end
    e2e = None
    if not args.no_e2e:
        bg_host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in w["background"]]
        du_h = torch.zeros((nz, ny, nx), dtype=torch.float64).pin_memory().numpy()
        dv_h = torch.zeros((nz, ny, nx), dtype=torch.float64).pin_memory().numpy()
        ke = e2e_steps
        # warm-up of the asynchronous path (its staging slots, second background set and the step
        # graphs of its output slots are allocated and captured on first use)
        for _ in range(3):
            T.set_background_async(*bg_host)
            if ghost:
                T.launch_ghost(w["source"], w["dt"])
            T.step_host_async(w["dt"], du_h, dv_h)
        T.synchronize()
        a0 = T.stats()["ray_steps"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            T.set_background_async(*bg_host)
            if ghost:
                T.launch_ghost(w["source"], w["dt"])
            T.step_host_async(w["dt"], du_h, dv_h)
        T.synchronize()
        t1 = time.perf_counter()
        rs = T.stats()["ray_steps"] - a0
        e2e_val = rs / (t1 - t0)
        _, _, e2e_val = whole_job(0.0, 0, e2e_val, dev, world)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * nz * ny * nx,
               "d2h_bytes_per_step": 2 * 8 * nz * ny * nx, "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ncpu, cpu_model = host_cpu()
        cval, sample = oracle_throughput(args.cpu_steps, 0,
                                         "sphere_columnar" if args.workload == "sphere_columnar" else "sphere")
        cpu = {"value": cval, "unit": UNIT, "cores": sample["threads"], "kind": "oracle", "cpu_model": cpu_model,
               "host_cores": ncpu,
               "sample": "%d oracle steps right after the launch of the full sphere workload (%d ray-volume steps, "
                         "%.1f s), per-ray loops on %d threads" % (sample["steps"], sample["ray_steps"],
                                                                   sample["seconds"], sample["threads"])}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 kinematics, f64 accumulation" if fp32
                      else "f64 state, sums and outputs; double-float (~48-bit) arithmetic on the FP32 pipes"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "sphere" else args.workload, "rays_live_start": s0["n_live"], "rays_live_end": s1["n_live"],
                       "ray_steps_timed": ray_steps, "timed_steps_of_run": step_window, "lead_in_steps": lead_in,
                       "run": whole_run,
                       "step_call": "gwam_step_graph (one CUDA graph launch per step)" if use_graph else "gwam_step",
                       "l2": "working set > L2 (ray state ~0.12-0.24 GB + "
                       "grid fields ~0.4 GB per step), no flush", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "gpu_launches": None,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
        }
        # per step: the kernel nodes of the step graph (counted by the library from the captured graph),
        # or the eager step's kernels; coupling adds the background set-up (2 kernels), a ghost-layer
        # launch its 2 launch passes, the 2 kernels of its slot scan, the tally fold and the close
        per_step = T.graph_kernel_count() if use_graph else launches_per_step(params, fp32)
        line["gpu_launches"] = args.steps * (per_step + (2 if coupled else 0) + (6 if ghost else 0))
        line["config"]["kernels_per_step"] = per_step
        print(json.dumps(line), flush=True)
    return 0


def ensemble_arm(args):
    """Batched ensemble: 16 independent spheres in one context; autotuned launch shapes; every
    timed step is one CUDA-graph launch."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2309_11257_gb300 import gwam, synth

    w = synth.ensemble_workload()
    grid, M = w["grid"], w["members"]
    nz, ny, nx = grid["nz"], grid["ny"], grid["nx"]
    nspec = sum(len(s) for s in w["specs"])
    n0 = M * 120 * nx * 32 + nspec
    T = gwam.Tracer(grid, w["params"], max_rays=int(2.2 * n0), members=M)
    for m in range(M):
        T.set_member_background(m, *[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in w["backgrounds"][m]])
    T.launch_sources(w["source"])
    T.launch_spectral(np.concatenate(w["specs"]))
    du = torch.zeros((M, nz, ny, nx), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    tuned = T.autotune(w["dt"], steps_per_candidate=1, dudt=du, dvdt=dv)
    for _ in range(args.warmup):
        T.step_graph(w["dt"], du, dv)
    s0 = T.stats()
    sampler = ClockSampler(0)
    sampler.start()
    sampler.settle()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        T.step_graph(w["dt"], du, dv)
    e1.record()
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    s1 = T.stats()
    rs = s1["ray_steps"] - s0["ray_steps"]
    line = {"metric": METRIC, "value": rs / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64 state, sums and outputs; double-float (~48-bit) arithmetic on the FP32 pipes",
            "data": "synthetic",
            "config": {"workload": "ensemble: %d spheres 256x128x90, background + convective sources" % M,
                       "rays_launched": s0["n_launched"], "rays_live_start": s0["n_live"],
                       "rays_live_end": s1["n_live"], "convective_specs": nspec, "launch_shapes": tuned,
                       "graph": "one CUDA graph launch per step"},
            "gpu_launches": args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


# Surrogate: algorithmic FLOPs of one column through the MLP 368 -> 4 x 512 (GELU) -> 180
SUR_DIMS = (368, 512, 512, 512, 512, 180)
SUR_FLOPS_PER_COLUMN = 2.0 * sum(a * b for a, b in zip(SUR_DIMS[:-1], SUR_DIMS[1:]))
SUR_BATCH = 32768


def surrogate_arm(args):
    """Surrogate inference: one step = one pass over a batch of 32 768 columns (normalisation and
    envelope test, 5 tensor-core GEMMs with fused bias/GELU, de-normalised drag scattered into the
    [nz][ny][nx] outputs).  The drag error is stated from a surrogate trained first on ray-tracer
    drag: 1 048 576 columns of 32 members of the 256 x 128 x 90 sphere (26 train, 2 validate the
    early stopping, 4 held out for the error)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2309_11257_gb300 import gwam, surrogate

    t_start = time.perf_counter()
    S = gwam.Surrogate(max_batch=SUR_BATCH, seed=1)
    te, base, train_cps, hist, infos, ntr, kept, nval, gen_s = None, None, None, [], None, 0, None, 0, None
    if args.train_steps > 0:
        X, Y, infos = surrogate.generate_1m()
        gen_s = time.perf_counter() - t_start
        ncol = infos[0]["ncol"]
        tr, va, tm = surrogate.member_split(4, 8, ncol)
        Xtr, Ytr = X[tr].contiguous(), Y[tr].contiguous()
        Xva, Yva = X[va].contiguous(), Y[va].contiguous()
        X, Y = X[tm].contiguous(), Y[tm].contiguous()          # the held-out members
        ntr, nval = Xtr.shape[0], Xva.shape[0]
        S.fit_normalization(Xtr, Ytr, margin=0.05)
        cfg = dict(surrogate.TRAIN_1M, max_steps=min(args.train_steps, surrogate.TRAIN_1M["max_steps"]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        best, kept, hist = surrogate.train_early_stopping(S, Xtr, Ytr, Xva, Yva, 90, **cfg)
        e1.record()
        e1.synchronize()
        steps_run = hist[-1][0] if hist else 0
        train_cps = steps_run * cfg["batch"] / (e0.elapsed_time(e1) / 1000.0)
        te = surrogate.drag_error(S, X, Y, 90)
        ref = Y.double()
        base = float(torch.linalg.norm(ref - Ytr.double().mean(dim=0)) / torch.linalg.norm(ref))
        del Xtr, Ytr, Xva, Yva
    else:
        # throughput only (profiling): untrained weights, unit normalisation, synthetic features
        X = torch.randn((SUR_BATCH, 368), device="cuda")
        Y = torch.zeros((SUR_BATCH, 180), device="cuda")
        one, zero = np.ones(368, np.float32), np.zeros(368, np.float32)
        S.set_normalization(zero, one, np.zeros(180, np.float32), np.ones(180, np.float32), one * -1e30, one * 1e30)
    prep_s = time.perf_counter() - t_start

    B = SUR_BATCH
    idx = torch.arange(B, device="cuda") % X.shape[0]
    Xb = X[idx].contiguous()
    du = torch.zeros((90, B), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    mask = torch.zeros(B, dtype=torch.int32, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        S.infer(Xb, du, dv, mask, nfb)
    S.status()
    S.profile(True)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.settle()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)                  # evict the batch from L2 between timed passes
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        S.infer(Xb, du, dv, mask, nfb)
        b.record()
        b.synchronize()
        tot += a.elapsed_time(b)
    clocks = sampler.stop()
    prof, passes = S.profile_read()
    S.profile(False)
    S.status()
    value = B * args.steps / (tot / 1000.0)
    gemm_ms = prof["gemm_ms"] / max(passes, 1)
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = SUR_FLOPS_PER_COLUMN * B / (gemm_ms / 1000.0) / 1e12
    roofline = {"bound": "tensor", "kernel": "k_gemm_bf16 (tcgen05, 5 launches per pass)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "measured burst bf16 (MEASURED_PEAKS.json bf16_tflops)",
                "gemm_ms_per_pass": gemm_ms, "pack_ms_per_pass": prof["pack_ms"] / max(passes, 1),
                "flops_per_column": SUR_FLOPS_PER_COLUMN}

    # end to end: features from pinned host memory, drag back to pinned host memory
    e2e = None
    if not args.no_e2e:
        Xh = Xb.cpu().pin_memory()
        duh = torch.zeros((90, B), dtype=torch.float64).pin_memory()
        dvh = torch.zeros_like(duh).pin_memory()
        Xd = torch.empty_like(Xb)
        ke = max(1, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            Xd.copy_(Xh, non_blocking=True)
            S.infer(Xd, du, dv, mask, nfb)
            duh.copy_(du, non_blocking=True)
            dvh.copy_(dv, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e = {"value": B * ke / (t1 - t0), "unit": "columns/s", "h2d_bytes_per_step": B * 368 * 4,
               "d2h_bytes_per_step": 2 * 90 * B * 8, "steps": ke}

    cpu = None
    if not args.no_cpu:
        from oracle import mlp
        p64 = [(W.astype(np.float64), b.astype(np.float64)) for W, b in S.params()]
        xs = np.random.default_rng(0).standard_normal((4096, 368))
        mlp.forward(p64, xs[:256])
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0:
            mlp.forward(p64, xs)
            reps += 1
        dtc = time.perf_counter() - t0
        cpu = {"value": 4096 * reps / dtc, "unit": "columns/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d FP64 forward passes of 4096 columns (%.1f s), numpy BLAS on all host cores" % (reps, dtc)}
    line = {"metric": "surrogate columns/s", "value": value, "unit": "columns/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "surrogate MLP 368-4x512-180 GELU, batch %d columns" % B,
                       "data": "1 048 576 columns from the FP64 tracer on 32 members of the 256x128x90 sphere "
                               "(sphere workload jets + ensemble jet distribution, background and convective "
                               "sources)" if te else "synthetic features, untrained",
                       "drag_rel_l2_heldout": te["rel_l2"] if te else None,
                       "drag_rel_l2_bound": 0.72, "drag_rel_l2_mean_baseline": base,
                       "fallback_heldout": te["n_fallback"] if te else None,
                       "heldout_columns": int(Y.shape[0]) if te else 0,
                       "train_columns": ntr, "validation_columns": nval, "kept_step": kept,
                       "train_columns_per_s": train_cps, "validation_history": hist,
                       "tracer_columns_per_s": (8 * infos[0]["ncol"] / (infos[0]["tracer_ms_per_step"] / 1000.0))
                       if infos else None,
                       "generation_seconds": gen_s, "prep_seconds": prep_s, "fallback_in_batch": int(nfb.item()),
                       "l2": "256 MB buffer written between timed passes"},
            "gpu_launches": args.steps * 6, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def launches_per_step(params, fp32=False) -> int:
    """Kernels of the library per eager gwam_step (memsets excluded): begin, advance, the two kernels
    that scan the new-id and per-cell counts together, scatter, segment sort, materialise, project,
    divergence, budget fold; the cap's find, apply and scan; the saturation's run list and kappa; in
    the FP64 form the smoothing, or without smoothing the split of the fields into double-float
    pairs; in the precision form the smoothing (which narrows the FP64 fields as it reads them), or
    without smoothing the narrowing pass."""
    n = 1 + 1 + 2 + 1 + 1 + 1 + 1 + 1 + 1
    if params.get("cap_per_column", 0) > 0:
        n += 2 + 2
    if params.get("saturation", 0):
        n += 2
    n += 1
    return n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--eager", action="store_true", help="time gwam_step calls instead of graph replays")
    ap.add_argument("--lead-in", type=int, default=-1,
                    help="untimed steps after the launch before the warm-up (default: half of the 200-step run)")
    ap.add_argument("--e2e-steps", type=int, default=50, help="steps of the end-to-end measurement")
    ap.add_argument("--cpu-steps", type=int, default=24,
                    help="oracle steps of the CPU baseline sample (about 10 s on 16 host cores)")
    ap.add_argument("--train-steps", type=int, default=1500,
                    help="surrogate workload: at most this many training steps (early stopping; 0: untrained "
                         "weights, throughput only)")
    ap.add_argument("--workload", default="sphere",
                    choices=["sphere", "sphere_half", "ensemble", "sphere_fp32", "sphere_half_fp32", "surrogate",
                             "sphere_columnar", "sphere_coupled", "sphere_ghost", "sphere_theta"],
                    help="sphere_half: the same physics on 128 x 64 columns (profiling captures); "
                         "sphere_columnar: the sphere in the single-column (MS-GWaM-1D) mode; "
                         "sphere_coupled: the sphere with u, v advanced by the drag after every step "
                         "(add on the device, then gwam_set_background, inside the timed region); "
                         "sphere_theta: the sphere with the potential-temperature flux projected too; "
                         "sphere_ghost: the source emitted through the ghost layer before every 60 s step, "
                         "from no rays (the count grows by up to 0.98 M per step); "
                         "ensemble: 16 members of the sphere with convective sources, graph-replayed steps; "
                         "surrogate: MLP inference over 32768 columns after training on tracer drag")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "ensemble":
        return ensemble_arm(args)
    if args.workload == "surrogate":
        return surrogate_arm(args)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = gpu_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
