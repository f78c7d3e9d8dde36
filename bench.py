#!/usr/bin/env python
"""Throughput benchmark of the particle model on GB300.

Workload (one bench "step" = one complete simulation on inputs resident in HBM): the
realistic plain-method configuration: 1e7 particles released continuously from a point
source over 24 h at dt = 30 s (2880 steps), hourly 200x200x30 weather (log profile plus
seeded mesoscale modes, K_z profile), 8-day half-life, dry and wet deposition, lateral
exit, hourly 400x400x20 concentration snapshots and a 400x400 deposition grid.
Metric: ACTIVE particle-steps per second (a particle advanced one dt while airborne).

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded particle sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s on 1 GB300, % of roofline; batched & adjoint vs plain step"
UNIT = "particle-steps/s"
WORKLOAD = ("plain method, realistic: 1e7 particles, 24 h at dt=30 s (2880 steps), hourly "
            "200x200x30 met, decay + dry/wet deposition + lateral exit, hourly 400x400x20 "
            "snapshots")

# Algorithmic 32-bit operations per active particle-step (FP32 + INT32 lane operations as
# the method states them; transcendental = 1): Philox4x32-10 twice (displacement and
# deposition streams) 2 x 98, uniforms 12, Box-Muller 11, 4D gather index and weight math
# 30, 16-corner lerps of 4 components 120, move 18, reflection/exit 8, deposition test 4.
OPS_PER_PARTICLE_STEP = 2 * 98 + 12 + 11 + 30 + 120 + 18 + 8 + 4
# The upper end of the coarser estimate of the same work (250-350 instructions per
# particle-step), reported beside it.
OPS_PER_PARTICLE_STEP_LOW = 350
# DRAM traffic per advance launch from an ncu capture of two mid-run 60-step launches
# (hours 10-11 of the realistic workload, persistent grid of 2 blocks per SM; read + write,
# mean of the two), valid while the kernel sources hash to the values below.
ADVANCE_TRAFFIC_BYTES = 0.5 * ((22.372096 + 0.0) + (23.778816 + 0.01792)) * 1e6
ADVANCE_TRAFFIC_SOURCES = {"lpm_advance.cuh": "fdaaeb52", "lpm_device.cuh": "c030129e"}
# Busiest hardware units of the same capture (% of peak, mean of the two launches): the
# L1 data pipe carrying the weather gathers, and the warp-instruction issue slots.
ADVANCE_BUSIEST_UNITS = {"l1tex_data_pipe": 0.5 * (82.04 + 82.09) / 100.0,
                         "issue_slots": 0.5 * (74.43 + 74.28) / 100.0}
LANES_PER_SM = 128          # 4 sub-partitions x 32 lanes issue one op per clock


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def capture_current():
    """Whether the kernel sources still hash to those of the committed ncu capture."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_0912_3223_gb300", "csrc")
    for name, digest in ADVANCE_TRAFFIC_SOURCES.items():
        with open(os.path.join(csrc, name), "rb") as f:
            if not hashlib.sha1(f.read()).hexdigest().startswith(digest):
                return False
    return True


def advance_traffic():
    """The captured per-launch DRAM traffic, or None once the kernel sources changed."""
    return ADVANCE_TRAFFIC_BYTES if capture_current() else None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts once the sampler has written its first row (bounded wait)
        t_end = time.monotonic() + 3.0
        while time.monotonic() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return parse_clock_rows(lines)


def parse_clock_rows(lines):
    """Summary of nvidia-smi rows (the ClockSampler fields, csv, no header or units): the
    median SM clock over the samples under load (above half the maximum), the maximum, and
    every throttle reason seen active in any sample."""
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return out
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for name, v in zip(names, r[5:9]):
            if v.lower() in ("active", "1"):
                reasons.add(name)
    loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
    out.update(sm_mhz=statistics.median(loaded) if loaded else None,
               sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
               samples=len(rows))
    return out


# ------------------------------------------------------------------------------------
# CPU baseline: the oracle on a deterministic particle sample of the same workload
# ------------------------------------------------------------------------------------
def oracle_sample(cfg, stride: int, offset: int = 0):
    import numpy as np
    import oracle
    oracle.build()
    sel = np.arange(offset, cfg.n_particles, stride, dtype=np.int64)
    t0 = time.perf_counter()
    r = oracle.run(cfg, sel=sel)
    dt = time.perf_counter() - t0
    return r["active_steps"], dt, sel.size


def _oracle_worker(job):
    """One process of the all-cores leg: the oracle on particles offset, offset + stride, ...
    of the realistic workload (regenerated from its seeds in the process)."""
    stride, offset = job
    import lpm_inputs as li
    return oracle_sample(li.make_cfg1(), stride, offset)


def _host_workers() -> int:
    """Host cores to use, at most one process per 1.5 GB of available memory (one process
    holds the 480 MB weather and about 0.1 GB of grids)."""
    n = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(ln.split()[1]) * 1024 for ln in f if ln.startswith("MemAvailable:"))
        n = min(n, max(1, int(avail // (1.5 * 2 ** 30))))
    except (OSError, StopIteration, ValueError):
        n = 1
    return n


def cpu_baseline(cfg, stride: int = 30, all_cores: bool = True):
    steps, dt, n = oracle_sample(cfg, stride)
    out = {"value": steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"every {stride}th particle ({n} particles) of the workload, all "
                     f"{cfg.n_steps} steps: {steps} active particle-steps in {dt:.1f} s, "
                     "FP64, single thread"}
    workers = _host_workers() if all_cores else 1
    if workers > 1:
        # the same oracle in `workers` spawned processes over interleaved particle subsets
        # (particles are independent), each process loaded with about half the single-thread
        # sample; throughput = summed particle-steps / the slowest process
        import multiprocessing as mp
        s_all = max(1, round(2 * stride / workers))
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(s_all * workers, r * s_all) for r in range(workers)])
        tot = sum(r[0] for r in res)
        slow = max(r[1] for r in res)
        out["all_cores"] = {
            "value": tot / slow, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"every {s_all}th particle ({sum(r[2] for r in res)} particles), all "
                      f"{cfg.n_steps} steps, in {workers} processes: {tot} active "
                      f"particle-steps, slowest process {slow:.1f} s, FP64"}
    return out


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import lpm_inputs as li
    cfg = li.make_cfg1()
    stride = args.ref_stride
    for _ in range(args.warmup):
        oracle_sample(cfg, stride * 10)
    tot_steps, tot_t, n = 0, 0.0, 0
    for _ in range(args.steps):
        s, dt, n = oracle_sample(cfg, stride)
        tot_steps += s
        tot_t += dt
    value = tot_steps / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_stride": stride},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"every {stride}th particle ({n} particles), all steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------
def measure_batched(args, stream, cfg=None):
    """The batched ensemble form: 256 scenarios (log-uniform 1e4..1e6 particles, own
    source, release height, 24-value emission series and wind offset), 12 h at dt = 30 s,
    particles of all scenarios sorted by cell every `sort_every` steps; the whole run (sorts
    and persistent launches) is one CUDA graph launch."""
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = cfg or li.make_cfg2()
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.batched_block, args.batched_ppt,
                                              args.batched_occ),
                  sort_every=args.batched_sort_every)
    tuned = None
    try:
        if args.autotune:
            # the autotuner's choice of launch shape and sort interval, timed fresh here
            from paper_0912_3223_gb300.autotune import autotune_with_sort
            shape, every, tried = autotune_with_sort(
                sim, shapes=[(512, 1, 2), (256, 1, 2), (128, 1, 2), (256, 1, 1), (256, 2, 1)],
                sort_intervals=(30, 60, 90), use_cache=False, reps=1)
            tuned = {"launch": list(shape), "sort_every": every,
                     "ms_per_run_tried": {k: round(v, 2) for k, v in tried.items()}}
        for _ in range(max(1, args.warmup)):
            sim.reset()
            sim.step(cfg.n_steps)
        torch.cuda.synchronize()
        lpm.lpm_stats(sim.ctx)
        times, active = [], 0
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            sim.reset()
            sim.step(cfg.n_steps)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            active += sum(int(sim.fixed_state(s)[2][4]) for s in range(cfg.n_scenarios))
        launches, adv, _ = lpm.lpm_stats(sim.ctx)
    finally:
        sim.close()
    t = sum(times) / 1e3
    out = {"value": active / t, "unit": UNIT, "ms_per_run": statistics.mean(times),
           "scenarios": cfg.n_scenarios, "particles": cfg.n_particles,
           "steps_per_run": cfg.n_steps, "graph_launches_per_run": adv // max(1, args.steps),
           "kernel_launches_per_run": launches / max(1, args.steps),
           "launch": tuned["launch"] if tuned else [args.batched_block, args.batched_ppt,
                                                    args.batched_occ],
           "sort_every": tuned["sort_every"] if tuned else args.batched_sort_every,
           "weather": "shared hourly fields + per-scenario hourly wind offset + 4 "
                      "perturbation modes (own phases and amplitudes)"}
    if tuned:
        out["autotuned"] = tuned
    return out


def measure_adjoint(args, stream, storage="checkpoints"):
    """The adjoint form: 1e6 particles, 6 h at dt = 20 s on the realistic met, 64 receptors
    (Gaussian kernel, 200 m), sampled every 18 steps; forward (receptors, keeping the states
    the backward needs) and backward (reverse sweep) per run. ``storage``: "checkpoints"
    keeps the state every 64 steps and recomputes each segment in the backward (the form
    the workload names; the segments in weather-cell order, one segment's states as
    scratch); "trajectory" keeps every particle-step (9.3 GB) instead."""
    import numpy as np
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = li.make_cfg3(n_particles=args.adjoint_particles)
    rec = li.make_receptors()
    w = np.linspace(-1.0, 1.0, rec.shape[0])[None, :]
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream)
    try:
        if storage == "checkpoints":
            lpm.lpm_set_adjoint_storage(sim.ctx, 0)
        sim.reset()
        sim.step(cfg.n_steps)
        active = int(sim.fixed_state()[2][4])         # same paths as the receptor run
        for _ in range(max(1, args.warmup)):
            lpm.lpm_receptors(sim.ctx, 1, rec, 200.0, 18)
            lpm.lpm_adjoint(sim.ctx, rec, 200.0, 18, w, 24)
        fwd, bwd = [], []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lpm.lpm_receptors(sim.ctx, 1, rec, 200.0, 18)
            t1 = time.perf_counter()
            lpm.lpm_adjoint(sim.ctx, rec, 200.0, 18, w, 24)
            t2 = time.perf_counter()
            fwd.append(t1 - t0)
            bwd.append(t2 - t1)
        traj, nbytes = lpm.lpm_adjoint_storage(sim.ctx)
    finally:
        sim.close()
    tf, tb = statistics.mean(fwd), statistics.mean(bwd)
    return {"value": active / (tf + tb), "unit": UNIT,
            "note": "active particle-steps of the run / (forward + backward) wall time",
            "ms_forward": 1e3 * tf, "ms_backward": 1e3 * tb, "particles": cfg.n_particles,
            "steps_per_run": cfg.n_steps, "receptors": int(rec.shape[0]),
            "active_particle_steps": active,
            "storage": "trajectory" if traj else "checkpoints every 64 steps",
            "storage_gb": nbytes / 1e9}


def measure_inversion(args, stream):
    """Batched source inversion: 64 candidate sources x 1e5 particles on the adjoint
    workload, 20 Adam iterations (one receptor forward + one adjoint launch for all
    candidates per iteration) against observations of a hidden source."""
    import numpy as np
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim, lpm
    from paper_0912_3223_gb300.inversion import invert, observe
    cand, obs, hidden = li.make_cfg4()
    rec = li.make_receptors()
    with torch.cuda.stream(stream):
        with Sim(obs, stream=stream) as so:
            c_obs = observe(so, rec, 200.0, 18)
        sim = Sim(cand, stream=stream)
    try:
        sim.reset()
        sim.step(cand.n_steps)
        active = sum(int(sim.fixed_state(s)[2][4]) for s in range(cand.n_scenarios))
        t0 = time.perf_counter()
        res = invert(sim, rec, c_obs, n_iter=20)
        t = time.perf_counter() - t0
        traj, nbytes = lpm.lpm_adjoint_storage(sim.ctx)
    finally:
        sim.close()
    h = np.array(hidden)
    d0 = np.linalg.norm(res.sources[0, :, :2] - h[:2], axis=1).min()
    d1 = float(np.linalg.norm(res.sources[-1, res.best, :2] - h[:2]))
    return {"value": 20 * active / t, "unit": UNIT,
            "note": "20 x (forward + adjoint) active particle-steps / wall time of the inversion",
            "candidates": cand.n_scenarios, "particles": cand.n_particles,
            "ms_per_iteration": 1e3 * t / 20,
            "ms_forward_total": 1e3 * res.timings["forward"],
            "ms_adjoint_total": 1e3 * res.timings["adjoint"],
            "best_loss_start": float(res.loss[0].min()), "best_loss_end": float(res.loss[-1].min()),
            "best_distance_start_m": float(d0), "best_distance_end_m": d1,
            "storage": "trajectory" if traj else "checkpoints every 64 steps",
            "storage_gb": nbytes / 1e9}


def measure_stress(args, stream):
    """Forward-only stress case: 1e8 particles, 48 h at dt = 30 s, 512x512x32 weather."""
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim
    cfg = li.make_stress()
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, args.ppt, args.occ))
    cfg.uvwk = None                                   # the host copy is no longer needed
    try:
        sim.reset()
        sim.step(cfg.n_steps)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.reset()
        sim.step(cfg.n_steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        active = int(sim.fixed_state()[2][4])
    finally:
        sim.close()
    return {"value": active / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
            "particles": cfg.n_particles, "steps_per_run": cfg.n_steps,
            "met": [cfg.n_met_t, cfg.nz, cfg.ny, cfg.nx], "active_particle_steps": active}


def measure_dosage(args, stream):
    """The plain realistic run with the time-integrated dosage sampled every 4 steps (the
    paper's smallest summation interval, Sec. 3.2) in the step kernel."""
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim
    cfg = li.make_cfg1()
    every = 4
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, args.ppt, args.occ),
                  sort_every=args.sort_every)
    try:
        times = []
        for i in range(max(1, args.warmup) + 2):
            sim.reset()
            sim.set_dosage(every)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(cfg.n_steps)
            e1.record(stream)
            e1.synchronize()
            if i >= max(1, args.warmup):
                times.append(e0.elapsed_time(e1))
        active = int(sim.fixed_state()[2][4])
        samples = sim.dosage()[2]
    finally:
        sim.close()
    ms = statistics.mean(times)
    return {"value": active / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
            "dose_every": every, "samples_per_run": samples, "particles": cfg.n_particles,
            "steps_per_run": cfg.n_steps}


def measure_kz_eq3(args, stream):
    """The plain realistic run with K_z computed in the step from Eq. 3 on hourly
    boundary-layer columns (u*, 1/L, H_z) instead of read from the gridded field."""
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim
    cfg = li.make_cfg1(kz_eq3=True)
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, 1, args.occ),
                  sort_every=args.sort_every)
    try:
        times = []
        for i in range(max(1, args.warmup) + 2):
            sim.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(cfg.n_steps)
            e1.record(stream)
            e1.synchronize()
            if i >= max(1, args.warmup):
                times.append(e0.elapsed_time(e1))
        active = int(sim.fixed_state()[2][4])
    finally:
        sim.close()
    ms = statistics.mean(times)
    return {"value": active / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
            "kz": "Eq. 3 in the step (Businger-Dyer Phi_h), hourly u*, 1/L, H_z columns",
            "particles": cfg.n_particles, "steps_per_run": cfg.n_steps}


def measure_decay_chain(args, stream):
    """The plain realistic run with a three-species decay chain (the 8-day parent, a
    12-hour daughter, a stable end): every snapshot and deposition also bins the
    daughters."""
    import dataclasses

    import numpy as np
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim
    base = li.make_cfg1()
    cfg = dataclasses.replace(base, chain_half_lives=np.array([base.half_life_s, 43200.0, 0.0]))
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, 1, args.occ),
                  sort_every=args.sort_every)
    try:
        times = []
        for i in range(max(1, args.warmup) + 2):
            sim.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(cfg.n_steps)
            e1.record(stream)
            e1.synchronize()
            if i >= max(1, args.warmup):
                times.append(e0.elapsed_time(e1))
        active = int(sim.fixed_state()[2][4])
    finally:
        sim.close()
    ms = statistics.mean(times)
    return {"value": active / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
            "species": [float(v) for v in cfg.chain_half_lives], "particles": cfg.n_particles,
            "steps_per_run": cfg.n_steps}


def measure_langevin(args, stream):
    """The plain realistic run with the vertical Langevin (velocity-memory) variant,
    T_L = 100 s."""
    import dataclasses

    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim
    cfg = dataclasses.replace(li.make_cfg1(), langevin=1, t_lagr=100.0)
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, 1, args.occ),
                  sort_every=args.sort_every)
    try:
        times = []
        for i in range(max(1, args.warmup) + 2):
            sim.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(cfg.n_steps)
            e1.record(stream)
            e1.synchronize()
            if i >= max(1, args.warmup):
                times.append(e0.elapsed_time(e1))
        active = int(sim.fixed_state()[2][4])
    finally:
        sim.close()
    ms = statistics.mean(times)
    return {"value": active / (ms / 1e3), "unit": UNIT, "ms_per_run": ms, "t_lagr_s": cfg.t_lagr,
            "particles": cfg.n_particles, "steps_per_run": cfg.n_steps}


def device_sm_count(index: int) -> int:
    """Streaming multiprocessors of the device (cudaDeviceProp.multiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(index).multi_processor_count)


def alu_roofline(active_steps, adv_ms, step_ms_total, sm_count, clk, peaks):
    """The advance kernel against its ALU roofline. achieved = algorithmic operations of the
    timed runs / the advance launches' summed CUDA-event time; peak = the device's SMs x 128
    lanes x the median SM clock sampled during the timed region (one 32-bit operation per
    lane per clock), falling back to the device's maximum clock when no sample was taken."""
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or peaks.get("sm_max_mhz")
    clock_source = "median of the timed region's samples" if clk.get("sm_mhz") else \
        "maximum SM clock (no samples)"
    peak = sm_count * LANES_PER_SM * mhz * 1e6 / 1e12 if mhz else None
    rate = active_steps / (adv_ms / 1e3) if adv_ms > 0 else None
    achieved = OPS_PER_PARTICLE_STEP * rate / 1e12 if rate else None
    achieved_low = OPS_PER_PARTICLE_STEP_LOW * rate / 1e12 if rate else None
    return {
        "bound": "alu", "kernel": "advance_kernel",
        "achieved": achieved, "peak": peak, "unit": "Tops/s",
        "frac": achieved / peak if achieved and peak else None,
        "traffic": advance_traffic(),
        "traffic_unit": "bytes per advance launch (ncu capture, mid-run launches)",
        "peak_source": (f"derived: {sm_count} SMs (queried from the device) x {LANES_PER_SM} "
                        f"lanes x {mhz:.0f} MHz ({clock_source}); one 32-bit op per lane per "
                        "clock") if mhz else None,
        "ops_per_particle_step": OPS_PER_PARTICLE_STEP,
        "advance_particle_steps_per_s": rate,
        "frac_at_350_ops": achieved_low / peak if achieved_low and peak else None,
        # the hardware view of the same kernel (ncu capture, % of each unit's peak): what
        # bounds it is the L1 data pipe and the issue slots, not DRAM
        "busiest_units": dict(ADVANCE_BUSIEST_UNITS,
                              source="ncu capture of the same kernel sources (hashes in "
                                     "ADVANCE_TRAFFIC_SOURCES)") if capture_current() else None,
        "advance_share_of_step": (adv_ms / 1e3) / (step_ms_total / 1e3) if step_ms_total else None,
        "hbm_gbs_measured_peak": peaks.get("hbm_gbs"),
    }


def run_gpu(args):
    import numpy as np
    import torch

    import lpm_inputs as li
    from paper_0912_3223_gb300 import Sim, lpm, parallel
    from paper_0912_3223_gb300 import build as pkg_build

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    store = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        store = dist.distributed_c10d._get_default_store()
    pkg_build.build()
    lpm.load()

    # weak scaling: N GPUs run one release of N x 1e7 particles, each rank holding a
    # contiguous range of 1e7 (the same keyed draws as a single run of the whole release);
    # at every hourly snapshot the ranks sum their fixed-point grids and counters on the
    # device (one int64 all-reduce over NCCL), the exchange step of a partitioned run
    per_rank = 10_000_000                        # the realistic workload's particles
    cfg = li.make_cfg1(n_particles=per_rank * world)
    part = parallel.partition(cfg.n_particles, world, rank) if world > 1 else None
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = Sim(cfg, stream=stream, launch=(args.block, args.ppt, args.occ),
                  sort_every=args.sort_every, part=part)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    exchange = parallel.SnapshotExchange(sim) if world > 1 else None
    ex_events = []
    runs = [0]

    def timed_exchange():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        exchange()
        e1.record(stream)
        ex_events.append((e0, e1))

    def one_run():
        sim.reset()
        if exchange is None:
            sim.step(cfg.n_steps)
        else:
            runs[0] += 1
            for _ in parallel.run_partitioned(sim, cfg.n_steps, cfg.bin_every, timed_exchange,
                                              store=store, world=world, rank=rank,
                                              timeout_s=60.0, run_tag=f"run{runs[0]}/"):
                pass

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()
    ex_events.clear()
    lpm.lpm_stats(sim.ctx)
    lpm.lpm_set_profiling(sim.ctx, True)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, active = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)                       # L2 flush between timed steps (256 MB > L2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        one_run()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        _, _, ctr, _ = sim.fixed_state()
        active.append(int(ctr[4]))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ex_ms = sum(a.elapsed_time(b) for a, b in ex_events)
    n_ex = len(ex_events)
    launches, adv_launches, adv_ms = lpm.lpm_stats(sim.ctx)
    lpm.lpm_set_profiling(sim.ctx, False)
    t_total = sum(times) / 1e3
    psteps = sum(active)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        p = torch.tensor([psteps], dtype=torch.float64, device="cuda")
        dist.all_reduce(p)
        t_total, psteps = float(t.item()), int(p.item())
    value = psteps / t_total

    # end to end through the C ABI with host buffers: met from pinned host memory in,
    # snapshots, deposition and budget out, every step
    pinned_uvwk = torch.from_numpy(cfg.uvwk).pin_memory()
    pinned_rain = torch.from_numpy(cfg.rain).pin_memory()
    conc_t = torch.empty((cfg.cz, cfg.cy, cfg.cx), dtype=torch.float64, pin_memory=True)
    dep_t = torch.empty((2, cfg.cy, cfg.cx), dtype=torch.float64, pin_memory=True)
    conc = conc_t.numpy()
    if exchange is not None:
        unit = 2.0 ** -int(sim.fixed_state()[3])         # fixed-point unit (mass)
        conc_f = unit / (cfg.cdx * cfg.cdy * cfg.cdz)
        dep_f = unit / (cfg.cdx * cfg.cdy)
    h2d = pinned_uvwk.numel() * 4 + pinned_rain.numel()
    d2h = conc.nbytes + 2 * cfg.cy * cfg.cx * 8 + 8 * 8
    e2e_t, e2e_p = 0.0, 0
    for i in range(max(1, args.warmup) + args.steps):   # warm-up passes first, untimed
        torch.cuda.synchronize()
        if world > 1 and i == max(1, args.warmup):
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for t in range(cfg.n_met_t):
            lpm.lpm_set_met(sim.ctx, t, pinned_uvwk[t], None, pinned_rain[t])
        one_run()
        if exchange is None:
            sim.concentration(out=conc)
            dry, wet = sim.deposition()
        else:
            # the whole release's grids, from the last exchange, converted on the device
            with torch.cuda.stream(stream):
                conc_t.copy_(exchange.conc.to(torch.float64) * conc_f)
                dep_t.copy_(exchange.dep.to(torch.float64) * dep_f)
            stream.synchronize()
        b = sim.budget()
        if i < max(1, args.warmup):
            continue
        e2e_t += time.perf_counter() - t0
        _, _, ctr, _ = sim.fixed_state()
        e2e_p += int(ctr[4])
    if world > 1:                                # whole job: max time, summed work
        import torch.distributed as dist
        t = torch.tensor([e2e_t], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        p = torch.tensor([e2e_p], dtype=torch.float64, device="cuda")
        dist.all_reduce(p)
        e2e_t, e2e_p = float(t.item()), int(p.item())
    e2e_value = e2e_p / e2e_t

    sim.close()
    peaks = read_peaks()
    roofline = alu_roofline(sum(active), adv_ms, sum(times), device_sm_count(local), clk, peaks)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": cfg.n_particles, "steps_per_run": cfg.n_steps,
                   "dt_s": cfg.dt, "met": [cfg.n_met_t, cfg.nz, cfg.ny, cfg.nx],
                   "launch": [args.block, args.ppt, args.occ], "sort_every": args.sort_every,
                   "l2": "flushed (256 MB write) between timed steps",
                   "active_particle_steps_per_run": sum(active) // max(1, len(active)),
                   "slot_steps_per_run": cfg.n_particles * cfg.n_steps},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world > 1:
        line["config"]["partition"] = (f"one release of {cfg.n_particles} particles, "
                                       f"{per_rank} per rank (contiguous id ranges)")
        line["exchange"] = {
            "what": "int64 all-reduce (NCCL) of the hourly snapshot, deposition grids and "
                    "counters, on the device",
            "per_run": n_ex // max(1, args.steps), "bytes_per_rank": exchange.bytes,
            "ms_per_run": ex_ms / max(1, args.steps),
            "share_of_step": ex_ms / max(1e-9, sum(times))}
    if not args.no_forms:
        forms = {"batched": measure_batched(args, stream),
                 "adjoint": measure_adjoint(args, stream, "checkpoints"),
                 "adjoint_trajectory": measure_adjoint(args, stream, "trajectory"),
                 "inversion": measure_inversion(args, stream),
                 "dosage": measure_dosage(args, stream),
                 "kz_eq3": measure_kz_eq3(args, stream),
                 "decay_chain": measure_decay_chain(args, stream),
                 "langevin": measure_langevin(args, stream)}
        if not args.no_stress:
            forms["stress"] = measure_stress(args, stream)
        for f in forms.values():
            f["vs_plain"] = f["value"] / value * world   # both per GPU
        line["forms"] = forms
        if world > 1:
            line["forms_scope"] = "rank 0's GPU"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_stride)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def relaunch_distributed(n: int) -> int:
    """``--gpus N`` outside a distributed launcher: run this command again as N ranks on
    this node (torch.distributed.run, rendezvous on 127.0.0.1) and return its status."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)]
    return subprocess.call(cmd + sys.argv[1:])


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block", type=int, default=512)
    ap.add_argument("--ppt", type=int, default=1)
    ap.add_argument("--occ", type=int, default=2)
    ap.add_argument("--sort-every", type=int, default=60,
                    help="re-order the particles by weather cell every N steps (0 = off)")
    ap.add_argument("--ref-stride", type=int, default=100,
                    help="particle sample stride of each --impl reference step")
    ap.add_argument("--cpu-stride", type=int, default=30,
                    help="particle sample stride of the cpu_baseline leg (about 10-20 s of oracle "
                         "work on one core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and adjoint forms")
    ap.add_argument("--no-stress", action="store_true", help="skip the 1e8-particle stress case")
    ap.add_argument("--only", choices=["batched", "adjoint", "adjoint_trajectory", "inversion",
                                       "stress", "dosage", "kz_eq3", "decay_chain", "langevin"],
                    default=None,
                    help="run one form alone and print its measurement (profiling aid)")
    ap.add_argument("--batched-block", type=int, default=512)
    ap.add_argument("--batched-ppt", type=int, default=1)
    ap.add_argument("--batched-occ", type=int, default=2)
    ap.add_argument("--adjoint-particles", type=int, default=1_000_000,
                    help="particles of the adjoint form (smaller for profiler captures)")
    ap.add_argument("--batched-sort-every", type=int, default=60,
                    help="steps between sorts by cell in the batched form (0: off)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the batched form with the given launch shape and sort interval "
                         "instead of the autotuner's choice")
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 0)
    if args.gpus > 1 and world == 0:
        return relaunch_distributed(args.gpus)
    if world and args.gpus != world:
        print(f"--gpus {args.gpus} does not match WORLD_SIZE={world}", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        from paper_0912_3223_gb300 import build as pkg_build
        pkg_build.build()
        stream = torch.cuda.Stream()
        fn = {"batched": measure_batched, "adjoint": measure_adjoint,
              "adjoint_trajectory": lambda a, st: measure_adjoint(a, st, "trajectory"),
              "inversion": measure_inversion, "stress": measure_stress,
              "dosage": measure_dosage, "kz_eq3": measure_kz_eq3,
              "decay_chain": measure_decay_chain, "langevin": measure_langevin}[args.only]
        print(json.dumps({"form": args.only, **fn(args, stream)}), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
