"""Launch-shape and sort-interval autotuner for the particle kernels.

Times complete runs (lpm_reset + lpm_step over the whole horizon, so the release ramp,
the exits and the end-of-run binning are all represented) for every supported
(threads per block, particles per thread, occupancy variant), and with
``autotune_with_sort`` also for several intervals of the re-ordering of the particles by
weather cell (the steps fused between two sorts), with CUDA events on the context stream,
and keeps the fastest. Results are cached per (GPU name, workload signature) in a JSON file
(``$LPM_AUTOTUNE_CACHE`` or ``~/.cache/lpm_gb300/autotune.json``). Every shape and sort
interval gives bit-identical results, so tuning never changes what is computed.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Iterable, Optional, Tuple

from . import lpm

BLOCKS = (128, 256, 512)
PPTS = (1, 2, 4)
OCCS = (0, 1, 2)
# shapes tried by default: every (block, particles per thread, occupancy variant)
DEFAULT_SHAPES = [(b, p, o) for b in BLOCKS for p in PPTS for o in OCCS]


def cache_path() -> str:
    return os.environ.get("LPM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lpm_gb300",
                                       "autotune.json"))


def signature(cfg) -> str:
    """Workload signature: the shapes and switches that change the kernel's work."""
    parts = [cfg.nx, cfg.ny, cfg.nz, cfg.n_met_t, cfg.cx, cfg.cy, cfg.cz, cfg.n_steps,
             cfg.bin_every, cfg.n_particles, cfg.n_scenarios, cfg.kh is None,
             cfg.rain is None, cfg.vd_dry > 0, cfg.wet_lambda > 0, cfg.lateral_exit,
             cfg.reflect_top, cfg.drift_correction, round(cfg.dt, 6),
             getattr(cfg, "kz_model", 0), getattr(cfg, "chain_half_lives", None) is not None,
             0 if getattr(cfg, "modes", None) is None else len(cfg.modes)]
    return hashlib.sha1(repr(parts).encode()).hexdigest()[:16]


def _load() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: Dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_shape(sim, shape, reps: int = 2) -> float:
    """Milliseconds of one complete run with the given launch shape (best of ``reps``)."""
    import torch
    lpm.lpm_set_launch(sim.ctx, *shape)
    stream = sim.stream
    best = float("inf")
    for _ in range(reps + 1):                # the first run builds graphs and warms up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.reset()
        sim.step(sim.cfg.n_steps - sim.k)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune(sim, shapes: Optional[Iterable[Tuple[int, int, int]]] = None, use_cache: bool = True,
             reps: int = 2) -> Tuple[int, int, int]:
    """Picks and applies the fastest launch shape for ``sim`` (a ``Sim``); returns it."""
    import torch
    key = f"{torch.cuda.get_device_name()}|{signature(sim.cfg)}"
    cache = _load() if use_cache else {}
    if key in cache:
        shape = tuple(cache[key]["shape"])
        lpm.lpm_set_launch(sim.ctx, *shape)
        return shape
    shapes = [tuple(v) for v in shapes] if shapes is not None else DEFAULT_SHAPES
    results = {}
    for shape in shapes:
        try:
            results["x".join(map(str, shape))] = time_shape(sim, shape, reps)
        except lpm.LpmError as e:
            # shapes the context's options do not run with (e.g. dosage, Eq. 3 K_z or a
            # decay chain need one particle per thread)
            if e.status != lpm.LPM_E_INVALID:
                raise
    if not results:
        raise RuntimeError("no launch shape runs with this context's options")
    best = min(results, key=results.get)
    shape = tuple(int(v) for v in best.split("x"))
    lpm.lpm_set_launch(sim.ctx, *shape)
    sim.reset()
    if use_cache:
        cache = _load()
        cache[key] = {"shape": list(shape), "ms": results}
        _store(cache)
    return shape


SORT_INTERVALS = (30, 60, 90)


def autotune_with_sort(sim, shapes: Optional[Iterable[Tuple[int, int, int]]] = None,
                       sort_intervals: Iterable[int] = SORT_INTERVALS, use_cache: bool = True,
                       reps: int = 2) -> Tuple[Tuple[int, int, int], int, Dict[str, float]]:
    """Picks and applies the fastest (launch shape, sort interval) for ``sim``; returns the
    shape, the interval and the measured milliseconds of every combination tried."""
    import torch
    intervals = [int(e) for e in sort_intervals]
    key = f"{torch.cuda.get_device_name()}|{signature(sim.cfg)}|sort{intervals}"
    cache = _load() if use_cache else {}
    if key in cache:
        shape = tuple(cache[key]["shape"])
        every = int(cache[key]["sort_every"])
        lpm.lpm_set_launch(sim.ctx, *shape)
        lpm.lpm_set_sort(sim.ctx, every)
        return shape, every, cache[key]["ms"]
    shapes = [tuple(v) for v in shapes] if shapes is not None else DEFAULT_SHAPES
    results = {}
    for every in intervals:
        lpm.lpm_set_sort(sim.ctx, every)
        for shape in shapes:
            try:
                results["x".join(map(str, shape)) + f"/sort{every}"] = time_shape(sim, shape, reps)
            except lpm.LpmError as e:
                if e.status != lpm.LPM_E_INVALID:
                    raise
    if not results:
        raise RuntimeError("no launch shape runs with this context's options")
    best = min(results, key=results.get)
    shape_s, every_s = best.split("/sort")
    shape = tuple(int(v) for v in shape_s.split("x"))
    every = int(every_s)
    lpm.lpm_set_launch(sim.ctx, *shape)
    lpm.lpm_set_sort(sim.ctx, every)
    sim.reset()
    if use_cache:
        cache = _load()
        cache[key] = {"shape": list(shape), "sort_every": every, "ms": results}
        _store(cache)
    return shape, every, results
