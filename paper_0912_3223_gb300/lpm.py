"""Python binding of the C ABI in include/lpm.h (argument marshalling only).

Functions keep the C names (``lpm_create``, ``lpm_set_met``, ``lpm_release``, ``lpm_step``,
``lpm_concentration``, ``lpm_deposition``, ``lpm_budget``, ...). Every step of the
particle method runs in the CUDA library; this module converts numpy arrays, torch
tensors and streams into plain pointers. It raises if the library has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblpm.so")
# The checked build (every kernel index tested against its array; see build.py), loaded
# instead when the environment sets LPM_CHECKED_BUILD=1 before the first call.
CHECKED_LIB_PATH = os.path.join(HERE, "liblpm_checked.so")


def library_path() -> str:
    return CHECKED_LIB_PATH if os.environ.get("LPM_CHECKED_BUILD") == "1" else LIB_PATH

LPM_OK, LPM_E_INVALID, LPM_E_OOM, LPM_E_CUDA, LPM_E_STATE, LPM_E_NUMERIC, LPM_E_TIMEOUT = range(7)
STATUS_NAMES = {0: "LPM_OK", 1: "LPM_E_INVALID", 2: "LPM_E_OOM", 3: "LPM_E_CUDA",
                4: "LPM_E_STATE", 5: "LPM_E_NUMERIC", 6: "LPM_E_TIMEOUT"}
B_RELEASED, B_AIR_IN, B_AIR_OUT, B_DRY, B_WET, B_EXITED, B_DECAYED, B_N_ACTIVE = range(8)

# Exported symbols declared in include/lpm.h.
SYMBOLS = ["lpm_create", "lpm_destroy", "lpm_last_error", "lpm_set_met", "lpm_set_source",
           "lpm_release", "lpm_step", "lpm_current_step", "lpm_concentration",
           "lpm_deposition", "lpm_budget", "lpm_particles", "lpm_fixed_state",
           "lpm_set_launch", "lpm_sync", "lpm_draws", "lpm_release_range", "lpm_reset",
           "lpm_set_profiling", "lpm_stats", "lpm_set_params", "lpm_set_emission",
           "lpm_receptors", "lpm_adjoint", "lpm_draws_static", "lpm_set_sort", "lpm_save",
           "lpm_load", "lpm_set_dosage", "lpm_dosage", "lpm_set_kz_model",
           "lpm_set_boundary_layer", "lpm_set_decay_chain", "lpm_species", "lpm_set_langevin",
           "lpm_particle_velocity", "lpm_set_adjoint_storage", "lpm_adjoint_storage",
           "lpm_set_modes", "lpm_set_mode_phases", "lpm_device_state"]


class LpmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lpm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("z_levels", C.POINTER(C.c_double)),
        ("n_met_t", C.c_int), ("met_t0", C.c_double), ("met_dt", C.c_double),
        ("cx", C.c_int), ("cy", C.c_int), ("cz", C.c_int),
        ("cx0", C.c_double), ("cy0", C.c_double), ("cz0", C.c_double),
        ("cdx", C.c_double), ("cdy", C.c_double), ("cdz", C.c_double),
        ("src_x", C.c_double), ("src_y", C.c_double), ("src_z", C.c_double),
        ("dt", C.c_double), ("n_steps", C.c_int64), ("seed", C.c_uint64),
        ("bin_every", C.c_int),
        ("half_life_s", C.c_double), ("vd_dry", C.c_double), ("h_mix", C.c_double),
        ("wet_lambda", C.c_double), ("kh_uniform", C.c_double),
        ("reflect_ground", C.c_int), ("reflect_top", C.c_int), ("z_top", C.c_double),
        ("lateral_exit", C.c_int), ("drift_correction", C.c_int),
        ("n_scenarios", C.c_int), ("max_particles", C.c_int64),
    ]


_lib = None


def load() -> C.CDLL:
    """Loads liblpm.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`"
                           + (" (the checked build: python paper_0912_3223_gb300/build.py "
                              "--checked)" if path == CHECKED_LIB_PATH else ""))
    L = C.CDLL(path)
    vp, i64, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
    L.lpm_create.argtypes = [C.POINTER(lpm_config), vp, C.POINTER(vp)]
    L.lpm_destroy.argtypes = [vp]
    L.lpm_destroy.restype = None
    L.lpm_last_error.argtypes = [vp]
    L.lpm_last_error.restype = C.c_char_p
    L.lpm_set_met.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
    L.lpm_set_source.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_double, vp]
    L.lpm_release.argtypes = [vp, C.c_int, i64, dp, C.c_int, C.c_double, i64, i64]
    L.lpm_step.argtypes = [vp, i64]
    L.lpm_current_step.argtypes = [vp, C.POINTER(i64)]
    L.lpm_concentration.argtypes = [vp, C.c_int, dp, C.c_size_t]
    L.lpm_deposition.argtypes = [vp, C.c_int, dp, dp, C.c_size_t]
    L.lpm_budget.argtypes = [vp, C.c_int, dp]
    L.lpm_particles.argtypes = [vp, i64, i64, C.POINTER(C.c_float), C.POINTER(C.c_uint32)]
    L.lpm_fixed_state.argtypes = [vp, C.c_int, C.POINTER(C.c_uint64), C.c_size_t,
                                  C.POINTER(C.c_uint64), C.c_size_t, C.POINTER(i64),
                                  C.POINTER(C.c_int)]
    L.lpm_set_launch.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.lpm_sync.argtypes = [vp]
    L.lpm_release_range.argtypes = [vp, C.c_int, i64, i64, i64, dp, C.c_int, C.c_double, i64,
                                    i64, i64]
    L.lpm_reset.argtypes = [vp]
    L.lpm_set_profiling.argtypes = [vp, C.c_int]
    L.lpm_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), dp]
    L.lpm_set_params.argtypes = [vp, C.c_double, C.c_double, C.c_double]
    L.lpm_set_sort.argtypes = [vp, C.c_int]
    L.lpm_set_dosage.argtypes = [vp, C.c_int]
    L.lpm_set_kz_model.argtypes = [vp, C.c_int, C.c_double]
    L.lpm_set_decay_chain.argtypes = [vp, C.c_int, dp]
    L.lpm_set_langevin.argtypes = [vp, C.c_int, C.c_double]
    L.lpm_particle_velocity.argtypes = [vp, i64, i64, C.POINTER(C.c_float)]
    L.lpm_species.argtypes = [vp, C.c_int, C.c_int, dp, dp, dp, C.POINTER(C.c_uint64),
                              C.POINTER(C.c_uint64)]
    L.lpm_set_boundary_layer.argtypes = [vp, C.c_int, vp, C.c_int]
    L.lpm_dosage.argtypes = [vp, C.c_int, dp, C.c_size_t, C.POINTER(C.c_uint64), C.POINTER(i64)]
    L.lpm_save.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.lpm_load.argtypes = [vp, vp, C.c_size_t]
    L.lpm_set_emission.argtypes = [vp, C.c_int, dp, C.c_int]
    L.lpm_receptors.argtypes = [vp, dp, C.c_int, C.c_double, C.c_int, dp]
    L.lpm_adjoint.argtypes = [vp, dp, C.c_int, C.c_double, C.c_int, dp, dp]
    L.lpm_set_adjoint_storage.argtypes = [vp, C.c_uint64]
    L.lpm_adjoint_storage.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_uint64)]
    L.lpm_device_state.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                   C.POINTER(i64)]
    L.lpm_set_modes.argtypes = [vp, C.c_int, dp, dp]
    L.lpm_set_mode_phases.argtypes = [vp, C.c_int, dp, dp]
    L.lpm_draws_static.argtypes = [C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32),
                                   C.c_uint32, i64, C.POINTER(C.c_uint32), C.POINTER(C.c_float)]
    L.lpm_draws.argtypes = [C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32),
                            C.c_uint32, i64, C.POINTER(C.c_uint32), C.POINTER(C.c_float)]
    for name in ("lpm_create", "lpm_set_met", "lpm_set_source", "lpm_release", "lpm_step",
                 "lpm_current_step", "lpm_concentration", "lpm_deposition", "lpm_budget",
                 "lpm_particles", "lpm_fixed_state", "lpm_set_launch", "lpm_sync",
                 "lpm_draws", "lpm_release_range", "lpm_reset", "lpm_set_profiling",
                 "lpm_stats", "lpm_set_params", "lpm_set_emission", "lpm_receptors",
                 "lpm_adjoint", "lpm_draws_static", "lpm_set_sort", "lpm_save", "lpm_load",
                 "lpm_set_dosage", "lpm_dosage", "lpm_set_kz_model", "lpm_set_boundary_layer",
                 "lpm_set_decay_chain", "lpm_species", "lpm_set_langevin",
                 "lpm_particle_velocity", "lpm_set_adjoint_storage", "lpm_adjoint_storage",
                 "lpm_set_modes", "lpm_set_mode_phases", "lpm_device_state"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def _check(ctx, status: int):
    if status != LPM_OK:
        msg = load().lpm_last_error(ctx)
        raise LpmError(status, msg.decode() if msg else "")


def config_struct(cfg, max_particles: Optional[int] = None):
    """C record for an ``lpm_inputs.LpmConfig``; returns (struct, keep-alive arrays)."""
    z = np.ascontiguousarray(cfg.z_levels, dtype=np.float64)
    s = lpm_config()
    for name in ("nx", "ny", "nz", "n_met_t", "cx", "cy", "cz", "bin_every", "reflect_ground",
                 "reflect_top", "lateral_exit", "drift_correction", "n_scenarios"):
        setattr(s, name, int(getattr(cfg, name)))
    for name in ("x0", "y0", "dx", "dy", "met_t0", "met_dt", "cx0", "cy0", "cz0", "cdx", "cdy",
                 "cdz", "src_x", "src_y", "src_z", "dt", "half_life_s", "vd_dry", "h_mix",
                 "wet_lambda", "kh_uniform", "z_top"):
        setattr(s, name, float(getattr(cfg, name)))
    s.n_steps = int(cfg.n_steps)
    s.seed = int(cfg.seed)
    s.z_levels = _ptr(z, C.c_double)
    s.max_particles = int(max_particles if max_particles is not None else cfg.n_particles)
    return s, [z]


def lpm_create(cfg, stream=None, max_particles: Optional[int] = None) -> int:
    L = load()
    s, keep = config_struct(cfg, max_particles)
    out = C.c_void_p()
    st = L.lpm_create(C.byref(s), C.c_void_p(int(stream or 0)), C.byref(out))
    del keep
    _check(None, st)
    return out.value


def lpm_destroy(ctx) -> None:
    load().lpm_destroy(C.c_void_p(ctx))


def _addr(a):
    """Host numpy array -> (address, on_device=0); torch CUDA tensor -> (address, 1)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    return a.ctypes.data, 0


def lpm_set_met(ctx, t_index: int, uvwk, kh=None, rain=None) -> None:
    """uvwk [nz][ny][nx][4] float32, kh [nz][ny][nx] float32, rain [ny][nx] uint8: all numpy
    (host) or all torch CUDA tensors (device)."""
    if not hasattr(uvwk, "data_ptr"):
        uvwk = np.ascontiguousarray(uvwk, dtype=np.float32)
        kh = None if kh is None else np.ascontiguousarray(kh, dtype=np.float32)
        rain = None if rain is None else np.ascontiguousarray(rain, dtype=np.uint8)
    a, dev = _addr(uvwk)
    b, _ = _addr(kh)
    r, _ = _addr(rain)
    _check(ctx, load().lpm_set_met(C.c_void_p(ctx), int(t_index), a, b, r, dev))


def lpm_device_state(ctx, scenario: int = 0):
    """Device addresses of a scenario's fixed-point conc grid, deposition grid and first
    counter, and the counters' stride (elements)."""
    conc, dep, ctr = C.c_void_p(), C.c_void_p(), C.c_void_p()
    stride = C.c_int64()
    _check(ctx, load().lpm_device_state(C.c_void_p(ctx), int(scenario), C.byref(conc),
                                        C.byref(dep), C.byref(ctr), C.byref(stride)))
    return conc.value, dep.value, ctr.value, stride.value


MAX_MODES = 4


def lpm_set_modes(ctx, modes, profile) -> None:
    """Perturbation modes shared by the scenarios: ``modes`` [n][5] = (fx, fy, omega, eu,
    ev), ``profile`` [nz]; an empty ``modes`` turns them off."""
    m = np.ascontiguousarray(np.zeros((0, 5)) if modes is None else modes,
                             dtype=np.float64).reshape(-1, 5)
    prof = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)
    _check(ctx, load().lpm_set_modes(C.c_void_p(ctx), m.shape[0], _ptr(m, C.c_double),
                                     _ptr(prof, C.c_double)))


def lpm_set_mode_phases(ctx, scenario: int, phase, amp) -> None:
    """A scenario's phases (cycles) and amplitudes (m/s) of the modes."""
    ph = np.ascontiguousarray(phase, dtype=np.float64)
    am = np.ascontiguousarray(amp, dtype=np.float64)
    _check(ctx, load().lpm_set_mode_phases(C.c_void_p(ctx), int(scenario), _ptr(ph, C.c_double),
                                           _ptr(am, C.c_double)))


def lpm_set_source(ctx, scenario: int, x: float, y: float, z: float, wind_offset=None) -> None:
    wo = None if wind_offset is None else np.ascontiguousarray(wind_offset, dtype=np.float32)
    _check(ctx, load().lpm_set_source(C.c_void_p(ctx), int(scenario), float(x), float(y),
                                      float(z), None if wo is None else wo.ctypes.data))


def lpm_release(ctx, scenario: int, n_particles: int, q, q_dt: float, first_step: int,
                last_step: int) -> None:
    qa = np.ascontiguousarray(q, dtype=np.float64)
    _check(ctx, load().lpm_release(C.c_void_p(ctx), int(scenario), int(n_particles),
                                   _ptr(qa, C.c_double), int(qa.size), float(q_dt),
                                   int(first_step), int(last_step)))


def lpm_release_range(ctx, scenario: int, n_total: int, first_particle: int, count: int, q,
                      q_dt: float, first_step: int, last_step: int, id_base: int = 0) -> None:
    qa = np.ascontiguousarray(q, dtype=np.float64)
    _check(ctx, load().lpm_release_range(C.c_void_p(ctx), int(scenario), int(n_total),
                                         int(first_particle), int(count), _ptr(qa, C.c_double),
                                         int(qa.size), float(q_dt), int(first_step),
                                         int(last_step), int(id_base)))


def lpm_reset(ctx) -> None:
    _check(ctx, load().lpm_reset(C.c_void_p(ctx)))


def lpm_set_profiling(ctx, on: bool) -> None:
    _check(ctx, load().lpm_set_profiling(C.c_void_p(ctx), int(bool(on))))


def lpm_stats(ctx):
    """(kernels launched, advance launches, advance device ms) since the last call."""
    a, b, ms = C.c_int64(), C.c_int64(), C.c_double()
    _check(ctx, load().lpm_stats(C.c_void_p(ctx), C.byref(a), C.byref(b), C.byref(ms)))
    return int(a.value), int(b.value), float(ms.value)


def lpm_save(ctx) -> bytes:
    """The run state as bytes (step, particles in index order, grids, counters)."""
    n = C.c_size_t(0)
    _check(ctx, load().lpm_save(C.c_void_p(ctx), None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, load().lpm_save(C.c_void_p(ctx), C.cast(buf, C.c_void_p), C.byref(n)))
    return buf.raw[:n.value]


def lpm_load(ctx, state: bytes) -> None:
    buf = C.create_string_buffer(state, len(state))
    _check(ctx, load().lpm_load(C.c_void_p(ctx), C.cast(buf, C.c_void_p), len(state)))


def lpm_set_sort(ctx, every_steps: int) -> None:
    _check(ctx, load().lpm_set_sort(C.c_void_p(ctx), int(every_steps)))


def lpm_set_params(ctx, k_scale: float = 1.0, bias_u: float = 0.0, bias_v: float = 0.0) -> None:
    _check(ctx, load().lpm_set_params(C.c_void_p(ctx), float(k_scale), float(bias_u),
                                      float(bias_v)))


def lpm_set_emission(ctx, scenario: int, q) -> None:
    qa = np.ascontiguousarray(q, dtype=np.float64)
    _check(ctx, load().lpm_set_emission(C.c_void_p(ctx), int(scenario), _ptr(qa, C.c_double),
                                        int(qa.size)))


def lpm_receptors(ctx, n_scenarios: int, receptors, bandwidth: float, sample_every: int):
    """Receptor concentrations [n_scenarios][R]."""
    rec = np.ascontiguousarray(receptors, dtype=np.float64).reshape(-1, 3)
    out = np.empty((n_scenarios, rec.shape[0]), dtype=np.float64)
    _check(ctx, load().lpm_receptors(C.c_void_p(ctx), _ptr(rec, C.c_double), rec.shape[0],
                                     float(bandwidth), int(sample_every), _ptr(out, C.c_double)))
    return out


def lpm_adjoint(ctx, receptors, bandwidth: float, sample_every: int, dL_dC, n_q: int):
    """Gradient [n_scenarios][3 + n_q + 3] of sum(dL_dC * C)."""
    rec = np.ascontiguousarray(receptors, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(dL_dC, dtype=np.float64)
    w = w.reshape(-1, rec.shape[0])
    out = np.empty((w.shape[0], 3 + n_q + 3), dtype=np.float64)
    _check(ctx, load().lpm_adjoint(C.c_void_p(ctx), _ptr(rec, C.c_double), rec.shape[0],
                                   float(bandwidth), int(sample_every), _ptr(w, C.c_double),
                                   _ptr(out, C.c_double)))
    return out


def lpm_set_adjoint_storage(ctx, max_bytes: int) -> None:
    """Largest trajectory the receptor forward may keep for the adjoint (0: checkpoints)."""
    _check(ctx, load().lpm_set_adjoint_storage(C.c_void_p(ctx), int(max_bytes)))


def lpm_adjoint_storage(ctx):
    """(kept the trajectory, device bytes held for the adjoint's states)."""
    t, b = C.c_int(), C.c_uint64()
    _check(ctx, load().lpm_adjoint_storage(C.c_void_p(ctx), C.byref(t), C.byref(b)))
    return bool(t.value), int(b.value)


def lpm_step(ctx, n: int) -> None:
    _check(ctx, load().lpm_step(C.c_void_p(ctx), int(n)))


def lpm_current_step(ctx) -> int:
    k = C.c_int64()
    _check(ctx, load().lpm_current_step(C.c_void_p(ctx), C.byref(k)))
    return int(k.value)


def lpm_concentration(ctx, scenario: int, shape, out=None) -> np.ndarray:
    """Concentration [cz][cy][cx]; ``out`` (a C-contiguous float64 array of that shape,
    e.g. over page-locked memory) receives it instead of a new array."""
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
        raise ValueError("out must be a C-contiguous float64 array of the grid's size")
    _check(ctx, load().lpm_concentration(C.c_void_p(ctx), int(scenario), _ptr(out, C.c_double),
                                         out.size))
    return out


def lpm_deposition(ctx, scenario: int, shape):
    dry = np.empty(shape, dtype=np.float64)
    wet = np.empty(shape, dtype=np.float64)
    _check(ctx, load().lpm_deposition(C.c_void_p(ctx), int(scenario), _ptr(dry, C.c_double),
                                      _ptr(wet, C.c_double), dry.size))
    return dry, wet


def lpm_budget(ctx, scenario: int = 0) -> np.ndarray:
    out = np.empty(8, dtype=np.float64)
    _check(ctx, load().lpm_budget(C.c_void_p(ctx), int(scenario), _ptr(out, C.c_double)))
    return out


def lpm_particles(ctx, first: int, count: int):
    xyz = np.empty((count, 3), dtype=np.float32)
    tag = np.empty(count, dtype=np.uint32)
    _check(ctx, load().lpm_particles(C.c_void_p(ctx), int(first), int(count),
                                     _ptr(xyz, C.c_float), _ptr(tag, C.c_uint32)))
    return xyz, tag


def lpm_fixed_state(ctx, scenario: int, conc_shape, dep_shape):
    conc = np.empty(conc_shape, dtype=np.uint64)
    dep = np.empty(dep_shape, dtype=np.uint64)
    ctr = np.empty(16, dtype=np.int64)
    sh = C.c_int()
    _check(ctx, load().lpm_fixed_state(C.c_void_p(ctx), int(scenario), _ptr(conc, C.c_uint64),
                                       conc.size, _ptr(dep, C.c_uint64), dep.size,
                                       _ptr(ctr, C.c_int64), C.byref(sh)))
    return conc, dep, ctr, int(sh.value)


def lpm_set_langevin(ctx, on: bool, t_lagr: float = 100.0) -> None:
    _check(ctx, load().lpm_set_langevin(C.c_void_p(ctx), int(bool(on)), float(t_lagr)))


def lpm_particle_velocity(ctx, first: int, count: int) -> np.ndarray:
    """Turbulent vertical velocity w' (m/s) of slots [first, first + count)."""
    w = np.empty(int(count), dtype=np.float32)
    _check(ctx, load().lpm_particle_velocity(C.c_void_p(ctx), int(first), int(count),
                                             _ptr(w, C.c_float)))
    return w


def lpm_set_decay_chain(ctx, half_lives) -> None:
    hl = np.ascontiguousarray(half_lives, dtype=np.float64)
    _check(ctx, load().lpm_set_decay_chain(C.c_void_p(ctx), int(hl.size), _ptr(hl, C.c_double)))


def lpm_species(ctx, scenario: int, species: int, conc_shape, dep_shape):
    """(conc, dry, wet, conc_fixed, dep_fixed) of one species of the decay chain."""
    conc = np.empty(conc_shape, dtype=np.float64)
    dry = np.empty(dep_shape, dtype=np.float64)
    wet = np.empty(dep_shape, dtype=np.float64)
    cf = np.empty(conc_shape, dtype=np.uint64)
    df = np.empty((2,) + tuple(dep_shape), dtype=np.uint64)
    _check(ctx, load().lpm_species(C.c_void_p(ctx), int(scenario), int(species),
                                   _ptr(conc, C.c_double), _ptr(dry, C.c_double),
                                   _ptr(wet, C.c_double), _ptr(cf, C.c_uint64),
                                   _ptr(df, C.c_uint64)))
    return conc, dry, wet, cf, df


def lpm_set_kz_model(ctx, model: int, kz_min: float = 0.1) -> None:
    _check(ctx, load().lpm_set_kz_model(C.c_void_p(ctx), int(model), float(kz_min)))


def lpm_set_boundary_layer(ctx, t_index: int, bl) -> None:
    """Hour t_index of the (u*, 1/L, H_z, unused) columns, [ny][nx][4] float32 (numpy
    array or CUDA tensor)."""
    if not hasattr(bl, "data_ptr"):
        bl = np.ascontiguousarray(bl, dtype=np.float32)
    a, dev = _addr(bl)
    _check(ctx, load().lpm_set_boundary_layer(C.c_void_p(ctx), int(t_index), a, dev))


def lpm_set_dosage(ctx, every_steps: int) -> None:
    _check(ctx, load().lpm_set_dosage(C.c_void_p(ctx), int(every_steps)))


def lpm_dosage(ctx, scenario: int, shape):
    """(dosage [mass s / m^3], raw fixed-point sums, number of samples) of a scenario."""
    out = np.empty(shape, dtype=np.float64)
    fixed = np.empty(shape, dtype=np.uint64)
    n = C.c_int64()
    _check(ctx, load().lpm_dosage(C.c_void_p(ctx), int(scenario), _ptr(out, C.c_double), out.size,
                                  _ptr(fixed, C.c_uint64), C.byref(n)))
    return out, fixed, int(n.value)


def lpm_set_launch(ctx, block: int, particles_per_thread: int, occupancy: int = 1) -> None:
    _check(ctx, load().lpm_set_launch(C.c_void_p(ctx), int(block), int(particles_per_thread),
                                      int(occupancy)))


def lpm_sync(ctx) -> None:
    _check(ctx, load().lpm_sync(C.c_void_p(ctx)))


def lpm_draws(seed: int, pid, step, stream: int = 0):
    """Philox words [n][4] (uint32) and the step's normals [n][3] (float32)."""
    pid = np.ascontiguousarray(pid, dtype=np.uint64)
    step = np.ascontiguousarray(np.broadcast_to(step, pid.shape), dtype=np.uint32)
    words = np.empty((pid.size, 4), dtype=np.uint32)
    nrm = np.empty((pid.size, 3), dtype=np.float32)
    _check(None, load().lpm_draws(int(seed), _ptr(pid, C.c_uint64), _ptr(step, C.c_uint32),
                                  int(stream), pid.size, _ptr(words, C.c_uint32),
                                  _ptr(nrm, C.c_float)))
    return words, nrm


DRAWS_STATIC_MAX = 65536


def lpm_draws_static(seed: int, pid, step, stream: int = 0):
    """As ``lpm_draws``, without device allocation (staged through the library's fixed
    device array; at most DRAWS_STATIC_MAX draws per call)."""
    pid = np.ascontiguousarray(pid, dtype=np.uint64)
    step = np.ascontiguousarray(np.broadcast_to(step, pid.shape), dtype=np.uint32)
    words = np.empty((pid.size, 4), dtype=np.uint32)
    nrm = np.empty((pid.size, 3), dtype=np.float32)
    _check(None, load().lpm_draws_static(int(seed), _ptr(pid, C.c_uint64), _ptr(step, C.c_uint32),
                                         int(stream), pid.size, _ptr(words, C.c_uint32),
                                         _ptr(nrm, C.c_float)))
    return words, nrm


# ------------------------------------------------------------------------------------
# Convenience wrapper
# ------------------------------------------------------------------------------------
class Sim:
    """One context set up from an ``lpm_inputs.LpmConfig``: met uploaded, sources set,
    releases declared. ``stream`` is a torch.cuda.Stream (default: current stream).
    ``part = (first, count)`` holds that particle range of a single release, and
    ``id_base`` sets the global id (generator counter) of its particle 0;
    ``scenarios = (first, count)`` holds that range of an ensemble's scenarios (local
    scenario i is ensemble scenario first + i) with the ensemble's global particle ids, so
    each held scenario draws the same random numbers as in the whole ensemble."""

    def __init__(self, cfg, stream=None, met_on_device: bool = False, launch=None,
                 part=None, sort_every: Optional[int] = None, scenarios=None,
                 id_base: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the particle model runs on a CUDA GPU; none is available")
        self.id_base = None
        if id_base and cfg.scenarios:
            raise ValueError("id_base applies to a single release; an ensemble's scenarios "
                             "take their ids from their order")
        if scenarios is not None:
            import dataclasses
            if not cfg.scenarios or part is not None:
                raise ValueError("a scenario range needs an ensemble and no particle range")
            first, count = (int(v) for v in scenarios)
            if first < 0 or count < 1 or first + count > len(cfg.scenarios):
                raise ValueError(f"scenario range ({first}, {count}) outside the "
                                 f"{len(cfg.scenarios)} scenarios")
            ids = [0]
            for sc in cfg.scenarios:
                ids.append(ids[-1] + int(sc.release.n_particles))
            self.id_base = ids[first:first + count]
            cfg = dataclasses.replace(cfg, n_scenarios=count,
                                      scenarios=list(cfg.scenarios[first:first + count]))
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.part = part
        n_slots = part[1] if part is not None else None
        self.ctx = lpm_create(cfg, self.stream.cuda_stream, max_particles=n_slots)
        try:
            if launch is not None:
                lpm_set_launch(self.ctx, *launch)
            if sort_every is not None:
                lpm_set_sort(self.ctx, sort_every)
            self._set_met(met_on_device)
            if getattr(cfg, "langevin", 0):
                lpm_set_langevin(self.ctx, True, cfg.t_lagr)
            if getattr(cfg, "chain_half_lives", None) is not None:
                lpm_set_decay_chain(self.ctx, cfg.chain_half_lives)
            if getattr(cfg, "kz_model", 0):
                lpm_set_kz_model(self.ctx, cfg.kz_model, cfg.kz_min)
                for t in range(cfg.n_met_t):
                    lpm_set_boundary_layer(self.ctx, t, cfg.bl[t])
            modes = getattr(cfg, "modes", None)
            if modes is not None and len(modes):
                lpm_set_modes(self.ctx, modes, cfg.mode_profile)
                for i, sc in enumerate(cfg.scenarios or [cfg]):
                    if getattr(sc, "mode_phase", None) is not None:
                        lpm_set_mode_phases(self.ctx, i, sc.mode_phase, sc.mode_amp)
            if cfg.scenarios:
                for i, sc in enumerate(cfg.scenarios):
                    lpm_set_source(self.ctx, i, sc.src_x, sc.src_y, sc.src_z, sc.wind_offset)
                for i, sc in enumerate(cfg.scenarios):
                    r = sc.release
                    if self.id_base is None:
                        lpm_release(self.ctx, i, r.n_particles, r.q, r.q_dt, r.first_step,
                                    r.last_step)
                    else:
                        lpm_release_range(self.ctx, i, r.n_particles, 0, r.n_particles, r.q,
                                          r.q_dt, r.first_step, r.last_step, self.id_base[i])
            elif part is not None or id_base:
                r = cfg.release
                first, count = part if part is not None else (0, r.n_particles)
                lpm_release_range(self.ctx, 0, r.n_particles, first, count, r.q, r.q_dt,
                                  r.first_step, r.last_step, int(id_base))
            else:
                r = cfg.release
                lpm_release(self.ctx, 0, r.n_particles, r.q, r.q_dt, r.first_step, r.last_step)
        except Exception:
            lpm_destroy(self.ctx)
            self.ctx = None
            raise

    def _set_met(self, on_device: bool):
        cfg = self.cfg
        if on_device:
            import torch
            dev = torch.device("cuda", torch.cuda.current_device())
            uvwk = torch.from_numpy(np.ascontiguousarray(cfg.uvwk)).to(dev)
            kh = None if cfg.kh is None else torch.from_numpy(np.ascontiguousarray(cfg.kh)).to(dev)
            rain = None if cfg.rain is None else torch.from_numpy(
                np.ascontiguousarray(cfg.rain)).to(dev)
            self._met_keep = (uvwk, kh, rain)
            for t in range(cfg.n_met_t):
                lpm_set_met(self.ctx, t, uvwk[t], None if kh is None else kh[t],
                            None if rain is None else rain[t])
        else:
            for t in range(cfg.n_met_t):
                lpm_set_met(self.ctx, t, cfg.uvwk[t], None if cfg.kh is None else cfg.kh[t],
                            None if cfg.rain is None else cfg.rain[t])

    def step(self, n: int):
        lpm_step(self.ctx, n)
        return self

    def reset(self):
        lpm_reset(self.ctx)
        return self

    @property
    def k(self) -> int:
        return lpm_current_step(self.ctx)

    def concentration(self, scenario: int = 0, out=None) -> np.ndarray:
        c = self.cfg
        return lpm_concentration(self.ctx, scenario, (c.cz, c.cy, c.cx), out=out)

    def deposition(self, scenario: int = 0):
        c = self.cfg
        return lpm_deposition(self.ctx, scenario, (c.cy, c.cx))

    def budget(self, scenario: int = 0) -> np.ndarray:
        return lpm_budget(self.ctx, scenario)

    def particles(self, first: int = 0, count: Optional[int] = None):
        if count is None:
            held = self.part[1] if self.part is not None else self.cfg.n_particles
            count = held - first
        return lpm_particles(self.ctx, first, count)

    def fixed_state(self, scenario: int = 0):
        c = self.cfg
        return lpm_fixed_state(self.ctx, scenario, (c.cz, c.cy, c.cx), (2, c.cy, c.cx))

    def velocity(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        """Langevin w' of the held particles."""
        if count is None:
            held = self.part[1] if self.part is not None else self.cfg.n_particles
            count = held - first
        return lpm_particle_velocity(self.ctx, first, count)

    def species(self, species: int, scenario: int = 0):
        """(conc, dry, wet, conc_fixed, dep_fixed) of a decay-chain species."""
        c = self.cfg
        return lpm_species(self.ctx, scenario, species, (c.cz, c.cy, c.cx), (c.cy, c.cx))

    def set_dosage(self, every_steps: int):
        lpm_set_dosage(self.ctx, every_steps)
        return self

    def dosage(self, scenario: int = 0):
        """(dosage [mass s / m^3], fixed-point sums, samples) of a scenario."""
        c = self.cfg
        return lpm_dosage(self.ctx, scenario, (c.cz, c.cy, c.cx))

    def sync(self):
        lpm_sync(self.ctx)

    def close(self):
        if self.ctx:
            lpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
