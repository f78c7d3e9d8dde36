"""FP64 CPU oracle of the stochastic Lagrangian particle model (test infrastructure).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may import this
package. The product library never imports, links or executes anything here, and this
package imports nothing from the product library: the two share only the seeded input
generators of ``lpm_inputs``.

The arithmetic lives in ``lpm_oracle.c`` (plain C, double precision, plain loops); this
module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OCfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("z_levels", C.POINTER(C.c_double)),
        ("n_met_t", C.c_int), ("met_t0", C.c_double), ("met_dt", C.c_double),
        ("uvwk", C.POINTER(C.c_float)), ("kh", C.POINTER(C.c_float)),
        ("rain", C.POINTER(C.c_uint8)), ("wind_offset", C.POINTER(C.c_float)),
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
        ("n_particles", C.c_int64), ("q", C.POINTER(C.c_double)), ("n_q", C.c_int),
        ("q_dt", C.c_double), ("first_step", C.c_int64), ("last_step", C.c_int64),
        ("pid_offset", C.c_int64),
        ("k_scale", C.c_double), ("bias_u", C.c_double), ("bias_v", C.c_double),
        ("dose_every", C.c_int),
        ("kz_model", C.c_int), ("kz_min", C.c_double), ("bl", C.POINTER(C.c_float)),
        ("n_species", C.c_int), ("chain_half_life", C.POINTER(C.c_double)),
        ("langevin", C.c_int), ("t_lagr", C.c_double),
        ("n_modes", C.c_int), ("modes", C.POINTER(C.c_double)),
        ("mode_profile", C.POINTER(C.c_double)), ("mode_phase", C.POINTER(C.c_double)),
        ("mode_amp", C.POINTER(C.c_double)),
    ]


class OOut(C.Structure):
    _fields_ = [
        ("pos", C.POINTER(C.c_double)), ("status", C.POINTER(C.c_int32)),
        ("release", C.POINTER(C.c_int64)), ("margin", C.POINTER(C.c_double)),
        ("conc", C.POINTER(C.c_double)), ("conc_fixed", C.POINTER(C.c_int64)),
        ("dep", C.POINTER(C.c_double)), ("dep_fixed", C.POINTER(C.c_int64)),
        ("budget", C.POINTER(C.c_double)), ("counters", C.POINTER(C.c_int64)),
        ("dose", C.POINTER(C.c_double)), ("dose_fixed", C.POINTER(C.c_int64)),
        ("dose_ctr", C.POINTER(C.c_int64)),
        ("sp_conc", C.POINTER(C.c_double)), ("sp_conc_fixed", C.POINTER(C.c_int64)),
        ("sp_dep", C.POINTER(C.c_double)), ("sp_dep_fixed", C.POINTER(C.c_int64)),
        ("wvel", C.POINTER(C.c_double)),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = configure(C.CDLL(_LIB))
    return _lib


def configure(L):
    """Declares the argument and result types of the oracle's exported functions on a
    loaded copy of the library."""
    u64p = C.POINTER(C.c_uint64)
    u32p = C.POINTER(C.c_uint32)
    L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.oracle_draw_many.argtypes = [C.c_uint64, u64p, u32p, C.c_uint32, C.c_int64, u32p]
    L.oracle_normals_many.argtypes = [C.c_uint64, u64p, u32p, C.c_int64,
                                      C.POINTER(C.c_double)]
    L.oracle_uniform.argtypes = [C.c_uint32]
    L.oracle_uniform.restype = C.c_double
    L.oracle_interp_many.argtypes = [C.POINTER(OCfg), C.POINTER(C.c_double), C.c_int64,
                                     C.POINTER(C.c_double)]
    L.oracle_release_many.argtypes = [C.c_int64, C.c_int64, C.c_int64,
                                      C.POINTER(C.c_int64), C.c_int64,
                                      C.POINTER(C.c_int64)]
    L.oracle_release_count.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64]
    L.oracle_release_count.restype = C.c_int64
    L.oracle_total_mass.argtypes = [C.POINTER(OCfg)]
    L.oracle_total_mass.restype = C.c_double
    L.oracle_fixed_shift.argtypes = [C.c_double]
    L.oracle_fixed_shift.restype = C.c_int
    L.oracle_initial_mass.argtypes = [C.POINTER(OCfg), C.c_int64]
    L.oracle_initial_mass.restype = C.c_double
    L.oracle_kz_eq3.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)]
    L.oracle_kz_eq3_partials.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)]
    L.oracle_interp_grad_many.argtypes = [C.POINTER(OCfg), C.POINTER(C.c_double), C.c_int64,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.oracle_chain_amount.argtypes = [C.POINTER(OCfg), C.c_int, C.c_double]
    L.oracle_chain_amount.restype = C.c_double
    L.oracle_threshold.argtypes = [C.c_double]
    L.oracle_threshold.restype = C.c_uint32
    L.oracle_run.argtypes = [C.POINTER(OCfg), C.POINTER(C.c_int64), C.c_int64, C.c_int64,
                             C.POINTER(OOut)]
    L.oracle_run.restype = C.c_int
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    L.oracle_receptors.argtypes = [C.POINTER(OCfg), dp, C.c_int, C.c_double, C.c_int, i64p,
                                   C.c_int64, C.c_int64, dp]
    L.oracle_adjoint.argtypes = [C.POINTER(OCfg), dp, C.c_int, C.c_double, C.c_int, dp, i64p,
                                 C.c_int64, C.c_int64, dp]
    L.oracle_sensitivity.argtypes = [C.POINTER(OCfg), i64p, C.c_int64, C.c_int64, dp]
    for f in (L.oracle_receptors, L.oracle_adjoint, L.oracle_sensitivity):
        f.restype = C.c_int
    return L


def _ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return C.POINTER(ct)()
    return a.ctypes.data_as(C.POINTER(ct))


class _Pinned:
    """Keeps the numpy arrays referenced by an OCfg alive."""

    def __init__(self):
        self.keep = []

    def arr(self, a, dtype):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        self.keep.append(a)
        return a


def make_ocfg(cfg, scenario: Optional[int] = None, k_scale: float = 1.0,
              bias=(0.0, 0.0), src=None, q=None, dose_every: int = 0,
              id_offset: Optional[int] = None):
    """Build the C record for one release of ``cfg`` (an ``lpm_inputs.LpmConfig``).
    ``scenario`` selects a member of a batched ensemble (its source, release, global id
    offset and wind offset). ``src``/``q`` override the source and emission series;
    ``dose_every`` > 0 samples the time-integrated dosage every that many steps;
    ``id_offset`` sets the global id (generator counter) of the release's particle 0."""
    pin = _Pinned()
    o = OCfg()
    for name in ("nx", "ny", "nz", "n_met_t", "cx", "cy", "cz", "bin_every",
                 "reflect_ground", "reflect_top", "lateral_exit", "drift_correction"):
        setattr(o, name, int(getattr(cfg, name)))
    for name in ("x0", "y0", "dx", "dy", "met_t0", "met_dt", "cx0", "cy0", "cz0", "cdx",
                 "cdy", "cdz", "src_x", "src_y", "src_z", "dt", "half_life_s", "vd_dry",
                 "h_mix", "wet_lambda", "kh_uniform", "z_top"):
        setattr(o, name, float(getattr(cfg, name)))
    o.n_steps = int(cfg.n_steps)
    o.seed = int(cfg.seed)
    o.z_levels = _ptr(pin.arr(cfg.z_levels, np.float64), C.c_double)
    o.uvwk = _ptr(pin.arr(cfg.uvwk, np.float32), C.c_float)
    o.kh = _ptr(pin.arr(cfg.kh, np.float32), C.c_float)
    o.rain = _ptr(pin.arr(cfg.rain, np.uint8), C.c_uint8)
    rel = cfg.release
    offset = 0
    wind_offset = None
    if scenario is not None:
        sc = cfg.scenarios[scenario]
        rel = sc.release
        offset = int(sum(s.release.n_particles for s in cfg.scenarios[:scenario]))
        o.src_x, o.src_y, o.src_z = sc.src_x, sc.src_y, sc.src_z
        wind_offset = sc.wind_offset
    if src is not None:
        o.src_x, o.src_y, o.src_z = (float(v) for v in src)
    o.wind_offset = _ptr(pin.arr(wind_offset, np.float32), C.c_float)
    # perturbation modes: the ensemble's waves and profile, the scenario's phases and
    # amplitudes (a plain configuration may carry them as scenario 0's)
    modes = getattr(cfg, "modes", None)
    o.n_modes = 0
    if modes is not None and len(modes):
        sc_modes = cfg.scenarios[scenario] if scenario is not None else cfg
        phase = getattr(sc_modes, "mode_phase", None)
        amp = getattr(sc_modes, "mode_amp", None)
        if phase is not None and amp is not None:
            o.n_modes = int(len(modes))
            o.modes = _ptr(pin.arr(modes, np.float64), C.c_double)
            o.mode_profile = _ptr(pin.arr(cfg.mode_profile, np.float64), C.c_double)
            o.mode_phase = _ptr(pin.arr(phase, np.float64), C.c_double)
            o.mode_amp = _ptr(pin.arr(amp, np.float64), C.c_double)
    qa = pin.arr(rel.q if q is None else q, np.float64)
    o.n_particles = int(rel.n_particles)
    o.q = _ptr(qa, C.c_double)
    o.n_q = int(qa.size)
    o.q_dt = float(rel.q_dt)
    o.first_step = int(rel.first_step)
    o.last_step = int(rel.last_step)
    o.pid_offset = offset if id_offset is None else int(id_offset)
    o.k_scale = float(k_scale)
    o.bias_u, o.bias_v = float(bias[0]), float(bias[1])
    o.dose_every = int(dose_every)
    o.kz_model = int(getattr(cfg, "kz_model", 0))
    o.kz_min = float(getattr(cfg, "kz_min", 0.1))
    o.bl = _ptr(pin.arr(getattr(cfg, "bl", None), np.float32), C.c_float)
    chain = getattr(cfg, "chain_half_lives", None)
    o.n_species = 0 if chain is None else len(chain)
    o.chain_half_life = _ptr(pin.arr(chain, np.float64), C.c_double)
    o.langevin = int(getattr(cfg, "langevin", 0))
    o.t_lagr = float(getattr(cfg, "t_lagr", 0.0))
    o._pin = pin  # keep arrays alive with the record
    return o


# ------------------------------------------------------------------------------------
# Thin wrappers
# ------------------------------------------------------------------------------------
def philox(key, ctr):
    L = lib()
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    o = (C.c_uint32 * 4)()
    L.oracle_philox4x32_10(k, c, o)
    return [int(v) for v in o]


def draws(seed: int, pid, step, stream: int = 0) -> np.ndarray:
    pid = np.ascontiguousarray(pid, dtype=np.uint64)
    step = np.ascontiguousarray(np.broadcast_to(step, pid.shape), dtype=np.uint32)
    out = np.empty((pid.size, 4), dtype=np.uint32)
    lib().oracle_draw_many(seed, _ptr(pid, C.c_uint64), _ptr(step, C.c_uint32), stream,
                           pid.size, _ptr(out, C.c_uint32))
    return out


def normals(seed: int, pid, step) -> np.ndarray:
    pid = np.ascontiguousarray(pid, dtype=np.uint64)
    step = np.ascontiguousarray(np.broadcast_to(step, pid.shape), dtype=np.uint32)
    out = np.empty((pid.size, 3), dtype=np.float64)
    lib().oracle_normals_many(seed, _ptr(pid, C.c_uint64), _ptr(step, C.c_uint32), pid.size,
                              _ptr(out, C.c_double))
    return out


def uniform(w: int) -> float:
    return lib().oracle_uniform(int(w) & 0xFFFFFFFF)


def interp(cfg, xyzt, **kw) -> np.ndarray:
    """Weather at points [N][4] = (x, y, z, t) -> [N][6] = (u, v, w, K_z, K_h, dK_z/dz)."""
    o = make_ocfg(cfg, **kw)
    pts = np.ascontiguousarray(xyzt, dtype=np.float64).reshape(-1, 4)
    out = np.empty((pts.shape[0], 6), dtype=np.float64)
    lib().oracle_interp_many(C.byref(o), _ptr(pts, C.c_double), pts.shape[0],
                             _ptr(out, C.c_double))
    return out


def interp_grad(cfg, xyzt, **kw):
    """(values [N][5] = (u, v, w, K_z, K_h), gradients [N][5][3] in x, y, z) of the
    interpolated weather, as the tangent-linear model uses them."""
    o = make_ocfg(cfg, **kw)
    pts = np.ascontiguousarray(xyzt, dtype=np.float64).reshape(-1, 4)
    val = np.empty((pts.shape[0], 5))
    grad = np.empty((pts.shape[0], 5, 3))
    lib().oracle_interp_grad_many(C.byref(o), _ptr(pts, C.c_double), pts.shape[0],
                                  _ptr(val, C.c_double), _ptr(grad, C.c_double))
    return val, grad


def release_steps(n: int, first: int, last: int, p) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.int64)
    out = np.empty_like(p)
    lib().oracle_release_many(n, first, last, _ptr(p, C.c_int64), p.size, _ptr(out, C.c_int64))
    return out


def release_count(n: int, first: int, last: int, step: int) -> int:
    return int(lib().oracle_release_count(n, first, last, step))


def kz_eq3(ustar: float, inv_l: float, hz: float, kz_min: float, z: float):
    """(K_z, dK_z/dz) of Eq. 3 at height z."""
    out = (C.c_double * 2)()
    lib().oracle_kz_eq3(float(ustar), float(inv_l), float(hz), float(kz_min), float(z), out)
    return float(out[0]), float(out[1])


def kz_eq3_partials(ustar: float, inv_l: float, hz: float, kz_min: float, z: float):
    """(K_z, dK/dz, dK/du*, dK/d(1/L), dK/dH_z, d2K/dz2) of Eq. 3 at height z."""
    out = (C.c_double * 6)()
    lib().oracle_kz_eq3_partials(float(ustar), float(inv_l), float(hz), float(kz_min), float(z),
                                 out)
    return tuple(float(v) for v in out)


def chain_amount(cfg, species: int, age: float) -> float:
    """Amount of ``species`` per unit of emitted parent after ``age`` seconds."""
    o = make_ocfg(cfg)
    return float(lib().oracle_chain_amount(C.byref(o), int(species), float(age)))


def threshold(p: float) -> int:
    return int(lib().oracle_threshold(float(p)))


def fixed_shift(cfg, **kw) -> int:
    o = make_ocfg(cfg, **kw)
    return int(lib().oracle_fixed_shift(lib().oracle_total_mass(C.byref(o))))


def total_mass(cfg, **kw) -> float:
    o = make_ocfg(cfg, **kw)
    return float(lib().oracle_total_mass(C.byref(o)))


def run(cfg, sel=None, n_run: Optional[int] = None, **kw) -> dict:
    """Run the oracle for steps [0, n_run) on the particles ``sel`` (local indices of the
    release; None = all). Returns positions, status, release steps, decision margins,
    the last concentration snapshot (FP64 and fixed point), the deposition grids, the
    budget and the fixed-point counters; with ``dose_every`` the dosage sums (dose,
    dose_fixed: summed mass per cell over the samples; dose_out: fixed-point mass outside
    the grid; dose_samples)."""
    o = make_ocfg(cfg, **kw)
    if n_run is None:
        n_run = int(cfg.n_steps)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        n = sel.size
    else:
        n = int(o.n_particles)
    ncell = cfg.cx * cfg.cy * cfg.cz
    out = dict(
        pos=np.zeros((n, 3)), status=np.zeros(n, np.int32), release=np.zeros(n, np.int64),
        margin=np.zeros(n), conc=np.zeros((cfg.cz, cfg.cy, cfg.cx)),
        conc_fixed=np.zeros((cfg.cz, cfg.cy, cfg.cx), np.int64),
        dep=np.zeros((2, cfg.cy, cfg.cx)), dep_fixed=np.zeros((2, cfg.cy, cfg.cx), np.int64),
        budget=np.zeros(8), counters=np.zeros(6, np.int64), wvel=np.zeros(n),
        dose=np.zeros((cfg.cz, cfg.cy, cfg.cx)),
        dose_fixed=np.zeros((cfg.cz, cfg.cy, cfg.cx), np.int64), dose_ctr=np.zeros(2, np.int64))
    n_sp = int(o.n_species)
    if n_sp > 1:
        out.update(sp_conc=np.zeros((n_sp, cfg.cz, cfg.cy, cfg.cx)),
                   sp_conc_fixed=np.zeros((n_sp, cfg.cz, cfg.cy, cfg.cx), np.int64),
                   sp_dep=np.zeros((n_sp, 2, cfg.cy, cfg.cx)),
                   sp_dep_fixed=np.zeros((n_sp, 2, cfg.cy, cfg.cx), np.int64))
    oo = OOut(_ptr(out["pos"], C.c_double), _ptr(out["status"], C.c_int32),
              _ptr(out["release"], C.c_int64), _ptr(out["margin"], C.c_double),
              _ptr(out["conc"], C.c_double), _ptr(out["conc_fixed"], C.c_int64),
              _ptr(out["dep"], C.c_double), _ptr(out["dep_fixed"], C.c_int64),
              _ptr(out["budget"], C.c_double), _ptr(out["counters"], C.c_int64),
              _ptr(out["dose"], C.c_double), _ptr(out["dose_fixed"], C.c_int64),
              _ptr(out["dose_ctr"], C.c_int64),
              _ptr(out.get("sp_conc"), C.c_double), _ptr(out.get("sp_conc_fixed"), C.c_int64),
              _ptr(out.get("sp_dep"), C.c_double), _ptr(out.get("sp_dep_fixed"), C.c_int64),
              _ptr(out["wvel"], C.c_double))
    assert ncell == out["conc"].size
    rc = lib().oracle_run(C.byref(o), _ptr(sel, C.c_int64), n, int(n_run), C.byref(oo))
    if rc != 0:
        raise ValueError(f"oracle_run rejected the configuration (code {rc})")
    out["active_steps"] = int(out["counters"][4])
    out["dose_out"] = int(out["dose_ctr"][0])
    out["dose_samples"] = int(out["dose_ctr"][1])
    return out


def receptors(cfg, rec, sigma: float, every: int, sel=None, n_run: Optional[int] = None,
              **kw) -> np.ndarray:
    """Receptor concentrations C[R] (Gaussian kernel of width sigma with the ground image,
    averaged over the sample steps (k+1) % every == 0)."""
    o = make_ocfg(cfg, **kw)
    rec = np.ascontiguousarray(rec, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(rec.shape[0])
    n_run = cfg.n_steps if n_run is None else n_run
    sel_a = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    rc = lib().oracle_receptors(C.byref(o), _ptr(rec, C.c_double), rec.shape[0], float(sigma),
                                int(every), _ptr(sel_a, C.c_int64),
                                0 if sel_a is None else sel_a.size, int(n_run),
                                _ptr(out, C.c_double))
    if rc:
        raise ValueError(f"oracle_receptors failed ({rc})")
    return out


def adjoint(cfg, rec, sigma: float, every: int, w, sel=None, n_run: Optional[int] = None,
            **kw) -> np.ndarray:
    """Gradient of sum_r w_r C_r with respect to (x_s, y_s, h, q[0..n_q-1], s_K, b_u, b_v)."""
    o = make_ocfg(cfg, **kw)
    rec = np.ascontiguousarray(rec, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(3 + int(o.n_q) + 3)
    n_run = cfg.n_steps if n_run is None else n_run
    sel_a = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    rc = lib().oracle_adjoint(C.byref(o), _ptr(rec, C.c_double), rec.shape[0], float(sigma),
                              int(every), _ptr(w, C.c_double), _ptr(sel_a, C.c_int64),
                              0 if sel_a is None else sel_a.size, int(n_run),
                              _ptr(out, C.c_double))
    if rc:
        raise ValueError(f"oracle_adjoint failed ({rc})")
    return out


SENS_FIELDS = 6


def sensitivity(cfg, sel=None, n_run: Optional[int] = None, **kw) -> np.ndarray:
    """Per particle [n][6]: the largest norms of d X_end / d (x_k, y_k) and of
    d X_end / d z_k over its steps k (finite-time perturbation growth), the sums over k of
    their squares, and the sums over k of the squared growth from X_{k+1} times the square
    of step k's horizontal and vertical displacement scale."""
    o = make_ocfg(cfg, **kw)
    n_run = cfg.n_steps if n_run is None else n_run
    sel_a = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    n = int(o.n_particles) if sel_a is None else sel_a.size
    out = np.zeros((n, SENS_FIELDS))
    rc = lib().oracle_sensitivity(C.byref(o), _ptr(sel_a, C.c_int64), 0 if sel_a is None else n,
                                  int(n_run), _ptr(out, C.c_double))
    if rc:
        raise ValueError(f"oracle_sensitivity failed ({rc})")
    return out


# Relative error of a displacement computed in FP32: about four roundings of 2^-24 (the
# interpolated wind, the normal and the diffusion scale each carry about one). Against GPU
# paths of the realistic workload (770 000 particles after 360 steps) the largest distance
# was 2.0 times this bound, where the position rounding alone gave 14.5 times.
DISP_REL_ERR = 2.0 ** -22


def growth_bound(sens: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """The expected distance between a path run in FP32 and the same path in FP64: per
    step, one rounding of the state (2^-24 of its magnitude) and the error of the computed
    displacement (DISP_REL_ERR of its scale), each grown to the end of the run by that
    step's growth factor, adding up as a random walk. Needs ``sensitivity``."""
    eps = 2.0 ** -24
    rh = np.maximum(np.abs(pos[:, 0]), np.abs(pos[:, 1]))
    rz = np.maximum(pos[:, 2], 1.0)
    state = eps ** 2 * (sens[:, 2] * rh ** 2 + sens[:, 3] * rz ** 2)
    disp = DISP_REL_ERR ** 2 * (sens[:, 4] + sens[:, 5]) if sens.shape[1] > 4 else 0.0
    return np.sqrt(state + disp)


def chaotic(cfg, sens: np.ndarray, pos: np.ndarray, pos_tol: float) -> np.ndarray:
    """Paths whose expected FP32-vs-FP64 distance (``growth_bound``) exceeds the position
    tolerance: their two realisations are not expected to stay within it."""
    return growth_bound(sens, pos) > pos_tol
