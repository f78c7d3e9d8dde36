"""Seeded synthetic inputs for the Lagrangian particle model.

This module builds the inputs that both the CUDA path and the FP64 oracle consume:
the configuration records, the gridded meteorology (wind, eddy diffusivity, rain mask),
the per-scenario sources and emission series of the batched ensemble, and the receptor
lattice. It performs no step of the particle method itself (no interpolation, no random
walk, no deposition test, no binning): it only writes input arrays.

The paper's own workloads used ALADIN numerical-weather-prediction fields and a uniform
"artificial" weather (Sec. 4, Fig. 3b caption); neither dataset exists here, so seeded
synthetic fields with the same shapes stand in for them.

Seeds: particles 1, meteorology 11, rain 12, scenarios 13, hidden source 14, receptors 15.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "LpmConfig", "Release", "Scenario",
    "make_cfg0", "make_cfg1", "make_cfg2", "make_cfg3", "make_cfg4", "make_stress",
    "make_artificial_weather", "make_receptors", "z_levels_stretched",
    "STATUS_ACTIVE", "STATUS_UNRELEASED", "STATUS_DEP_DRY", "STATUS_DEP_WET",
    "STATUS_EXITED",
]

# Particle status codes (the 4-bit field of the particle tag). Shared vocabulary only.
STATUS_ACTIVE = 0
STATUS_UNRELEASED = 1
STATUS_DEP_DRY = 2
STATUS_DEP_WET = 3
STATUS_EXITED = 4

SEED_PARTICLES = 1
SEED_MET = 11
SEED_RAIN = 12
SEED_SCENARIOS = 13
SEED_HIDDEN = 14
SEED_RECEPTORS = 15
SEED_BOUNDARY_LAYER = 16
SEED_MODES = 17


@dataclasses.dataclass
class Release:
    """A continuous release: ``n_particles`` spread over steps [first_step, last_step),
    emission rate ``q[h]`` (mass/s) for hour-bin h of width ``q_dt`` seconds."""
    n_particles: int
    q: np.ndarray
    q_dt: float
    first_step: int
    last_step: int


@dataclasses.dataclass
class Scenario:
    """One member of a batched ensemble: own source, release and wind perturbation."""
    src_x: float
    src_y: float
    src_z: float
    release: Release
    # Domain-uniform wind offset (du, dv) per met hour, [n_met_t][2] float32.
    wind_offset: Optional[np.ndarray] = None
    # The scenario's realisation of the ensemble's perturbation modes (LpmConfig.modes):
    # phase (cycles) and amplitude (m/s) of each mode, float64 [n_modes].
    mode_phase: Optional[np.ndarray] = None
    mode_amp: Optional[np.ndarray] = None


@dataclasses.dataclass
class LpmConfig:
    """Mirror of the C ``lpm_config`` record plus the input arrays."""
    # meteorology grid (node-centred), x/y uniform, z stretched
    nx: int
    ny: int
    nz: int
    x0: float
    y0: float
    dx: float
    dy: float
    z_levels: np.ndarray
    n_met_t: int
    met_t0: float
    met_dt: float
    # concentration grid (cell-centred, uniform)
    cx: int
    cy: int
    cz: int
    cx0: float
    cy0: float
    cz0: float
    cdx: float
    cdy: float
    cdz: float
    # point source
    src_x: float
    src_y: float
    src_z: float
    # time stepping
    dt: float
    n_steps: int
    seed: int
    bin_every: int
    # physics
    half_life_s: float          # <= 0: no decay
    vd_dry: float               # dry deposition velocity (m/s), 0: off
    h_mix: float                # mixing-layer height (m)
    wet_lambda: float           # scavenging coefficient (1/s), 0: off
    kh_uniform: float           # < 0: gridded K_h field
    reflect_ground: int
    reflect_top: int
    z_top: float
    lateral_exit: int
    drift_correction: int
    n_scenarios: int
    release: Release
    # input arrays
    uvwk: np.ndarray            # float32 [n_met_t][nz][ny][nx][4] = (u, v, w, K_z)
    kh: Optional[np.ndarray] = None     # float32 [n_met_t][nz][ny][nx]
    rain: Optional[np.ndarray] = None   # uint8  [n_met_t][ny][nx]
    scenarios: List[Scenario] = dataclasses.field(default_factory=list)
    # K_z model: 0 = the gridded K_z of uvwk, 1 = Eq. 3 from the boundary-layer columns
    kz_model: int = 0
    kz_min: float = 0.1
    bl: Optional[np.ndarray] = None     # float32 [n_met_t][ny][nx][4] = (u*, 1/L, H_z, 0)
    # decay chain: half-lives (s) of parent -> daughter -> ..., the first = half_life_s,
    # 0 = stable (last only); None: one species
    chain_half_lives: Optional[np.ndarray] = None
    # vertical Langevin variant (velocity memory over the Lagrangian time scale t_lagr, s)
    langevin: int = 0
    t_lagr: float = 100.0
    # perturbation modes of the wind (plane waves of a streamfunction), shared by the
    # scenarios: float64 [n_modes][5] = (fx, fy (cycles/m), omega (cycles/s), eu, ev (unit
    # velocity direction)) and the height profile [nz] they are scaled by; each scenario
    # (or, for a plain run, mode_phase / mode_amp here) gives its phases and amplitudes
    modes: Optional[np.ndarray] = None
    mode_profile: Optional[np.ndarray] = None
    mode_phase: Optional[np.ndarray] = None
    mode_amp: Optional[np.ndarray] = None
    name: str = ""

    @property
    def n_particles(self) -> int:
        if self.scenarios:
            return int(sum(s.release.n_particles for s in self.scenarios))
        return int(self.release.n_particles)


def z_levels_stretched(nz: int = 30, top: float = 3000.0) -> np.ndarray:
    """Stretched vertical levels z_k = top*(k/(nz-1))^2 (k = 0..nz-1)."""
    k = np.arange(nz, dtype=np.float64)
    return top * (k / (nz - 1)) ** 2


def make_artificial_weather(nx: int = 2, ny: int = 2, nz: int = 2, n_t: int = 2,
                            u: float = 5.0, v: float = 0.0, w: float = 0.0,
                            kz: float = 10.0, z_top: float = 400.0):
    """Homogeneous, constant fields (the paper's 'artificial' weather, Fig. 3b caption)."""
    uvwk = np.empty((n_t, nz, ny, nx, 4), dtype=np.float32)
    uvwk[..., 0] = u
    uvwk[..., 1] = v
    uvwk[..., 2] = w
    uvwk[..., 3] = kz
    z_levels = np.linspace(0.0, z_top, nz)
    return uvwk, z_levels


def make_cfg0(n_particles: int = 10_000, n_steps: int = 360, seed: int = SEED_PARTICLES,
              kh: float = 50.0, kz: float = 10.0, u: float = 5.0,
              src=(0.0, 0.0, 50.0)) -> LpmConfig:
    """Plain method, small: uniform wind u along x, constant K_h, K_z, reflecting ground,
    no decay or deposition, dt = 10 s, 100x100x20 grid of 100 m x 100 m x 20 m cells."""
    uvwk, z_levels = make_artificial_weather(u=u, kz=kz, z_top=400.0)
    return LpmConfig(
        nx=2, ny=2, nz=2, x0=-1000.0, y0=-5000.0, dx=10000.0, dy=10000.0,
        z_levels=z_levels, n_met_t=2, met_t0=0.0, met_dt=3600.0,
        cx=100, cy=100, cz=20, cx0=-1000.0, cy0=-5000.0, cz0=0.0,
        cdx=100.0, cdy=100.0, cdz=20.0,
        src_x=src[0], src_y=src[1], src_z=src[2],
        dt=10.0, n_steps=n_steps, seed=seed, bin_every=n_steps,
        half_life_s=0.0, vd_dry=0.0, h_mix=0.0, wet_lambda=0.0, kh_uniform=kh,
        reflect_ground=1, reflect_top=0, z_top=0.0, lateral_exit=0, drift_correction=0,
        n_scenarios=1,
        release=Release(n_particles=n_particles, q=np.array([1.0]), q_dt=3600.0,
                        first_step=0, last_step=n_steps),
        uvwk=uvwk, name="cfg0 plain small")


# ----------------------------------------------------------------------------------------
# Realistic synthetic meteorology (stand-in for the ALADIN fields of Sec. 4)
# ----------------------------------------------------------------------------------------
VON_KARMAN = 0.4


def _log_wind(z: np.ndarray, ustar: float, z0: float) -> np.ndarray:
    out = np.zeros_like(z)
    m = z > z0
    out[m] = ustar / VON_KARMAN * np.log(z[m] / z0)
    return out


def _kz_profile(z: np.ndarray, ustar: float, hz: float, kmin: float) -> np.ndarray:
    """Neutral similarity profile k u* z (1 - z/H_z)^2 (Eq. 3 with Phi = 1), floored at
    kmin and set to kmin at and above H_z. Evaluated here, at the met nodes, as met
    preprocessing: the particle step reads the gridded result."""
    kz = VON_KARMAN * ustar * z * (1.0 - z / hz) ** 2
    kz = np.where(z >= hz, kmin, kz)
    return np.maximum(kz, kmin)


def make_met_realistic(nx: int = 200, ny: int = 200, nz: int = 30, n_t: int = 25,
                       dx: float = 250.0, dy: float = 250.0, z_top: float = 3000.0,
                       ustar: float = 0.4, z0: float = 0.1, pbl: float = 1000.0,
                       n_modes: int = 16, rms: float = 1.5, seed: int = SEED_MET):
    """Hourly wind = log profile along +x plus a non-divergent mesoscale perturbation
    built from random-phase Fourier modes of a streamfunction (wavelengths log-uniform in
    5..50 km, rms ``rms`` m/s, scaled with height by u(z)/u(100 m), phases advancing per
    hour); w = 0; K_z from the similarity profile; returns float32 [n_t][nz][ny][nx][4]."""
    rng = np.random.default_rng(seed)
    z_levels = z_levels_stretched(nz, z_top)
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    X, Y = np.meshgrid(x, y)                 # [ny][nx]
    u_base = _log_wind(z_levels, ustar, z0)  # [nz]
    u100 = _log_wind(np.array([100.0]), ustar, z0)[0]
    hscale = u_base / u100                   # height scaling of the perturbation
    kz = _kz_profile(z_levels, ustar, pbl, 0.1)

    lam = np.exp(rng.uniform(np.log(5000.0), np.log(50000.0), n_modes))
    theta = rng.uniform(0.0, 2 * np.pi, n_modes)
    phase0 = rng.uniform(0.0, 2 * np.pi, n_modes)
    dphase = rng.uniform(0.0, 0.5 * np.pi, n_modes)
    amp = rms * math.sqrt(2.0 / n_modes)
    kvec = 2 * np.pi / lam

    uvwk = np.empty((n_t, nz, ny, nx, 4), dtype=np.float32)
    for h in range(n_t):
        up = np.zeros((ny, nx))
        vp = np.zeros((ny, nx))
        for m in range(n_modes):
            kx = kvec[m] * math.cos(theta[m])
            ky = kvec[m] * math.sin(theta[m])
            s = np.sin(kx * X + ky * Y + phase0[m] + h * dphase[m])
            # psi = (amp/|k|) cos(k.x + phi): u' = dpsi/dy, v' = -dpsi/dx
            up += -amp * math.sin(theta[m]) * s
            vp += amp * math.cos(theta[m]) * s
        for k in range(nz):
            uvwk[h, k, :, :, 0] = u_base[k] + hscale[k] * up
            uvwk[h, k, :, :, 1] = hscale[k] * vp
            uvwk[h, k, :, :, 2] = 0.0
            uvwk[h, k, :, :, 3] = kz[k]
    return uvwk, z_levels


def make_boundary_layer(nx: int = 200, ny: int = 200, n_t: int = 25, dx: float = 250.0,
                        dy: float = 250.0, seed: int = SEED_BOUNDARY_LAYER) -> np.ndarray:
    """Hourly boundary-layer columns for Eq. 3, float32 [n_t][ny][nx][4] = (u*, 1/L, H_z, 0):
    a diurnal cycle starting at 06 h (stable night to unstable day: 1/L from +0.01 to
    -0.03 1/m, H_z from 400 m to 1600 m) modulated by seeded smooth fields (4 Fourier modes,
    wavelengths 10..40 km): u* = 0.4 (1 + 0.25 g1) m/s, 1/L + 0.004 g2, H_z (1 + 0.15 g3)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    X, Y = np.meshgrid(x, y)

    def smooth():
        g = np.zeros((ny, nx))
        for _ in range(4):
            lam = rng.uniform(10000.0, 40000.0)
            th = rng.uniform(0.0, 2 * np.pi)
            ph = rng.uniform(0.0, 2 * np.pi)
            g += np.sin(2 * np.pi / lam * (np.cos(th) * X + np.sin(th) * Y) + ph)
        return g / 2.0                       # roughly in [-1, 1]

    g1, g2, g3 = smooth(), smooth(), smooth()
    out = np.zeros((n_t, ny, nx, 4), dtype=np.float32)
    for h in range(n_t):
        day = math.sin(2 * np.pi * (h - 6) / 24.0)        # > 0 by day
        inv_l = (0.01 - 0.02 * (day + 1.0)) if day > 0 else 0.01 * (1.0 + day)
        hz = 1000.0 + 600.0 * day
        out[h, :, :, 0] = np.clip(0.4 * (1.0 + 0.25 * g1), 0.1, 0.8)
        out[h, :, :, 1] = inv_l + 0.004 * g2
        out[h, :, :, 2] = np.clip(hz * (1.0 + 0.15 * g3), 200.0, 2500.0)
    return out


def make_rain(nx: int = 200, ny: int = 200, n_t: int = 25, dx: float = 250.0,
              dy: float = 250.0, n_discs: int = 8, u_adv: float = None,
              seed: int = SEED_RAIN) -> np.ndarray:
    """Rain mask [n_t][ny][nx] (uint8): seeded discs of radius 2..5 km advected hourly
    at the 100 m mean wind along +x."""
    rng = np.random.default_rng(seed)
    if u_adv is None:
        u_adv = _log_wind(np.array([100.0]), 0.4, 0.1)[0]
    lx = (nx - 1) * dx
    ly = (ny - 1) * dy
    cx = rng.uniform(-0.5 * lx, lx, n_discs)
    cy = rng.uniform(0.0, ly, n_discs)
    r = rng.uniform(2000.0, 5000.0, n_discs)
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    X, Y = np.meshgrid(x, y)
    out = np.zeros((n_t, ny, nx), dtype=np.uint8)
    for h in range(n_t):
        for d in range(n_discs):
            # advected along +x, periodic over [-lx/2, 3lx/2) so rain stays in view
            ccx = (cx[d] + u_adv * 3600.0 * h + 0.5 * lx) % (2.0 * lx) - 0.5 * lx
            m = (X - ccx) ** 2 + (Y - cy[d]) ** 2 <= r[d] ** 2
            out[h][m] = 1
    return out


def make_cfg1(n_particles: int = 10_000_000, n_steps: int = 2880, n_hours: int = None,
              seed: int = SEED_PARTICLES, with_rain: bool = True,
              kz_eq3: bool = False) -> LpmConfig:
    """Plain method, realistic: 24 h at dt = 30 s on a 200x200x30 hourly met grid
    (250 m spacing, stretched levels to 3 km), 8-day half-life, dry deposition velocity
    0.002 m/s below a 1000 m mixing layer, wet scavenging 1e-4 1/s inside the rain mask,
    400x400x20 concentration grid (125 m x 125 m x 50 m) plus a 400x400 deposition grid.
    ``n_hours`` limits the generated met slabs (default: enough for ``n_steps``).
    ``kz_eq3`` takes K_z from Eq. 3 on seeded boundary-layer columns instead of the grid."""
    dt = 30.0
    if n_hours is None:
        n_hours = int(math.ceil(n_steps * dt / 3600.0)) + 1
    n_hours = max(2, min(n_hours, 25))
    uvwk, z_levels = make_met_realistic(n_t=n_hours)
    rain = make_rain(n_t=n_hours) if with_rain else None
    return LpmConfig(
        nx=200, ny=200, nz=30, x0=0.0, y0=0.0, dx=250.0, dy=250.0,
        z_levels=z_levels, n_met_t=n_hours, met_t0=0.0, met_dt=3600.0,
        cx=400, cy=400, cz=20, cx0=0.0, cy0=0.0, cz0=0.0, cdx=125.0, cdy=125.0, cdz=50.0,
        src_x=5000.0, src_y=24875.0, src_z=50.0,
        dt=dt, n_steps=n_steps, seed=seed, bin_every=120,
        half_life_s=8 * 86400.0, vd_dry=0.002, h_mix=1000.0,
        wet_lambda=1e-4 if with_rain else 0.0, kh_uniform=100.0,
        reflect_ground=1, reflect_top=1, z_top=3000.0, lateral_exit=1, drift_correction=0,
        n_scenarios=1,
        release=Release(n_particles=n_particles, q=np.array([1.0]), q_dt=3600.0,
                        first_step=0, last_step=n_steps),
        uvwk=uvwk, kh=None, rain=rain, name="cfg1 plain realistic",
        kz_model=1 if kz_eq3 else 0,
        bl=make_boundary_layer(n_t=n_hours) if kz_eq3 else None)


def make_modes(z_levels: np.ndarray, n_modes: int = 4, ustar: float = 0.4, z0: float = 0.1,
               seed: int = SEED_MODES):
    """Perturbation modes shared by an ensemble: ``n_modes`` plane waves of a horizontal
    streamfunction with wavelengths log-uniform in 5..50 km, seeded directions, phase rates
    of 0..1/4 cycle per hour, velocity perpendicular to the wavenumber (non-divergent), and
    the height profile u(z)/u(100 m) of the log wind at the levels. Returns (modes [M][5],
    profile [nz])."""
    rng = np.random.default_rng(seed)
    lam = np.exp(rng.uniform(np.log(5000.0), np.log(50000.0), n_modes))
    theta = rng.uniform(0.0, 2 * np.pi, n_modes)
    omega = rng.uniform(0.0, 0.25, n_modes) / 3600.0
    modes = np.stack([np.cos(theta) / lam, np.sin(theta) / lam, omega, -np.sin(theta),
                      np.cos(theta)], axis=1)
    u100 = _log_wind(np.array([100.0]), ustar, z0)[0]
    profile = _log_wind(np.asarray(z_levels, dtype=np.float64), ustar, z0) / u100
    # values representable in FP32, so that a single-precision consumer reads them exactly
    return _fp32_exact(modes), _fp32_exact(profile)


def _fp32_exact(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def make_cfg2(n_scenarios: int = 256, n_steps: int = 1440, n_min: float = 1e4,
              n_max: float = 1e6, seed: int = SEED_SCENARIOS,
              base: Optional[LpmConfig] = None, n_modes: int = 4,
              mode_rms: float = 1.0) -> LpmConfig:
    """Batched ensemble: ``n_scenarios`` scenarios on the realistic met grid, particle
    counts log-uniform in [n_min, n_max], own source (x, y, release height 10..300 m),
    24-value hourly emission series and perturbed meteorology: a seeded, domain-uniform
    hourly wind offset (AR(1), rms 1.5 m/s per component) plus the scenario's own
    realisation of ``n_modes`` shared perturbation modes (seeded phases, amplitudes
    (0.5..1.5) x mode_rms sqrt(2 / n_modes)); 12 h at dt = 30 s; one surface-layer
    concentration layer (0..50 m) plus dry/wet deposition per scenario."""
    if base is None:
        base = make_cfg1(n_particles=1, n_steps=n_steps)
    modes = profile = None
    mrng = np.random.default_rng(SEED_MODES + 1)
    if n_modes > 0:
        modes, profile = make_modes(base.z_levels, n_modes)
    rng = np.random.default_rng(seed)
    scen = []
    for _ in range(n_scenarios):
        n = int(math.floor(10 ** rng.uniform(math.log10(n_min), math.log10(n_max))))
        sx = rng.uniform(2000.0, 15000.0)
        sy = rng.uniform(10000.0, 40000.0)
        sz = rng.uniform(10.0, 300.0)
        q = np.exp(rng.normal(0.0, 0.5, 24))
        off = np.empty((base.n_met_t, 2), dtype=np.float32)
        a = rng.normal(0.0, 1.5, 2)
        for h in range(base.n_met_t):
            off[h] = a
            a = 0.8 * a + math.sqrt(1 - 0.64) * rng.normal(0.0, 1.5, 2)
        sc = Scenario(sx, sy, sz, Release(n, q, 3600.0, 0, n_steps), off)
        if n_modes > 0:
            sc.mode_phase = _fp32_exact(mrng.uniform(0.0, 1.0, n_modes))
            sc.mode_amp = _fp32_exact(mode_rms * math.sqrt(2.0 / n_modes) *
                                      mrng.uniform(0.5, 1.5, n_modes))
        scen.append(sc)
    cfg = dataclasses.replace(base, n_steps=n_steps, bin_every=n_steps,
                              cz=1, n_scenarios=n_scenarios, scenarios=scen,
                              modes=modes, mode_profile=profile,
                              name="cfg2 batched ensemble")
    return cfg


def make_receptors(src=(5000.0, 24875.0), n_side: int = 8, z: float = 2.0,
                   down=(2000.0, 20000.0), cross: float = 5000.0) -> np.ndarray:
    """8x8 receptor lattice at height z, 2..20 km downstream (+x) of the source and
    +-5 km cross-wind; returns float64 [R][3]."""
    xs = src[0] + np.linspace(down[0], down[1], n_side)
    ys = src[1] + np.linspace(-cross, cross, n_side)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)


def make_cfg3(n_particles: int = 1_000_000, n_steps: int = 1080,
              seed: int = SEED_PARTICLES) -> LpmConfig:
    """Adjoint workload: 6 h at dt = 20 s on the realistic met grid, source
    (5 km, 24.875 km, 50 m), 24-value hourly emission series (seeded)."""
    base = make_cfg1(n_particles=n_particles, n_steps=n_steps)
    rng = np.random.default_rng(SEED_RECEPTORS)
    q = np.exp(rng.normal(0.0, 0.3, 24))
    n_steps = int(n_steps)
    base = dataclasses.replace(base, dt=20.0, n_steps=n_steps, bin_every=n_steps,
                               release=Release(n_particles, q, 3600.0, 0, n_steps),
                               name="cfg3 adjoint")
    return base


def make_cfg4(n_candidates: int = 64, n_per: int = 100_000, n_steps: int = 1080,
              seed: int = SEED_HIDDEN, n_obs: int = 1_000_000):
    """Batched source inversion on the adjoint workload's weather and receptors:
    returns (candidates, observation) configurations and the hidden source. The
    candidates are ``n_candidates`` scenarios of ``n_per`` particles with seeded starting
    sources; the observation is a plain release of ``n_obs`` particles from the hidden
    seeded source with another key, so its noise is independent of the candidates'."""
    base = make_cfg3(n_particles=n_per, n_steps=n_steps)
    rng = np.random.default_rng(seed)
    hidden = (float(rng.uniform(3000.0, 8000.0)), float(rng.uniform(20000.0, 30000.0)),
              float(rng.uniform(20.0, 150.0)))
    cands = np.stack([rng.uniform(2000.0, 10000.0, n_candidates),
                      rng.uniform(18000.0, 32000.0, n_candidates),
                      rng.uniform(10.0, 300.0, n_candidates)], axis=1)
    rel = base.release
    scen = [Scenario(float(c[0]), float(c[1]), float(c[2]),
                     Release(n_per, rel.q, rel.q_dt, 0, n_steps)) for c in cands]
    cand_cfg = dataclasses.replace(base, n_scenarios=n_candidates, scenarios=scen,
                                   name="batched source inversion (candidates)")
    obs_cfg = dataclasses.replace(base, src_x=hidden[0], src_y=hidden[1], src_z=hidden[2],
                                  seed=base.seed + 1000,
                                  release=Release(n_obs, rel.q, rel.q_dt, 0, n_steps),
                                  name="batched source inversion (observation)")
    return cand_cfg, obs_cfg, hidden


def make_stress(n_particles: int = 100_000_000, n_steps: int = 5760, seed: int = SEED_PARTICLES):
    """Forward-only throughput stress case: 1e8 particles released continuously over 48 h at
    dt = 30 s on a 512x512x32 hourly weather grid (250 m spacing, 128 km domain, levels to
    3 km), source (10 km, 64 km, 50 m); the realistic physics; 512x512x20 concentration grid
    of 250 m x 250 m x 50 m cells, hourly snapshots."""
    n_hours = int(math.ceil(n_steps * 30.0 / 3600.0)) + 1
    uvwk, z_levels = make_met_realistic(nx=512, ny=512, nz=32, n_t=n_hours)
    rain = make_rain(nx=512, ny=512, n_t=n_hours)
    return LpmConfig(
        nx=512, ny=512, nz=32, x0=0.0, y0=0.0, dx=250.0, dy=250.0,
        z_levels=z_levels, n_met_t=n_hours, met_t0=0.0, met_dt=3600.0,
        cx=512, cy=512, cz=20, cx0=0.0, cy0=0.0, cz0=0.0, cdx=250.0, cdy=250.0, cdz=50.0,
        src_x=10000.0, src_y=64000.0, src_z=50.0,
        dt=30.0, n_steps=n_steps, seed=seed, bin_every=120,
        half_life_s=8 * 86400.0, vd_dry=0.002, h_mix=1000.0, wet_lambda=1e-4,
        kh_uniform=100.0, reflect_ground=1, reflect_top=1, z_top=3000.0, lateral_exit=1,
        drift_correction=0, n_scenarios=1,
        release=Release(n_particles=n_particles, q=np.array([1.0]), q_dt=3600.0,
                        first_step=0, last_step=n_steps),
        uvwk=uvwk, kh=None, rain=rain, name="stress 1e8 x 48 h")
