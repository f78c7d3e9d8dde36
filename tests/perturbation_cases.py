"""Configurations with closed-form paths in perturbed weather (no diffusion): the hourly
wind offset and the perturbation modes. Shared by the oracle pins and the GPU tests; the
expected paths are computed in the tests themselves."""
import dataclasses
import math

import numpy as np

import lpm_inputs as li

HOUR = 3600.0


def offset_cfg(offsets, dt=70.0, n_steps=150, n_particles=50, rel_last=100, u=5.0):
    n_t = offsets.shape[0]
    uvwk, z_levels = li.make_artificial_weather(u=u, v=0.0, w=0.0, kz=0.0, n_t=n_t,
                                                z_top=400.0)
    base = li.make_cfg0(n_particles=n_particles, n_steps=n_steps, kh=0.0, kz=0.0, u=u)
    rel = li.Release(n_particles, np.array([1.0]), HOUR, 0, rel_last)
    sc = li.Scenario(base.src_x + 120.0, base.src_y - 75.0, base.src_z, rel,
                     offsets.astype(np.float32))
    return dataclasses.replace(base, uvwk=uvwk, z_levels=z_levels, n_met_t=n_t, dt=dt,
                               release=rel, scenarios=[sc], n_scenarios=1)


def offsets():
    return np.random.default_rng(41).normal(0.0, 2.0, (4, 2))


Z_LEVELS = np.array([0.0, 100.0, 200.0, 300.0, 400.0])
PROFILE = np.array([0.0, 0.5, 1.0, 1.3, 1.5])


def mode(theta=0.7, lam=3000.0, omega=0.0):
    return np.array([[math.cos(theta) / lam, math.sin(theta) / lam, omega, -math.sin(theta),
                      math.cos(theta)]])


def mode_cfg(modes, phase, amp, src=(1234.0, -567.0, 130.0), dt=30.0, n_steps=120,
             n_particles=30, rel_last=60):
    nz = Z_LEVELS.size
    uvwk = np.zeros((2, nz, 2, 2, 4), np.float32)      # no base wind, no diffusion
    base = li.make_cfg0(n_particles=n_particles, n_steps=n_steps, kh=0.0, kz=0.0)
    rel = li.Release(n_particles, np.array([1.0]), HOUR, 0, rel_last)
    sc = li.Scenario(src[0], src[1], src[2], rel, None, mode_phase=np.asarray(phase, float),
                     mode_amp=np.asarray(amp, float))
    return dataclasses.replace(base, uvwk=uvwk, z_levels=Z_LEVELS, nz=nz, dt=dt, release=rel,
                               scenarios=[sc], n_scenarios=1, modes=np.asarray(modes, float),
                               mode_profile=PROFILE)


def release_steps(sc):
    n = sc.release.n_particles
    return np.arange(n) * sc.release.last_step // n
