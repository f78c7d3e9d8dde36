"""Perturbed weather on the CUDA path (through the C ABI): the hourly wind offset and the
perturbation modes follow their closed-form paths in weather without diffusion, a plain
context with modes matches the oracle element by element, and the adjoint refuses a
context with modes (it does not differentiate them)."""
import dataclasses
import math

import numpy as np
import pytest

import lpm_inputs as li
import oracle
from parity_util import compare, run_gpu
from perturbation_cases import (HOUR, PROFILE, Z_LEVELS, mode, mode_cfg, offset_cfg, offsets,
                                release_steps)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# FP32 state: each step rounds x to half an ulp (2e-3 m at 50 km); over 150 steps the
# rounding adds up, as a random walk, to a few cm. 0.1 m still separates the correct
# path from an hour taken off by one (du differences of metres per second over an hour).
PATH_TOL_M = 0.1


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    oracle.build()


def _gpu_positions(cfg):
    from paper_0912_3223_gb300 import Sim
    with Sim(cfg) as sim:
        sim.step(cfg.n_steps)
        xyz, tag = sim.particles()
    return xyz.astype(np.float64), tag


def test_wind_offset_paths_gpu():
    cfg = offset_cfg(offsets())
    sc = cfg.scenarios[0]
    xyz, _ = _gpu_positions(cfg)
    off = sc.wind_offset.astype(np.float64)
    hours = np.arange(off.shape[0], dtype=np.float64)
    worst = 0.0
    for p, s_p in enumerate(release_steps(sc)):
        t = np.arange(s_p, cfg.n_steps) * cfg.dt / HOUR
        x = sc.src_x + np.sum((5.0 + np.interp(t, hours, off[:, 0])) * cfg.dt)
        y = sc.src_y + np.sum(np.interp(t, hours, off[:, 1]) * cfg.dt)
        worst = max(worst, abs(xyz[p, 0] - x), abs(xyz[p, 1] - y))
    print(f"offset paths: max deviation {worst:.4f} m")
    assert worst < PATH_TOL_M


def test_mode_paths_gpu():
    # steady mode: straight line along the crest
    modes = mode()
    cfg = mode_cfg(modes, [0.05], [2.0])
    sc = cfg.scenarios[0]
    xyz, _ = _gpu_positions(cfg)
    fx, fy, _, eu, ev = modes[0]
    p = np.interp(sc.src_z, Z_LEVELS, PROFILE)
    speed = 2.0 * p * math.sin(2 * math.pi * (fx * sc.src_x + fy * sc.src_y + 0.05))
    n_moves = cfg.n_steps - release_steps(sc)
    dev = np.maximum(np.abs(xyz[:, 0] - (sc.src_x + n_moves * cfg.dt * speed * eu)),
                     np.abs(xyz[:, 1] - (sc.src_y + n_moves * cfg.dt * speed * ev)))
    print(f"steady mode: max deviation {dev.max():.4f} m")
    assert dev.max() < PATH_TOL_M
    # moving phase: the sum of a sine over an arithmetic progression
    omega = 0.2 / HOUR
    modes = mode(theta=-1.1, lam=4500.0, omega=omega)
    cfg = mode_cfg(modes, [0.8], [1.5], n_steps=300, rel_last=150)
    sc = cfg.scenarios[0]
    xyz, _ = _gpu_positions(cfg)
    fx, fy, _, eu, ev = modes[0]
    c0 = fx * sc.src_x + fy * sc.src_y + 0.8
    d = 2 * math.pi * omega * cfg.dt
    worst = 0.0
    for i, s in enumerate(release_steps(sc)):
        M = cfg.n_steps - s
        a = 2 * math.pi * (c0 + omega * s * cfg.dt)
        disp = 1.5 * p * cfg.dt * math.sin(M * d / 2) / math.sin(d / 2) * math.sin(a + (M - 1) * d / 2)
        worst = max(worst, abs(xyz[i, 0] - (sc.src_x + disp * eu)),
                    abs(xyz[i, 1] - (sc.src_y + disp * ev)))
    print(f"moving mode: max deviation {worst:.4f} m")
    assert worst < PATH_TOL_M


def _plain_with_modes(n_particles=20_000, n_steps=2880):
    base = li.make_cfg1(n_particles=n_particles, n_steps=n_steps, n_hours=25)
    modes, prof = li.make_modes(base.z_levels)
    return dataclasses.replace(base, modes=modes, mode_profile=prof,
                               mode_phase=np.array([0.25, 0.5, 0.75, 0.125]),
                               mode_amp=np.array([0.75, 0.5, 1.0, 0.625]))


def test_plain_context_with_modes_matches_oracle():
    """The realistic weather plus four modes on a one-scenario context (the extended step
    kernel, release-ordered and cell-sorted tiles): all particles after 360 steps, then
    the first hourly snapshot's grids, against the oracle."""
    cfg = _plain_with_modes()
    g = run_gpu(cfg, n_run=360)
    o = oracle.run(cfg, n_run=360)
    rep = compare(cfg, g, o, check_grid=False, sens=oracle.sensitivity(cfg, n_run=360))
    print("modes, 360 steps:", rep)
    g = run_gpu(cfg, n_run=120)
    o = oracle.run(cfg, n_run=120)
    rep = compare(cfg, g, o, sens=oracle.sensitivity(cfg, n_run=120))
    print("modes, 120 steps:", rep)
    assert int(g["counters"][4]) == o["active_steps"]


def test_adjoint_refuses_perturbation_modes():
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = _plain_with_modes(n_particles=1000, n_steps=120)
    rec = li.make_receptors()
    with Sim(cfg) as sim:
        sim.step(cfg.n_steps)
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_receptors(sim.ctx, 1, rec, 200.0, 18)
        assert e.value.status == lpm.LPM_E_INVALID and "modes" in str(e.value)


def test_modes_alone_and_in_the_extended_kernel_agree():
    """The perturbation modes run in a kernel of their own, or, with any extended option
    on (the dosage here, which moves no particle), in the extended kernel: particles and
    grids are the same bits either way, for mixed-scenario lanes and per-scenario tiles."""
    from paper_0912_3223_gb300 import Sim
    cfg = li.make_cfg2(n_scenarios=5, n_steps=240, n_min=300, n_max=1500)

    def run(dose, sort_every):
        with Sim(cfg, sort_every=sort_every) as sim:
            if dose:
                sim.set_dosage(6)
            sim.step(cfg.n_steps)
            xyz, tag = sim.particles()
            grids = [sim.fixed_state(s)[:2] for s in range(cfg.n_scenarios)]
        return xyz, tag, grids

    for sort_every in (0, 30):
        a, b = run(False, sort_every), run(True, sort_every)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        for (ca, da), (cb, db) in zip(a[2], b[2]):
            assert np.array_equal(ca, cb) and np.array_equal(da, db)
