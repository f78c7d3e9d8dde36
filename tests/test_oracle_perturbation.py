"""Pins of the oracle's perturbed weather (the batched ensemble's per-scenario wind):

- the domain-uniform hourly wind offset: with uniform wind and no diffusion every path is
  the Euler sum of the wind plus the offset blended linearly between the hours (Eq. 1 with
  the linear time interpolation of Sec. 3.2), computed here with numpy's own linear
  interpolation;
- the perturbation modes (plane waves of a streamfunction): a particle carried along a
  wave crest keeps its phase, so it moves in a straight line; with a moving phase its
  Euler sum is the sum of a sine over an arithmetic progression; the field has zero
  divergence; its tangent-linear gradient matches central differences;
- the adjoint's wind-bias and source gradients against central differences with both
  perturbations present.

Each pin is also run against copies of the oracle with a planted mistake (an hour off by
one, u and v swapped, a dropped weight, a swapped direction, cos for sin, a dropped phase
or 2 pi) and must fail on them. No expected value comes from the CUDA path.
"""
import dataclasses
import math

import numpy as np
import pytest

import lpm_inputs as li
import oracle
from oracle_variants import fails

from perturbation_cases import (HOUR, PROFILE, Z_LEVELS, mode as _mode, mode_cfg as _mode_cfg,
                               offset_cfg as _offset_cfg, offsets as _offsets,
                               release_steps as _release_steps)


# ------------------------------------------------------------------------------------
# Domain-uniform hourly wind offset
# ------------------------------------------------------------------------------------
def _check_offset_paths():
    off = _offsets()
    cfg = _offset_cfg(off)
    sc = cfg.scenarios[0]
    r = oracle.run(cfg, scenario=0)
    off32 = sc.wind_offset.astype(np.float64)
    hours = np.arange(off32.shape[0], dtype=np.float64)
    n = sc.release.n_particles
    for p in range(n):
        s_p = p * sc.release.last_step // n
        t = np.arange(s_p, cfg.n_steps) * cfg.dt / HOUR
        du = np.interp(t, hours, off32[:, 0])
        dv = np.interp(t, hours, off32[:, 1])
        x = sc.src_x + np.sum((5.0 + du) * cfg.dt)
        y = sc.src_y + np.sum(dv * cfg.dt)
        assert abs(r["pos"][p, 0] - x) < 1e-9, (p, r["pos"][p, 0], x)
        assert abs(r["pos"][p, 1] - y) < 1e-9, (p, r["pos"][p, 1], y)
        assert r["pos"][p, 2] == sc.src_z


def test_wind_offset_paths_follow_the_closed_form():
    """Uniform wind u = 5 m/s, K = 0, four hourly offsets (du, dv), dt = 70 s (steps
    straddle the hours): every particle ends at x_s + sum_k (u + du(t_k)) dt,
    y_s + sum_k dv(t_k) dt, to 1e-9 m."""
    _check_offset_paths()


@pytest.mark.parametrize("mistake", [
    # the hour off by one: the later slab's offset in place of the earlier one's
    [("(1.0 - f) * (double)c->wind_offset[2 * h0]", "(1.0 - f) * (double)c->wind_offset[2 * h1]")],
    # u and v swapped
    [("c->wind_offset[2 * h0] + f * (double)c->wind_offset[2 * h1];",
      "c->wind_offset[2 * h0 + 1] + f * (double)c->wind_offset[2 * h1 + 1];")],
    # the time weight of the earlier hour dropped
    [("acc[0] += (1.0 - f) * (double)c->wind_offset[2 * h0]",
      "acc[0] += (double)c->wind_offset[2 * h0]")],
], ids=["hour_off_by_one", "u_v_swapped", "weight_dropped"])
def test_wind_offset_pin_catches_planted_mistakes(mistake):
    assert fails(_check_offset_paths, *mistake)


# ------------------------------------------------------------------------------------
# Perturbation modes
# ------------------------------------------------------------------------------------
def _check_steady_mode_paths():
    """omega = 0: the velocity (eu, ev) is perpendicular to the wavenumber, so the phase
    fx x + fy y of a particle never changes and it moves in a straight line at
    amp p(z) sin(2 pi (fx x_s + fy y_s + phase))."""
    modes = _mode()
    cfg = _mode_cfg(modes, [0.05], [2.0])
    sc = cfg.scenarios[0]
    r = oracle.run(cfg, scenario=0)
    fx, fy, _, eu, ev = modes[0]
    p = np.interp(sc.src_z, Z_LEVELS, PROFILE)
    speed = 2.0 * p * math.sin(2 * math.pi * (fx * sc.src_x + fy * sc.src_y + 0.05))
    assert abs(speed) > 0.5
    n_moves = cfg.n_steps - _release_steps(sc)
    np.testing.assert_allclose(r["pos"][:, 0], sc.src_x + n_moves * cfg.dt * speed * eu,
                               rtol=0, atol=1e-6)
    np.testing.assert_allclose(r["pos"][:, 1], sc.src_y + n_moves * cfg.dt * speed * ev,
                               rtol=0, atol=1e-6)
    np.testing.assert_array_equal(r["pos"][:, 2], sc.src_z)


def _check_moving_mode_paths():
    """omega != 0, still along a crest: x_end - x_s = amp p dt eu sum_{k=s}^{S-1}
    sin(a + (k - s) d) with a = 2 pi (phase_s + omega s dt), d = 2 pi omega dt, which is
    sin(M d / 2) / sin(d / 2) sin(a + (M - 1) d / 2) for M steps."""
    omega = 0.2 / HOUR
    modes = _mode(theta=-1.1, lam=4500.0, omega=omega)
    cfg = _mode_cfg(modes, [0.8], [1.5], n_steps=300, rel_last=150)
    sc = cfg.scenarios[0]
    r = oracle.run(cfg, scenario=0)
    fx, fy, _, eu, ev = modes[0]
    p = np.interp(sc.src_z, Z_LEVELS, PROFILE)
    c0 = fx * sc.src_x + fy * sc.src_y + 0.8
    d = 2 * math.pi * omega * cfg.dt
    for i, s in enumerate(_release_steps(sc)):
        M = cfg.n_steps - s
        a = 2 * math.pi * (c0 + omega * s * cfg.dt)
        total = math.sin(M * d / 2) / math.sin(d / 2) * math.sin(a + (M - 1) * d / 2)
        disp = 1.5 * p * cfg.dt * total
        assert abs(r["pos"][i, 0] - (sc.src_x + disp * eu)) < 1e-6
        assert abs(r["pos"][i, 1] - (sc.src_y + disp * ev)) < 1e-6


def test_steady_mode_moves_particles_along_the_crest():
    _check_steady_mode_paths()


def test_moving_mode_paths_follow_the_progression_sum():
    _check_moving_mode_paths()


def _field_cfg():
    modes, _ = li.make_modes(Z_LEVELS, n_modes=4)
    phase = np.array([0.1, 0.45, 0.7, 0.9])
    amp = np.array([0.8, 1.2, 0.6, 1.0])
    return _mode_cfg(modes, phase, amp)


def _points(n=64):
    rng = np.random.default_rng(43)
    return np.stack([rng.uniform(-5000, 30000, n), rng.uniform(-8000, 8000, n),
                     rng.uniform(5.0, 395.0, n), rng.uniform(0.0, 7000.0, n)], axis=1)


def _check_field_divergence_and_gradient():
    cfg = _field_cfg()
    pts = _points()
    h = 0.5
    f = lambda q: oracle.interp(cfg, q, scenario=0)                   # noqa: E731
    ex, ey = np.array([h, 0, 0, 0]), np.array([0, h, 0, 0])
    dudx = (f(pts + ex)[:, 0] - f(pts - ex)[:, 0]) / (2 * h)
    dvdy = (f(pts + ey)[:, 1] - f(pts - ey)[:, 1]) / (2 * h)
    dvdx = (f(pts + ex)[:, 1] - f(pts - ex)[:, 1]) / (2 * h)
    dudy = (f(pts + ey)[:, 0] - f(pts - ey)[:, 0]) / (2 * h)
    scale = np.abs(dudx).max()
    assert scale > 1e-4
    assert np.abs(dudx + dvdy).max() < 1e-6 * scale              # non-divergent
    assert np.abs(dvdx - dudy).max() > 0.1 * scale               # and not trivial
    # the tangent-linear gradient of the oracle against central differences
    _, grad = oracle.interp_grad(cfg, pts, scenario=0)
    ez = np.array([0, 0, 1e-3, 0])
    dz = (f(pts + ez)[:, :2] - f(pts - ez)[:, :2]) / 2e-3
    np.testing.assert_allclose(grad[:, 0, 0], dudx, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(grad[:, 0, 1], dudy, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(grad[:, 1, 0], dvdx, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(grad[:, 1, 1], dvdy, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(grad[:, :2, 2], dz, rtol=1e-5, atol=1e-9)


def test_modes_are_non_divergent_and_their_gradient_matches_differences():
    _check_field_divergence_and_gradient()


def test_mode_profile_at_the_levels():
    """At a level the scale is the profile's value there; halfway between two levels the
    mean of the two (steady mode, the particle's speed)."""
    modes = _mode()
    for z, p in [(100.0, 0.5), (300.0, 1.3), (250.0, 1.15), (50.0, 0.25)]:
        cfg = _mode_cfg(modes, [0.3], [2.0], src=(1234.0, -567.0, z), n_steps=1,
                        n_particles=1, rel_last=1)
        fx, fy, _, eu, _ = modes[0]
        v = oracle.interp(cfg, [[1234.0, -567.0, z, 0.0]], scenario=0)[0]
        s = 2.0 * math.sin(2 * math.pi * (fx * 1234.0 + fy * -567.0 + 0.3))
        assert v[0] == pytest.approx(p * s * eu, rel=1e-12)


@pytest.mark.parametrize("check,mistake", [
    (_check_steady_mode_paths, [("s_u += a * md[3] * sn;", "s_u += a * md[4] * sn;")]),
    (_check_steady_mode_paths, [("const double sn = sin(arg), cs = cos(arg)",
                                 "const double sn = cos(arg), cs = cos(arg)")]),
    (_check_steady_mode_paths, [(" + c->mode_phase[m]", "")]),
    (_check_steady_mode_paths, [("(1.0 - cz) * c->mode_profile[k] + cz * c->mode_profile[k + 1]",
                                 "(1.0 - cz) * c->mode_profile[k + 1] + cz * c->mode_profile[k]")]),
    (_check_moving_mode_paths, [(" + md[2] * t)", ")")]),
    (_check_field_divergence_and_gradient,
     [("d_u[d] += a * md[3] * cs * two_pi * md[d];", "d_u[d] += a * md[3] * cs * md[d];")]),
    (_check_field_divergence_and_gradient, [("g[0][2] = dp * s_u;", "g[0][2] = 0.0;")]),
], ids=["direction_swapped", "cos_for_sin", "phase_dropped", "profile_weights_swapped",
        "phase_rate_dropped", "gradient_2pi_dropped", "profile_derivative_dropped"])
def test_mode_pins_catch_planted_mistakes(check, mistake):
    assert fails(check, *mistake)


# ------------------------------------------------------------------------------------
# The adjoint with the perturbations present
# ------------------------------------------------------------------------------------
def test_adjoint_bias_and_source_gradient_with_perturbed_weather():
    """Realistic sheared weather plus a scenario's hourly offsets and four modes: the
    oracle adjoint's source and wind-bias gradients against central differences of its
    receptor loss (same seeds), 2 % of the largest component as in the unperturbed case."""
    base = li.make_cfg1(n_particles=600, n_steps=120, n_hours=3, with_rain=False)
    modes, prof = li.make_modes(base.z_levels, n_modes=4)
    rel = li.Release(600, np.array([1.0, 3.0]), 1800.0, 0, 120)
    off = np.random.default_rng(44).normal(0.0, 1.5, (base.n_met_t, 2)).astype(np.float32)
    sc = li.Scenario(base.src_x, base.src_y, base.src_z, rel, off,
                     mode_phase=np.array([0.2, 0.5, 0.9, 0.4]),
                     mode_amp=np.array([0.9, 0.7, 1.1, 0.5]))
    cfg = dataclasses.replace(base, vd_dry=0.0, lateral_exit=0, half_life_s=3600.0,
                              release=rel, scenarios=[sc], n_scenarios=1, modes=modes,
                              mode_profile=prof)
    rec = np.array([[9000.0, 24875.0, 2.0], [12000.0, 25500.0, 30.0], [7000.0, 24000.0, 80.0]])
    w = np.array([1.0, 0.5, -1.0])
    g = oracle.adjoint(cfg, rec, 200.0, 12, w, scenario=0)

    def L(**kw):
        return float(w @ oracle.receptors(cfg, rec, 200.0, 12, scenario=0, **kw))

    h = 1e-2
    s = (sc.src_x, sc.src_y, sc.src_z)
    fd = np.array([
        (L(src=(s[0] + h, s[1], s[2])) - L(src=(s[0] - h, s[1], s[2]))) / (2 * h),
        (L(src=(s[0], s[1] + h, s[2])) - L(src=(s[0], s[1] - h, s[2]))) / (2 * h),
        (L(src=(s[0], s[1], s[2] + h)) - L(src=(s[0], s[1], s[2] - h))) / (2 * h),
        (L(bias=(1e-3, 0)) - L(bias=(-1e-3, 0))) / 2e-3,
        (L(bias=(0, 1e-3)) - L(bias=(0, -1e-3))) / 2e-3,
    ])
    got = np.concatenate([g[:3], g[-2:]])
    assert np.abs(fd).max() > 0
    np.testing.assert_allclose(got, fd, atol=0.02 * np.abs(fd).max())
