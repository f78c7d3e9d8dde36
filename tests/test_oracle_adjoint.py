"""Pins of the oracle's receptor concentration and its adjoint gradient.

- central finite differences of the oracle forward with the same seeds (common random
  numbers), uniform and realistic weather;
- the analytic gradient of the expected receptor concentration for uniform weather
  (Gaussian puffs with the ground image), within Monte-Carlo error;
- exact structure: linearity in the emission series, zero gradient for emission hours
  after the run, the uniform-weather Jacobian.
"""
import dataclasses
import math

import numpy as np
import pytest

import lpm_inputs as li
import oracle

SIGMA = 200.0


def _uniform_cfg(n=2000, steps=120, u=5.0, kh=50.0, kz=10.0, q=None):
    cfg = li.make_cfg0(n_particles=n, n_steps=steps, u=u, kh=kh, kz=kz)
    if q is not None:
        cfg = dataclasses.replace(cfg, release=dataclasses.replace(cfg.release, q=np.asarray(q),
                                                                    q_dt=300.0))
    return cfg


REC = np.array([[2000.0, 0.0, 2.0], [2500.0, 300.0, 10.0], [1500.0, -200.0, 40.0],
                [3000.0, 150.0, 80.0]])
W = np.array([1.0, -0.5, 2.0, 0.7])


def _loss(cfg, every, **kw):
    return float(W @ oracle.receptors(cfg, REC, SIGMA, every, **kw))


def _fd(cfg, every, base_src, h=1e-3):
    x, y, z = base_src
    fd = [(_loss(cfg, every, src=(x + h, y, z)) - _loss(cfg, every, src=(x - h, y, z))) / (2 * h),
          (_loss(cfg, every, src=(x, y + h, z)) - _loss(cfg, every, src=(x, y - h, z))) / (2 * h),
          (_loss(cfg, every, src=(x, y, z + h)) - _loss(cfg, every, src=(x, y, z - h))) / (2 * h)]
    q0 = np.asarray(cfg.release.q, dtype=float)
    for i in range(q0.size):
        qp, qm = q0.copy(), q0.copy()
        qp[i] += h
        qm[i] -= h
        fd.append((_loss(cfg, every, q=qp) - _loss(cfg, every, q=qm)) / (2 * h))
    fd.append((_loss(cfg, every, k_scale=1 + h) - _loss(cfg, every, k_scale=1 - h)) / (2 * h))
    fd.append((_loss(cfg, every, bias=(h, 0)) - _loss(cfg, every, bias=(-h, 0))) / (2 * h))
    fd.append((_loss(cfg, every, bias=(0, h)) - _loss(cfg, every, bias=(0, -h))) / (2 * h))
    return np.array(fd)


def test_adjoint_matches_central_fd_uniform_weather():
    """Uniform weather: the step is affine in the state, so the pathwise gradient equals
    the finite difference up to the rare reflections that switch under the perturbation
    (catches a wrong sign of the fold, a missing sqrt(s_K) factor, a wrong sample)."""
    cfg = _uniform_cfg(q=[1.0, 2.0, 0.5, 1.5])
    g = oracle.adjoint(cfg, REC, SIGMA, 10, W)
    fd = _fd(cfg, 10, (cfg.src_x, cfg.src_y, cfg.src_z))
    scale = np.abs(fd).max()
    np.testing.assert_allclose(g, fd, rtol=2e-3, atol=1e-4 * scale)


def test_adjoint_matches_central_fd_realistic_weather():
    """Sheared, perturbed, height-dependent weather (no deposition or exit): the
    interpolation kinks at cell faces make the finite difference a slightly different
    average, so the bar is 2 % of the largest component."""
    base = li.make_cfg1(n_particles=600, n_steps=120, n_hours=3, with_rain=False)
    cfg = dataclasses.replace(base, vd_dry=0.0, lateral_exit=0, half_life_s=3600.0,
                              release=li.Release(600, np.array([1.0, 3.0]), 1800.0, 0, 120))
    rec = np.array([[9000.0, 24875.0, 2.0], [12000.0, 25500.0, 30.0], [7000.0, 24000.0, 80.0]])
    w = np.array([1.0, 0.5, -1.0])
    g = oracle.adjoint(cfg, rec, SIGMA, 12, w)

    def L(**kw):
        return float(w @ oracle.receptors(cfg, rec, SIGMA, 12, **kw))

    h = 1e-2
    s = (cfg.src_x, cfg.src_y, cfg.src_z)
    fd = np.array([
        (L(src=(s[0] + h, s[1], s[2])) - L(src=(s[0] - h, s[1], s[2]))) / (2 * h),
        (L(src=(s[0], s[1] + h, s[2])) - L(src=(s[0], s[1] - h, s[2]))) / (2 * h),
        (L(src=(s[0], s[1], s[2] + h)) - L(src=(s[0], s[1], s[2] - h))) / (2 * h),
        (L(k_scale=1 + 1e-3) - L(k_scale=1 - 1e-3)) / 2e-3,
        (L(bias=(1e-3, 0)) - L(bias=(-1e-3, 0))) / 2e-3,
        (L(bias=(0, 1e-3)) - L(bias=(0, -1e-3))) / 2e-3,
    ])
    got = np.concatenate([g[:3], g[-3:]])
    np.testing.assert_allclose(got, fd, atol=0.02 * np.abs(fd).max())


def _expected_loss(theta, cfg, every, rec, w):
    """E[sum_r w_r C_r] for uniform wind u and constant K: cohort j (mass q dt) at age
    tau is a Gaussian puff N(x_s + (u + b_u) tau, 2 s_K K_h tau) x N(y_s + b_v tau, ...)
    x reflected N(h, 2 s_K K_z tau); convolved with the receptor kernel (width s) each
    axis becomes a Gaussian of variance 2 s_K K tau + s^2 and the image terms add."""
    xs, ys, h, sk, bu, bv = theta
    u, kh, kz = 5.0, 50.0, 10.0
    S, dt = cfg.n_steps, cfg.dt
    n_s = S // every
    tot = 0.0

    def nrm(d, var):
        return np.exp(-d * d / (2 * var)) / np.sqrt(2 * np.pi * var)

    for k in range(S):
        if (k + 1) % every:
            continue
        j = np.arange(k + 1)
        tau = (k + 1 - j) * dt
        vh = 2 * sk * kh * tau + SIGMA ** 2
        vz = 2 * sk * kz * tau + SIGMA ** 2
        for r in range(rec.shape[0]):
            xr, yr, zr = rec[r]
            e = (nrm(xr - xs - (u + bu) * tau, vh) * nrm(yr - ys - bv * tau, vh) *
                 (nrm(h - zr, vz) + nrm(h + zr, vz)))
            tot += w[r] * np.sum(1.0 * dt * e) / n_s
    return tot


def test_adjoint_matches_analytic_plume_gradient():
    """Monte-Carlo pathwise gradient (100k particles, same seeds) against the exact
    gradient of the expected loss, within 5 standard errors from interleaved batches
    (catches a biased estimator: e.g. a missing image term or a wrong mass)."""
    n, S, every = 100_000, 60, 6
    cfg = _uniform_cfg(n=n, steps=S)
    rec = np.array([[900.0, 0.0, 2.0], [1200.0, 250.0, 60.0], [600.0, -150.0, 25.0]])
    w = np.array([1.0, 1.5, -0.8])
    B = 20
    per = []
    for b in range(B):
        sel = np.arange(b, n, B)
        g = oracle.adjoint(cfg, rec, SIGMA, every, w, sel=sel)
        per.append(B * np.concatenate([g[:3], g[-3:]]))
    per = np.array(per)
    mc = per.mean(axis=0)
    se = per.std(axis=0, ddof=1) / math.sqrt(B)
    theta = np.array([0.0, 0.0, 50.0, 1.0, 0.0, 0.0])
    exact = []
    for i in range(6):
        hstep = 1e-3 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += hstep
        tm[i] -= hstep
        exact.append((_expected_loss(tp, cfg, every, rec, w) -
                      _expected_loss(tm, cfg, every, rec, w)) / (2 * hstep))
    exact = np.array(exact)
    assert np.all(np.abs(mc - exact) < 5 * se + 1e-3 * np.abs(exact).max()), (mc, exact, se)


def test_emission_gradient_linear_and_zero_after_the_run():
    """C is linear in q, so dL/dq_h = L(q = e_h); hours after the run have zero gradient."""
    cfg = _uniform_cfg(n=500, steps=60, q=[1.0, 2.0, 0.5, 1.5, 3.0])   # 300 s bins, 600 s run
    g = oracle.adjoint(cfg, REC, SIGMA, 6, W)
    nq = 5
    for hq in range(nq):
        e = np.zeros(nq)
        e[hq] = 1.0
        assert g[3 + hq] == pytest.approx(_loss(cfg, 6, q=e), rel=1e-12, abs=1e-300)
    assert g[3 + 2] == 0.0 and g[3 + 3] == 0.0 and g[3 + 4] == 0.0
    q = np.asarray(cfg.release.q)
    assert float(g[3:3 + nq] @ q) == pytest.approx(_loss(cfg, 6), rel=1e-12)


def test_sensitivity_uniform_and_fd():
    """Uniform weather: every step Jacobian is diag(1, 1, +-1), so the horizontal and
    vertical growth factors are exactly sqrt(2) and 1. Realistic weather: the growth of a
    perturbation of the release height (a finite difference of the final position) never
    exceeds the reported vertical factor."""
    cfg = _uniform_cfg(n=300, steps=50)
    s = oracle.sensitivity(cfg)
    np.testing.assert_allclose(s[:, 0], math.sqrt(2.0), rtol=1e-12)
    np.testing.assert_allclose(s[:, 1], 1.0, rtol=1e-12)
    # realistic weather: the growth of a vertical perturbation from the release step is
    # bounded by the reported maximum; check it against a finite difference of the source
    base = li.make_cfg1(n_particles=40, n_steps=60, n_hours=2, with_rain=False)
    cfg = dataclasses.replace(base, vd_dry=0.0, lateral_exit=0)
    s = oracle.sensitivity(cfg, n_run=60)
    assert np.all(s >= 1.0) and np.all(np.isfinite(s))
    h = 1e-6
    a = oracle.run(cfg, src=(cfg.src_x, cfg.src_y, cfg.src_z + h))["pos"]
    b = oracle.run(cfg, src=(cfg.src_x, cfg.src_y, cfg.src_z - h))["pos"]
    growth = np.linalg.norm(a - b, axis=1) / (2 * h)
    assert np.all(growth <= s[:, 1] * (1 + 1e-3) + 1e-6)
