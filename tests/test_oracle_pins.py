"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No expected value here comes from the CUDA path; every check is a closed form, an exact
invariant, a distributional law of the discrete scheme, or brute force on a tiny case.
Each test names the plausible oracle mistakes it would catch.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import stats

import lpm_inputs as li
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------------------------------------
# Counter-based generator (replaces the Mersenne Twister of Sec. 2 / Sec. 3.2)
# ------------------------------------------------------------------------------------
def _bits(a):
    return np.unpackbits(np.ascontiguousarray(a, dtype=">u4").view(np.uint8)).reshape(
        a.shape[0], -1)


def test_philox_uniform_bytes_chi2():
    """Every byte lane of every output word is uniform (catches a dropped round or a
    stuck/duplicated output word)."""
    w = oracle.draws(7, np.arange(1 << 16), 3, 0)
    for col in range(4):
        for shift in (0, 8, 16, 24):
            b = (w[:, col] >> shift) & 0xFF
            cnt = np.bincount(b, minlength=256)
            chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
            assert stats.chi2.sf(chi2, 255) > 1e-4, (col, shift, chi2)


def test_philox_avalanche_counter_and_key():
    """Flipping any single bit of the counter or the key flips each output bit with
    probability 1/2 (catches fewer than 10 rounds, a missing key mix or a word that
    bypasses the multipliers)."""
    rng = np.random.default_rng(0)
    n = 400
    base_ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    base_key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    ref = np.array([oracle.philox(k, c) for k, c in zip(base_key, base_ctr)], dtype=np.uint32)
    rb = _bits(ref)
    for word in range(6):
        for bit in (0, 13, 31):
            ctr = base_ctr.copy()
            key = base_key.copy()
            if word < 4:
                ctr[:, word] ^= (1 << bit)
            else:
                key[:, word - 4] ^= (1 << bit)
            out = np.array([oracle.philox(k, c) for k, c in zip(key, ctr)], dtype=np.uint32)
            frac = (rb != _bits(out)).mean(axis=0)          # per output bit
            assert np.all(np.abs(frac - 0.5) < 0.13), (word, bit, frac.min(), frac.max())
            assert abs(frac.mean() - 0.5) < 0.01


_TRITON_PHILOX = r"""
import json, sys
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def philox_rows(seed, ctr_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(ctr_ptr + 4 * i), tl.load(ctr_ptr + 4 * i + 1),
                               tl.load(ctr_ptr + 4 * i + 2), tl.load(ctr_ptr + 4 * i + 3))
    tl.store(out_ptr + 4 * i, r0)
    tl.store(out_ptr + 4 * i + 1, r1)
    tl.store(out_ptr + 4 * i + 2, r2)
    tl.store(out_ptr + 4 * i + 3, r3)

res = []
for seed, ctr in json.load(sys.stdin):
    ctr = np.ascontiguousarray(np.array(ctr, dtype=np.uint32))
    out = torch.empty(ctr.shape, dtype=torch.int32)
    philox_rows[(1,)](seed, torch.from_numpy(ctr.view(np.int32)), out, N=ctr.shape[0])
    res.append(out.numpy().view(np.uint32).tolist())
print(json.dumps(res))
"""


def test_philox_matches_an_independent_library_implementation():
    """Bit identity with Triton's own Philox4x32-10 (``tl.philox``, 10 rounds, key = the
    seed's low and high 32-bit halves), run by Triton's CPU interpreter in a child process
    (the interpreter must be chosen before Triton is imported): a second implementation of
    the SC'11 generator written by other people. Catches swapped multipliers or Weyl
    constants, a wrong round count, swapped key halves, a word permutation in the round and
    a dropped high or low product half, none of which the statistical pins above need to
    see."""
    pytest.importorskip("triton")
    import json
    import os
    import subprocess
    import sys

    n = 64
    edge = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]], np.uint32)
    rand = np.random.default_rng(3).integers(0, 2 ** 32, (n - len(edge), 4), dtype=np.uint64)
    ctr = np.vstack([edge, rand.astype(np.uint32)])
    seeds = (0, 1, 7, 0x0123456789ABCDEF, (1 << 63) - 1, (1 << 64) - 1)
    # the particle draw puts (particle id low, high, step, stream) in the counter
    pid = np.array([0, 1, 123456789, (1 << 40) + 5], dtype=np.uint64)
    draw_seed, step, stream = 0x0123456789ABCDEF, 77, 1
    draw_ctr = np.stack([pid & 0xFFFFFFFF, pid >> 32, np.full(4, step), np.full(4, stream)],
                        1).astype(np.uint32)
    jobs = [[s, ctr.tolist()] for s in seeds] + [[draw_seed, draw_ctr.tolist()]]
    env = dict(os.environ, TRITON_INTERPRET="1")
    run = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(jobs),
                         capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stderr[-2000:]
    lib = [np.array(r, dtype=np.uint32) for r in json.loads(run.stdout.splitlines()[-1])]
    for seed, got in zip(seeds, lib):
        ours = np.array([oracle.philox([seed & 0xFFFFFFFF, seed >> 32], c) for c in ctr],
                        dtype=np.uint32)
        np.testing.assert_array_equal(ours, got, err_msg=hex(seed))
    np.testing.assert_array_equal(oracle.draws(draw_seed, pid, step, stream), lib[-1])


def test_philox_no_collisions_and_streams_independent():
    """Distinct counters give distinct outputs (the round is a bijection), and the
    deposition stream is uncorrelated with the displacement stream."""
    pid = np.arange(200_000)
    w0 = oracle.draws(1, pid, 5, 0)
    w1 = oracle.draws(1, pid, 5, 1)
    as_int = [tuple(r) for r in w0[:50_000]]
    assert len(set(as_int)) == len(as_int)
    u0 = w0[:, 0].astype(np.float64)
    u1 = w1[:, 0].astype(np.float64)
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 5 / math.sqrt(pid.size)
    # consecutive steps of one particle are uncorrelated too
    ws = oracle.draws(1, np.full(100_000, 12345), np.arange(100_000), 0)
    a = ws[:-1, 1].astype(np.float64)
    b = ws[1:, 1].astype(np.float64)
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(a.size)


def test_uniform_mapping_closed_form():
    """u = (2*(w>>9)+1)*2^-24: endpoints, symmetry and exactness."""
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.uniform(1 << 9) == 3 * 2.0 ** -24
    for w in (0, 511, 512, 0x80000000, 0xDEADBEEF):
        u = oracle.uniform(w)
        assert oracle.uniform(w ^ 0xFFFFFE00) == pytest.approx(1.0 - u, abs=0.0)
        assert np.float32(u) == u                      # exactly representable in FP32


def test_box_muller_normals_law():
    """N(0,1): moments, KS against the normal CDF, zero correlation between the three
    components, and the bound |n| <= sqrt(2 ln 2^24) from the smallest uniform."""
    n = oracle.normals(42, np.arange(150_000), 17)
    assert np.abs(n).max() <= math.sqrt(2 * 24 * math.log(2)) + 1e-12
    for c in range(3):
        x = n[:, c]
        assert abs(x.mean()) < 5 / math.sqrt(x.size)
        assert abs(x.var() - 1) < 5 * math.sqrt(2 / x.size)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    cc = np.corrcoef(n.T)
    assert np.all(np.abs(cc - np.eye(3)) < 5 / math.sqrt(n.shape[0]))
    # n0, n1 share a radius: n0^2+n1^2 is exactly -2 ln u0 ~ Exp(1/2)
    r2 = n[:, 0] ** 2 + n[:, 1] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-4


# ------------------------------------------------------------------------------------
# Release schedule and mass assignment (Sec. 3.2)
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,first,last", [(10_000, 0, 360), (7, 3, 10), (1000, 5, 2880),
                                          (360, 0, 360), (12345, 0, 1)])
def test_release_schedule_counts(n, first, last):
    p = np.arange(n)
    s = oracle.release_steps(n, first, last, p)
    assert s[0] == first and np.all(np.diff(s) >= 0) and s[-1] < last
    direct = np.bincount(s - first, minlength=last - first)
    counts = np.array([oracle.release_count(n, first, last, first + j)
                       for j in range(last - first)])
    assert np.array_equal(direct, counts)
    assert counts.sum() == n
    if n >= last - first:
        assert counts.max() - counts.min() <= 1
    assert oracle.release_count(n, first, last, last) == 0
    assert oracle.release_count(n, first, last, first - 1) == 0


def test_total_mass_and_fixed_shift():
    cfg = li.make_cfg0()
    assert oracle.total_mass(cfg) == pytest.approx(3600.0, rel=1e-15)   # q=1 over 3600 s
    sh = oracle.fixed_shift(cfg)
    assert 3600.0 * 2.0 ** sh < 2.0 ** 61 <= 2 * 3600.0 * 2.0 ** sh


# ------------------------------------------------------------------------------------
# 4D linear interpolation (Sec. 3.2)
# ------------------------------------------------------------------------------------
def _linear_met(nx=7, ny=5, nz=6, nt=3, coef=(1.5, 0.01, -0.02, 0.3, 1e-4)):
    z_levels = li.z_levels_stretched(nz, 1200.0)
    x = -500.0 + 100.0 * np.arange(nx)
    y = 200.0 + 150.0 * np.arange(ny)
    t = 60.0 + 900.0 * np.arange(nt)
    T, Z, Y, X = np.meshgrid(t, z_levels, y, x, indexing="ij")
    a, bx, by, bz, bt = coef
    uvwk = np.empty((nt, nz, ny, nx, 4), np.float64)
    uvwk[..., 0] = a + bx * X + by * Y + bz * Z + bt * T
    uvwk[..., 1] = -a + 2 * bx * X - by * Y
    uvwk[..., 2] = 0.1 * bz * Z - bt * T
    uvwk[..., 3] = 5.0 + 0.01 * Z + 0.001 * X
    kh = (50.0 + 0.02 * X + 0.03 * Y + 0.01 * Z).astype(np.float32)
    cfg = li.make_cfg0()
    cfg = dataclasses.replace(cfg, nx=nx, ny=ny, nz=nz, x0=-500.0, y0=200.0, dx=100.0,
                              dy=150.0, z_levels=z_levels, n_met_t=nt, met_t0=60.0,
                              met_dt=900.0, uvwk=uvwk.astype(np.float32), kh=kh,
                              kh_uniform=-1.0)
    return cfg, coef


def test_interp_reproduces_linear_fields():
    """A field linear in x, y, z and t is reproduced exactly anywhere inside the grid
    (catches swapped axes, a wrong weight complement, an off-by-one cell or a wrong
    level search)."""
    cfg, (a, bx, by, bz, bt) = _linear_met()
    rng = np.random.default_rng(3)
    n = 2000
    pts = np.stack([rng.uniform(-500, 100, n), rng.uniform(200, 800, n),
                    rng.uniform(0, 1200, n), rng.uniform(60, 1860, n)], axis=1)
    X, Y, Z, T = pts.T
    got = oracle.interp(cfg, pts)
    # the float32 node values carry ~1e-7 relative rounding
    np.testing.assert_allclose(got[:, 0], a + bx * X + by * Y + bz * Z + bt * T, rtol=1e-6,
                               atol=1e-5)
    np.testing.assert_allclose(got[:, 1], -a + 2 * bx * X - by * Y, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(got[:, 2], 0.1 * bz * Z - bt * T, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(got[:, 3], 5.0 + 0.01 * Z + 0.001 * X, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(got[:, 4], 50.0 + 0.02 * X + 0.03 * Y + 0.01 * Z, rtol=1e-6,
                               atol=1e-5)
    np.testing.assert_allclose(got[:, 5], 0.01, rtol=1e-4)      # dK_z/dz


def test_interp_nodes_and_clamping():
    """Node values are returned exactly at nodes (ties go to the upper cell) and the
    field is extended as a constant beyond the grid."""
    cfg, _ = _linear_met()
    node = (2, 3, 4, 1)   # (i, j, k, h)
    x = cfg.x0 + node[0] * cfg.dx
    y = cfg.y0 + node[1] * cfg.dy
    z = cfg.z_levels[node[2]]
    t = cfg.met_t0 + node[3] * cfg.met_dt
    got = oracle.interp(cfg, [[x, y, z, t]])[0]
    want = cfg.uvwk[node[3], node[2], node[1], node[0]].astype(np.float64)
    np.testing.assert_array_equal(got[:4], want)
    # beyond the last node: clamped to the edge
    far = oracle.interp(cfg, [[1e6, -1e6, 1e5, 1e7]])[0]
    edge = cfg.uvwk[-1, -1, 0, -1].astype(np.float64)
    np.testing.assert_array_equal(far[:4], edge)
    assert far[5] == 0.0          # no vertical derivative above the top level


# ------------------------------------------------------------------------------------
# The random walk: closed forms of the discrete scheme (Eq. 1-2, uniform weather)
# ------------------------------------------------------------------------------------
def _pit_uniform(u):
    return stats.kstest(u, "uniform").pvalue


def test_uniform_weather_exact_laws():
    """With uniform wind u and constant K, after age tau = m*dt (sums of Gaussian steps):
    x - x_s ~ N(u tau, 2 K_h tau), y - y_s ~ N(0, 2 K_h tau), and the reflected chain
    z_{k+1} = |z_k + xi| has exactly the image-source law |h + N(0, 2 K_z tau)|.
    Probability-integral transforms of all particles must be uniform (catches a wrong
    factor in sqrt(2 K dt), a sign error, a missing reflection or a wrong time step)."""
    cfg = li.make_cfg0(n_particles=20_000, n_steps=120)
    r = oracle.run(cfg)
    tau = (cfg.n_steps - r["release"]) * cfg.dt
    x, y, z = r["pos"].T
    sx = np.sqrt(2 * 50.0 * tau)
    sz = np.sqrt(2 * 10.0 * tau)
    assert _pit_uniform(stats.norm.cdf((x - 5.0 * tau) / sx)) > 1e-3
    assert _pit_uniform(stats.norm.cdf(y / sx)) > 1e-3
    h = 50.0
    Fz = stats.norm.cdf((z - h) / sz) - stats.norm.cdf((-z - h) / sz)
    assert _pit_uniform(Fz) > 1e-3
    assert np.all(z >= 0)
    assert np.all(r["status"] == li.STATUS_ACTIVE)
    assert r["active_steps"] == int(tau.sum() / cfg.dt)


def _cell_prob(edges, mean, sd):
    c = stats.norm.cdf((edges - mean[:, None]) / sd[:, None])
    return np.diff(c, axis=1)


def test_cfg0_concentration_matches_cell_integrated_plume():
    """The binned field equals in expectation the cell-integrated puff sum
    E[mass in cell] = sum_cohorts n_j m0 P_x P_y P_z (image source for z); a chi-square
    statistic over well-populated cells must be consistent with sampling noise."""
    n = 200_000
    cfg = li.make_cfg0(n_particles=n)
    r = oracle.run(cfg)
    S, dt = cfg.n_steps, cfg.dt
    j = np.arange(S)
    counts = np.array([oracle.release_count(n, 0, S, s) for s in j])
    m0 = 1.0 * dt / counts                                 # q = 1
    tau = (S - j) * dt
    ex = cfg.cx0 + cfg.cdx * np.arange(cfg.cx + 1)
    ey = cfg.cy0 + cfg.cdy * np.arange(cfg.cy + 1)
    ez = cfg.cz0 + cfg.cdz * np.arange(cfg.cz + 1)
    sh = np.sqrt(2 * 50.0 * tau)
    sz = np.sqrt(2 * 10.0 * tau)
    Px = _cell_prob(ex, cfg.src_x + 5.0 * tau, sh)
    Py = _cell_prob(ey, np.full(S, cfg.src_y), sh)
    Pz = _cell_prob(ez, np.full(S, cfg.src_z), sz) + _cell_prob(-ez[::-1], np.full(S, cfg.src_z),
                                                               sz)[:, ::-1]
    # expected particle counts and mass per cell
    npart = np.einsum("s,sx,sy,sz->zyx", counts.astype(float), Px, Py, Pz)
    emass = np.einsum("s,sx,sy,sz->zyx", counts * m0, Px, Py, Pz)
    emass2 = np.einsum("s,sx,sy,sz->zyx", counts * m0 ** 2, Px, Py, Pz)
    sel = npart >= 10
    assert sel.sum() > 400
    chi2 = ((r["conc"][sel] - emass[sel]) ** 2 / emass2[sel]).sum()
    nu = sel.sum()
    assert abs(chi2 / nu - 1.0) < 6 * math.sqrt(2.0 / nu), chi2 / nu
    # total mass in the grid equals the exact airborne-in-grid budget
    assert r["conc"].sum() == pytest.approx(r["budget"][1], rel=1e-10)


def test_deterministic_paths_reflection_and_exit():
    """K = 0 removes the random walk: positions follow the closed form, reflections
    fold at the ground and the top, and the lateral exit happens at the predicted
    step (catches a reflection sign error, the wrong fold order, an exit off by one)."""
    def one(w, n_run, **kw):
        uvwk, z_levels = li.make_artificial_weather(u=7.0, w=w, kz=0.0, z_top=1000.0)
        cfg = li.make_cfg0(n_particles=1, n_steps=100, kh=0.0, kz=0.0)
        cfg = dataclasses.replace(cfg, uvwk=uvwk, z_levels=z_levels, x0=-1000.0, dx=5000.0,
                                  y0=-5000.0, dy=10000.0, src_z=50.0, reflect_top=1,
                                  z_top=80.0, **kw)
        return oracle.run(cfg, n_run=n_run)

    # ground: 50 -> 20 -> |-10| = 10 -> |-20| = 20 -> 10 (hand-computed, dt = 10 s)
    for n_run, z in [(1, 20.0), (2, 10.0), (3, 20.0), (4, 10.0)]:
        r = one(-3.0, n_run)
        assert r["pos"][0, 2] == pytest.approx(z, abs=1e-9)
        assert r["pos"][0, 0] == pytest.approx(70.0 * n_run, abs=1e-9)
    # top at 80 m: 50 -> 90 -> 160-90 = 70 ... with w = +4: 50, 90->70, 110->50, 90->70
    for n_run, z in [(1, 70.0), (2, 50.0), (3, 70.0)]:
        assert one(4.0, n_run)["pos"][0, 2] == pytest.approx(z, abs=1e-9)
    # a step longer than the column folds more than once: w = -25 from 50 m:
    # 50-250 = -200 -> 200 -> 2*80-200 = -40 -> 40
    assert one(-25.0, 1)["pos"][0, 2] == pytest.approx(40.0, abs=1e-9)
    # x_hi = -1000 + 5000 = 4000; from x = 0 at 70 m per step the particle first lies
    # beyond 4000 m after step k with 70*(k+1) > 4000, i.e. k = 57 (58 steps taken)
    re = one(0.0, 100, lateral_exit=1)
    assert re["status"][0] == li.STATUS_EXITED
    assert re["pos"][0, 0] == pytest.approx(70.0 * 58, abs=1e-9)
    assert re["active_steps"] == 58
    assert re["budget"][5] == pytest.approx(10.0, rel=1e-15)   # all of the mass exited


def test_decay_total_closed_form():
    """Without deposition the airborne mass after S steps is exactly
    sum_j q dt exp(-lambda (S - j) dt) (deterministic decay from the time since
    emission, Sec. 3.2); the budget identity holds to rounding."""
    cfg = li.make_cfg0(n_particles=5000, n_steps=200)
    cfg = dataclasses.replace(cfg, half_life_s=1800.0)
    r = oracle.run(cfg)
    lam = math.log(2) / 1800.0
    j = np.arange(cfg.n_steps)
    want = np.sum(1.0 * cfg.dt * np.exp(-lam * (cfg.n_steps - j) * cfg.dt))
    b = r["budget"]
    assert b[1] + b[2] == pytest.approx(want, rel=1e-12)
    assert b[0] - b[6] == pytest.approx(b[1] + b[2] + b[3] + b[4] + b[5], rel=1e-12)
    assert b[0] == pytest.approx(cfg.n_steps * cfg.dt, rel=1e-12)


def _mixed_column(n, steps, vd=0.0, lam_wet=0.0, rain_value=1):
    uvwk, z_levels = li.make_artificial_weather(u=2.0, kz=50.0, z_top=500.0)
    cfg = li.make_cfg0(n_particles=n, n_steps=steps)
    rain = np.full((2, 2, 2), rain_value, np.uint8)
    return dataclasses.replace(cfg, uvwk=uvwk, z_levels=z_levels, reflect_top=1, z_top=500.0,
                               vd_dry=vd, h_mix=500.0 if vd > 0 else 0.0, wet_lambda=lam_wet,
                               rain=rain if lam_wet > 0 else None, half_life_s=3600.0)


def test_dry_deposition_binomial():
    """Inside a reflecting column capped at h_mix every step is a Bernoulli trial with
    p = 1 - exp(-v_d dt / h_mix): the deposited count is a sum of independent
    geometric-survival indicators (mean and variance known exactly)."""
    n, S = 20_000, 150
    cfg = _mixed_column(n, S, vd=0.5)
    r = oracle.run(cfg)
    p = 1 - math.exp(-0.5 * cfg.dt / 500.0)
    age = S - r["release"]
    q = 1 - (1 - p) ** age
    ndep = int((r["status"] == li.STATUS_DEP_DRY).sum())
    assert abs(ndep - q.sum()) < 5 * math.sqrt((q * (1 - q)).sum())
    assert not np.any(r["status"] == li.STATUS_DEP_WET)
    # the deposition grid holds the decayed mass at the deposition step
    b = r["budget"]
    assert r["dep"][0].sum() + 0.0 <= b[3] * (1 + 1e-12)
    assert b[0] - b[6] == pytest.approx(b[1] + b[2] + b[3] + b[4] + b[5], rel=1e-12)


def test_wet_deposition_binomial_and_rain_mask():
    n, S = 20_000, 150
    cfg = _mixed_column(n, S, lam_wet=2e-4)
    r = oracle.run(cfg)
    p = 1 - math.exp(-2e-4 * cfg.dt)
    age = S - r["release"]
    q = 1 - (1 - p) ** age
    ndep = int((r["status"] == li.STATUS_DEP_WET).sum())
    assert abs(ndep - q.sum()) < 5 * math.sqrt((q * (1 - q)).sum())
    dry = _mixed_column(n, S, lam_wet=2e-4, rain_value=0)
    r0 = oracle.run(dry)
    assert not np.any(r0["status"] == li.STATUS_DEP_WET)


def test_binning_brute_force_and_integer_identity():
    """Floor-index binning equals an O(N * cells) point-in-box enumeration; the
    fixed-point grid plus the out-of-grid counter equals the sum of the per-particle
    rounded masses exactly."""
    cfg = li.make_cfg0(n_particles=300, n_steps=60)
    cfg = dataclasses.replace(cfg, cx=12, cy=9, cz=5, cx0=-100.0, cy0=-400.0, cdx=40.0,
                              cdy=90.0, cdz=25.0, half_life_s=900.0)
    r = oracle.run(cfg)
    lam = math.log(2) / 900.0
    S = cfg.n_steps
    counts = {s: oracle.release_count(300, 0, S, s) for s in range(S)}
    m = np.array([cfg.dt / counts[s] * math.exp(-lam * (S - s) * cfg.dt) for s in r["release"]])
    grid = np.zeros((cfg.cz, cfg.cy, cfg.cx))
    for p in range(r["pos"].shape[0]):
        x, y, z = r["pos"][p]
        for k in range(cfg.cz):
            for jj in range(cfg.cy):
                for ii in range(cfg.cx):
                    x0 = cfg.cx0 + ii * cfg.cdx
                    y0 = cfg.cy0 + jj * cfg.cdy
                    z0 = cfg.cz0 + k * cfg.cdz
                    if x0 <= x < x0 + cfg.cdx and y0 <= y < y0 + cfg.cdy and z0 <= z < z0 + cfg.cdz:
                        grid[k, jj, ii] += m[p]
    np.testing.assert_allclose(r["conc"], grid, rtol=1e-13, atol=1e-15)
    sh = oracle.fixed_shift(cfg)
    fixed = np.array([int(np.rint(np.ldexp(v, sh))) for v in m], dtype=np.int64)
    assert int(r["conc_fixed"].sum()) + int(r["counters"][0]) == int(fixed.sum())


def test_drift_correction_well_mixed_condition():
    """K_z = K0 + K1 z in a reflecting column, no wind: the random walk of Eq. 2 (no drift)
    relaxes to the stationary law of dz = sqrt(2K) dW with zero-flux walls, density
    proportional to 1/K(z); adding (dK_z/dz) dt (drift_correction) gives the uniform,
    well-mixed state. KS tests pin both (catches a wrong sign, factor or missing drift)."""
    H, nz, K0, K1 = 100.0, 11, 10.0, 0.1
    z_levels = np.linspace(0.0, H, nz)
    uvwk = np.zeros((2, nz, 2, 2, 4), np.float32)
    uvwk[..., 3] = (K0 + K1 * z_levels)[None, :, None, None]
    res = {}
    for drift in (1, 0):
        cfg = li.make_cfg0(n_particles=8000, n_steps=2000, kh=0.0, kz=0.0, u=0.0,
                           src=(0.0, 0.0, 50.0))
        cfg = dataclasses.replace(cfg, uvwk=uvwk, z_levels=z_levels, nz=nz, dt=2.0,
                                  reflect_top=1, z_top=H, drift_correction=drift,
                                  release=li.Release(8000, np.array([1.0]), 3600.0, 0, 10))
        z = oracle.run(cfg)["pos"][:, 2]
        uniform = stats.kstest(z / H, "uniform").pvalue
        inv_k = stats.kstest(np.log((K0 + K1 * z) / K0) / np.log((K0 + K1 * H) / K0),
                             "uniform").pvalue
        res[drift] = (uniform, inv_k)
    assert res[1][0] > 1e-3 and res[1][1] < 1e-6, res
    assert res[0][1] > 1e-3 and res[0][0] < 1e-6, res


# ------------------------------------------------------------------------------------
# Time-integrated dosage (the post-processing of the n-th-step summations, Sec. 3.2)
# ------------------------------------------------------------------------------------
def test_dosage_total_closed_form():
    """In uniform weather with no lateral boundary, no deposition and a reflecting ground,
    every particle released at s_p <= k is airborne after step k, so the dosage summed
    over all cells plus the out-of-grid part is sum over the samples (k+1) % n == 0 of
    sum_{s_p <= k} round(m0(s_p) exp(-lambda (k+1-s_p) dt) 2^shift), with s_p and m0 from
    the release reading. Catches a sample taken at the wrong step, a missed sample, the
    mass of the wrong time, or a dropped out-of-grid part."""
    n_p, steps, every = 700, 90, 4
    cfg = dataclasses.replace(li.make_cfg0(n_particles=n_p, n_steps=steps), half_life_s=1800.0)
    r = oracle.run(cfg, dose_every=every)
    # fixed point of the dosage: the snapshot's shift less ceil(log2(S // n)) bits
    shift = oracle.fixed_shift(cfg) - math.ceil(math.log2(steps // every))
    lam = math.log(2.0) / 1800.0
    sp = (np.arange(n_p) * steps) // n_p                      # s_p = floor(p S / N)
    counts = np.bincount(sp, minlength=steps)
    want, samples = 0, 0
    for k in range(steps):
        if (k + 1) % every:
            continue
        samples += 1
        for s in sp[sp <= k]:
            m = (1.0 * cfg.dt / counts[s]) * math.exp(-lam * ((k + 1 - s) * cfg.dt))
            want += int(np.rint(math.ldexp(m, shift)))
    got = int(r["dose_fixed"].sum()) + r["dose_out"]
    assert r["dose_samples"] == samples == steps // every
    assert got == want < 2 ** 61


def test_dosage_is_the_sum_of_the_snapshots():
    """The dosage grid equals, cell by cell, the sum of the concentration snapshots taken
    at the same steps (each snapshot pinned separately against the plume law), and its
    out-of-grid part the sum of theirs. Catches a wrong cell index or a sample whose
    positions are not those of the snapshot at the same time."""
    every, steps = 5, 40                      # 8 samples: the dosage drops b = 3 bits
    base = dataclasses.replace(li.make_cfg0(n_particles=400, n_steps=steps), half_life_s=3600.0,
                               bin_every=every, cx=15)        # the plume leaves x > 500 m
    whole = oracle.run(base, dose_every=every)
    total = np.zeros_like(whole["dose"])
    out = 0.0
    for end in range(every, steps + 1, every):
        r = oracle.run(base, n_run=end)             # its last snapshot is at step end - 1
        total += r["conc"]
        out += r["budget"][2]                       # airborne mass outside the grid
    np.testing.assert_allclose(whole["dose"], total, rtol=1e-12, atol=0.0)
    # the fixed-point sums are the snapshots' on a scale 2^3 coarser
    shift = oracle.fixed_shift(base) - 3
    ulp = 2.0 ** -shift                             # each of <= 3200 terms rounds by <= ulp/2
    np.testing.assert_allclose(whole["dose_fixed"] * ulp, total, rtol=0.0, atol=1600 * ulp)
    assert out > 0
    assert whole["dose_out"] * ulp == pytest.approx(out, rel=0, abs=1600 * ulp)


# ------------------------------------------------------------------------------------
# K_z from Eq. 3 in the step (k u* z (1 - z/H_z)^2 / Phi_h(z/L), Sec. 2)
# ------------------------------------------------------------------------------------
def test_kz_eq3_closed_forms():
    """Neutral (1/L = 0): K_z = k u* z (1 - z/H)^2 with its maximum 4 k u* H / 27 at
    z = H/3; stable and unstable layers scale it by 1/(1 + 5 z/L) and (1 - 16 z/L)^(1/2);
    zero (then the floor) at and above H_z and at the ground. Catches a wrong von Karman
    constant, exponent, sign of the stability correction or a missing cut at H_z."""
    k, u, H, kmin = 0.4, 0.37, 900.0, 1e-3
    kz, dkz = oracle.kz_eq3(u, 0.0, H, kmin, H / 3.0)
    assert kz == pytest.approx(4.0 * k * u * H / 27.0, rel=1e-12)
    assert abs(dkz) < 1e-9
    rng = np.random.default_rng(5)
    for z in rng.uniform(1.0, H - 1.0, 20):
        neutral = k * u * z * (1.0 - z / H) ** 2
        assert oracle.kz_eq3(u, 0.0, H, kmin, z)[0] == pytest.approx(max(kmin, neutral),
                                                                      rel=1e-12)
        for inv_l in (0.004, 0.02):
            assert oracle.kz_eq3(u, inv_l, H, kmin, z)[0] == pytest.approx(
                max(kmin, neutral / (1.0 + 5.0 * z * inv_l)), rel=1e-12)
            assert oracle.kz_eq3(u, -inv_l, H, kmin, z)[0] == pytest.approx(
                max(kmin, neutral * math.sqrt(1.0 + 16.0 * z * inv_l)), rel=1e-12)
    for z in (H, H + 50.0, 0.0):
        assert oracle.kz_eq3(u, 0.0, H, 0.25, z) == (0.25, 0.0)


def test_kz_eq3_derivative_against_differences():
    """dK_z/dz (the drift term) against central differences of K_z, in stable, neutral
    and unstable layers. Catches a dropped product-rule term or a wrong Phi_h derivative."""
    rng = np.random.default_rng(6)
    for _ in range(60):
        u = rng.uniform(0.1, 0.8)
        inv_l = rng.uniform(-0.04, 0.04)
        H = rng.uniform(300.0, 2000.0)
        z = rng.uniform(0.02, 0.98) * H
        if abs(z * inv_l) < 1e-6:
            continue
        h = 1e-4 * H
        fd = (oracle.kz_eq3(u, inv_l, H, 0.0, z + h)[0] -
              oracle.kz_eq3(u, inv_l, H, 0.0, z - h)[0]) / (2 * h)
        # central-difference truncation ~ h^2 K'''/6 ~ 1e-8 k u*
        assert oracle.kz_eq3(u, inv_l, H, 0.0, z)[1] == pytest.approx(fd, rel=1e-6,
                                                                       abs=1e-7 * 0.4 * u)


def _bl_column(u, inv_l, H, n_t=2, nx=2, ny=2):
    bl = np.zeros((n_t, ny, nx, 4), np.float32)
    bl[..., 0], bl[..., 1], bl[..., 2] = u, inv_l, H
    return bl


def test_kz_eq3_columns_interpolated_like_the_weather():
    """With 1/L = 0, K_z is linear in u*: a u* field linear in x, y and t must give
    K_z = k u*(x, y, t) z (1 - z/H)^2 exactly (bilinear-in-space, linear-in-time
    interpolation of the columns)."""
    cfg = li.make_cfg0(n_particles=10, n_steps=10)
    bl = _bl_column(0.0, 0.0, 800.0)
    a0, ax, ay, at = 0.3, 1e-5, -2e-5, 3e-6
    for h in range(2):
        for j in range(2):
            for i in range(2):
                bl[h, j, i, 0] = a0 + ax * (cfg.x0 + i * cfg.dx) + ay * (cfg.y0 + j * cfg.dy) \
                    + at * (cfg.met_t0 + h * cfg.met_dt)
    cfg = dataclasses.replace(cfg, kz_model=1, kz_min=0.0, bl=bl)
    rng = np.random.default_rng(7)
    pts = np.stack([rng.uniform(cfg.x0, cfg.x0 + cfg.dx, 50), rng.uniform(cfg.y0, cfg.y0 + cfg.dy, 50),
                    rng.uniform(1.0, 799.0, 50), rng.uniform(0.0, cfg.met_dt, 50)], axis=1)
    got = oracle.interp(cfg, pts)
    ustar = (a0 + ax * pts[:, 0] + ay * pts[:, 1] + at * pts[:, 3]).astype(np.float32)
    # the columns hold float32 values; compare with the float32-rounded field tolerance
    want = 0.4 * ustar.astype(np.float64) * pts[:, 2] * (1.0 - pts[:, 2] / 800.0) ** 2
    np.testing.assert_allclose(got[:, 3], want, rtol=2e-6)


@pytest.mark.parametrize("inv_l", [0.0, 0.02, -0.02])
def test_kz_eq3_drift_keeps_a_column_well_mixed(inv_l):
    """A reflecting 100 m column under Eq. 3 (K_z from ~0 at the ground): with the drift
    term the uniform state is stationary (KS uniform); in the neutral case the walk
    without it piles particles up where K_z is small (rejected)."""
    H = 100.0
    cfg = li.make_cfg0(n_particles=8000, n_steps=2000, kh=0.0, kz=0.0, u=0.0, src=(0.0, 0.0, 50.0))
    cfg = dataclasses.replace(cfg, dt=2.0, reflect_top=1, z_top=H, kz_model=1, kz_min=0.1,
                              bl=_bl_column(0.5, inv_l, 1000.0),
                              release=li.Release(8000, np.array([1.0]), 3600.0, 0, 10))
    for drift in ((1, 0) if inv_l == 0.0 else (1,)):
        z = oracle.run(dataclasses.replace(cfg, drift_correction=drift))["pos"][:, 2]
        p = stats.kstest(z / H, "uniform").pvalue
        if drift:
            assert p > 1e-3, p
        else:
            assert p < 1e-6, p


def test_kz_eq3_gradient_of_the_tangent_linear_model():
    """The x, y, z gradient of K_z that the tangent-linear model (adjoint, sensitivity)
    uses, against central differences of the interpolated Eq. 3 K_z on the realistic
    boundary-layer columns. Catches a missing chain-rule term through u*, 1/L or H_z."""
    cfg = li.make_cfg1(n_particles=10, n_steps=240, n_hours=3, kz_eq3=True)
    cfg = dataclasses.replace(cfg, kz_min=0.0)
    rng = np.random.default_rng(8)
    n = 200
    pts = np.stack([rng.uniform(1000.0, 48000.0, n), rng.uniform(1000.0, 48000.0, n),
                    rng.uniform(5.0, 300.0, n), rng.uniform(0.0, 7000.0, n)], axis=1)
    val, grad = oracle.interp_grad(cfg, pts)
    np.testing.assert_allclose(val[:, 3], oracle.interp(cfg, pts)[:, 3], rtol=1e-12)
    for d, h in enumerate((1e-2, 1e-2, 1e-3)):
        e = np.zeros(4)
        e[d] = h
        fd = (oracle.interp(cfg, pts + e)[:, 3] - oracle.interp(cfg, pts - e)[:, 3]) / (2 * h)
        # cell faces (kinks of the bilinear columns) within h are skipped
        f = (pts[:, d] - (0.0 if d < 2 else 0.0)) / 250.0
        ok = np.abs(f - np.round(f)) * 250.0 > 2 * h if d < 2 else np.ones(n, bool)
        np.testing.assert_allclose(grad[ok, 3, d], fd[ok], rtol=1e-5, atol=1e-9)


def test_kz_eq3_second_derivative_and_partials():
    """d2K_z/dz2 (the drift term's derivative in the tangent-linear model) and the
    partials in u*, 1/L, H_z against central differences of Eq. 3."""
    rng = np.random.default_rng(10)
    for _ in range(60):
        u, inv_l, H = rng.uniform(0.1, 0.8), rng.uniform(-0.04, 0.04), rng.uniform(300.0, 2000.0)
        z = rng.uniform(0.05, 0.95) * H
        p = oracle.kz_eq3_partials(u, inv_l, H, 0.0, z)
        h = 1e-4 * H
        fd2 = (oracle.kz_eq3(u, inv_l, H, 0.0, z + h)[1] -
               oracle.kz_eq3(u, inv_l, H, 0.0, z - h)[1]) / (2 * h)
        assert p[5] == pytest.approx(fd2, rel=1e-5, abs=1e-7 * 0.4 * u / H)
        for idx, (du, args) in enumerate([(1e-6, lambda e: (u + e, inv_l, H)),
                                          (1e-7, lambda e: (u, inv_l + e, H)),
                                          (1e-3, lambda e: (u, inv_l, H + e))]):
            fd = (oracle.kz_eq3(*args(du), 0.0, z)[0] - oracle.kz_eq3(*args(-du), 0.0, z)[0]) / (2 * du)
            assert p[2 + idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


# ------------------------------------------------------------------------------------
# Decay chains (Sec. 2: particles transform to other species by radioactive decay)
# ------------------------------------------------------------------------------------
def _chain_cfg(half_lives, n_particles=300, n_steps=60):
    cfg = li.make_cfg0(n_particles=n_particles, n_steps=n_steps)
    return dataclasses.replace(cfg, half_life_s=float(half_lives[0]),
                               chain_half_lives=np.asarray(half_lives, dtype=np.float64))


@pytest.mark.parametrize("half_lives", [(3600.0, 1200.0, 0.0), (900.0, 5400.0, 300.0, 0.0),
                                        (7200.0, 600.0)])
def test_chain_amounts_solve_the_rate_equations(half_lives):
    """The closed-form amounts against a numerical integration of dN_1/dt = -l_1 N_1,
    dN_j/dt = l_{j-1} N_{j-1} - l_j N_j (N_1(0) = 1); with a stable last species the total
    stays 1, otherwise it decays. Catches a wrong product, sign or index in the formula."""
    from scipy.integrate import solve_ivp
    cfg = _chain_cfg(half_lives)
    lam = np.array([math.log(2.0) / h if h > 0 else 0.0 for h in half_lives])
    n = len(lam)

    def rhs(t, y):
        d = -lam * y
        d[1:] += lam[:-1] * y[:-1]
        return d

    ages = np.array([0.0, 120.0, 1800.0, 7200.0, 30000.0])
    sol = solve_ivp(rhs, (0.0, ages[-1]), np.eye(n)[0], t_eval=ages, rtol=1e-12, atol=1e-15,
                    method="DOP853")
    for a_i, age in enumerate(ages):
        got = np.array([oracle.chain_amount(cfg, j, age) for j in range(n)])
        np.testing.assert_allclose(got, sol.y[:, a_i], rtol=1e-8, atol=1e-12)
        if lam[-1] == 0.0:
            assert got.sum() == pytest.approx(1.0, abs=1e-12)


def test_chain_grids_per_species():
    """Uniform weather, every particle inside the grid: species 0 is the single-species
    snapshot exactly, and each species' grid total is the sum over the airborne particles
    of m0 N_j(age) with N_j from the numerically integrated rate equations."""
    from scipy.integrate import solve_ivp
    half_lives = (1800.0, 600.0, 0.0)
    n_p, steps = 300, 60
    cfg = dataclasses.replace(_chain_cfg(half_lives, n_p, steps), cx0=-1000.0, cx=100)
    r = oracle.run(cfg)
    assert np.array_equal(r["sp_conc_fixed"][0], r["conc_fixed"])
    np.testing.assert_allclose(r["sp_conc"][0], r["conc"], rtol=0, atol=0)
    assert r["counters"][0] == 0                       # nothing outside the grid
    lam = np.array([math.log(2.0) / h if h > 0 else 0.0 for h in half_lives])

    def rhs(t, y):
        d = -lam * y
        d[1:] += lam[:-1] * y[:-1]
        return d

    sp = (np.arange(n_p) * steps) // n_p
    ages = (steps - sp) * cfg.dt                        # the snapshot after the last step
    sol = solve_ivp(rhs, (0.0, ages.max()), [1.0, 0.0, 0.0], t_eval=np.unique(ages),
                    rtol=1e-12, atol=1e-15, method="DOP853")
    amount = {a: sol.y[:, i] for i, a in enumerate(np.unique(ages))}
    counts = np.bincount(sp, minlength=steps)
    for j in range(3):
        want = sum((1.0 * cfg.dt / counts[s]) * amount[a][j] for s, a in zip(sp, ages))
        assert r["sp_conc"][j].sum() == pytest.approx(want, rel=1e-9)


# ------------------------------------------------------------------------------------
# Vertical Langevin (velocity-memory) variant of the random walk
# ------------------------------------------------------------------------------------
def _langevin_column(K_of_z, H, n, steps, dt, t_lagr, src_z, reflect=True, nz=21):
    z_levels = np.linspace(0.0, H, nz)
    uvwk = np.zeros((2, nz, 2, 2, 4), np.float32)
    uvwk[..., 3] = K_of_z(z_levels)[None, :, None, None]
    cfg = li.make_cfg0(n_particles=n, n_steps=steps, kh=0.0, kz=0.0, u=0.0, src=(0.0, 0.0, src_z))
    return dataclasses.replace(cfg, uvwk=uvwk, z_levels=z_levels, nz=nz, dt=dt,
                               reflect_ground=int(reflect), reflect_top=int(reflect), z_top=H,
                               langevin=1, t_lagr=t_lagr,
                               release=li.Release(n, np.array([1.0]), 3600.0, 0, 1))


def test_langevin_discrete_laws_in_homogeneous_turbulence():
    """Constant K_z far from the walls: w' and z after m steps are jointly Gaussian with the
    covariance of the linear update w <- (1 - dt/T_L) w + sqrt(2 s2 dt / T_L) n,
    z <- z + dt w (w starting as sqrt(s2) n' at release, s2 = K_z / T_L), propagated here
    exactly; KS tests on w' and z. Catches a wrong relaxation, kick or initial variance,
    or the position following the old velocity."""
    K, T, dt, m, n = 20.0, 50.0, 2.0, 60, 6000
    cfg = _langevin_column(lambda z: np.full_like(z, K), 20000.0, n, m, dt, T, 10000.0,
                           reflect=False)
    r = oracle.run(cfg)
    s2 = K / T
    a, b = 1.0 - dt / T, math.sqrt(2.0 * s2 * dt / T)
    A = np.array([[a, 0.0], [dt * a, 1.0]])
    B = np.array([[b], [dt * b]])
    C = np.array([[s2, 0.0], [0.0, 0.0]])              # (w', z) at release, before the step
    for _ in range(m):
        C = A @ C @ A.T + B @ B.T
    assert stats.kstest(r["wvel"] / math.sqrt(C[0, 0]), "norm").pvalue > 1e-3
    assert stats.kstest((r["pos"][:, 2] - 10000.0) / math.sqrt(C[1, 1]), "norm").pvalue > 1e-3
    # and the velocity keeps its memory: lag-m correlation a^m against the release draw
    assert np.corrcoef(r["wvel"], r["pos"][:, 2])[0, 1] == pytest.approx(
        C[0, 1] / math.sqrt(C[0, 0] * C[1, 1]), abs=0.05)


def test_langevin_well_mixed_in_an_inhomogeneous_column():
    """K_z = K0 + K1 z in a reflecting column: with the drift term of the well-mixed model
    a uniform state stays uniform and the turbulent velocity at height z has variance
    K_z(z) / T_L. Catches a missing or mis-signed drift term and a wrong reflection."""
    H, K0, K1, T, dt = 100.0, 2.0, 0.3, 20.0, 1.0
    n, steps = 8000, 3000
    cfg = _langevin_column(lambda z: K0 + K1 * z, H, n, steps, dt, T, 50.0)
    r = oracle.run(cfg)
    z, w = r["pos"][:, 2], r["wvel"]
    assert stats.kstest(z / H, "uniform").pvalue > 1e-3
    for lo in (0.0, 40.0, 80.0):
        sel = (z >= lo) & (z < lo + 20.0)
        want = (K0 + K1 * (lo + 10.0)) / T
        assert np.var(w[sel]) == pytest.approx(want, rel=0.12)
