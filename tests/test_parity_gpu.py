"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element, plus exact integer identities of the
fixed-point binning. Bars: Philox words bit-exact; per-particle positions within
0.5 m after 360 steps; grids within 1e-4 relative L1 outside face-ambiguous cells."""
import dataclasses
import math

import numpy as np
import pytest

import lpm_inputs as li
import oracle
from parity_util import (POS_TOL_M, artificial_weather_cfg, compare, run_gpu)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    oracle.build()


def _integer_identity(g):
    """Right after a bin step: the budget kernel's per-particle fixed-point masses (in and
    out of the grid) equal the binned grid plus its out-of-grid counter, exactly."""
    ctr = g["counters"]
    assert int(g["conc_fixed"].sum()) + int(ctr[0]) == int(ctr[6]) + int(ctr[7])


def test_draws_bit_exact():
    rng = np.random.default_rng(5)
    pid = np.concatenate([np.arange(1000), rng.integers(0, 2 ** 40, 3000)]).astype(np.uint64)
    step = rng.integers(0, 2 ** 28, pid.size).astype(np.uint32)
    from paper_0912_3223_gb300 import lpm
    for seed in (1, 0xDEADBEEF12345678):
        for stream in (0, 1):
            w, n = lpm.lpm_draws(seed, pid, step, stream)
            ref = oracle.draws(seed, pid, step, stream)
            assert np.array_equal(w, ref)
        ref_n = oracle.normals(seed, pid, step)
        w, n = lpm.lpm_draws(seed, pid, step, 0)
        assert np.abs(n.astype(np.float64) - ref_n).max() < 4e-6


def test_cfg0_full_parity():
    """Plain method, small: 1e4 particles, 360 steps, uniform weather."""
    cfg = li.make_cfg0()
    g = run_gpu(cfg)
    o = oracle.run(cfg)
    rep = compare(cfg, g, o)
    assert rep["ambiguous"] == 0
    assert rep["grid_rel_l1"] <= 1e-4
    _integer_identity(g)
    assert int(g["counters"][4]) == o["active_steps"] == 1_805_160
    np.testing.assert_allclose(g["budget"][:6], o["budget"][:6], rtol=1e-5)
    assert g["budget"][7] == o["budget"][7]


def test_artificial_weather_of_the_paper():
    """The paper's homogeneous case (Fig. 3b): 2160 particles, dt = 10 s. Per-particle
    distances are gated after 360 steps and reported after 6 h."""
    cfg = artificial_weather_cfg()
    g = run_gpu(cfg, n_run=360)
    o = oracle.run(cfg, n_run=360)
    compare(cfg, g, o)
    gf = run_gpu(cfg)
    of = oracle.run(cfg)
    rep = compare(cfg, gf, of, pos_tol=5.0, grid_tol=1e-3, max_excluded_frac=0.05)
    print("artificial weather after 6 h:", rep)
    _integer_identity(gf)


@pytest.fixture(scope="module")
def cfg1_small():
    return li.make_cfg1(n_particles=20_000, n_steps=2880, n_hours=25)


def test_cfg1_parity_360_steps(cfg1_small):
    """Realistic weather (log profile + mesoscale modes, K_z profile, decay, dry and wet
    deposition, lateral exit), all 20000 particles after 360 steps."""
    g = run_gpu(cfg1_small, n_run=360)
    o = oracle.run(cfg1_small, n_run=360)
    sens = oracle.sensitivity(cfg1_small, n_run=360)
    rep = compare(cfg1_small, g, o, check_grid=False, sens=sens)
    print("cfg1 360 steps:", rep)
    # budget after 360 steps (not a bin step: compare the airborne + event totals)
    np.testing.assert_allclose(g["budget"][0], o["budget"][0], rtol=1e-6)
    assert abs(g["budget"][7] - o["budget"][7]) <= rep["ambiguous"]


def test_cfg1_parity_bin_step(cfg1_small):
    """Same inputs stepped to the first hourly snapshot: grids and deposition compared."""
    g = run_gpu(cfg1_small, n_run=120)
    o = oracle.run(cfg1_small, n_run=120)
    rep = compare(cfg1_small, g, o, sens=oracle.sensitivity(cfg1_small, n_run=120))
    print("cfg1 120 steps:", rep)
    _integer_identity(g)
    assert int(g["counters"][4]) == o["active_steps"]


def test_cfg1_full_run_report(cfg1_small):
    """24 h: events and chaotic divergence in non-uniform wind (Sec. 4.1) make the late
    distances grow; they are reported, with a loose bar, and the exact invariants hold."""
    g = run_gpu(cfg1_small)
    o = oracle.run(cfg1_small)
    rep = compare(cfg1_small, g, o, pos_tol=10.0, check_grid=False, max_excluded_frac=0.3)
    print("cfg1 24 h:", rep)
    _integer_identity(g)
    b = g["budget"]
    assert b[0] - b[6] == pytest.approx(b[1] + b[2] + b[3] + b[4] + b[5], rel=1e-12)
    np.testing.assert_allclose(b[0], o["budget"][0], rtol=1e-6)


def test_cfg1_full_size_sampled():
    """1e7 particles x 2880 steps in the benchmark's launch shape; a deterministic sample
    of particle ids is recomputed one by one by the oracle."""
    cfg = li.make_cfg1()
    from paper_0912_3223_gb300 import Sim
    sel = np.arange(0, cfg.n_particles, 9973, dtype=np.int64)
    with Sim(cfg) as sim:
        sim.step(360)
        xyz, tag = sim.particles()
        g360 = dict(pos=xyz[sel].astype(np.float64), tag=tag[sel])
        sim.step(cfg.n_steps - 360)
        xyz, tag = sim.particles()
        cfix, dfix, ctr, shift = sim.fixed_state()
        b = sim.budget()
        cfix2, _, ctr2, _ = sim.fixed_state()
    o360 = oracle.run(cfg, sel=sel, n_run=360)
    sens = oracle.sensitivity(cfg, sel=sel, n_run=360)
    ch = oracle.chaotic(cfg, sens, o360["pos"], POS_TOL_M)
    ok = (o360["margin"] >= POS_TOL_M) & (o360["status"] != li.STATUS_UNRELEASED) & ~ch
    assert ch.mean() <= 0.01
    st = (g360["tag"] >> 28).astype(np.int32)
    assert np.array_equal(st[ok], o360["status"][ok])
    d = np.linalg.norm(g360["pos"][ok] - o360["pos"][ok], axis=1)
    print(f"1e7 sample after 360 steps: max {d.max():.3g} m over {ok.sum()} particles")
    assert d.max() <= POS_TOL_M
    # integer identity at the final bin step, and the budget identity
    assert int(cfix2.sum()) + int(ctr2[0]) == int(ctr2[6]) + int(ctr2[7])
    assert b[0] - b[6] == pytest.approx(b[1] + b[2] + b[3] + b[4] + b[5], rel=1e-12)
    assert b[0] == pytest.approx(oracle.total_mass(cfg), rel=1e-9)


@pytest.mark.parametrize("block,ppt,occ", [(128, 1, 0), (128, 1, 2), (256, 2, 1), (256, 4, 0),
                                           (512, 1, 2), (512, 4, 1), (128, 4, 2)])
def test_launch_shape_does_not_change_results(block, ppt, occ):
    """Results are bit-identical for every launch shape (integer binning, per-particle
    keyed draws)."""
    cfg = li.make_cfg1(n_particles=3001, n_steps=240, n_hours=5)
    ref = run_gpu(cfg, launch=(256, 2, 0))
    g = run_gpu(cfg, launch=(block, ppt, occ))
    assert np.array_equal(g["pos"], ref["pos"]) and np.array_equal(g["tag"], ref["tag"])
    assert np.array_equal(g["conc_fixed"], ref["conc_fixed"])
    assert np.array_equal(g["dep_fixed"], ref["dep_fixed"])
    assert np.array_equal(g["counters"], ref["counters"])


def test_stepping_in_pieces_is_identical():
    cfg = li.make_cfg1(n_particles=2000, n_steps=300, n_hours=4)
    a = run_gpu(cfg)
    b = run_gpu(cfg, pieces=[1, 7, 112, 3, 57, 120])
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["tag"], b["tag"])
    assert np.array_equal(a["conc_fixed"], b["conc_fixed"])
    assert np.array_equal(a["dep_fixed"], b["dep_fixed"])


@pytest.mark.parametrize("n,first,last", [(1, 0, 50), (37, 0, 120), (1025, 3, 77),
                                          (4099, 10, 200)])
def test_ragged_and_sparse_releases(n, first, last):
    """One particle, fewer particles than release steps (empty steps), ragged tile
    tails and a delayed release window."""
    base = li.make_cfg1(n_particles=n, n_steps=200, n_hours=4)
    cfg = dataclasses.replace(base, bin_every=50,
                              release=li.Release(n, np.array([1.0, 3.0, 0.5]), 1800.0,
                                                 first, last))
    g = run_gpu(cfg)
    o = oracle.run(cfg)
    compare(cfg, g, o, sens=oracle.sensitivity(cfg))
    _integer_identity(g)


@pytest.mark.parametrize("id_base", [(1 << 32) - 1000, (1 << 40) + 7])
def test_particle_ids_beyond_32_bits(id_base):
    """Global particle ids past 2^32: the generator counter's high word is non-zero (and,
    for the first base, the release straddles the boundary), yet the particle path still
    matches the oracle drawing with the same ids, and differs from the ids-from-0 run."""
    cfg = li.make_cfg1(n_particles=3000, n_steps=240, n_hours=5)
    g = run_gpu(cfg, id_base=id_base)
    o = oracle.run(cfg, id_offset=id_base)
    rep = compare(cfg, g, o, sens=oracle.sensitivity(cfg, id_offset=id_base))
    print(f"ids from {id_base:#x}:", rep)
    _integer_identity(g)
    assert not np.array_equal(run_gpu(cfg)["pos"], g["pos"])


def test_maximum_levels_match_oracle():
    """64 stretched levels, the most the kernel parameters carry (the lowest 0.76 m apart,
    so the level table would need over 4096 bins and the lookup bisects): the realistic
    run against the oracle."""
    base = li.make_cfg1(n_particles=3000, n_steps=240, n_hours=5)
    uvwk, z = li.make_met_realistic(nz=64, n_t=5)
    cfg = dataclasses.replace(base, nz=64, z_levels=z, uvwk=uvwk)
    g = run_gpu(cfg)
    o = oracle.run(cfg)
    rep = compare(cfg, g, o, sens=oracle.sensitivity(cfg))
    print("64 levels:", rep)
    _integer_identity(g)


def test_degenerate_zero_emission_and_stable_tracer():
    """Two degenerate cases of the method. An all-zero emission series: the particles still
    move exactly as the oracle's, every grid and budget entry is zero, and the run reports
    no error. A stable tracer (no decay) with no deposition and no lateral exit: nothing
    leaves the air, so the airborne mass equals the released mass up to the FP32 storage of
    the initial masses, and the fixed-point identity holds."""
    base = li.make_cfg1(n_particles=2000, n_steps=120, n_hours=3)
    zero = dataclasses.replace(base, release=li.Release(2000, np.zeros(3), 3600.0, 0, 120))
    g = run_gpu(zero)
    o = oracle.run(zero)
    compare(zero, g, o, check_grid=False, sens=oracle.sensitivity(zero))
    assert not g["conc_fixed"].any() and not g["dep_fixed"].any()
    assert not np.any(g["budget"][:7])
    stable = dataclasses.replace(base, half_life_s=0.0, vd_dry=0.0, wet_lambda=0.0,
                                 lateral_exit=0)
    g = run_gpu(stable)
    _integer_identity(g)
    b = g["budget"]
    assert b[0] > 0 and b[3] == b[4] == b[5] == 0.0
    assert abs(b[1] + b[2] - b[0]) <= 1e-6 * b[0] and abs(b[6]) <= 1e-6 * b[0]
    assert int(b[7]) == 2000                     # every particle released and still airborne


def _linear_wind(X, Y, Z, T):
    u = 4.0 + 1e-4 * X - 5e-5 * Y + 2e-3 * Z + 1e-4 * T
    v = -1.0 + 5e-5 * X + 1e-4 * Y - 1e-3 * Z + 5e-5 * T
    w = 1e-3 - 1e-6 * Z + 1e-7 * X
    return u, v, w


def test_linear_weather_paths_follow_the_closed_form():
    """No diffusion and no sinks: every particle follows the Euler map
    x_{k+1} = x_k + u(x_k, t_k) dt (Eq. 1-2 with K = 0). For weather linear in x, y, z
    and t the multilinear interpolation is exact, so the GPU paths must follow the map
    iterated in FP64 on the closed-form field, independently of the oracle, to FP32
    rounding of the positions (0.1 m after up to 120 steps at x <= 14 km). Catches
    swapped axes, a wrong weight complement, an off-by-one cell or level and a wrong time
    fraction, each worth metres per step."""
    nx, ny, nz, nt = 25, 21, 12, 2
    z_levels = li.z_levels_stretched(nz, 2000.0)
    T, Z, Y, X = np.meshgrid(np.arange(nt) * 3600.0, z_levels, 1000.0 * np.arange(ny),
                             1000.0 * np.arange(nx), indexing="ij")
    uvwk = np.zeros((nt, nz, ny, nx, 4))
    uvwk[..., 0], uvwk[..., 1], uvwk[..., 2] = _linear_wind(X, Y, Z, T)
    n = 120
    base = li.make_cfg0(n_particles=n, n_steps=n, kh=0.0, kz=0.0)
    cfg = dataclasses.replace(base, nx=nx, ny=ny, nz=nz, x0=0.0, y0=0.0, dx=1000.0,
                              dy=1000.0, z_levels=z_levels, n_met_t=nt, met_t0=0.0,
                              met_dt=3600.0, uvwk=uvwk.astype(np.float32), dt=20.0,
                              src_x=2000.0, src_y=10000.0, src_z=300.0,
                              release=li.Release(n, np.array([1.0]), 3600.0, 0, n))
    want = np.empty((n, 3))
    for p in range(n):                           # particle p leaves at step p
        x = np.array([cfg.src_x, cfg.src_y, cfg.src_z])
        for k in range(p, n):
            x = x + np.array(_linear_wind(x[0], x[1], x[2], k * cfg.dt)) * cfg.dt
        want[p] = x
    g = run_gpu(cfg)
    assert np.all(g["status"] == 0)
    d = np.abs(g["pos"] - want).max()
    print(f"linear weather: max deviation from the closed-form paths {d:.3g} m")
    assert d < 0.1


def test_gridded_kh_drift_and_emission_series():
    """Gridded K_h, the drift-corrected variant and a 24-value emission series."""
    base = li.make_cfg1(n_particles=5000, n_steps=240, n_hours=5)
    rng = np.random.default_rng(9)
    kh = (80.0 + 40.0 * rng.random(base.uvwk.shape[:-1])).astype(np.float32)
    cfg = dataclasses.replace(base, kh=kh, kh_uniform=-1.0, drift_correction=1,
                              release=li.Release(5000, np.exp(rng.normal(0, 0.5, 24)), 600.0,
                                                 0, 240))
    g = run_gpu(cfg)
    o = oracle.run(cfg)
    rep = compare(cfg, g, o)
    print("gridded K_h + drift:", rep)


def test_met_from_device_tensors():
    cfg = li.make_cfg1(n_particles=2000, n_steps=120, n_hours=3)
    a = run_gpu(cfg)
    b = run_gpu(cfg, met_on_device=True)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["conc_fixed"], b["conc_fixed"])


def test_error_paths():
    from paper_0912_3223_gb300 import lpm
    cfg = li.make_cfg0(n_particles=100, n_steps=20)
    ctx = lpm.lpm_create(cfg)
    try:
        # releasing out of order / stepping before every scenario is released
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_step(ctx, 1)
        assert e.value.status == lpm.LPM_E_STATE
        lpm.lpm_step(ctx, 0)                        # an empty step is a no-op
        # empty, oversized and ill-formed releases are refused and change nothing
        for args in [(0, [1.0], 3600.0, 0, 20), (cfg.n_particles + 1, [1.0], 3600.0, 0, 20),
                     (100, [1.0], 3600.0, 5, 5), (100, [1.0], 3600.0, 0, 21),
                     (100, [-1.0], 3600.0, 0, 20), (100, [1.0], 0.0, 0, 20)]:
            with pytest.raises(lpm.LpmError) as e:
                lpm.lpm_release(ctx, 0, *args)
            assert e.value.status == lpm.LPM_E_INVALID, args
        lpm.lpm_release(ctx, 0, 100, [1.0], 3600.0, 0, 20)
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_release(ctx, 0, 100, [1.0], 3600.0, 0, 20)
        assert e.value.status == lpm.LPM_E_STATE
        # met slab missing
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_step(ctx, 1)
        assert e.value.status == lpm.LPM_E_STATE and "met slab" in str(e.value)
        for t in range(cfg.n_met_t):
            lpm.lpm_set_met(ctx, t, cfg.uvwk[t])
        lpm.lpm_step(ctx, 20)
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_step(ctx, 1)
        assert e.value.status == lpm.LPM_E_STATE
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_set_met(ctx, 5, cfg.uvwk[0])
        assert e.value.status == lpm.LPM_E_INVALID
    finally:
        lpm.lpm_destroy(ctx)
    # a NaN in the weather is reported as LPM_E_NUMERIC, the context stays usable
    bad = dataclasses.replace(cfg, uvwk=cfg.uvwk.copy())
    bad.uvwk[..., 0] = np.nan
    from paper_0912_3223_gb300 import Sim
    with Sim(bad) as sim:
        sim.step(5)
        with pytest.raises(lpm.LpmError) as e:
            sim.sync()
        assert e.value.status == lpm.LPM_E_NUMERIC
    with Sim(cfg) as sim:
        sim.step(cfg.n_steps)
        sim.sync()


def test_partitioned_contexts_sum_to_single_run():
    """Three contexts holding disjoint particle ranges of one release: their integer grids
    and counters add up bit for bit to the single-context run (the exchange step of a
    multi-GPU run, here sequential on one GPU)."""
    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.parallel import partition
    cfg = li.make_cfg1(n_particles=9001, n_steps=240, n_hours=5)
    full = run_gpu(cfg)
    conc = np.zeros_like(full["conc_fixed"])
    dep = np.zeros_like(full["dep_fixed"])
    ctr = np.zeros(6, np.int64)
    pos = []
    for r in range(3):
        first, count = partition(cfg.n_particles, 3, r)
        with Sim(cfg, part=(first, count)) as sim:
            sim.step(cfg.n_steps)
            c, d, k, _ = sim.fixed_state()
            xyz, tag = sim.particles()
        conc += c
        dep += d
        ctr += k[:6]
        pos.append(xyz)
    assert np.array_equal(conc, full["conc_fixed"])
    assert np.array_equal(dep, full["dep_fixed"])
    assert np.array_equal(ctr[[0, 1, 2, 3, 4]], full["counters"][[0, 1, 2, 3, 4]])
    assert np.array_equal(np.concatenate(pos).astype(np.float64), full["pos"])


@pytest.mark.parametrize("every", [7, 60])
def test_sorting_particles_by_cell_changes_nothing(every):
    """Re-ordering the released particles by weather cell is a layout change only: the
    particles (read back in index order), grids, counters and budget are bit-identical. The
    read-backs go through the slot map the sorts leave stale; reading back in mid-run,
    sorting on and reading back again rebuilds it twice."""
    cfg = li.make_cfg1(n_particles=7001, n_steps=300, n_hours=4)
    from paper_0912_3223_gb300 import Sim
    ref = run_gpu(cfg, sort_every=0)
    with Sim(cfg, sort_every=0) as sim:
        sim.step(137)
        mid_ref = sim.particles()
        mid_budget_ref = sim.budget()
    with Sim(cfg, sort_every=every) as sim:
        sim.step(137)
        mid = sim.particles()
        mid_budget = sim.budget()
        sim.step(cfg.n_steps - 137)
        xyz, tag = sim.particles()
        part = sim.particles(1234, 99)
        cfix, dfix, ctr, _ = sim.fixed_state()
        budget = sim.budget()
    assert np.array_equal(mid[0], mid_ref[0]) and np.array_equal(mid[1], mid_ref[1])
    assert np.array_equal(mid_budget, mid_budget_ref)
    assert np.array_equal(budget, ref["budget"])
    assert np.array_equal(xyz.astype(np.float64), ref["pos"]) and np.array_equal(tag, ref["tag"])
    assert np.array_equal(part[0], xyz[1234:1333]) and np.array_equal(part[1], tag[1234:1333])
    assert np.array_equal(cfix, ref["conc_fixed"]) and np.array_equal(dfix, ref["dep_fixed"])
    assert np.array_equal(ctr[:6], ref["counters"][:6])


@pytest.mark.parametrize("sort_every", [0, 60])
def test_save_and_resume_is_bit_identical(sort_every):
    """Checkpoint after 150 steps, resume in a fresh context: the continued run equals the
    uninterrupted one bit for bit (particles, grids, counters)."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = li.make_cfg1(n_particles=6007, n_steps=330, n_hours=4)
    with Sim(cfg, sort_every=sort_every) as a:
        if sort_every:
            a.set_dosage(8)                  # the dosage state travels with the checkpoint
        a.step(150)
        saved = lpm.lpm_save(a.ctx)
        a.step(cfg.n_steps - 150)
        ref_xyz, ref_tag = a.particles()
        ref = a.fixed_state()
        ref_dose = a.dosage() if sort_every else None
    with Sim(cfg, sort_every=sort_every) as b:
        lpm.lpm_load(b.ctx, saved)
        assert b.k == 150
        b.step(cfg.n_steps - 150)
        xyz, tag = b.particles()
        got = b.fixed_state()
        if sort_every:
            dose = b.dosage()
            assert np.array_equal(dose[1], ref_dose[1]) and dose[2] == ref_dose[2] == 330 // 8
    assert np.array_equal(xyz, ref_xyz) and np.array_equal(tag, ref_tag)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert np.array_equal(got[2][:6], ref[2][:6]) and got[2][11] == ref[2][11]
    with Sim(li.make_cfg1(n_particles=100, n_steps=330, n_hours=4)) as other:
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_load(other.ctx, saved)
        assert e.value.status == lpm.LPM_E_INVALID
    # headers with impossible snapshot or dosage counts are refused before anything is
    # loaded: the context keeps its own run (header: 8-byte magic, then int64 k, n_bins,
    # n_slots, n_scen, ncell, ndep, n_ctr, dose_every, n_dose, ...)
    import struct
    bad_fields = [(16, -1), (16, 151)]                 # n_bins < 0, n_bins > k
    bad_fields += [(72, 150 // 8 + 1), (72, -1)] if sort_every else [(72, 1)]
    with Sim(cfg, sort_every=sort_every) as c:
        c.step(10)
        before = c.fixed_state()
        for off, val in bad_fields:
            bad = bytearray(saved)
            struct.pack_into("<q", bad, off, val)
            with pytest.raises(lpm.LpmError) as e:
                lpm.lpm_load(c.ctx, bytes(bad))
            assert e.value.status == lpm.LPM_E_INVALID
            assert c.k == 10
        after = c.fixed_state()
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[2], after[2])


def test_allocation_failure_is_reported():
    """A context too large for the device fails cleanly with LPM_E_OOM."""
    from paper_0912_3223_gb300 import lpm
    cfg = li.make_cfg0(n_particles=10, n_steps=10)
    # 32 scenarios of a 2e9-cell concentration grid: 512 GB of 64-bit counters
    huge = dataclasses.replace(cfg, cx=2000, cy=2000, cz=500, n_scenarios=32)
    with pytest.raises(lpm.LpmError) as e:
        lpm.lpm_create(huge)
    assert e.value.status == lpm.LPM_E_OOM
    with pytest.raises(lpm.LpmError) as e:          # beyond the 31-bit slot indices
        lpm.lpm_create(cfg, max_particles=1 << 40)
    assert e.value.status == lpm.LPM_E_INVALID
    ctx = lpm.lpm_create(cfg)           # the device is still usable
    lpm.lpm_destroy(ctx)


def test_met_from_pinned_host_memory_overlaps_and_matches():
    """Weather from page-locked host memory is uploaded asynchronously (hours arrive while
    earlier ones are computed); the results equal those of pageable uploads bit for bit,
    also when the same context re-uploads between runs."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = li.make_cfg1(n_particles=5003, n_steps=480, n_hours=5)
    ref = run_gpu(cfg)
    uvwk = torch.from_numpy(cfg.uvwk).pin_memory()
    rain = torch.from_numpy(cfg.rain).pin_memory()
    with Sim(cfg) as sim:
        for rep in range(2):
            sim.reset()
            for t in range(cfg.n_met_t):
                lpm.lpm_set_met(sim.ctx, t, uvwk[t], None, rain[t])
            sim.step(cfg.n_steps)
            xyz, tag = sim.particles()
            assert np.array_equal(xyz.astype(np.float64), ref["pos"]) and np.array_equal(tag, ref["tag"])
            assert np.array_equal(sim.fixed_state()[0], ref["conc_fixed"])


def test_level_bisection_path_matches_oracle():
    """Levels whose smallest spacing would need more than 4096 table bins (a 3 mm first
    layer) take the bisection path of the vertical cell search; realistic weather, 360
    steps, against the oracle with the same exclusions as the table path."""
    cfg = li.make_cfg1(n_particles=5000, n_steps=360)
    z = np.array(cfg.z_levels, dtype=np.float64)
    z[1] = 0.003
    cfg = dataclasses.replace(cfg, z_levels=z)
    g = run_gpu(cfg, n_run=360)
    o = oracle.run(cfg, n_run=360)
    sens = oracle.sensitivity(cfg, n_run=360)
    # the 3 mm layer makes the wind's vertical gradient near the ground a hundred times
    # steeper than in the realistic levels: more paths are chaotic, so up to 2 % may be set
    # apart (each still held to its own growth bound)
    rep = compare(cfg, g, o, check_grid=False, sens=sens, max_excluded_frac=0.02)
    print("bisection levels, 360 steps:", rep)
    np.testing.assert_allclose(g["budget"][0], o["budget"][0], rtol=1e-6)
