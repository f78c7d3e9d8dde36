"""Batched ensemble: many scenarios (own source, release, emission series and perturbed
weather: an hourly wind offset plus the scenario's realisation of the perturbation modes)
in one persistent launch replayed from a CUDA graph, checked against the oracle scenario
by scenario, against single-scenario contexts bit for bit, and across graph replays."""
import dataclasses

import numpy as np
import pytest

import lpm_inputs as li
import oracle
from parity_util import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def small_ensemble():
    return li.make_cfg2(n_scenarios=6, n_steps=240, n_min=500, n_max=3000)


def _run(cfg, launch=None, repeat=1, sort_every=None, pieces=None):
    from paper_0912_3223_gb300 import Sim
    out = []
    with Sim(cfg, launch=launch, sort_every=sort_every) as sim:
        for _ in range(repeat):
            sim.reset()
            if pieces:
                for n in pieces:
                    sim.step(n)
            else:
                sim.step(cfg.n_steps)
            xyz, tag = sim.particles()
            scen = []
            for s in range(cfg.n_scenarios):
                c, d, k, sh = sim.fixed_state(s)
                scen.append(dict(conc=sim.concentration(s), dep=sim.deposition(s),
                                 conc_fixed=c, dep_fixed=d, counters=k, budget=sim.budget(s)))
            out.append((xyz, tag, scen))
    return out


def test_batched_matches_oracle_per_scenario(small_ensemble):
    cfg = small_ensemble
    (xyz, tag, scen), = _run(cfg)
    off = 0
    vol = cfg.cdx * cfg.cdy * cfg.cdz
    area = cfg.cdx * cfg.cdy
    for s, sc in enumerate(cfg.scenarios):
        n = sc.release.n_particles
        o = oracle.run(cfg, scenario=s)
        sens = oracle.sensitivity(cfg, scenario=s)
        g = dict(pos=xyz[off:off + n].astype(np.float64), tag=tag[off:off + n],
                 status=(tag[off:off + n] >> 28).astype(np.int32),
                 release=(tag[off:off + n] & 0x0FFFFFFF).astype(np.int64),
                 conc_mass=scen[s]["conc"] * vol,
                 dep_mass=np.stack(scen[s]["dep"]) * area)
        rep = compare(cfg, g, o, sens=sens)
        print(f"scenario {s}: {rep}")
        c = scen[s]["counters"]
        assert int(c[4]) == o["active_steps"]
        off += n


def test_scenario_ranges_reproduce_the_ensemble(small_ensemble):
    """Contexts holding contiguous scenario ranges of the ensemble, as the ranks of a
    partitioned batched run would, reproduce every scenario's particles, grids and
    counters bit for bit (global particle ids carried over; no exchange needed)."""
    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.parallel import partition
    cfg = small_ensemble
    (xyz, tag, scen), = _run(cfg)
    offs = np.cumsum([0] + [sc.release.n_particles for sc in cfg.scenarios])
    for r in range(3):
        first, count = partition(cfg.n_scenarios, 3, r)
        with Sim(cfg, scenarios=(first, count)) as sim:
            sim.step(cfg.n_steps)
            pxyz, ptag = sim.particles()
            a, b = offs[first], offs[first + count]
            assert np.array_equal(pxyz, xyz[a:b]) and np.array_equal(ptag, tag[a:b])
            for i in range(count):
                c, d, k, _ = sim.fixed_state(i)
                ref = scen[first + i]
                assert np.array_equal(c, ref["conc_fixed"])
                assert np.array_equal(d, ref["dep_fixed"])
                # the counters the steps accumulate (the airborne ones are written by the
                # budget pass, compared through the budget itself)
                step_ctr = [0, 1, 2, 3, 4, 5, 9, 10]
                assert np.array_equal(k[step_ctr], ref["counters"][step_ctr])
                assert np.array_equal(sim.budget(i), ref["budget"])


def test_graph_replay_is_identical(small_ensemble):
    a, b = _run(small_ensemble, repeat=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for sa, sb in zip(a[2], b[2]):
        assert np.array_equal(sa["conc_fixed"], sb["conc_fixed"])
        assert np.array_equal(sa["dep_fixed"], sb["dep_fixed"])


def test_scenario_equals_single_context(small_ensemble):
    """Scenario s of the ensemble equals a plain context holding the same release with the
    same global ids (id_base), source, wind offset and perturbation modes."""
    from paper_0912_3223_gb300 import lpm
    cfg = small_ensemble
    (xyz, tag, scen), = _run(cfg)
    s = 3
    sc = cfg.scenarios[s]
    off = sum(x.release.n_particles for x in cfg.scenarios[:s])
    one = dataclasses.replace(cfg, n_scenarios=1, scenarios=[], src_x=sc.src_x, src_y=sc.src_y,
                              src_z=sc.src_z, release=sc.release)
    ctx = lpm.lpm_create(one, torch.cuda.current_stream().cuda_stream,
                         max_particles=sc.release.n_particles)
    try:
        for t in range(one.n_met_t):
            lpm.lpm_set_met(ctx, t, one.uvwk[t], None, one.rain[t])
        lpm.lpm_set_source(ctx, 0, sc.src_x, sc.src_y, sc.src_z, sc.wind_offset)
        if cfg.modes is not None:
            lpm.lpm_set_modes(ctx, cfg.modes, cfg.mode_profile)
            lpm.lpm_set_mode_phases(ctx, 0, sc.mode_phase, sc.mode_amp)
        r = sc.release
        lpm.lpm_release_range(ctx, 0, r.n_particles, 0, r.n_particles, r.q, r.q_dt,
                              r.first_step, r.last_step, off)
        lpm.lpm_step(ctx, one.n_steps)
        pxyz, ptag = lpm.lpm_particles(ctx, 0, r.n_particles)
        c, d, k, _ = lpm.lpm_fixed_state(ctx, 0, (one.cz, one.cy, one.cx), (2, one.cy, one.cx))
    finally:
        lpm.lpm_destroy(ctx)
    n = sc.release.n_particles
    assert np.array_equal(pxyz, xyz[off:off + n]) and np.array_equal(ptag, tag[off:off + n])
    assert np.array_equal(c, scen[s]["conc_fixed"])
    assert np.array_equal(d, scen[s]["dep_fixed"])


def test_autotuner_keeps_results(small_ensemble, tmp_path, monkeypatch):
    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.autotune import autotune
    monkeypatch.setenv("LPM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ref = _run(small_ensemble)[0]
    with Sim(small_ensemble) as sim:
        shapes = [(128, 1, 2), (256, 2, 1), (512, 4, 0)]
        shape = autotune(sim, shapes=shapes, reps=1)
        assert shape in shapes
        sim.step(small_ensemble.n_steps)
        xyz, tag = sim.particles()
        again = autotune(sim)                        # served from the cache
        assert again == shape
    assert np.array_equal(xyz, ref[0]) and np.array_equal(tag, ref[1])


def test_autotuner_with_sort_interval_keeps_results(small_ensemble, tmp_path, monkeypatch):
    """Tuning the launch shape together with the sort interval picks one of the tried
    combinations, applies it, and the run it leaves is bit-identical to the default one."""
    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.autotune import autotune_with_sort
    monkeypatch.setenv("LPM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ref = _run(small_ensemble)[0]
    with Sim(small_ensemble) as sim:
        shape, every, tried = autotune_with_sort(sim, shapes=[(128, 1, 2), (512, 1, 2)],
                                                 sort_intervals=(20, 60), reps=1)
        assert shape in [(128, 1, 2), (512, 1, 2)] and every in (20, 60)
        assert len(tried) == 4
        sim.step(small_ensemble.n_steps)
        xyz, tag = sim.particles()
        assert autotune_with_sort(sim, shapes=[(128, 1, 2), (512, 1, 2)],
                                  sort_intervals=(20, 60))[:2] == (shape, every)   # cached
    assert np.array_equal(xyz, ref[0]) and np.array_equal(tag, ref[1])


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for sa, sb in zip(a[2], b[2]):
        assert np.array_equal(sa["conc_fixed"], sb["conc_fixed"])
        assert np.array_equal(sa["dep_fixed"], sb["dep_fixed"])
        assert np.array_equal(sa["counters"], sb["counters"])
        assert np.array_equal(sa["budget"], sb["budget"])


@pytest.mark.parametrize("every", [1, 37, 60])
def test_sorting_mixes_scenarios_without_changing_results(small_ensemble, every):
    """Sorting by cell puts particles of different scenarios into one warp (each lane with
    its own scenario's wind offset, masses and grids): every bit stays the same."""
    ref = _run(small_ensemble, sort_every=0)[0]
    got = _run(small_ensemble, sort_every=every)[0]
    _same(ref, got)


def test_sorted_batched_in_pieces_and_replayed(small_ensemble):
    ref = _run(small_ensemble, sort_every=0)[0]
    a, b = _run(small_ensemble, sort_every=30, repeat=2, pieces=[45, 15, 100, 80])
    _same(ref, a)
    _same(ref, b)


def test_sorted_batched_save_resume_and_resort(small_ensemble):
    """Checkpoint in the middle of a sorted batched run, resume in a fresh context, and
    change the sort interval on the way (the sorted set goes home first)."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = small_ensemble
    ref = _run(cfg, sort_every=0)[0]
    with Sim(cfg, sort_every=40) as sim:
        sim.reset()
        sim.step(100)
        blob = lpm.lpm_save(sim.ctx)
    with Sim(cfg, sort_every=25) as sim:
        sim.reset()
        lpm.lpm_load(sim.ctx, blob)
        sim.step(50)
        lpm.lpm_set_sort(sim.ctx, 0)
        sim.step(30)
        lpm.lpm_set_sort(sim.ctx, 20)
        sim.step(cfg.n_steps - 180)
        xyz, tag = sim.particles()
        assert np.array_equal(xyz, ref[0]) and np.array_equal(tag, ref[1])
        for s in range(cfg.n_scenarios):
            c, d, k, _ = sim.fixed_state(s)
            assert np.array_equal(c, ref[2][s]["conc_fixed"])
            assert np.array_equal(d, ref[2][s]["dep_fixed"])
            assert np.array_equal(sim.budget(s), ref[2][s]["budget"])
