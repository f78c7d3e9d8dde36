"""GPU parity of the time-integrated dosage (the summations of every n-th step, integrated
in time as Sec. 3.2 describes) against the FP64 oracle, and its invariance under the
particle order, stepping in pieces and scenario mixing."""
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


def _gpu(cfg, every, n_run=None, sort_every=None, pieces=None):
    from paper_0912_3223_gb300 import Sim
    n_run = cfg.n_steps if n_run is None else n_run
    with Sim(cfg, sort_every=sort_every) as sim:
        sim.set_dosage(every)
        for n in (pieces or [n_run]):
            sim.step(n)
        dose, fixed, samples = sim.dosage()
        ctr = sim.fixed_state()[2]
        xyz, tag = sim.particles()
    return dict(dose=dose, fixed=fixed, samples=samples, out=int(ctr[11]),
                pos=xyz.astype(np.float64), tag=tag, status=(tag >> 28).astype(np.int32),
                release=(tag & 0x0FFFFFFF).astype(np.int64))


def _rel_l1(got, ref):
    return float(np.abs(got - ref).sum() / np.abs(ref).sum())


def test_dosage_uniform_weather():
    """Uniform wind and diffusivity with decay, a sample every 4 steps for 360 steps: the
    dosage grid against the oracle's FP64 sums, and the fixed-point total (grid plus the
    out-of-grid part) to the rounding of FP32 masses."""
    cfg = dataclasses.replace(li.make_cfg0(n_particles=10_000, n_steps=360), half_life_s=3600.0)
    every = 4
    g = _gpu(cfg, every)
    o = oracle.run(cfg, dose_every=every)
    assert g["samples"] == o["dose_samples"] == cfg.n_steps // every
    ref = o["dose"] * (every * cfg.dt) / (cfg.cdx * cfg.cdy * cfg.cdz)
    rel = _rel_l1(g["dose"], ref)
    tot_g = int(g["fixed"].sum()) + g["out"]
    tot_o = int(o["dose_fixed"].sum()) + o["dose_out"]
    print(f"uniform dosage: rel L1 {rel:.2e}, totals {tot_g} / {tot_o}")
    assert abs(tot_g - tot_o) <= 1e-6 * tot_o
    assert rel <= 1e-4


def test_dosage_realistic_weather():
    """Realistic weather (decay, dry and wet deposition, lateral exit), a sample every 6
    steps for 360 steps. A particle the comparison excludes (a decision within the position
    tolerance, or a chaotic path) may put its mass into other cells at every sample, so the
    bar is the excluded particles' share, doubled, plus 1e-4."""
    cfg = li.make_cfg1(n_particles=20_000, n_steps=2880, n_hours=25)
    every, n_run = 6, 360
    g = _gpu(cfg, every, n_run=n_run)
    o = oracle.run(cfg, n_run=n_run, dose_every=every)
    sens = oracle.sensitivity(cfg, n_run=n_run)
    rep = compare(cfg, g, o, check_grid=False, sens=sens)
    released = int((o["status"] != li.STATUS_UNRELEASED).sum())
    share = rep["ambiguous"] / released
    ref = o["dose"] * (every * cfg.dt) / (cfg.cdx * cfg.cdy * cfg.cdz)
    rel = _rel_l1(g["dose"], ref)
    tot_g = int(g["fixed"].sum()) + g["out"]
    tot_o = int(o["dose_fixed"].sum()) + o["dose_out"]
    print(f"realistic dosage: rel L1 {rel:.2e}, totals {tot_g} / {tot_o}, excluded {rep}")
    assert g["samples"] == o["dose_samples"] == n_run // every
    assert abs(tot_g - tot_o) <= (2 * share + 1e-6) * tot_o
    assert rel <= 2 * share + 1e-4


def test_dosage_is_independent_of_order_and_pieces():
    """Sorting the particles by cell and stepping in pieces change no bit of the dosage."""
    cfg = li.make_cfg1(n_particles=5003, n_steps=400, n_hours=7)
    ref = _gpu(cfg, 7, sort_every=0)
    for kw in (dict(sort_every=30), dict(sort_every=60, pieces=[45, 100, 255])):
        got = _gpu(cfg, 7, **kw)
        assert np.array_equal(got["fixed"], ref["fixed"]) and got["out"] == ref["out"]
        assert got["samples"] == ref["samples"] == cfg.n_steps // 7


def test_batched_dosage_mixed_scenarios():
    """Batched ensemble sorted by cell (lanes of several scenarios in one warp) against the
    unsorted run bit for bit, and one scenario against the oracle."""
    from paper_0912_3223_gb300 import Sim
    cfg = li.make_cfg2(n_scenarios=5, n_steps=200, n_min=500, n_max=2000)
    every = 5
    runs = []
    for se in (0, 25):
        with Sim(cfg, sort_every=se) as sim:
            sim.set_dosage(every)
            sim.step(cfg.n_steps)
            runs.append([(sim.dosage(s)[1], int(sim.fixed_state(s)[2][11]))
                         for s in range(cfg.n_scenarios)])
    for (fa, oa), (fb, ob) in zip(*runs):
        assert np.array_equal(fa, fb) and oa == ob
    s = 2
    o = oracle.run(cfg, scenario=s, dose_every=every)
    fixed, out = runs[1][s]
    tot_g, tot_o = int(fixed.sum()) + out, int(o["dose_fixed"].sum()) + o["dose_out"]
    assert abs(tot_g - tot_o) <= 1e-3 * tot_o


def test_dosage_survives_save_and_resume():
    """A dosage run checkpointed after 150 steps and resumed in a fresh context, which takes
    the sampling interval, the sums, the out-of-grid counter and the sample count from the
    checkpoint, ends bit-identical to the uninterrupted run."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = li.make_cfg1(n_particles=5003, n_steps=400, n_hours=7)
    ref = _gpu(cfg, 7)
    with Sim(cfg) as a:
        a.set_dosage(7)
        a.step(150)
        blob = lpm.lpm_save(a.ctx)
    with Sim(cfg) as b:
        lpm.lpm_load(b.ctx, blob)
        b.step(cfg.n_steps - 150)
        dose, fixed, samples = b.dosage()
        out = int(b.fixed_state()[2][11])
    assert samples == ref["samples"] == cfg.n_steps // 7
    assert np.array_equal(fixed, ref["fixed"]) and out == ref["out"]
    assert np.array_equal(dose, ref["dose"])
