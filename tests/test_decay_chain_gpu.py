"""GPU parity of decay chains (particles transforming to other species, Sec. 2): the
daughters' concentration and deposition grids against the FP64 oracle, and their
invariance under the particle order, scenario mixing and checkpoint/resume."""
import dataclasses

import numpy as np
import pytest

import lpm_inputs as li
import oracle
from parity_util import compare, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHAIN = (7200.0, 1800.0, 0.0)          # parent (2 h) -> daughter (30 min) -> stable


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    oracle.build()


def _chain(cfg, half_lives=CHAIN):
    return dataclasses.replace(cfg, half_life_s=half_lives[0],
                               chain_half_lives=np.asarray(half_lives, np.float64))


def _species_run(cfg, n_run, sort_every=None):
    from paper_0912_3223_gb300 import Sim
    with Sim(cfg, sort_every=sort_every) as sim:
        sim.step(n_run)
        xyz, tag = sim.particles()
        sp = [sim.species(j) for j in range(len(cfg.chain_half_lives))]
        fixed = sim.fixed_state()
    return xyz, tag, sp, fixed


def test_chain_grids_against_the_oracle():
    """Realistic weather (decay, dry and wet deposition, lateral exit) stepped to the first
    hourly snapshot with a three-species chain: every species' concentration and
    deposition grid against the oracle outside face-ambiguous cells; species 0 equals the
    single-species grids bit for bit."""
    cfg = _chain(li.make_cfg1(n_particles=20_000, n_steps=2880, n_hours=3))
    n_run = 120
    g = run_gpu(cfg, n_run=n_run)
    _, _, sp, fixed = _species_run(cfg, n_run)
    o = oracle.run(cfg, n_run=n_run)
    sens = oracle.sensitivity(cfg, n_run=n_run)
    assert np.array_equal(sp[0][3], g["conc_fixed"]) and np.array_equal(sp[0][4], g["dep_fixed"])
    vol, area = cfg.cdx * cfg.cdy * cfg.cdz, cfg.cdx * cfg.cdy
    for j in range(3):
        conc, dry, wet = sp[j][:3]
        gj = dict(g, conc_mass=conc * vol, dep_mass=np.stack([dry, wet]) * area)
        oj = dict(o, conc=o["sp_conc"][j], dep=o["sp_dep"][j])
        rep = compare(cfg, gj, oj, sens=sens)
        print(f"species {j}: mass {oj['conc'].sum():.4g}, deposited {oj['dep'].sum():.4g}, {rep}")
        assert oj["conc"].sum() > 0 and oj["dep"].sum() > 0


def test_chain_invariant_under_order_mixing_and_resume():
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = _chain(li.make_cfg1(n_particles=4001, n_steps=300, n_hours=6))
    ref = _species_run(cfg, cfg.n_steps, sort_every=0)
    got = _species_run(cfg, cfg.n_steps, sort_every=40)
    for a, b in zip(ref[2], got[2]):
        assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])
    assert np.array_equal(ref[3][2], got[3][2])
    with Sim(cfg) as s1:
        s1.step(130)
        blob = lpm.lpm_save(s1.ctx)
    with Sim(cfg) as s2:
        lpm.lpm_load(s2.ctx, blob)
        s2.step(cfg.n_steps - 130)
        for j, a in enumerate(ref[2]):
            b = s2.species(j)
            assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])
    ens = li.make_cfg2(n_scenarios=4, n_steps=200, n_min=500, n_max=1500)
    ens = _chain(ens, (ens.half_life_s, 3600.0, 0.0))
    runs = []
    for se in (0, 25):
        with Sim(ens, sort_every=se) as sim:
            sim.step(ens.n_steps)
            runs.append([sim.species(j, s)[3] for s in range(4) for j in range(3)])
    assert all(np.array_equal(a, b) for a, b in zip(*runs))


def test_chain_errors():
    from paper_0912_3223_gb300 import Sim, lpm
    cfg = li.make_cfg1(n_particles=100, n_steps=60, n_hours=2)
    with Sim(cfg) as sim:
        for bad in ([1.0, 60.0], [cfg.half_life_s, cfg.half_life_s], [cfg.half_life_s, 0.0, 60.0]):
            with pytest.raises(lpm.LpmError) as e:
                lpm.lpm_set_decay_chain(sim.ctx, bad)
            assert e.value.status == lpm.LPM_E_INVALID
        sim.step(5)
        with pytest.raises(lpm.LpmError) as e:
            lpm.lpm_set_decay_chain(sim.ctx, [cfg.half_life_s, 60.0])
        assert e.value.status == lpm.LPM_E_STATE
