"""Small runs covering every kernel family of the library (plain and sorted advance,
batched mixed-scenario lanes with perturbation modes, the extended options, the sort, the
budget, the adjoint's trajectory and checkpoint forms, cell-sorted and in release order), returning their outputs: the
checked-build test runs them once with each library and compares."""
import dataclasses

import numpy as np

import lpm_inputs as li


def run_cases() -> dict:
    from paper_0912_3223_gb300 import Sim, lpm
    out = {}
    plain = li.make_cfg1(n_particles=4001, n_steps=240, n_hours=5)
    for name, cfg, kw in [
        ("plain", plain, {}),
        ("plain_unsorted", plain, {"sort_every": 0}),
        ("ensemble", li.make_cfg2(n_scenarios=5, n_steps=240, n_min=300, n_max=1500), {}),
        ("options", dataclasses.replace(plain, langevin=1, t_lagr=100.0,
                                        chain_half_lives=np.array([plain.half_life_s, 3600.0,
                                                                   0.0])), {}),
        ("launch_ppt4", plain, {"launch": (256, 4, 0)}),
    ]:
        with Sim(cfg, **kw) as sim:
            if name == "options":
                sim.set_dosage(8)
            sim.step(cfg.n_steps)
            xyz, tag = sim.particles()
            out[f"{name}_xyz"], out[f"{name}_tag"] = xyz, tag
            for s in range(cfg.n_scenarios):
                c, d, k, _ = sim.fixed_state(s)
                out[f"{name}_conc{s}"], out[f"{name}_dep{s}"] = c, d
                out[f"{name}_budget{s}"] = sim.budget(s)
    adj = li.make_cfg3(n_particles=3000, n_steps=240)
    rec = li.make_receptors()
    w = np.linspace(-1.0, 1.0, rec.shape[0])[None, :]
    for name, storage, sort in [("adj_traj", None, 60), ("adj_ckpt", 0, 60),
                                ("adj_traj_release", None, 0), ("adj_ckpt_release", 0, 0)]:
        with Sim(adj) as sim:
            lpm.lpm_set_sort(sim.ctx, sort)
            if storage is not None:
                lpm.lpm_set_adjoint_storage(sim.ctx, storage)
            out[f"{name}_C"] = lpm.lpm_receptors(sim.ctx, 1, rec, 200.0, 18)
            out[f"{name}_grad"] = lpm.lpm_adjoint(sim.ctx, rec, 200.0, 18, w, 24)
    # a batch of candidates: segments sorted by scenario, then cell tile
    cand, _, _ = li.make_cfg4(n_candidates=3, n_per=2000, n_steps=200, n_obs=500)
    wb = np.linspace(-1.0, 1.0, cand.n_scenarios * rec.shape[0]).reshape(cand.n_scenarios, -1)
    for name, storage in [("adj_batch_traj", None), ("adj_batch_ckpt", 0)]:
        with Sim(cand) as sim:
            if storage is not None:
                lpm.lpm_set_adjoint_storage(sim.ctx, storage)
            out[f"{name}_C"] = lpm.lpm_receptors(sim.ctx, cand.n_scenarios, rec, 200.0, 18)
            out[f"{name}_grad"] = lpm.lpm_adjoint(sim.ctx, rec, 200.0, 18, wb, 24)
    return out
