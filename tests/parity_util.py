"""Shared helpers of the GPU parity tests: run both sides on the same seeded inputs and
compare element by element with the stated exclusions."""
import dataclasses
import math

import numpy as np

import lpm_inputs as li
import oracle

POS_TOL_M = 0.5          # per-particle distance after 360 steps
GRID_REL_L1 = 1e-4       # concentration / deposition grids, relative L1
FACE_EPS_M = 1e-3        # a particle closer than this (or than the measured distance) to a
                         # cell face makes the cell's bin ambiguous


def artificial_weather_cfg(n_particles=2160, n_steps=2160, nz=25):
    """The paper's homogeneous case (Fig. 3b caption) with the readings listed in
    tests/golden/artificial_weather.txt."""
    vals = {}
    for line in open(__file__.replace("parity_util.py", "golden/artificial_weather.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    k = 0.4
    ustar = k * vals["wind_u_m_s"] / math.log(vals["source_height_m"] / vals["z0_m"])
    hm = vals["h_mix_m"]
    z_levels = np.linspace(0.0, 300.0, nz)
    kz = k * ustar * z_levels * (1 - z_levels / hm) ** 2
    kz = np.where(z_levels >= hm, 0.1, np.maximum(kz, 0.1))
    uvwk = np.zeros((2, nz, 2, 2, 4), np.float32)
    uvwk[..., 0] = vals["wind_u_m_s"]
    uvwk[..., 1] = vals["wind_v_m_s"]
    uvwk[..., 2] = vals["wind_w_m_s"]
    uvwk[..., 3] = kz[None, :, None, None]
    cfg = li.make_cfg0(n_particles=int(vals["n_particles"]), n_steps=n_steps,
                       kh=vals["kh_m2_s"], src=(0.0, 0.0, vals["source_height_m"]))
    cfg = dataclasses.replace(
        cfg, z_levels=z_levels, uvwk=uvwk, nz=nz, dt=vals["dt_s"], vd_dry=0.002, h_mix=hm,
        x0=-1000.0, dx=200000.0, cx=100, cy=60, cz=15, cx0=-1000.0, cy0=-6000.0, cdx=1200.0,
        cdy=200.0, cdz=20.0, bin_every=360, reflect_top=1, z_top=300.0,
        release=li.Release(int(vals["n_particles"]), np.array([1.0]), 3600.0, 0, n_steps),
        name="artificial weather (Fig. 3b)")
    if n_particles != int(vals["n_particles"]):
        cfg = dataclasses.replace(cfg, release=dataclasses.replace(cfg.release,
                                                                   n_particles=n_particles))
    return cfg


def run_gpu(cfg, n_run=None, launch=None, pieces=None, met_on_device=False, sort_every=None,
            id_base=0):
    from paper_0912_3223_gb300 import Sim
    n_run = cfg.n_steps if n_run is None else n_run
    sim = Sim(cfg, launch=launch, met_on_device=met_on_device, sort_every=sort_every,
              id_base=id_base)
    try:
        if pieces:
            for n in pieces:
                sim.step(n)
        else:
            sim.step(n_run)
        xyz, tag = sim.particles()
        conc = sim.concentration()
        dry, wet = sim.deposition()
        budget = sim.budget()
        cfix, dfix, ctr, shift = sim.fixed_state()
    finally:
        sim.close()
    vol = cfg.cdx * cfg.cdy * cfg.cdz
    area = cfg.cdx * cfg.cdy
    return dict(pos=xyz.astype(np.float64), tag=tag, status=(tag >> 28).astype(np.int32),
                release=(tag & 0x0FFFFFFF).astype(np.int64), conc_mass=conc * vol,
                dep_mass=np.stack([dry, wet]) * area, budget=budget, conc_fixed=cfix,
                dep_fixed=dfix, counters=ctr, shift=shift)


def face_distance(cfg, pos):
    """Distance of each position to the nearest face of the concentration grid's cells."""
    d = np.full(pos.shape[0], np.inf)
    for axis, (c0, cd) in enumerate([(cfg.cx0, cfg.cdx), (cfg.cy0, cfg.cdy), (cfg.cz0, cfg.cdz)]):
        f = (pos[:, axis] - c0) / cd
        d = np.minimum(d, np.abs(f - np.round(f)) * cd)
    return d


def cell_index(cfg, pos, horizontal=False):
    ix = np.floor((pos[:, 0] - cfg.cx0) / cfg.cdx).astype(np.int64)
    iy = np.floor((pos[:, 1] - cfg.cy0) / cfg.cdy).astype(np.int64)
    iz = np.floor((pos[:, 2] - cfg.cz0) / cfg.cdz).astype(np.int64)
    ok = (ix >= 0) & (ix < cfg.cx) & (iy >= 0) & (iy < cfg.cy)
    if horizontal:
        return np.where(ok, iy * cfg.cx + ix, -1)
    ok &= (iz >= 0) & (iz < cfg.cz)
    return np.where(ok, (iz * cfg.cy + iy) * cfg.cx + ix, -1)


def compare(cfg, g, o, pos_tol=POS_TOL_M, grid_tol=GRID_REL_L1, check_grid=True,
            max_excluded_frac=0.01, sens=None, max_chaotic_frac=0.01):
    """Element-wise comparison of a GPU run ``g`` with an oracle run ``o`` over the same
    particles (all of the release). ``sens`` (the oracle's perturbation growth per
    particle) marks chaotic paths, which are reported and excluded like ambiguous ones.
    Returns a report dict; asserts the bars."""
    rep = {}
    assert np.array_equal(g["release"], o["release"]), "release steps differ"
    released = o["status"] != li.STATUS_UNRELEASED
    assert np.array_equal(g["status"] == li.STATUS_UNRELEASED, ~released)
    # particles that took a decision within pos_tol of its boundary may branch either way
    ambiguous = (o["margin"] < pos_tol) & released
    if sens is not None:
        ch = oracle.chaotic(cfg, sens, o["pos"], pos_tol) & released & ~ambiguous
        rep["chaotic"] = int(ch.sum())
        assert ch.mean() <= max_chaotic_frac, rep
        ambiguous = ambiguous | ch
    rep["ambiguous"] = int(ambiguous.sum())
    assert ambiguous.mean() <= max_excluded_frac, rep
    ok = ~ambiguous & released
    st_eq = g["status"][ok] == o["status"][ok]
    assert st_eq.all(), f"{(~st_eq).sum()} status mismatches"
    dist = np.linalg.norm(g["pos"][ok] - o["pos"][ok], axis=1)
    rep["max_dist"] = float(dist.max()) if dist.size else 0.0
    rep["median_dist"] = float(np.median(dist)) if dist.size else 0.0
    assert rep["max_dist"] <= pos_tol, rep
    if not check_grid:
        return rep
    # grid: exclude cells touched by ambiguous particles or by particles near a face
    eps = max(FACE_EPS_M, rep["max_dist"])
    active = (o["status"] == li.STATUS_ACTIVE) | (g["status"] == li.STATUS_ACTIVE)
    near = (face_distance(cfg, o["pos"]) < eps) | ambiguous
    bad = set()
    for pos in (o["pos"], g["pos"]):
        idx = cell_index(cfg, pos[near & active])
        bad.update(int(i) for i in idx[idx >= 0])
    mask = np.ones(cfg.cz * cfg.cy * cfg.cx, bool)
    mask[list(bad)] = False
    mask = mask.reshape(cfg.cz, cfg.cy, cfg.cx)
    rep["excluded_cells"] = int((~mask).sum())
    ref = o["conc"][mask]
    got = g["conc_mass"][mask]
    denom = np.abs(ref).sum()
    rep["grid_rel_l1"] = float(np.abs(got - ref).sum() / denom) if denom > 0 else 0.0
    assert rep["grid_rel_l1"] <= grid_tol, rep
    # deposition grids (horizontal cells of deposited particles)
    dep_near = ambiguous | (face_distance(cfg, o["pos"]) < eps)
    dmask = np.ones(cfg.cy * cfg.cx, bool)
    for pos in (o["pos"], g["pos"]):
        idx = cell_index(cfg, pos[dep_near], horizontal=True)
        dmask[idx[idx >= 0]] = False
    dmask = dmask.reshape(cfg.cy, cfg.cx)
    for kind in range(2):
        ref = o["dep"][kind][dmask]
        got = g["dep_mass"][kind][dmask]
        denom = np.abs(ref).sum()
        if denom > 0:
            rel = float(np.abs(got - ref).sum() / denom)
            rep[f"dep{kind}_rel_l1"] = rel
            assert rel <= grid_tol, rep
    return rep
