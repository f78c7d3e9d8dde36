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
CHAOS_MULT = 4.0         # a path's distance must stay within this multiple of its growth
                         # bound where that exceeds the position tolerance


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


def _cell_mask(cfg, near, g, o):
    """Cells of the concentration grid not touched (on either side) by an active particle
    flagged in ``near``."""
    active = (o["status"] == li.STATUS_ACTIVE) | (g["status"] == li.STATUS_ACTIVE)
    mask = np.ones(cfg.cz * cfg.cy * cfg.cx, bool)
    for pos in (o["pos"], g["pos"]):
        idx = cell_index(cfg, pos[near & active])
        mask[idx[idx >= 0]] = False
    return mask.reshape(cfg.cz, cfg.cy, cfg.cx)


def _grid_l1(cfg, g, o, mask):
    ref = o["conc"][mask]
    denom = np.abs(ref).sum()
    return float(np.abs(g["conc_mass"][mask] - ref).sum() / denom) if denom > 0 else 0.0


def compare(cfg, g, o, pos_tol=POS_TOL_M, grid_tol=GRID_REL_L1, check_grid=True,
            max_excluded_frac=0.01, sens=None, max_chaotic_frac=0.01):
    """Element-wise comparison of a GPU run ``g`` with an oracle run ``o`` over the same
    particles (all of the release). A particle held to the position tolerance is within
    ``pos_tol``; one whose path the oracle's perturbation growth (``sens``) shows to be
    chaotic is held to CHAOS_MULT times its growth bound instead; one that met an event
    boundary within ``pos_tol`` may branch either way and is held to its distance only
    while it still moves on both sides. Returns a report dict; asserts the bars."""
    rep = {}
    assert np.array_equal(g["release"], o["release"]), "release steps differ"
    released = o["status"] != li.STATUS_UNRELEASED
    assert np.array_equal(g["status"] == li.STATUS_UNRELEASED, ~released)
    # particles that took a decision within pos_tol of its boundary may branch either way
    near_event = (o["margin"] < pos_tol) & released
    all_dist = np.linalg.norm(g["pos"] - o["pos"], axis=1)
    same_status = g["status"] == o["status"]
    # the distance each particle is held to: pos_tol, or, on a path whose FP32 rounding is
    # expected (growth bound) to grow past it, CHAOS_MULT times that bound
    allowed = np.full(all_dist.shape, float(pos_tol))
    ch = np.zeros_like(released)
    if sens is not None:
        bound = oracle.growth_bound(sens, o["pos"])
        widened = (CHAOS_MULT * bound > pos_tol) & released
        allowed = np.where(widened, CHAOS_MULT * bound, allowed)
        ch = (bound > pos_tol) & released & ~near_event
        rep["chaotic"] = int(ch.sum())
        assert ch.mean() <= max_chaotic_frac, rep
        rep["growth_widened"] = int((widened & ~near_event).sum())
        rep["chaotic_status_mismatch"] = int((ch & ~same_status).sum())
        cs = widened & same_status & ~near_event
        if cs.any():
            rep["widened_max_ratio"] = float((all_dist[cs] / bound[cs]).max())
    # a particle that met an event boundary within pos_tol may branch either way; one still
    # moving on both sides took the same branches, and is held to its distance as well
    # (one that ended on both sides may have ended at different steps)
    rep["near_event"] = int(near_event.sum())
    rep["near_event_status_mismatch"] = int((near_event & ~same_status).sum())
    ne = near_event & same_status & (o["status"] == li.STATUS_ACTIVE)
    if sens is not None and ne.any():
        rep["near_event_max_ratio"] = float((all_dist[ne] / allowed[ne]).max())
        assert rep["near_event_max_ratio"] <= 1.0, rep
    ambiguous = near_event | ch
    rep["ambiguous"] = int(ambiguous.sum())
    rep["excluded_frac"] = float(ambiguous.sum() / max(1, released.sum()))
    assert ambiguous.mean() <= max_excluded_frac, rep
    # every other released particle: the same status (a chaotic path may have crossed an
    # event boundary the other way), within its distance
    ok = ~near_event & released
    st_eq = g["status"][ok & ~ch] == o["status"][ok & ~ch]
    assert st_eq.all(), f"{(~st_eq).sum()} status mismatches"
    ok &= same_status
    strict = ok & ~ch & (allowed <= pos_tol)
    dist = all_dist[strict]
    rep["max_dist"] = float(dist.max()) if dist.size else 0.0
    rep["median_dist"] = float(np.median(dist)) if dist.size else 0.0
    assert rep["max_dist"] <= pos_tol, rep
    over = all_dist[ok] > allowed[ok]
    rep["over_allowed"] = int(over.sum())
    assert not over.any(), rep
    if not check_grid:
        return rep
    # the grid with only the stated face band excluded (cells holding a particle within
    # 1e-3 m of a face), every particle included: reported beside the gated figure below
    rep["grid_rel_l1_face_band_only"] = _grid_l1(cfg, g, o, _cell_mask(
        cfg, (face_distance(cfg, o["pos"]) < FACE_EPS_M), g, o))
    # grid: exclude cells touched by ambiguous particles or by particles nearer to a face
    # than the larger of 1e-3 m and their own distance (only those can be binned apart)
    eps = np.maximum(FACE_EPS_M, all_dist)
    mask = _cell_mask(cfg, (face_distance(cfg, o["pos"]) < eps) | ambiguous, g, o)
    rep["excluded_cells"] = int((~mask).sum())
    rep["cells_with_mass"] = int((o["conc"] > 0).sum())
    rep["grid_rel_l1"] = _grid_l1(cfg, g, o, mask)
    assert rep["grid_rel_l1"] <= grid_tol, rep
    # deposition grids (horizontal cells of deposited particles)
    dep_near = ambiguous | ~same_status | (face_distance(cfg, o["pos"]) < eps)
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


def oracle_sharded(cfg, n_run, n_particles, with_sens=True, threads=None, chunks=None, **kw):
    """The oracle over particles [0, n_particles) of the release, run in contiguous shards
    on host threads (the oracle's C calls release the interpreter lock and share no
    state), put together as one run: per-particle arrays concatenated in particle order;
    grids, budgets and counters summed (the fixed-point grids exactly); the snapshot count
    taken once. With ``with_sens`` the per-particle perturbation growth of the same run
    comes back as ``sens``."""
    import concurrent.futures as cf
    import os
    threads = threads or os.cpu_count() or 1
    chunks = chunks or 4 * threads
    bounds = np.linspace(0, n_particles, chunks + 1).astype(np.int64)
    jobs = [np.arange(a, b, dtype=np.int64) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]

    def one(sel):
        r = oracle.run(cfg, sel=sel, n_run=n_run, **kw)
        if with_sens:
            r["sens"] = oracle.sensitivity(cfg, sel=sel, n_run=n_run, **kw)
        return r

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, jobs))
    out = {}
    per_particle = ["pos", "status", "release", "margin", "wvel"] + (["sens"] if with_sens else [])
    for key in per_particle:
        out[key] = np.concatenate([p[key] for p in parts])
    for key in ("conc", "conc_fixed", "dep", "dep_fixed", "budget", "dose", "dose_fixed"):
        out[key] = sum(p[key] for p in parts)
    ctr = sum(p["counters"] for p in parts)
    ctr[5] = parts[0]["counters"][5]              # snapshots taken: the same in every shard
    out["counters"] = ctr
    out["active_steps"] = int(ctr[4])
    return out


def gpu_state(sim, cfg, n, grids=True):
    """Particles [0, n) of a running one-scenario context and (with ``grids``) its last
    snapshot and deposition grids in the form ``compare`` takes."""
    xyz, tag = sim.particles(0, n)
    g = dict(pos=xyz.astype(np.float64), tag=tag, status=(tag >> 28).astype(np.int32),
             release=(tag & 0x0FFFFFFF).astype(np.int64))
    if grids:
        vol = cfg.cdx * cfg.cdy * cfg.cdz
        dry, wet = sim.deposition()
        g.update(conc_mass=sim.concentration() * vol,
                 dep_mass=np.stack([dry, wet]) * cfg.cdx * cfg.cdy, budget=sim.budget())
        g["conc_fixed"], g["dep_fixed"], g["counters"], g["shift"] = sim.fixed_state()
    return g
