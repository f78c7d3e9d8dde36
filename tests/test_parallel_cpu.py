"""Partitioned runs: contiguous particle ranges per rank and one integer all-reduce give
exactly the single-run grids; the receptor concentrations and adjoint gradients, FP64 sums
over particles, are reduced in fixed point and match the single run to rounding.
Exercised on CPU ranks (gloo, world size 2 and 3) with the oracle standing in for each
rank's particle kernel."""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import lpm_inputs as li
import oracle
from paper_0912_3223_gb300.parallel import (allreduce_fixed, allreduce_float_fixed,
                                            partition, sum_float_fixed)


def test_partition_covers_every_id_once():
    for n, w in [(10, 1), (10, 3), (10_000_000, 8), (7, 7), (1001, 4)]:
        ranges = [partition(n, w, r) for r in range(w)]
        assert ranges[0][0] == 0
        for (a, na), (b, _) in zip(ranges, ranges[1:]):
            assert a + na == b
        assert sum(c for _, c in ranges) == n
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        partition(3, 4, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = li.make_cfg1(n_particles=600, n_steps=150, n_hours=4)
    first, count = partition(cfg.n_particles, world, rank)
    r = oracle.run(cfg, sel=np.arange(first, first + count))
    conc = allreduce_fixed(r["conc_fixed"])
    dep = allreduce_fixed(r["dep_fixed"])
    ctr = allreduce_fixed(r["counters"][:5])
    if rank == 0:
        np.savez(os.path.join(out_dir, "reduced.npz"), conc=conc, dep=dep, ctr=ctr)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_partitioned_reduction_matches_single_run(tmp_path, world):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    red = np.load(tmp_path / "reduced.npz")
    cfg = li.make_cfg1(n_particles=600, n_steps=150, n_hours=4)
    full = oracle.run(cfg)
    assert np.array_equal(red["conc"], full["conc_fixed"])
    assert np.array_equal(red["dep"], full["dep_fixed"])
    assert np.array_equal(red["ctr"], full["counters"][:5])
    assert full["conc_fixed"].sum() > 0


# ------------------------------------------------------------------------------------
# Receptors and adjoint gradients of a partitioned run (FP64 sums reduced in fixed point)
# ------------------------------------------------------------------------------------
SIGMA = 200.0
EVERY = 12
REC = np.array([[9000.0, 24875.0, 2.0], [12000.0, 25500.0, 30.0], [7000.0, 24000.0, 80.0],
                [15000.0, 24500.0, 10.0]])


def _adjoint_cfg():
    base = li.make_cfg1(n_particles=500, n_steps=120, n_hours=3, with_rain=False)
    return dataclasses.replace(base, release=li.Release(500, np.array([1.0, 3.0]), 1800.0, 0, 120))


def _obs(c):
    return 0.5 * c + 1e-12                       # a misfit that is not linear in C


def _adjoint_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _adjoint_cfg()
    first, count = partition(cfg.n_particles, world, rank)
    sel = np.arange(first, first + count)
    c = allreduce_float_fixed(oracle.receptors(cfg, REC, SIGMA, EVERY, sel=sel))
    w = 2.0 * (c - _obs(c))                      # dL/dC of sum (C - obs)^2, the same on all ranks
    g = allreduce_float_fixed(oracle.adjoint(cfg, REC, SIGMA, EVERY, w, sel=sel))
    if rank == 0:
        np.savez(os.path.join(out_dir, "adjoint.npz"), c=c, g=g)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_partitioned_receptors_and_adjoint_match_single_run(tmp_path, world):
    """Receptor sums reduced first, then every rank forms the same dL/dC and the gradients
    are reduced: both match the single run to FP64 rounding, and equal bit for bit the
    fixed-point sum of the partitions computed in one process (order independence)."""
    mp.start_processes(_adjoint_worker, args=(world, _free_port(), str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    red = np.load(tmp_path / "adjoint.npz")
    cfg = _adjoint_cfg()
    c_full = oracle.receptors(cfg, REC, SIGMA, EVERY)
    assert np.abs(c_full).max() > 0
    np.testing.assert_allclose(red["c"], c_full, rtol=1e-12, atol=1e-15 * np.abs(c_full).max())
    w = 2.0 * (red["c"] - _obs(red["c"]))
    g_full = oracle.adjoint(cfg, REC, SIGMA, EVERY, w)
    assert np.count_nonzero(g_full) == g_full.size
    np.testing.assert_allclose(red["g"], g_full, rtol=1e-10, atol=1e-12 * np.abs(g_full).max())
    ranges = [partition(cfg.n_particles, world, r) for r in range(world)]
    parts = [oracle.adjoint(cfg, REC, SIGMA, EVERY, w, sel=np.arange(a, a + n)) for a, n in ranges]
    assert np.array_equal(sum_float_fixed(parts), red["g"])
    assert np.array_equal(sum_float_fixed(parts[::-1]), red["g"])


def test_fixed_point_float_sum_is_order_independent_and_exact_to_rounding():
    """Per-element scales from the largest magnitude: elements spanning 1e-30..1e30 keep
    full relative precision, zeros stay zero, and any order of the parts gives the same
    bits."""
    rng = np.random.default_rng(5)
    mags = 10.0 ** rng.integers(-30, 30, size=16)
    parts = [rng.normal(size=16) * mags for _ in range(5)]
    for p in parts:
        p[3] = 0.0
    ref = np.sum(np.array(parts, dtype=np.longdouble), axis=0).astype(np.float64)
    got = sum_float_fixed(parts)
    assert got[3] == 0.0
    np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)
    for perm in ([4, 3, 2, 1, 0], [2, 0, 4, 1, 3]):
        assert np.array_equal(sum_float_fixed([parts[i] for i in perm]), got)
    with pytest.raises(ValueError):
        sum_float_fixed([np.array([1.0, np.inf])])


def _nan_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = np.array([1.0, 2.0, 3.0])
    if rank == 1:
        vals[1] = np.nan
    try:
        allreduce_float_fixed(vals)
        outcome = "reduced"
    except ValueError:
        outcome = "raised"
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(outcome)
    dist.destroy_process_group()


def test_gloo_non_finite_value_on_one_rank_raises_on_every_rank(tmp_path):
    """A NaN held by one rank makes every rank raise before the integer sum, so no rank is
    left waiting in a collective the others never enter."""
    world = 3
    mp.start_processes(_nan_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        assert (tmp_path / f"rank{r}.txt").read_text() == "raised"


# ------------------------------------------------------------------------------------
# A rank that leaves between steps
# ------------------------------------------------------------------------------------
def _leaving_worker(rank, world, store_port, out_dir, leaver):
    import datetime

    import torch.distributed as dist
    from paper_0912_3223_gb300.parallel import RankLost, check_ranks
    store = dist.TCPStore("127.0.0.1", store_port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    cfg = li.make_cfg1(n_particles=300, n_steps=150, n_hours=4)
    first, count = partition(cfg.n_particles, world, rank)
    sel = np.arange(first, first + count)
    log = []
    try:
        for k in (50, 100, 150):                 # three exchange steps
            r = oracle.run(cfg, sel=sel, n_run=k)
            check_ranks(store, f"step{k}", world, rank, timeout_s=5.0)
            allreduce_fixed(r["conc_fixed"])
            log.append(f"exchanged {k}")
            if rank == leaver and k == 50:
                log.append("left")               # leaves between steps, nothing in flight
                break
    except RankLost as e:
        log.append(f"lost {e.missing} at {e.tag}")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write("\n".join(log))
    if rank != 0:
        return                                   # rank 0 keeps the store up for the others
    import time
    time.sleep(2.0)


def test_gloo_rank_leaving_between_steps_is_reported_by_the_others(tmp_path):
    """Three CPU ranks exchange after every 50 steps; rank 2 leaves after the first
    exchange. The others detect it on the host before the next exchange (their store
    announcements go unanswered within the time limit) and report the missing rank
    instead of waiting in a collective it will never join."""
    world, leaver = 3, 2
    mp.start_processes(_leaving_worker, args=(world, _free_port(), str(tmp_path), leaver),
                       nprocs=world, join=True, start_method="spawn")
    logs = {r: (tmp_path / f"rank{r}.txt").read_text().splitlines() for r in range(world)}
    assert logs[leaver] == ["exchanged 50", "left"]
    for r in range(world):
        if r != leaver:
            assert logs[r] == ["exchanged 50", f"lost [{leaver}] at step100"], logs[r]
