"""Partitioned runs: contiguous particle ranges per rank and one integer all-reduce give
exactly the single-run grids. Exercised on CPU ranks (gloo, world size 2 and 3) with the
oracle standing in for each rank's particle kernel."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import lpm_inputs as li
import oracle
from paper_0912_3223_gb300.parallel import allreduce_fixed, partition


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
