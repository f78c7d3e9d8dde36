"""The exchange step of a partitioned run on the CUDA path: two ranks (processes with
their own CUDA contexts on this GPU, gloo between them, no kernel waiting on the other
rank), each holding a contiguous particle range of one release, sum their hourly
snapshots, deposition grids and counters on the device (``SnapshotExchange``); the reduced
state equals a single context's bit for bit at every snapshot."""
import datetime
import os
import socket

import numpy as np
import pytest

import lpm_inputs as li

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_PARTICLES, N_STEPS, EVERY = 6007, 360, 120
STEP_COUNTERS = [0, 1, 2, 3, 4, 9, 10]         # the counters the steps accumulate


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()


def _cfg():
    return li.make_cfg1(n_particles=N_PARTICLES, n_steps=N_STEPS, n_hours=5)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.parallel import SnapshotExchange, partition, run_partitioned
    torch.cuda.set_device(0)
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=120))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    cfg = _cfg()
    out = {}
    with Sim(cfg, part=partition(cfg.n_particles, world, rank)) as sim:
        ex = SnapshotExchange(sim)
        for k in run_partitioned(sim, N_STEPS, EVERY, ex, store=store, world=world, rank=rank,
                                 timeout_s=60.0):
            sim.stream.synchronize()
            out[f"conc{k}"] = ex.conc.cpu().numpy()
            out[f"dep{k}"] = ex.dep.cpu().numpy()
            out[f"ctr{k}"] = ex.counters.cpu().numpy()
    if rank == 0:
        np.savez(os.path.join(out_dir, "exchange.npz"), **out)
    dist.barrier()
    dist.destroy_process_group()


def test_device_exchange_of_two_ranks_equals_a_single_context(tmp_path):
    import torch.multiprocessing as mp

    from paper_0912_3223_gb300 import Sim
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    red = np.load(tmp_path / "exchange.npz")
    cfg = _cfg()
    with Sim(cfg) as sim:
        for k in range(EVERY, N_STEPS + 1, EVERY):
            sim.step(EVERY)
            conc, dep, ctr, _ = sim.fixed_state()
            assert conc.sum() > 0
            assert np.array_equal(red[f"conc{k}"].view(np.uint64), conc), k
            assert np.array_equal(red[f"dep{k}"].view(np.uint64), dep), k
            assert np.array_equal(red[f"ctr{k}"][STEP_COUNTERS], ctr[STEP_COUNTERS]), k
