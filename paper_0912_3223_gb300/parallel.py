"""Particle-range partitioning across ranks and the one exchange step of a partitioned run.

Particles never interact (Sec. 4.2), so a release of N particles splits into contiguous
id ranges, one per rank; each rank's context holds its range (``lpm_release_range``),
draws the same keyed random numbers as a single run would, and bins with the scale of
the whole release. The only exchange is an integer sum of the fixed-point grids and
counters, which is associative, so the reduced result is bit-identical to the
single-context run whatever the rank count or reduction order. A batched ensemble
shards by scenario instead: ``partition(n_scenarios, world, rank)`` gives each rank a
contiguous scenario range (``Sim(cfg, scenarios=...)``, global particle ids kept), whose
grids are final without any exchange.

The receptor concentrations and the adjoint's parameter gradients are FP64 sums over
particles, so a partitioned run adds the ranks' partial sums. They are exchanged in fixed
point as well: each element is scaled by a power of two fitted to the largest magnitude of
that element over the ranks (a MAX reduction), rounded to int64, summed as integers and
scaled back, so the reduced value does not depend on the order in which ranks are added.
For a loss that is not linear in the concentrations, the receptor sums are reduced first,
every rank forms the same dL/dC from them, and the gradients taken with it are reduced
second.

On GPUs the exchange works on the library's device grids directly (``SnapshotExchange``:
one device copy into a staging buffer and one integer all-reduce, NCCL between GPUs). A
rank that leaves between steps is detected on the host before the next exchange: every
rank announces each exchange in the process group's store and waits, for a bounded time,
for the others' announcements (``check_ranks``), so the survivors raise ``RankLost``
naming the missing ranks instead of entering a collective that cannot complete.
"""
from __future__ import annotations

import time
from typing import Iterable, List, Tuple

import numpy as np


def partition(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous range [first, first + count) of ``n_total`` ids (particles, or the
    scenarios of an ensemble) held by ``rank``; range sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    if n_total < world:
        raise ValueError("fewer particles than ranks")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def allreduce_fixed(values: np.ndarray, group=None, device=None) -> np.ndarray:
    """Integer sum over all ranks of a fixed-point array (uint64 or int64 values below
    2^63) through torch.distributed; returns an array of the input dtype."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(values)
    t = torch.from_numpy(a.view(np.int64).copy())
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(a.dtype).reshape(a.shape)


FIXED_BITS = 62          # |reduced sum| * 2^scale stays below 2^62 whatever the rank count


def fixed_exponents(max_abs: np.ndarray, world: int) -> np.ndarray:
    """Per-element power-of-two exponent e such that world * max_abs * 2^e <= 2^FIXED_BITS
    (0 where the element is zero on every rank)."""
    m = np.asarray(max_abs, dtype=np.float64)
    if not np.all(np.isfinite(m)):
        raise ValueError("non-finite value in a fixed-point reduction")
    bound = m * world
    e = np.zeros(m.shape, dtype=np.int64)
    nz = bound > 0
    e[nz] = FIXED_BITS - np.ceil(np.log2(bound[nz])).astype(np.int64)
    return e


def to_fixed(values: np.ndarray, e: np.ndarray) -> np.ndarray:
    """round(values * 2^e) as int64 (exact scaling by a power of two, one rounding)."""
    return np.rint(np.ldexp(np.asarray(values, dtype=np.float64), e)).astype(np.int64)


def from_fixed(q: np.ndarray, e: np.ndarray) -> np.ndarray:
    return np.ldexp(np.asarray(q, dtype=np.int64).astype(np.float64), -e)


def sum_float_fixed(parts) -> np.ndarray:
    """The fixed-point sum of FP64 partial arrays held by one process (one per partition),
    with the same arithmetic as ``allreduce_float_fixed`` over that many ranks."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    e = fixed_exponents(np.max(np.abs(np.stack(parts)), axis=0), len(parts))
    return from_fixed(np.sum(np.stack([to_fixed(p, e) for p in parts]), axis=0), e)


def allreduce_float_fixed(values: np.ndarray, group=None, device=None) -> np.ndarray:
    """Sum over all ranks of an FP64 array, reduced in fixed point: a MAX reduction of the
    magnitudes fixes each element's scale, then an int64 SUM reduction adds the rounded
    values; the result is independent of the reduction order."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(values, dtype=np.float64)
    world = dist.get_world_size(group)
    mag = np.abs(a)
    mag[~np.isfinite(mag)] = np.inf              # MAX carries inf to every rank (NaN may not),
    m = torch.from_numpy(mag)                    # so all ranks raise before the SUM together
    if device is not None:
        m = m.to(device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    e = fixed_exponents(m.cpu().numpy(), world)
    q = torch.from_numpy(to_fixed(a, e))
    if device is not None:
        q = q.to(device)
    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return from_fixed(q.cpu().numpy(), e)


def receptors_partitioned(sim, receptors, bandwidth: float, sample_every: int, group=None,
                          device=None) -> np.ndarray:
    """Receptor concentrations [n_scenarios][R] of the whole release, from each rank's
    context holding its particle range."""
    from . import lpm
    c = lpm.lpm_receptors(sim.ctx, sim.cfg.n_scenarios, receptors, bandwidth, sample_every)
    return allreduce_float_fixed(c, group, device)


def adjoint_partitioned(sim, receptors, bandwidth: float, sample_every: int, dL_dC, n_q: int,
                        group=None, device=None) -> np.ndarray:
    """Gradient [n_scenarios][3 + n_q + 3] of sum(dL_dC * C) for the whole release; dL_dC
    must be the same on every rank (formed from ``receptors_partitioned``)."""
    from . import lpm
    g = lpm.lpm_adjoint(sim.ctx, receptors, bandwidth, sample_every, dL_dC, n_q)
    return allreduce_float_fixed(g, group, device)


# ------------------------------------------------------------------------------------
# The exchange on the device, and rank liveness
# ------------------------------------------------------------------------------------
N_COUNTERS = 16


class _DeviceWords:
    """A library-owned device array described by the CUDA array interface (no copy; the
    exchange only reads it)."""

    def __init__(self, ptr: int, n: int, stride: int = 1):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False),
                                         "strides": (8 * stride,), "version": 2}


class SnapshotExchange:
    """The exchange step of a run partitioned by particle ranges, on the device: the
    context's last snapshot, cumulative deposition grids and counters (scenario 0) are
    copied, on the context stream, into one staging buffer and summed over the ranks by
    one int64 all-reduce; the context's own state is left as it is (the deposition grids
    keep accumulating each rank's own deposits). After ``__call__`` the attributes
    ``conc``, ``dep`` and ``counters`` hold the whole release's fixed-point state."""

    def __init__(self, sim, group=None):
        import torch
        from . import lpm
        self.sim, self.group = sim, group
        cfg = sim.cfg
        conc, dep, ctr, stride = lpm.lpm_device_state(sim.ctx, 0)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.n_conc = cfg.cz * cfg.cy * cfg.cx
        self.n_dep = 2 * cfg.cy * cfg.cx
        self._src = [torch.as_tensor(_DeviceWords(conc, self.n_conc), device=dev),
                     torch.as_tensor(_DeviceWords(dep, self.n_dep), device=dev),
                     torch.as_tensor(_DeviceWords(ctr, N_COUNTERS, stride), device=dev)]
        self.buf = torch.empty(self.n_conc + self.n_dep + N_COUNTERS, dtype=torch.int64,
                               device=dev)
        self.conc = self.buf[:self.n_conc].view(cfg.cz, cfg.cy, cfg.cx)
        self.dep = self.buf[self.n_conc:self.n_conc + self.n_dep].view(2, cfg.cy, cfg.cx)
        self.counters = self.buf[self.n_conc + self.n_dep:]

    @property
    def bytes(self) -> int:
        """Bytes each rank contributes to one exchange."""
        return int(self.buf.numel() * 8)

    def __call__(self):
        import torch
        import torch.distributed as dist
        with torch.cuda.stream(self.sim.stream):
            torch.cat(self._src, out=self.buf)
            if dist.is_initialized() and dist.get_world_size(self.group) > 1:
                dist.all_reduce(self.buf, op=dist.ReduceOp.SUM, group=self.group)
        return self


class RankLost(RuntimeError):
    """Ranks that did not reach an exchange within the time limit (they left the run)."""

    def __init__(self, missing: List[int], tag: str):
        self.missing = list(missing)
        self.tag = tag
        super().__init__(f"rank(s) {self.missing} did not reach exchange {tag!r}: they left "
                         "the partitioned run")


def check_ranks(store, tag: str, world: int, rank: int, timeout_s: float = 10.0,
                poll_s: float = 0.01) -> None:
    """Announces that this rank reached the exchange ``tag`` and waits, at most
    ``timeout_s``, for every other rank's announcement; raises ``RankLost`` with the ranks
    still missing. Host only: nothing waits on the device."""
    store.set(f"lpm/alive/{tag}/{rank}", "1")
    missing = set(range(world)) - {rank}
    deadline = time.monotonic() + timeout_s
    while missing:
        for r in sorted(missing):
            if store.check([f"lpm/alive/{tag}/{r}"]):
                missing.discard(r)
        if not missing:
            break
        if time.monotonic() >= deadline:
            raise RankLost(sorted(missing), tag)
        time.sleep(poll_s)


def run_partitioned(sim, n_steps: int, exchange_every: int, exchange, store=None,
                    world: int = 1, rank: int = 0, timeout_s: float = 10.0,
                    run_tag: str = "") -> Iterable[int]:
    """Steps ``sim`` through ``n_steps`` in pieces of ``exchange_every`` steps; after each
    piece the ranks check one another's presence (with a ``store``; ``run_tag`` keeps the
    announcements of repeated runs apart) and run ``exchange``. Yields the step count
    after each exchange."""
    k = sim.k
    while k < n_steps:
        n = min(exchange_every - k % exchange_every, n_steps - k)
        sim.step(n)
        k += n
        if store is not None and world > 1:
            check_ranks(store, f"{run_tag}step{k}", world, rank, timeout_s)
        exchange()
        yield k
