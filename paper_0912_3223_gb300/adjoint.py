"""Differentiable receptor concentrations (torch.autograd.Function over the C ABI).

Forward: ``lpm_receptors`` (Gaussian-kernel receptor concentrations of every scenario,
keeping the states the backward needs: the whole trajectory, or 64-step checkpoints when
it does not fit). Backward: ``lpm_adjoint`` (hand-written reverse sweep of the
particle step with common random numbers and frozen events). Parameters per scenario:
the source (x_s, y_s, h) and the emission series q; shared: the diffusivity scale s_K
and the wind bias (b_u, b_v).
"""
from __future__ import annotations

import numpy as np
import torch

from . import lpm


def _apply(sim, sources, q, k_scale, bias):
    cfg = sim.cfg
    lpm.lpm_reset(sim.ctx)
    n_s = cfg.n_scenarios
    src = sources.detach().cpu().double().numpy().reshape(n_s, 3)
    qq = q.detach().cpu().double().numpy().reshape(n_s, -1)
    for s in range(n_s):
        woff = cfg.scenarios[s].wind_offset if cfg.scenarios else None
        lpm.lpm_set_source(sim.ctx, s, *src[s], woff)
        lpm.lpm_set_emission(sim.ctx, s, qq[s])
    b = bias.detach().cpu().double().numpy().reshape(2)
    lpm.lpm_set_params(sim.ctx, float(k_scale.detach().cpu()), float(b[0]), float(b[1]))


class ReceptorConcentrations(torch.autograd.Function):
    """C[s, r] = receptor concentrations; inputs sources [S, 3], q [S, n_q], k_scale [],
    bias [2] (float64 CPU tensors), then the ``Sim``, receptors [R, 3], the kernel
    bandwidth (m) and the sampling interval (steps)."""

    @staticmethod
    def forward(ctx, sources, q, k_scale, bias, sim, receptors, bandwidth, every):
        _apply(sim, sources, q, k_scale, bias)
        rec = np.ascontiguousarray(receptors, dtype=np.float64).reshape(-1, 3)
        C = lpm.lpm_receptors(sim.ctx, sim.cfg.n_scenarios, rec, bandwidth, every)
        ctx.sim, ctx.rec, ctx.bw, ctx.every, ctx.nq = sim, rec, float(bandwidth), int(every), q.shape[-1]
        ctx.state = (sources.detach().clone(), q.detach().clone(), k_scale.detach().clone(),
                     bias.detach().clone())
        return torch.from_numpy(C)

    @staticmethod
    def backward(ctx, dC):
        sim = ctx.sim
        sources, q, k_scale, bias = ctx.state
        _apply(sim, sources, q, k_scale, bias)      # the context may have moved on since
        g = lpm.lpm_adjoint(sim.ctx, ctx.rec, ctx.bw, ctx.every,
                            dC.detach().cpu().double().numpy(), ctx.nq)
        g = torch.from_numpy(g)
        nq = ctx.nq
        return (g[:, :3].reshape(sources.shape), g[:, 3:3 + nq].reshape(q.shape),
                g[:, 3 + nq].sum().reshape(k_scale.shape), g[:, 4 + nq:].sum(0).reshape(bias.shape),
                None, None, None, None)


def receptor_concentrations(sim, sources, q, k_scale, bias, receptors, bandwidth, every):
    return ReceptorConcentrations.apply(sources, q, k_scale, bias, sim, receptors, bandwidth, every)
