"""Batched source inversion: many candidate sources fitted at once to receptor data.

Every candidate is one scenario of a batched context (own source, same emission series,
weather and receptors). One iteration runs the receptor forward of all candidates
(``lpm_receptors``), forms each candidate's normalised misfit
L_s = sum_r (C_sr - C_obs_r)^2 / sum_r C_obs_r^2, and runs the adjoint of all candidates
with dL_s/dC_sr = 2 (C_sr - C_obs_r) / sum_r C_obs_r^2 (``lpm_adjoint``); the sources move
by Adam steps on (x_s, y_s, h). The forward and the adjoint are one launch each for all
candidates; the adjoint needs the complete forward sums, so they cannot share a launch.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional

import numpy as np

from . import lpm


@dataclasses.dataclass
class InversionResult:
    sources: np.ndarray          # [n_iter + 1][S][3] source estimates
    loss: np.ndarray             # [n_iter + 1][S] misfit (last row: final sources)
    grad: np.ndarray             # [n_iter][S][3]
    timings: Dict[str, float]    # seconds: forward, adjoint (summed over iterations)

    @property
    def best(self) -> int:
        return int(np.argmin(self.loss[-1]))


def observe(sim, receptors, bandwidth: float, every: int) -> np.ndarray:
    """Receptor concentrations of a (plain) context: the synthetic observations."""
    return lpm.lpm_receptors(sim.ctx, sim.cfg.n_scenarios, receptors, bandwidth, every)[0]


def invert(sim, receptors, c_obs, n_iter: int = 20, bandwidth: float = 200.0, every: int = 18,
           lr=(250.0, 250.0, 15.0), bounds: Optional[np.ndarray] = None,
           beta1: float = 0.9, beta2: float = 0.999) -> InversionResult:
    """Adam on every candidate's source; ``sim`` is a batched ``Sim`` whose scenarios are the
    candidates (their current sources are the starting points). ``bounds`` [3][2] clips the
    sources (default: the weather domain, heights 1..1000 m)."""
    import time
    cfg = sim.cfg
    S = cfg.n_scenarios
    rec = np.ascontiguousarray(receptors, dtype=np.float64).reshape(-1, 3)
    c_obs = np.asarray(c_obs, dtype=np.float64).reshape(-1)
    norm = float(np.sum(c_obs ** 2))
    if not norm > 0:
        raise ValueError("observations are all zero")
    nq = max(len(sc.release.q) for sc in cfg.scenarios)
    if bounds is None:
        bounds = np.array([[cfg.x0, cfg.x0 + (cfg.nx - 1) * cfg.dx],
                           [cfg.y0, cfg.y0 + (cfg.ny - 1) * cfg.dy], [1.0, 1000.0]])
    theta = np.array([[sc.src_x, sc.src_y, sc.src_z] for sc in cfg.scenarios], dtype=np.float64)
    lr = np.asarray(lr, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    srcs, losses, grads = [theta.copy()], [], []
    t_fwd = t_adj = 0.0

    def set_sources(th):
        for s in range(S):
            lpm.lpm_set_source(sim.ctx, s, *th[s], cfg.scenarios[s].wind_offset)

    for it in range(n_iter + 1):
        set_sources(theta)
        t0 = time.perf_counter()
        C = lpm.lpm_receptors(sim.ctx, S, rec, bandwidth, every)
        t_fwd += time.perf_counter() - t0
        resid = C - c_obs[None, :]
        losses.append(np.sum(resid ** 2, axis=1) / norm)
        if it == n_iter:
            break
        t0 = time.perf_counter()
        g = lpm.lpm_adjoint(sim.ctx, rec, bandwidth, every, 2.0 * resid / norm, nq)[:, :3]
        t_adj += time.perf_counter() - t0
        grads.append(g)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** (it + 1))
        vh = v / (1 - beta2 ** (it + 1))
        theta = theta - lr[None, :] * mh / (np.sqrt(vh) + 1e-30)
        theta = np.clip(theta, bounds[:, 0], bounds[:, 1])
        srcs.append(theta.copy())
    return InversionResult(np.array(srcs), np.array(losses), np.array(grads),
                           {"forward": t_fwd, "adjoint": t_adj})
