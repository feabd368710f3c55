"""FP64 oracle of the grain-growth example (test infrastructure only).

Sec. 3.3.1, Eq. grain-growth-equations: the multi-order-parameter Allen-Cahn system of Fan and Chen,
    d eta_i / dt = -L_i ( -alpha eta_i + beta eta_i^3 + 2 gamma eta_i sum_{j != i} eta_j^2
                          - kappa_i Lap eta_i ),   i = 1..q,
with L_i = 1, alpha = beta = gamma = 1, kappa_i = 2, periodic boundaries in every direction (reading
A17 of cell_centred), h = 2, dt = 0.25, initial values U(-0.001, 0.001).

Readings (the paper prints no time discretisation for this example):
  GG1 Linearly implicit backward Euler: the diffusion term is implicit, the local terms explicit,
          (1 - dt L_i kappa_i Lap_h) eta_i^{n+1}
              = eta_i^n - dt L_i ( -alpha eta_i^n + beta (eta_i^n)^3 + 2 gamma eta_i^n (phi^n - (eta_i^n)^2) ),
      phi^n = sum_j (eta_j^n)^2. Each order parameter is then one solve of the cell-centred operator
      with alpha' = 1, beta' = dt L_i kappa_i and constant diffusivity: the solver of this package,
      applied to q independent right-hand sides (a batched workload).
  GG2 The sum over j != i is written phi - eta_i^2 with phi formed once per step from the old values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cell_centred as cc


@dataclass
class GrainParams:
    """Model constants of Sec. 3.3.1 (the paper's values as defaults) and the step."""

    L: float = 1.0
    alpha: float = 1.0
    beta: float = 1.0
    gamma: float = 1.0
    kappa: float = 2.0
    dt: float = 0.25
    h: float = 2.0


def local_rate(etas: np.ndarray, p: GrainParams) -> np.ndarray:
    """The local (non-diffusive) part of the bracket for every i:
    -alpha eta_i + beta eta_i^3 + 2 gamma eta_i (phi - eta_i^2) (readings GG1, GG2)."""
    phi = np.sum(etas * etas, axis=0)
    return -p.alpha * etas + p.beta * etas ** 3 + 2.0 * p.gamma * etas * (phi[None] - etas * etas)


def step_operator(shape, p: GrainParams) -> cc.Operator:
    """(1 - dt L kappa Lap_h) on the periodic grid: alpha' = 1, beta' = dt L kappa."""
    return cc.Operator(shape, p.h, 1.0, p.dt * p.L * p.kappa, 1.0, (cc.PERIODIC,) * (2 * len(shape)))


def step(etas: np.ndarray, p: GrainParams, params: cc.Params = None):
    """One step of reading GG1 for all q order parameters (etas: shape (q, ...grid...)); returns
    the new fields and the solver reports. Each solve starts from the old field."""
    params = params or cc.Params(tol=1e-12, kmax=50, coarsest=4)
    op = step_operator(etas.shape[1:], p)
    levels = cc.build_levels(op, params.coarsest)
    rhs = etas - p.dt * p.L * local_rate(etas, p)
    out = np.array(etas, dtype=np.float64, copy=True)
    infos = []
    for i in range(etas.shape[0]):
        infos.append(cc.solve(levels, out[i], rhs[i], params))
    return out, infos
