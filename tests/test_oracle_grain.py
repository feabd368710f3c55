"""Pins of the grain-growth oracle (Sec. 3.3.1, readings GG1-GG2 of oracle/grain_growth.py) against
what the mathematics fixes: the step on spatially uniform fields (no diffusion, the local terms
written out with an explicit sum over j != i), the steady state eta = (1, 0, ..., 0), the growth
factor of a small single Fourier mode on the periodic grid, and the equivariance under relabelling of
the order parameters."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from oracle import grain_growth as gg
from workloads import grain_growth_fields, uniform

PRM = cc.Params(tol=1e-13, kmax=60, coarsest=4)


def test_uniform_fields_follow_the_local_equation():
    p = gg.GrainParams()
    q, shape = 4, (16, 16)
    c = uniform(41, 1, q) * 1.6 - 0.8
    etas = np.broadcast_to(c[:, None, None], (q,) + shape).copy()
    new, infos = gg.step(etas, p, PRM)
    assert all(i.converged for i in infos)
    for i in range(q):
        others = sum(c[j] ** 2 for j in range(q) if j != i)
        rate = -p.alpha * c[i] + p.beta * c[i] ** 3 + 2.0 * p.gamma * c[i] * others
        np.testing.assert_allclose(new[i], c[i] - p.dt * p.L * rate, rtol=0, atol=1e-13)


def test_single_grain_state_is_steady():
    p = gg.GrainParams()
    etas = np.zeros((3, 16, 16))
    etas[1] = 1.0  # alpha = beta: eta = 1 solves -alpha eta + beta eta^3 = 0; the others stay 0
    new, _ = gg.step(etas, p, PRM)
    np.testing.assert_allclose(new, etas, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [(1, 0), (2, 3), (7, 5)])
def test_small_mode_growth_factor(k):
    """Linearised about eta = 0 (amplitude 1e-7, cubic terms below 1e-20): one step multiplies the
    mode cos(2 pi k . x / (n h)) by (1 + dt L alpha) / (1 + dt L kappa lambda_k), with
    lambda_k = (4 / h^2) sum_a sin^2(pi k_a / n), the periodic eigenvalue of -Lap_h."""
    p = gg.GrainParams()
    n = 32
    y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    eta = 1e-7 * np.cos(2.0 * np.pi * (k[0] * x + k[1] * y) / n)
    new, _ = gg.step(eta[None], p, PRM)
    lam = 4.0 / p.h ** 2 * (np.sin(np.pi * k[0] / n) ** 2 + np.sin(np.pi * k[1] / n) ** 2)
    g = (1.0 + p.dt * p.L * p.alpha) / (1.0 + p.dt * p.L * p.kappa * lam)
    np.testing.assert_allclose(new[0], g * eta, rtol=0, atol=1e-9 * 1e-7)


def test_relabelling_order_parameters():
    p = gg.GrainParams()
    etas = grain_growth_fields(5, (16, 16), seed=7) * 300.0  # O(0.3) fields, the nonlinear regime
    perm = [3, 0, 4, 1, 2]
    a, _ = gg.step(etas, p, PRM)
    b, _ = gg.step(etas[perm], p, PRM)
    np.testing.assert_allclose(b, a[perm], rtol=0, atol=1e-12)


def test_disordered_start_crystallises():
    """Sec. 3.3.1: from the U(-0.001, 0.001) start the order parameters grow (crystallisation) before
    coarsening. The finest modes of the start decay first (their growth factor above is below one);
    after that transient the largest phi = sum_i eta_i^2 grows monotonically, by orders of magnitude."""
    p = gg.GrainParams()
    etas = grain_growth_fields(4, (32, 32), seed=5)
    phis = []
    for _ in range(30):
        etas, _ = gg.step(etas, p, cc.Params(tol=1e-10, kmax=40, coarsest=4))
        phis.append(float(np.max(np.sum(etas ** 2, axis=0))))
    late = phis[8:]
    assert all(b > a for a, b in zip(late, late[1:]))
    assert phis[-1] > 1e3 * phis[3]
