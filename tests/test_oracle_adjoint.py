"""Pins of the oracle's adjoint of backward-Euler heat stepping: central finite differences of the
forward model (solved to 1e-14) along random directions, for u0, f and kappa, with Neumann and
Dirichlet faces. Loss L = ||u^N - u_target||^2 (sum of squares)."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import random_field

N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _loss(op, u0, f, dt, steps, target, prm):
    uN, _ = cc.heat_run(op, u0, f, dt, steps, prm)
    return float(np.sum((uN - target) ** 2))


@pytest.mark.parametrize("bc", [(N_,) * 4, (D_, N_, N_, D_)])
def test_adjoint_matches_central_differences(bc):
    n, steps, dt = 16, 4, 2e-3
    shape = (n, n)
    h = 1.0 / n
    kappa = 1.0 + 0.5 * np.tanh(random_field(shape, 601, -2, 2))
    u0 = random_field(shape, 602, -1, 1)
    f = random_field(shape, 603, -1, 1)
    target = random_field(shape, 604, -1, 1)
    prm = cc.Params(tol=1e-14, kmax=80, coarsest=2)
    op = cc.Operator(shape, h, 1.0, dt, kappa, bc)
    uN, g_u0, g_f, g_k = cc.adjoint_heat(op, u0, f, dt, steps, 2.0 * (
        cc.heat_run(op, u0, f, dt, steps, prm)[0] - target), prm)
    for k, (name, g) in enumerate((("u0", g_u0), ("f", g_f), ("kappa", g_k))):
        d = random_field(shape, 610 + k, -1, 1)
        base = {"u0": u0, "f": f, "kappa": kappa}[name]
        eps = 1e-6 * np.linalg.norm(base) / np.linalg.norm(d)

        def L(x):
            args = {"u0": u0, "f": f, "kappa": kappa}
            args[name] = x
            o = cc.Operator(shape, h, 1.0, dt, args["kappa"], bc)
            return _loss(o, args["u0"], args["f"], dt, steps, target, prm)

        fd = (L(base + eps * d) - L(base - eps * d)) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (name, fd, ad)


def test_kappa_gradient_is_minus_derivative_of_bilinear_form():
    """kappa_gradient(u, mu) = -d(mu^T A(kappa) u)/d kappa, checked by differencing A itself."""
    shape = (6, 8)
    h = 1.0 / 8
    kappa = 0.7 + random_field(shape, 621)
    u = random_field(shape, 622, -1, 1)
    mu = random_field(shape, 623, -1, 1)
    op = cc.Operator(shape, h, 0.4, 0.03, kappa, (D_, N_, D_, D_))
    g = cc.kappa_gradient(op, u, mu)
    d = random_field(shape, 624, -1, 1)
    eps = 1e-6

    def form(k):
        return float(np.sum(mu * cc.apply_A(cc.Operator(shape, h, 0.4, 0.03, k, op.bc), u)))

    fd = (form(kappa + eps * d) - form(kappa - eps * d)) / (2 * eps)
    assert abs(-fd - np.sum(g * d)) <= 1e-8 * abs(fd)
