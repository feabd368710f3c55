"""The hand-written adjoint of backward-Euler heat stepping (gradients of a final-state loss with
respect to u0, the source and the diffusivity): against the oracle's adjoint, across checkpoint
intervals, against central differences at the full 1024^2 / 50-step workload, and through
torch.autograd."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import adjoint_heat, random_field

pytestmark = pytest.mark.gpu
N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(n, seed):
    shape = (n, n)
    return dict(shape=shape, h=1.0 / n, kappa=1.0 + 0.5 * np.tanh(random_field(shape, seed, -2, 2)),
                u0=random_field(shape, seed + 1, -1, 1), f=random_field(shape, seed + 2, -1, 1),
                target=random_field(shape, seed + 3, -1, 1))


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("bc", [(N_,) * 4, (D_, N_, N_, D_)])
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_oracle(cuda_lib, bc, precision):
    """The final state and the three gradients against the oracle's adjoint within 1e-10 relative
    max-norm, every solve on both sides taken to 1e-13 relative residual (the gradients are sums
    over steps of products of solved fields, so the comparison needs solves well past the bar)."""
    fas = cuda_lib
    c = _case(64, 701)
    dt, steps = 2e-3, 6
    prm = cc.Params(tol=1e-13, kmax=80, coarsest=4)
    op = cc.Operator(c["shape"], c["h"], 1.0, dt, c["kappa"], bc)
    uT_ref, _ = cc.heat_run(op, c["u0"], c["f"], dt, steps, prm)
    seed = 2.0 * (uT_ref - c["target"])
    _, gu_ref, gf_ref, gk_ref = cc.adjoint_heat(op, c["u0"], c["f"], dt, steps, seed, prm)
    ctx = fas.fas_create(fas.make_params(c["shape"], c["h"], beta=dt, bc=bc, coarsest=4, tol=1e-13, kmax=80,
                                         precision=precision), kappa=_t(c["kappa"]))
    outs = [_t(np.zeros(c["shape"])) for _ in range(4)]
    fas.fas_heat_adjoint(ctx, _t(c["u0"]), _t(c["f"]), dt, steps, _t(seed), *outs, ckpt_every=4)
    uT, gu, gf, gk = (o.cpu().numpy() for o in outs)
    assert _rel(uT, uT_ref) <= 1e-10, _rel(uT, uT_ref)
    for name, g, ref in (("u0", gu, gu_ref), ("f", gf, gf_ref), ("kappa", gk, gk_ref)):
        assert _rel(g, ref) <= 1e-10, (name, _rel(g, ref))


def test_checkpoint_interval_does_not_change_gradients(cuda_lib):
    fas = cuda_lib
    c = _case(128, 711)
    dt, steps = 1e-3, 7
    ctx = fas.fas_create(fas.make_params(c["shape"], c["h"], beta=dt, coarsest=4), kappa=_t(c["kappa"]))
    res = []
    for k in (0, 3, 10):
        outs = [_t(np.zeros(c["shape"])) for _ in range(4)]
        fas.fas_heat_adjoint(ctx, _t(c["u0"]), _t(c["f"]), dt, steps, _t(c["target"]), *outs, ckpt_every=k)
        res.append([o.cpu().numpy() for o in outs])
    for other in res[1:]:
        for a, b in zip(res[0], other):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_workload_central_differences(cuda_lib, precision):
    """1024^2, 50 steps, kappa = 1 + 0.5 tanh(8 Gaussians), loss ||u_T - u_target||^2, checkpoints
    every 10 steps: directional derivatives along random u0, f and kappa directions from the adjoint
    agree with central differences of forward runs to 1e-6 relative, with float64 solves and with
    mixed-precision solves (forward runs and adjoint alike, each solve to 1e-12)."""
    fas = cuda_lib
    w = adjoint_heat()
    shape, h, dt, steps = w["shape"], w["h"], w["dt"], w["nsteps"]
    opts = dict(beta=dt, coarsest=4, tol=1e-12, kmax=60, precision=precision)

    def run(u0, f, kappa):
        ctx = fas.fas_create(fas.make_params(shape, h, **opts), kappa=_t(kappa))
        u = _t(u0)
        fas.fas_heat_run(ctx, u, _t(f), dt, steps)
        uT = u.cpu().numpy()
        return float(np.sum((uT - w["target"]) ** 2)), uT

    L0, uT = run(w["u0"], w["fsrc"], w["kappa"])
    ctx = fas.fas_create(fas.make_params(shape, h, **opts), kappa=_t(w["kappa"]))
    outs = [_t(np.zeros(shape)) for _ in range(4)]
    fas.fas_heat_adjoint(ctx, _t(w["u0"]), _t(w["fsrc"]), dt, steps, _t(2.0 * (uT - w["target"])), *outs,
                         ckpt_every=10)
    grads = {"u0": outs[1].cpu().numpy(), "f": outs[2].cpu().numpy(), "kappa": outs[3].cpu().numpy()}
    base = {"u0": w["u0"], "f": w["fsrc"], "kappa": w["kappa"]}
    for k, name in enumerate(("u0", "f", "kappa")):
        d = random_field(shape, 720 + k, -1, 1)
        # L is exactly quadratic in (u0, f): a central difference is exact for any step, so a large
        # step keeps the solves' rounding out of it; kappa enters nonlinearly: small step
        rel_step = 1e-4 if name == "kappa" else 1.0
        eps = rel_step * np.linalg.norm(base[name]) / np.linalg.norm(d)
        args_p = dict(base)
        args_m = dict(base)
        args_p[name] = base[name] + eps * d
        args_m[name] = base[name] - eps * d
        fd = (run(args_p["u0"], args_p["f"], args_p["kappa"])[0] - run(args_m["u0"], args_m["f"], args_m["kappa"])[0]) \
            / (2 * eps)
        ad = float(np.sum(grads[name] * d))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (name, fd, ad)


def test_autograd_function(cuda_lib):
    import torch
    from paper_2510_11152_gb300.autograd import HeatSolve
    fas = cuda_lib
    c = _case(64, 731)
    dt, steps = 1e-3, 5
    u0 = _t(c["u0"]).requires_grad_(True)
    f = _t(c["f"]).requires_grad_(True)
    kap = _t(c["kappa"]).requires_grad_(True)
    uT = HeatSolve.apply(u0, f, kap, c["h"], dt, steps, 2, {"coarsest": 4})
    loss = ((uT - _t(c["target"])) ** 2).sum()
    loss.backward()
    ctx = fas.fas_create(fas.make_params(c["shape"], c["h"], beta=dt, coarsest=4), kappa=_t(c["kappa"]))
    outs = [_t(np.zeros(c["shape"])) for _ in range(4)]
    seed = 2.0 * (uT.detach() - _t(c["target"]))
    fas.fas_heat_adjoint(ctx, _t(c["u0"]), _t(c["f"]), dt, steps, seed, *outs, ckpt_every=2)
    for g, o in ((u0.grad, outs[1]), (f.grad, outs[2]), (kap.grad, outs[3])):
        assert torch.equal(g, o)
