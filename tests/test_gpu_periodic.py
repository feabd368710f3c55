"""Periodic axes on the GPU (FAS_BC_PERIODIC; the grain-growth example of Sec. 3.3.1 imposes periodic
boundaries in every direction) and the grain-growth step, through the C ABI, against the oracle.

Bars: single operators within a few ulps (1e-13 relative); float64 V-cycle iterates within 1e-12
relative max-norm for cycles 1..8; solutions solved to 1e-12 (float64 and mixed precision) within
1e-10 relative max-norm of the exact discrete Fourier solution; the grain-growth step's right-hand
sides within 1e-14 and its float64 steps within 1e-12 (mixed precision 1e-10) of the oracle's steps.
"""
import numpy as np
import pytest

from oracle import cell_centred as cc
from oracle import grain_growth as gg
from workloads import grain_growth_fields, random_field

pytestmark = pytest.mark.gpu
N_, D_, P_ = cc.NEUMANN, cc.DIRICHLET, cc.PERIODIC


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _pair(fas, shape, h, alpha, beta, kappa, bc, **kw):
    op = cc.Operator(shape, h, alpha, beta, kappa, bc)
    ctx = fas.fas_create(fas.make_params(shape, h, alpha=alpha, beta=beta, kappa_const=kappa, bc=bc, **kw))
    return op, ctx


BCS = {
    "periodic": lambda d: (P_,) * (2 * d),
    "periodic_x": lambda d: (P_, P_, N_, D_, D_, N_)[: 2 * d],
    "periodic_y": lambda d: (D_, N_, P_, P_, P_, P_)[: 2 * d],
}
SHAPES = [(2, 2), (8, 8), (16, 64), (128, 128), (4, 4, 4), (8, 16, 32), (32, 32, 32)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc_kind", sorted(BCS))
def test_periodic_single_operators(cuda_lib, shape, bc_kind):
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    op, ctx = _pair(fas, shape, h, 0.8, 3e-3, 1.3, BCS[bc_kind](dim), coarsest=2)
    u = random_field(shape, 801, -1, 1)
    f = random_field(shape, 802, -1, 1)
    out = _t(np.zeros(shape))
    nrm = fas.fas_residual(ctx, 0, _t(u), _t(f), out)
    r_ref = cc.residual(op, u, f)
    assert _rel(_n(out), r_ref) < 1e-13
    assert abs(nrm - cc.norm2(r_ref)) <= 1e-6 * cc.norm2(r_ref)
    for sweeps in (1, 3):
        ug = _t(u)
        fas.fas_smooth(ctx, 0, ug, _t(f), sweeps)
        uo = u.copy()
        cc.smooth(op, uo, f, sweeps)
        assert _rel(_n(ug), uo) < 1e-13, sweeps


@pytest.mark.parametrize("shape,coarsest", [((64, 64), 4), ((256, 256), 2), ((64, 128), 4), ((32, 32, 32), 2),
                                            ((16, 32, 32), 4)])
@pytest.mark.parametrize("bc_kind", ["periodic", "periodic_x"])
def test_periodic_vcycle_iterates(cuda_lib, shape, coarsest, bc_kind):
    """Cycles 1..8 of the float64 V-cycle against the oracle's (Algorithm 1 + recursion), the
    per-operation kernels on the large levels and the single-CTA kernel on the small ones."""
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    op, ctx = _pair(fas, shape, h, 1.0, 2e-3, 1.0, BCS[bc_kind](dim), coarsest=coarsest)
    levels = cc.build_levels(op, coarsest)
    assert fas.fas_num_levels(ctx) == len(levels)
    u = random_field(shape, 811)
    f = random_field(shape, 812, -1, 1)
    ug, fg = _t(u), _t(f)
    for k in range(8):
        fas.fas_vcycle(ctx, ug, fg)
        cc.vcycle(levels, u, f, cc.Params(coarsest=coarsest))
        assert _rel(_n(ug), u) < 1e-12, "cycle %d" % (k + 1)


def _fourier_solution(shape, h, alpha, beta, f):
    """Exact solution of the all-periodic system by the discrete Fourier transform (alpha = 0: the
    mean-free solution of the mean-free right-hand side)."""
    lam = np.full(shape, float(alpha))
    for ax, n in enumerate(shape):
        l1 = beta * 4.0 / h ** 2 * np.sin(np.pi * np.arange(n) / n) ** 2
        sh = [1] * len(shape)
        sh[ax] = n
        lam = lam + l1.reshape(sh)
    fh = np.fft.fftn(f)
    if alpha == 0.0:
        lam.flat[0] = 1.0
        fh.flat[0] = 0.0
    return np.real(np.fft.ifftn(fh / lam))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,alpha,beta", [((256, 256), 1.0, 1e-3), ((1024, 1024), 1.0, 1e-4),
                                              ((128, 128), 0.0, 1.0), ((64, 64, 64), 1.0, 1e-3),
                                              ((32, 32, 32), 0.0, 1.0)])
def test_periodic_solution_matches_fourier(cuda_lib, precision, shape, alpha, beta):
    """Solved to 1e-12 relative residual, within 1e-10 relative max-norm of the exact DFT solution;
    alpha = 0 is the singular all-periodic problem (mean-free, reading G7), with a dense coarsest solve."""
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    exact = alpha == 0.0
    op, ctx = _pair(fas, shape, h, alpha, beta, 1.0, (P_,) * (2 * dim), coarsest=4, coarse_exact=int(exact),
                    precision=precision, tol=1e-12, kmax=100)
    f = random_field(shape, 821, -1, 1)
    if exact:
        f -= f.mean()
    ref = _fourier_solution(shape, h, alpha, beta, f)
    ug = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, ug, _t(f))
    assert info.converged and info.rel <= 1e-12
    assert _rel(_n(ug), ref) <= 1e-10, _rel(_n(ug), ref)
    if exact:
        assert abs(float(_n(ug).mean())) <= 1e-12 * np.max(np.abs(ref))


def test_periodic_rejections(cuda_lib):
    fas = cuda_lib
    with pytest.raises(fas.FasError) as e:  # periodic faces come in pairs
        fas.fas_create(fas.make_params((32, 32), 1.0 / 32, bc=(P_, N_, N_, N_)))
    assert e.value.status == fas.FAS_EINVAL
    import torch
    kap = torch.ones((32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(fas.make_params((32, 32), 1.0 / 32, bc=(P_,) * 4), kappa=kap)
    assert e.value.status == fas.FAS_EUNSUPPORTED
    with pytest.raises(fas.FasError) as e:
        fas.fas_vcycle_small_static(fas.make_params((32, 32), 1.0 / 32, bc=(P_,) * 4), _t(np.zeros((32, 32))),
                                    _t(np.zeros((32, 32))), 1)
    assert e.value.status == fas.FAS_EUNSUPPORTED


# ---------------------------------------------------------------------------------------------
# grain growth (Sec. 3.3.1)
# ---------------------------------------------------------------------------------------------

def _gg_solver(fas, precision, tol):
    p = fas.fas_default_params()
    p.precision, p.tol, p.kmax, p.coarsest = precision, tol, 50, 4
    return p


def test_grain_rhs_matches_oracle(cuda_lib):
    fas = cuda_lib
    shape, q = (64, 64), 7
    p = gg.GrainParams()
    etas = random_field((q,) + shape, 831, -1, 1)
    ctx = fas.gg_create(shape, p.h, p.dt, q)
    rhs = _t(np.zeros((q,) + shape))
    fas.gg_rhs(ctx, _t(etas), rhs)
    ref = etas - p.dt * p.L * gg.local_rate(etas, p)
    assert _rel(_n(rhs), ref) <= 1e-14


@pytest.mark.parametrize("precision,bar", [(0, 1e-12), (1, 1e-10)])
@pytest.mark.parametrize("shape,q,batch", [((64, 64), 6, 4), ((32, 64), 3, 0), ((16, 16, 16), 4, 0)])
def test_grain_steps_match_oracle(cuda_lib, precision, bar, shape, q, batch):
    """Three steps of the linearly implicit grain-growth step from the paper's disordered start
    (scaled up so that the local terms matter), every solve to 1e-12 on both sides, against the
    oracle's steps; batch 4 runs the q solves in two graph launches."""
    fas = cuda_lib
    p = gg.GrainParams()
    etas = grain_growth_fields(q, shape, seed=9) * 300.0  # U(-0.3, 0.3)
    ctx = fas.gg_create(shape, p.h, p.dt, q, solver=_gg_solver(fas, precision, 1e-12), batch=batch)
    eg = _t(etas)
    ref = etas.copy()
    for step in range(3):
        infos = fas.gg_step(ctx, eg)
        ref, infos_ref = gg.step(ref, p, cc.Params(tol=1e-12, kmax=50, coarsest=4))
        assert all(i.converged for i in infos)
        if precision == 0:
            assert [i.cycles for i in infos] == [i.cycles for i in infos_ref]
        assert _rel(_n(eg), ref) <= bar, (step, _rel(_n(eg), ref))


def test_grain_uniform_state_is_steady_and_modes_grow(cuda_lib):
    """eta = (1, 0, ..., 0) is a steady state of the model; a small single Fourier mode of eta_1 about
    0 grows by (1 + dt L alpha) / (1 + dt L kappa lambda_k) per step (the closed forms the oracle is
    pinned by)."""
    fas = cuda_lib
    shape, q = (64, 64), 3
    p = gg.GrainParams()
    ctx = fas.gg_create(shape, p.h, p.dt, q, solver=_gg_solver(fas, 0, 1e-13))
    e = np.zeros((q,) + shape)
    e[0] = 1.0
    eg = _t(e)
    fas.gg_step(ctx, eg)
    assert _rel(_n(eg), e) <= 1e-13
    n = shape[0]
    x = (np.arange(n) + 0.5) * p.h
    k = 3
    mode = 1e-6 * np.cos(2 * np.pi * k * x / (n * p.h))[None, :] * np.ones((n, 1))
    e = np.zeros((q,) + shape)
    e[0] = mode
    eg = _t(e)
    fas.gg_step(ctx, eg)
    lam = 4.0 / p.h ** 2 * np.sin(np.pi * k / n) ** 2
    g = (1 + p.dt * p.L * p.alpha) / (1 + p.dt * p.L * p.kappa * lam)
    # the cubic terms are of relative size 1e-12 at this amplitude
    assert _rel(_n(eg)[0], g * mode) <= 1e-10
    assert np.max(np.abs(_n(eg)[1:])) == 0.0
