"""Parity of the CUDA path (through the C ABI) with the CPU oracle, on the same seeded inputs.

Bars: float64 single operators within a few ulps (1e-14 relative); float64 V-cycle iterates within
1e-12 relative max-norm for cycles 1..8; converged float64 and mixed-precision solutions within 1e-10
relative max-norm of the oracle's converged solution (where two solves stopped at the 1e-10 residual
could differ by more, the GPU side is solved tighter, never the bar widened).
"""
import math

import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import heat2d_small, noisy_cos_mode, random_field

pytestmark = pytest.mark.gpu

N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _bc(kind, dim):
    return {"neumann": (N_,) * (2 * dim), "dirichlet": (D_,) * (2 * dim),
            "mixed": (D_, N_, N_, D_, N_, D_)[: 2 * dim]}[kind]


def _pair(fas, shape, h, alpha, beta, kappa, bc, **kw):
    """Oracle operator and GPU context for the same problem."""
    op = cc.Operator(shape, h, alpha, beta, kappa, bc)
    kap_t = None if np.isscalar(kappa) else _t(kappa)
    p = fas.make_params(shape, h, alpha=alpha, beta=beta,
                        kappa_const=kappa if np.isscalar(kappa) else 1.0, bc=bc, **kw)
    ctx = fas.fas_create(p, kappa=kap_t)
    return op, ctx


SHAPES = [(2, 2), (8, 8), (16, 64), (128, 128), (4, 4, 4), (8, 16, 32), (32, 32, 32)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc_kind", ["neumann", "dirichlet", "mixed"])
@pytest.mark.parametrize("var_kappa", [False, True])
def test_single_operators(cuda_lib, shape, bc_kind, var_kappa):
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    kappa = (0.5 + random_field(shape, 201)) if var_kappa else 1.3
    op, ctx = _pair(fas, shape, h, 0.8, 3e-3, kappa, _bc(bc_kind, dim), coarsest=2)
    u = random_field(shape, 202, -1, 1)
    f = random_field(shape, 203, -1, 1)
    # residual
    out = _t(np.zeros(shape))
    nrm = fas.fas_residual(ctx, 0, _t(u), _t(f), out)
    r_ref = cc.residual(op, u, f)
    assert _rel(_n(out), r_ref) < 1e-13
    assert abs(nrm - cc.norm2(r_ref)) <= 1e-6 * cc.norm2(r_ref)
    # one and three sweeps
    for sweeps in (1, 3):
        ug = _t(u)
        fas.fas_smooth(ctx, 0, ug, _t(f), sweeps)
        uo = u.copy()
        cc.smooth(op, uo, f, sweeps)
        assert _rel(_n(ug), uo) < 1e-13
    # transfers
    if fas.fas_num_levels(ctx) > 1:
        cshape = tuple(n // 2 for n in shape)
        uc = _t(np.zeros(cshape))
        fas.fas_restrict(ctx, 0, _t(u), uc)
        assert _rel(_n(uc), cc.restrict(u)) < 1e-15
        c = random_field(cshape, 204, -1, 1)
        ug = _t(u)
        fas.fas_prolong_add(ctx, 0, ug, _t(c))
        assert _rel(_n(ug), u + cc.prolong(c)) < 1e-15


@pytest.mark.parametrize("shape,coarsest,exact", [((64, 64), 4, False), ((64, 256), 4, False),
                                                   ((256, 256), 2, False), ((512, 512), 4, True),
                                                   ((16, 16, 16), 2, False), ((32, 64, 64), 4, True)])
@pytest.mark.parametrize("bc_kind", ["neumann", "mixed"])
def test_vcycle_iterates(cuda_lib, shape, coarsest, exact, bc_kind):
    """Cycles 1..8 of the float64 V-cycle against the oracle's (Algorithm 1 + recursion)."""
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    op, ctx = _pair(fas, shape, h, 1.0, 2e-3, 1.0, _bc(bc_kind, dim), coarsest=coarsest,
                    coarse_exact=int(exact))
    prm = cc.Params(coarsest=coarsest, coarse_exact=exact)
    levels = cc.build_levels(op, coarsest)
    assert fas.fas_num_levels(ctx) == len(levels)
    u = random_field(shape, 211)
    f = random_field(shape, 212, -1, 1)
    ug, fg = _t(u), _t(f)
    for k in range(8):
        fas.fas_vcycle(ctx, ug, fg)
        cc.vcycle(levels, u, f, prm)
        assert _rel(_n(ug), u) < 1e-12, "cycle %d" % (k + 1)


@pytest.mark.parametrize("shape,coarsest", [((256, 256), 4), ((64, 128), 2), ((32, 32, 32), 2)])
def test_symmetric_ordering_iterates(cuda_lib, shape, coarsest):
    """The "1234-4321" X-MCGS ordering (Sec. 2.3): float64 V-cycles against the oracle's, and the
    mixed-precision solve to the same converged solution; the sweeps alternate direction on every
    level, the single-CTA levels included."""
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    op, ctx = _pair(fas, shape, h, 1.0, 2e-3, 1.0, _bc("mixed", dim), coarsest=coarsest,
                    ordering=fas.FAS_ORDER_SYMMETRIC)
    prm = cc.Params(coarsest=coarsest, ordering="1234-4321")
    levels = cc.build_levels(op, coarsest)
    u = random_field(shape, 221)
    f = random_field(shape, 222, -1, 1)
    ug, fg = _t(u), _t(f)
    for k in range(6):
        fas.fas_vcycle(ctx, ug, fg)
        cc.vcycle(levels, u, f, prm)
        assert _rel(_n(ug), u) < 1e-12, "cycle %d" % (k + 1)
    # a forward-ordering context gives different iterates
    _, ctx_fwd = _pair(fas, shape, h, 1.0, 2e-3, 1.0, _bc("mixed", dim), coarsest=coarsest)
    uf = _t(random_field(shape, 221))
    fas.fas_vcycle(ctx_fwd, uf, fg)
    um = _t(random_field(shape, 221))
    fas.fas_vcycle(ctx, um, fg)
    assert _rel(_n(um), _n(uf)) > 1e-8
    # mixed precision reaches the oracle's converged solution: both sides are solved past the 1e-10
    # bar (GPU 1e-12, oracle 1e-13) so that the max-norm comparison measures the solver, not where two
    # iterations that both satisfy a 1e-10 residual happened to stop
    _, ctx_m = _pair(fas, shape, h, 1.0, 2e-3, 1.0, _bc("mixed", dim), coarsest=coarsest,
                     ordering=fas.FAS_ORDER_SYMMETRIC, precision=fas.FAS_MIXED, tol=1e-12, kmax=60)
    u_ref = np.zeros(shape)
    assert cc.solve(levels, u_ref, f, cc.Params(coarsest=coarsest, ordering="1234-4321", tol=1e-13,
                                                kmax=60)).converged
    um = _t(np.zeros(shape))
    assert fas.fas_solve(ctx_m, um, fg).converged
    assert _rel(_n(um), u_ref) <= 1e-10


def test_symmetric_ordering_argument_checks(cuda_lib):
    fas = cuda_lib
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(fas.make_params((64, 64), 1.0 / 64, ordering=2))
    assert e.value.status == fas.FAS_EINVAL
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(fas.make_params((64, 64), 1.0 / 64, ordering=fas.FAS_ORDER_SYMMETRIC,
                                       location=fas.FAS_FACE_X))
    assert e.value.status == fas.FAS_EUNSUPPORTED


def test_vcycle_iterates_variable_kappa(cuda_lib):
    fas = cuda_lib
    shape = (128, 128)
    kappa = 1.0 + 0.5 * np.tanh(random_field(shape, 221, -2, 2))
    op, ctx = _pair(fas, shape, 1.0 / 128, 1.0, 1e-3, kappa, _bc("mixed", 2), coarsest=4)
    levels = cc.build_levels(op, 4)
    u = random_field(shape, 222)
    f = random_field(shape, 223, -1, 1)
    ug, fg = _t(u), _t(f)
    for k in range(6):
        fas.fas_vcycle(ctx, ug, fg)
        cc.vcycle(levels, u, f, cc.Params(coarsest=4))
        assert _rel(_n(ug), u) < 1e-12, "cycle %d" % (k + 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [(256, 256), (1024, 1024), (64, 64, 64)])
def test_converged_solution(cuda_lib, precision, shape):
    """Solve to 1e-10 relative residual; compare with the oracle solved to 1e-13, within 1e-10
    relative max-norm."""
    fas = cuda_lib
    h = 1.0 / shape[-1]
    op, ctx = _pair(fas, shape, h, 1.0, 1e-3, 1.0, (N_,) * (2 * len(shape)), coarsest=4, precision=precision)
    f = noisy_cos_mode(shape, 231)
    u_ref = np.zeros(shape)
    cc.solve(cc.build_levels(op, 4), u_ref, f, cc.Params(tol=1e-13, kmax=60, coarsest=4))
    ug = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, ug, _t(f))
    assert info.converged and info.rel <= 1e-10
    assert _rel(_n(ug), u_ref) <= 1e-10
    # the residual the library reports agrees with the oracle's residual of the returned field
    r = cc.residual(op, _n(ug), f)
    assert cc.norm2(r) <= 1e-10 * cc.norm2(f) * (1 + 1e-6)


def test_heat_run_small_matches_oracle(cuda_lib):
    """128^2 heat: Neumann, kappa 1, dt 1e-3, 10 steps, each to 1e-10 relative (float64)."""
    fas = cuda_lib
    w = heat2d_small()
    shape = w["shape"]
    op, ctx = _pair(fas, shape, w["h"], 1.0, w["dt"], 1.0, (N_,) * 4, coarsest=4)
    u_ref, infos_ref = cc.heat_run(op, w["u0"], None, w["dt"], w["nsteps"], cc.Params(tol=1e-10, coarsest=4))
    ug = _t(w["u0"])
    infos = fas.fas_heat_run(ctx, ug, None, w["dt"], w["nsteps"])
    assert all(i.converged for i in infos)
    assert [i.cycles for i in infos] == [i.cycles for i in infos_ref]
    assert _rel(_n(ug), u_ref) <= 1e-10


def test_singular_poisson_coarse_exact(cuda_lib):
    """Singular all-Neumann Poisson (alpha = 0, reading G7), float64: the GPU solve to 1e-13 relative
    residual (the operator's conditioning, about (2/(pi h))^2, turns a residual of 1e-13 into a
    solution error of about 1e-10) against the oracle's to 1e-14, within 1e-10 relative max-norm."""
    fas = cuda_lib
    shape = (64, 64)
    op, ctx = _pair(fas, shape, 1.0 / 64, 0.0, 1.0, 1.0, (N_,) * 4, coarsest=4, coarse_exact=1, kmax=200,
                    tol=1e-13)
    f = random_field(shape, 241, -1, 1)
    u_ref = np.zeros(shape)
    cc.solve(cc.build_levels(op, 4), u_ref, f, cc.Params(tol=1e-14, kmax=300, coarsest=4, coarse_exact=True))
    ug = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, ug, _t(f))
    assert info.converged
    assert abs(float(_n(ug).mean())) < 1e-12
    assert _rel(_n(ug), u_ref) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_right_hand_side(cuda_lib, precision):
    """f = 0. From u = 0 the solve returns u = 0 exactly after one cycle: the relative test falls back
    to the initial residual, which is 0. From a nonzero guess it drives the residual 1e10 times below
    the initial one (the oracle evaluates both residuals)."""
    fas = cuda_lib
    shape = (128, 128)
    op, ctx = _pair(fas, shape, 1.0 / 128, 1.0, 1e-3, 1.0, (N_,) * 4, coarsest=4, precision=precision)
    zero = np.zeros(shape)
    u = _t(zero)
    info = fas.fas_solve(ctx, u, _t(zero))
    assert info.converged and info.cycles == 1
    assert not np.any(_n(u))
    u0 = random_field(shape, 271, -1, 1)
    u = _t(u0)
    info = fas.fas_solve(ctx, u, _t(zero))
    assert info.converged
    r0 = cc.norm2(cc.residual(op, u0, zero))
    assert cc.norm2(cc.residual(op, _n(u), zero)) <= 1e-10 * r0 * (1 + 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,coarsest,exact", [((2, 2), 2, True), ((4, 4), 2, False), ((2, 16), 2, True),
                                                  ((4, 256), 4, True), ((2, 2, 2), 2, True), ((4, 4, 4), 2, False),
                                                  ((2, 4, 8), 2, True)])
def test_smallest_and_thinnest_grids(cuda_lib, precision, shape, coarsest, exact):
    """Grids of one level (2 x 2, 2 x 16, 4 x 256: the shortest axis is already the coarsest size) and
    two levels, smoothed or solved exactly on the coarsest: the GPU solve to 1e-12 against the oracle's
    to 1e-13, within 1e-10 relative max-norm."""
    fas = cuda_lib
    h = 1.0 / shape[-1]
    bc = (D_, N_, N_, D_, N_, D_)[: 2 * len(shape)]
    op, ctx = _pair(fas, shape, h, 1.0, 1e-2, 1.0, bc, coarsest=coarsest, coarse_exact=int(exact),
                    precision=precision, tol=1e-12, kmax=100)
    f = random_field(shape, 281, -1, 1)
    u_ref = np.zeros(shape)
    cc.solve(cc.build_levels(op, coarsest), u_ref, f,
             cc.Params(tol=1e-13, kmax=200, coarsest=coarsest, coarse_exact=exact))
    ug = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, ug, _t(f))
    assert info.converged
    assert _rel(_n(ug), u_ref) <= 1e-10


def test_error_statuses(cuda_lib):
    import torch
    fas = cuda_lib
    p = fas.make_params((48, 64), 1.0 / 64)
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(p)
    assert e.value.status == fas.FAS_EINVAL
    p = fas.make_params((64, 64), -1.0)
    with pytest.raises(fas.FasError):
        fas.fas_create(p)
    ctx = fas.fas_create(fas.make_params((64, 64), 1.0 / 64, beta=1e-3, kmax=1, tol=1e-14))
    f = _t(random_field((64, 64), 251))
    ug = _t(np.zeros((64, 64)))
    info = fas.fas_solve(ctx, ug, f, allow_notconv=True)
    assert info.cycles == 1 and not info.converged
    with pytest.raises(fas.FasError) as e:
        fas.fas_solve(ctx, _t(np.zeros((64, 64))), f)
    assert e.value.status == fas.FAS_ENOTCONV
    bad = random_field((64, 64), 252)
    bad[5, 7] = math.nan
    ctx2 = fas.fas_create(fas.make_params((64, 64), 1.0 / 64, beta=1e-3))
    with pytest.raises(fas.FasError) as e:
        fas.fas_solve(ctx2, _t(np.zeros((64, 64))), _t(bad))
    assert e.value.status in (fas.FAS_ENONFINITE, fas.FAS_ENOTCONV)
    # fields are moved in 16-byte vectors: a view starting at an odd element is rejected, not run
    big = _t(np.zeros(64 * 64 + 1))
    with pytest.raises(fas.FasError) as e:
        fas.fas_solve(ctx2, big[1:], f)
    assert e.value.status == fas.FAS_EINVAL and "aligned" in str(e.value)
    with pytest.raises(fas.FasError) as e:
        fas.fas_residual_ir(ctx2, ug, big[1:], torch.empty(64 * 64, dtype=torch.float32, device="cuda"))
    assert e.value.status == fas.FAS_EINVAL


@pytest.mark.parametrize("pinned,with_src,alias", [(True, True, False), (False, True, False), (True, False, True),
                                                   (False, False, True)])
def test_heat_run_host_matches_device_run(cuda_lib, pinned, with_src, alias):
    """fas_heat_run_host (host buffers in and out; page-locked buffers are copied by the GPU's own
    loads and stores, pageable ones by cudaMemcpyAsync) equals fas_heat_run on device buffers bit for
    bit, including uT_host aliasing u0_host."""
    import torch
    fas = cuda_lib
    shape = (256, 256)
    dt = 1e-3
    u0 = noisy_cos_mode(shape, 261)
    src = random_field(shape, 262, -1, 1) if with_src else None
    params = dict(alpha=1.0, beta=dt, precision=fas.FAS_MIXED)
    ref_ctx = fas.fas_create(fas.make_params(shape, 1.0 / 256, **params))
    ud = _t(u0)
    fas.fas_heat_run(ref_ctx, ud, None if src is None else _t(src), dt, 3)
    ctx = fas.fas_create(fas.make_params(shape, 1.0 / 256, **params))

    keep = []  # the host tensors behind the numpy views stay alive for the whole test

    def host(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        t = t.pin_memory() if pinned else t.clone()
        keep.append(t)
        return t.numpy()

    u0h = host(u0)
    outh = u0h if alias else host(np.zeros(shape))
    fh = None if src is None else host(src)
    for _ in range(2):  # the second call reuses the context's device buffers
        if alias:
            u0h[...] = u0
        fas.fas_heat_run_host(ctx, u0h, outh, fh, dt, 3)
        assert np.array_equal(outh, ud.cpu().numpy())


@pytest.mark.parametrize("shape,bc_kind,var_kappa", [((64, 128), "dirichlet", False), ((32, 64), "mixed", True),
                                                     ((16, 16, 32), "dirichlet", True),
                                                     ((16, 32, 16), "mixed", False)])
def test_fold_dirichlet_matches_oracle(cuda_lib, shape, bc_kind, var_kappa):
    """Inhomogeneous Dirichlet values moved into the right-hand side (Eq. boundry1 with a value,
    reading G10): the same additions as the oracle's fold, bit for bit (corners take every face)."""
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    kappa = (0.5 + random_field(shape, 241)) if var_kappa else 1.3
    op, ctx = _pair(fas, shape, h, 1.0, 3e-3, kappa, _bc(bc_kind, dim))
    values = [0.3, -1.2, 2.5, 0.7, -0.4, 1.1][: 2 * dim]
    f = random_field(shape, 242, -1, 1)
    ref = cc.fold_dirichlet_rhs(op, f, values)
    fg = _t(f)
    fas.fas_fold_dirichlet(ctx, fg, values)
    assert np.array_equal(_n(fg), ref)


def test_fold_dirichlet_rejects_face_grids(cuda_lib):
    fas = cuda_lib
    fctx = fas.fas_create(fas.make_params((32, 32), 1.0 / 32, alpha=1.0, beta=3e-3, bc=(D_,) * 4,
                                          location=fas.FAS_FACE_X))
    with pytest.raises(fas.FasError) as e:
        fas.fas_fold_dirichlet(fctx, _t(np.zeros((32, 32))), [1.0] * 4)
    assert e.value.status == fas.FAS_EUNSUPPORTED


def test_one_call_solve(cuda_lib):
    """fas.solve: context created, used and freed in one call; the same solution as a Solver."""
    fas = cuda_lib
    shape = (128, 128)
    f = random_field(shape, 251, -1, 1)
    u1 = _t(np.zeros(shape))
    info = fas.solve(u1, _t(f), 1.0 / 128, alpha=1.0, beta=1e-3, bc=_bc("mixed", 2), precision=fas.FAS_MIXED)
    assert info.converged and info.rel <= 1e-10
    s = fas.Solver(shape, 1.0 / 128, alpha=1.0, beta=1e-3, bc=_bc("mixed", 2), precision=fas.FAS_MIXED)
    u2 = _t(np.zeros(shape))
    s.solve(u2, _t(f))
    s.close()
    assert np.array_equal(_n(u1), _n(u2))
    assert fas.HeatSolve is not None
