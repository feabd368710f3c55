"""The allocation-free entry point fas_vcycle_small_static.

It serves callers that cannot allocate device memory when they need a solve (programs whose
allocator has reserved all device memory up front, applications that give a solver a fixed budget,
real-time loops). It must compute what the context-based fas_vcycle computes, and what the oracle's
V-cycle (Algorithm 1 with its recursion) computes, call after call, while its scratch lives in a
static device array shared by all calls. This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import random_field

pytestmark = pytest.mark.gpu
N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape,bc,coarsest", [((64, 64), (N_,) * 4, 4), ((32, 64), (D_, N_, N_, D_), 2),
                                               ((16, 16, 16), (D_, N_, N_, N_, D_, D_), 2)])
def test_static_entry_matches_context_vcycle_two_calls(cuda_lib, shape, bc, coarsest):
    fas = cuda_lib
    h = 1.0 / shape[-1]
    params = fas.make_params(shape, h, alpha=1.0, beta=2e-3, bc=bc, coarsest=coarsest)
    ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=2e-3, bc=bc, coarsest=coarsest))
    u0 = random_field(shape, 401)
    f = _t(random_field(shape, 402, -1, 1))
    u_ref, u_new = _t(u0), _t(u0)
    for call, ncycles in enumerate((2, 3)):
        for _ in range(ncycles):
            fas.fas_vcycle(ctx, u_ref, f)
        res = fas.fas_vcycle_small_static(params, u_new, f, ncycles)
        ref = u_ref.cpu().numpy()
        assert _rel(u_new.cpu().numpy(), ref) <= 1e-12, "call %d" % (call + 1)
        res_ref = fas.fas_residual(ctx, 0, u_ref, f)
        assert abs(res - res_ref) <= 1e-6 * res_ref, (call + 1, res, res_ref)


def test_static_entry_second_problem_after_first(cuda_lib):
    """Two calls in a row on different problems: the second must not see the first's scratch."""
    fas = cuda_lib
    outs = []
    for shape, beta in (((64, 64), 1e-3), ((8, 16), 5e-2)):
        h = 1.0 / shape[-1]
        params = fas.make_params(shape, h, beta=beta, coarsest=2)
        ctx = fas.fas_create(fas.make_params(shape, h, beta=beta, coarsest=2))
        u0 = random_field(shape, 411)
        f = _t(random_field(shape, 412, -1, 1))
        u_ref, u_new = _t(u0), _t(u0)
        fas.fas_vcycle(ctx, u_ref, f)
        fas.fas_vcycle_small_static(params, u_new, f, 1)
        outs.append(_rel(u_new.cpu().numpy(), u_ref.cpu().numpy()))
    assert max(outs) <= 1e-12


def test_static_entry_rejects_grids_beyond_its_limit(cuda_lib):
    fas = cuda_lib
    shape = (256, 256)
    params = fas.make_params(shape, 1.0 / 256, beta=1e-3)
    with pytest.raises(fas.FasError) as e:
        fas.fas_vcycle_small_static(params, _t(np.zeros(shape)), _t(np.zeros(shape)), 1)
    assert e.value.status == fas.FAS_EINVAL
    assert "too large" in fas.fas_last_error()


def test_static_entry_symmetric_ordering(cuda_lib):
    """The allocation-free entry with the "1234-4321" ordering computes what the context does."""
    fas = cuda_lib
    shape = (32, 32)
    h = 1.0 / 32
    kw = dict(alpha=1.0, beta=2e-3, coarsest=2, ordering=fas.FAS_ORDER_SYMMETRIC)
    ctx = fas.fas_create(fas.make_params(shape, h, **kw))
    u0 = random_field(shape, 421)
    f = _t(random_field(shape, 422, -1, 1))
    u_ref, u_new = _t(u0), _t(u0)
    for _ in range(3):
        fas.fas_vcycle(ctx, u_ref, f)
    fas.fas_vcycle_small_static(fas.make_params(shape, h, **kw), u_new, f, 3)
    assert _rel(u_new.cpu().numpy(), u_ref.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("shape,bc,coarsest,ordering", [((64, 64), (N_,) * 4, 4, 0),
                                                        ((64, 64), (D_, N_, N_, D_), 2, 1),
                                                        ((16, 16, 16), (N_,) * 6, 2, 0),
                                                        ((16, 16, 16), (D_, N_, N_, N_, D_, D_), 4, 1)])
def test_static_entry_matches_oracle_iterates(cuda_lib, shape, bc, coarsest, ordering):
    """Cycles 1..6 of the allocation-free entry (one call per cycle) against the oracle's V-cycle
    iterates within 1e-12 relative max-norm, and its reported residual against the oracle's."""
    fas = cuda_lib
    h = 1.0 / shape[-1]
    params = fas.make_params(shape, h, alpha=1.0, beta=2e-3, bc=bc, coarsest=coarsest, ordering=ordering)
    op = cc.Operator(shape, h, 1.0, 2e-3, 1.0, bc)
    levels = cc.build_levels(op, coarsest)
    prm = cc.Params(coarsest=coarsest, ordering="1234-4321" if ordering else "1234-1234")
    u = random_field(shape, 431)
    f = random_field(shape, 432, -1, 1)
    ug, fg = _t(u), _t(f)
    for k in range(6):
        res = fas.fas_vcycle_small_static(params, ug, fg, 1)
        cc.vcycle(levels, u, f, prm)
        assert _rel(ug.cpu().numpy(), u) <= 1e-12, "cycle %d" % (k + 1)
        res_ref = cc.norm2(cc.residual(op, u, f))
        assert abs(res - res_ref) <= 1e-6 * res_ref, (k + 1, res, res_ref)
