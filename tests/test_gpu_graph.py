"""The solve captured as one CUDA graph (a while node whose body is one cycle, the stopping decision
taken on the device) computes exactly what the host-driven loop computes."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import heat2d_small, noisy_cos_mode, random_field

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("shape,precision", [((256, 256), 0), ((1024, 1024), 1), ((512, 128), 1),
                                             ((32, 32, 32), 0), ((32, 64, 64), 1)])
def test_graph_solve_equals_host_loop(cuda_lib, shape, precision):
    fas = cuda_lib
    h = 1.0 / shape[-1]
    f = noisy_cos_mode(shape, 501)
    u0 = random_field(shape, 502)
    outs, infos = [], []
    for graph in (1, 0):
        ctx = fas.fas_create(fas.make_params(shape, h, beta=1e-3, precision=precision, use_graph=graph))
        u = _t(u0)
        infos.append(fas.fas_solve(ctx, u, _t(f)).as_dict())
        u2 = _t(u0)  # a second solve reuses the captured graph only for the same pointers
        fas.fas_solve(ctx, u2, _t(f))
        outs.append((u.cpu().numpy(), u2.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert infos[0] == infos[1]
    assert infos[0]["converged"] == 1


def test_graph_heat_run_equals_host_loop_and_oracle(cuda_lib):
    fas = cuda_lib
    w = heat2d_small()
    shape, h, dt, steps = w["shape"], w["h"], w["dt"], w["nsteps"]
    res = []
    for graph in (1, 0):
        ctx = fas.fas_create(fas.make_params(shape, h, beta=dt, coarsest=4, use_graph=graph))
        u = _t(w["u0"])
        infos = fas.fas_heat_run(ctx, u, None, dt, steps)
        res.append((u.cpu().numpy(), [i.as_dict() for i in infos]))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
    op = cc.heat_operator(shape, h, dt)
    u_ref, infos_ref = cc.heat_run(op, w["u0"], None, dt, steps, cc.Params(tol=1e-10, coarsest=4))
    assert [i["cycles"] for i in res[0][1]] == [i.cycles for i in infos_ref]


def test_graph_kmax_exhaustion_and_launch_count(cuda_lib):
    fas = cuda_lib
    shape = (128, 128)
    ctx = fas.fas_create(fas.make_params(shape, 1.0 / 128, beta=1e-3, kmax=2, tol=1e-15))
    u = _t(np.zeros(shape))
    fas.fas_launch_count(ctx, reset=True)
    info = fas.fas_solve(ctx, u, _t(random_field(shape, 511)), allow_notconv=True)
    assert info.cycles == 2 and not info.converged
    assert fas.fas_launch_count(ctx) > 0
