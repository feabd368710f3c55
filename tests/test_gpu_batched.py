"""Batched solves of independent Helmholtz problems (I - dt kappa Lap) u = f of uneven sizes in one
graph launch (mixed precision), checked against one-at-a-time solves (bit for bit), the float64
oracle's solutions (small sizes) and the oracle's residual of every result (full workload)."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import batched_helmholtz, batched_problem_rhs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _problems(count, sizes):
    return batched_helmholtz(count=count, seed=3, sizes=sizes)


def _ctx(fas, pr, **kw):
    n = pr["n"]
    return fas.fas_create(fas.make_params((n, n), 1.0 / n, alpha=1.0, beta=pr["dt"], kappa_const=pr["kappa"],
                                          coarsest=4, precision=1, **kw))


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
def test_batched_equals_one_at_a_time_and_oracle(cuda_lib, tol):
    """Batched = one at a time bit for bit; each result against the oracle's solution to 1e-13:
    solved to the workload's 1e-10, within 1e-10 relative in the 2-norm (the norm a 1e-10 relative
    residual bounds); solved to 1e-12, within 1e-10 relative max-norm."""
    fas = cuda_lib
    probs = _problems(10, (64, 128, 256))
    fs = [batched_problem_rhs(p) for p in probs]
    ctxs = [_ctx(fas, p, tol=tol, kmax=40) for p in probs]
    us = [_t(np.zeros((p["n"], p["n"]))) for p in probs]
    infos = fas.fas_solve_batched(ctxs, us, [_t(f) for f in fs])
    assert all(i.converged and i.rel <= tol for i in infos)
    for p, f, u, inf in zip(probs, fs, us, infos):
        n = p["n"]
        ctx1 = _ctx(fas, p, tol=tol, kmax=40)
        u1 = _t(np.zeros((n, n)))
        inf1 = fas.fas_solve(ctx1, u1, _t(f))
        np.testing.assert_array_equal(u.cpu().numpy(), u1.cpu().numpy())
        assert inf1.as_dict() == inf.as_dict()
        op = cc.Operator((n, n), 1.0 / n, 1.0, p["dt"], p["kappa"])
        ref = np.zeros((n, n))
        cc.solve(cc.build_levels(op, 4), ref, f, cc.Params(tol=1e-13, kmax=60, coarsest=4))
        ug = u.cpu().numpy()
        if tol >= 1e-10:
            assert np.linalg.norm(ug - ref) <= 1e-10 * np.linalg.norm(ref)
        else:
            assert np.max(np.abs(ug - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_batched_graph_reuse_and_errors(cuda_lib):
    fas = cuda_lib
    probs = _problems(4, (64, 128))
    fs = [_t(batched_problem_rhs(p)) for p in probs]
    ctxs = [_ctx(fas, p) for p in probs]
    runs = []
    for _ in range(2):
        us = [_t(np.zeros((p["n"], p["n"]))) for p in probs]
        infos = fas.fas_solve_batched(ctxs, us, fs)
        runs.append(([u.cpu().numpy() for u in us], [i.as_dict() for i in infos]))
    for a, b in zip(runs[0][0], runs[1][0]):
        np.testing.assert_array_equal(a, b)
    assert runs[0][1] == runs[1][1]
    with pytest.raises(fas.FasError) as e:
        fas.fas_solve_batched([ctxs[0], ctxs[0]], us[:1] * 2, fs[:1] * 2)
    assert e.value.status == fas.FAS_EINVAL


def test_batched_full_workload_residuals(cuda_lib):
    """96 problems, n uniform over 64..2048, kappa ~ U(0.5, 2), dt in {1e-4, 1e-3}, smoothed N(0,1)
    right-hand sides; every result's residual (evaluated by the oracle) within the tolerance."""
    fas = cuda_lib
    probs = batched_helmholtz()
    fs = [batched_problem_rhs(p) for p in probs]
    ctxs = [_ctx(fas, p) for p in probs]
    us = [_t(np.zeros((p["n"], p["n"]))) for p in probs]
    infos = fas.fas_solve_batched(ctxs, us, [_t(f) for f in fs])
    assert len(infos) == 96 and all(i.converged for i in infos)
    for p, f, u in zip(probs, fs, us):
        n = p["n"]
        op = cc.Operator((n, n), 1.0 / n, 1.0, p["dt"], p["kappa"])
        r = cc.residual(op, u.cpu().numpy(), f)
        assert cc.norm2(r) <= 1e-10 * cc.norm2(f) * (1 + 1e-5)


def test_autotune_choice_is_cached_and_converges(cuda_lib):
    fas = cuda_lib
    n = 1024
    p = {"n": n, "kappa": 1.3, "dt": 1e-3}
    f = _t(batched_problem_rhs({"n": n, "seed": 77}))
    ctx = _ctx(fas, p)
    scratch = _t(np.zeros((n, n)))
    r1 = fas.fas_autotune(ctx, scratch, f)
    assert r1["candidates"] == 15 and r1["inner_cycles"] in (1, 2, 3) and r1["seg_rows"] in (0, 16, 32, 64, 128)
    ctx2 = _ctx(fas, p)
    r2 = fas.fas_autotune(ctx2, scratch, f)
    assert r2["candidates"] == 0 and (r2["inner_cycles"], r2["seg_rows"]) == (r1["inner_cycles"], r1["seg_rows"])
    u = _t(np.zeros((n, n)))
    assert fas.fas_solve(ctx2, u, f).converged
