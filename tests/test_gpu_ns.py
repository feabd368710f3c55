"""The staggered (MAC) grid on the GPU, through the C ABI, against the CPU oracle.

Face-grid multigrid (fas_params.location = FAS_FACE_X/Y/Z): each single operation within a few ulps,
V-cycle iterates within 1e-12 relative max-norm, converged float64 and mixed-precision solutions
within 1e-10 relative of the oracle's. The first-order projection step (ns_projection_step) against
oracle.staggered.projection_step field by field, step after step. At the 256^3 cavity size, where
the oracle cannot run whole steps in seconds, properties that hold at any size: the solver residuals
recomputed by the oracle from the returned fields, the divergence identity, the projection identity.
"""
import numpy as np
import pytest

from oracle import cell_centred as cc
from oracle import staggered as st
from workloads import NS_NAMES, ns_cavity, ns_state, random_field, zero_wall_slot

pytestmark = pytest.mark.gpu
D_ = cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _face_pair(fas, shape, comp, beta, **kw):
    h = 1.0 / shape[-1]
    op = st.FaceOperator(shape, h, 1.0, beta, comp)
    p = fas.make_params(shape, h, alpha=1.0, beta=beta, bc=(D_,) * (2 * len(shape)),
                        location=fas.FAS_FACE_X + comp, **kw)
    return op, fas.fas_create(p)


def _face_field(shape, comp, seed, lo=-1.0, hi=1.0):
    return zero_wall_slot(random_field(shape, seed, lo, hi), comp)


FACE_CASES = [((32, 64), 0), ((32, 64), 1), ((64, 16), 0), ((16, 16, 32), 0), ((16, 16, 32), 1),
              ((16, 16, 32), 2), ((8, 32, 16), 2)]


@pytest.mark.parametrize("shape,comp", FACE_CASES)
def test_face_single_operators(cuda_lib, shape, comp):
    fas = cuda_lib
    op, ctx = _face_pair(fas, shape, comp, 2e-3, coarsest=2)
    u = _face_field(shape, comp, 501)
    f = _face_field(shape, comp, 502)
    # residual (the wall slot is 0)
    out = _t(np.zeros(shape))
    nrm = fas.fas_residual(ctx, 0, _t(u), _t(f), out)
    r = st.residual_face(op, u, f)
    assert _rel(_n(out), r) <= 1e-14
    assert abs(nrm - cc.norm2(r)) <= 1e-6 * cc.norm2(r)
    # one X-MCGS sweep
    ug = _t(u)
    fas.fas_smooth(ctx, 0, ug, _t(f), 1)
    uo = u.copy()
    st.xmcgs_sweep_face(op, uo, f)
    assert _rel(_n(ug), uo) <= 1e-14
    # Appendix D restriction and prolongation
    cshape = tuple(n // 2 for n in shape)
    uc = _t(np.zeros(cshape))
    fas.fas_restrict(ctx, 0, _t(u), uc)
    assert _rel(_n(uc), st.restrict_face(op, u)) <= 1e-14
    c = _face_field(cshape, comp, 503)
    up = _t(u)
    fas.fas_prolong_add(ctx, 0, up, _t(c))
    ref = u + st.prolong_face(op, c)
    assert _rel(_n(up), ref) <= 1e-14
    # a non-zero value in the coarse wall slot is never read
    c2 = c.copy()
    c2[tuple(slice(None) if k != len(shape) - 1 - comp else cshape[k] - 1 for k in range(len(shape)))] = 7.0
    up2 = _t(u)
    fas.fas_prolong_add(ctx, 0, up2, _t(c2))
    assert np.array_equal(_n(up2), _n(up))


@pytest.mark.parametrize("shape,comp", [((256, 256), 0), ((256, 256), 1), ((64, 128), 1), ((32, 32, 32), 0),
                                        ((32, 32, 32), 2), ((16, 32, 64), 1)])
def test_face_vcycle_iterates(cuda_lib, shape, comp):
    """Grids above the single-CTA switch level run the per-operation face kernels on the top levels."""
    fas = cuda_lib
    beta = 1e-3 / 100.0 * (shape[-1] / 64.0) ** 2  # dt/Re scaled so that beta/h^2 stays O(1)
    op, ctx = _face_pair(fas, shape, comp, beta, coarsest=4)
    levels = st.build_levels_face(op, 4)
    u = _face_field(shape, comp, 511)
    f = _face_field(shape, comp, 512)
    ug, fg = _t(u), _t(f)
    for k in range(5):
        fas.fas_vcycle(ctx, ug, fg)
        st.vcycle_face(levels, u, f, cc.Params(coarsest=4))
        assert _rel(_n(ug), u) < 1e-12, "cycle %d" % (k + 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,comp", [((256, 256), 0), ((512, 256), 1), ((32, 64, 32), 2)])
def test_face_converged_solution(cuda_lib, precision, shape, comp):
    fas = cuda_lib
    beta = 1e-5 * (shape[-1] / 64.0) ** 2
    op, ctx = _face_pair(fas, shape, comp, beta, coarsest=4, precision=precision, kmax=40)
    f = _face_field(shape, comp, 521)
    u_ref = np.zeros(shape)
    info_ref = st.solve_face(st.build_levels_face(op, 4), u_ref, f, cc.Params(tol=1e-10, kmax=40, coarsest=4))
    ug = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, ug, _t(f))
    assert info.converged and info.rel <= 1e-10
    if precision == 0:
        assert info.cycles == info_ref.cycles
        assert _rel(_n(ug), u_ref) <= 1e-12
    r = st.residual_face(op, _n(ug), f)
    assert cc.norm2(r) <= 1e-10 * cc.norm2(f) * (1 + 1e-6)
    # against the oracle's solution to 1e-13, within 1e-10 relative max-norm: the GPU side solved
    # to 1e-12 (a 1e-10 residual bounds the error only in the 2-norm)
    _, ctx_t = _face_pair(fas, shape, comp, beta, coarsest=4, precision=precision, kmax=60, tol=1e-12)
    u_tight = np.zeros(shape)
    st.solve_face(st.build_levels_face(op, 4), u_tight, f, cc.Params(tol=1e-13, kmax=60, coarsest=4))
    ut = _t(np.zeros(shape))
    assert fas.fas_solve(ctx_t, ut, _t(f)).converged
    assert _rel(_n(ut), u_tight) <= 1e-10


def test_face_grid_rejections(cuda_lib):
    fas = cuda_lib
    shape = (32, 32)
    p = fas.make_params(shape, 1.0 / 32, bc=(cc.NEUMANN,) * 4, location=fas.FAS_FACE_X)
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(p)
    assert e.value.status == fas.FAS_EINVAL
    p = fas.make_params(shape, 1.0 / 32, bc=(D_,) * 4, location=fas.FAS_FACE_Z)
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(p)
    assert e.value.status == fas.FAS_EINVAL
    p = fas.make_params(shape, 1.0 / 32, bc=(D_,) * 4, location=fas.FAS_FACE_Y, coarse_exact=1)
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(p)
    assert e.value.status == fas.FAS_EUNSUPPORTED


# ---------------------------------------------------------------------------------------------
# projection step
# ---------------------------------------------------------------------------------------------

def _fas_params(fas, precision, kmax, coarse_exact=0, tol=1e-10):
    p = fas.fas_default_params()
    p.precision = precision
    p.kmax = kmax
    p.coarse_exact = coarse_exact
    p.coarsest = 4
    p.tol = tol
    return p


def _ns_pair(fas, shape, precision, Re=100.0, dt=1e-3, lid=(1.0, 0.0, 0.0), order=1, tol=1e-10):
    h = 1.0 / shape[-1]
    ns = fas.ns_create(shape, h, Re, dt, lid=lid, order=order, solver=_fas_params(fas, precision, 40, tol=tol),
                       pressure=_fas_params(fas, precision, 60, 1, tol=tol))
    prm = st.NSParams(Re=Re, dt=dt, lid=lid, solver=cc.Params(tol=tol, kmax=40, coarsest=4),
                      pressure=cc.Params(tol=tol, kmax=60, coarsest=4, coarse_exact=True))
    return ns, prm, h


def _fields_dim(dim):
    return [NS_NAMES[a] + k for a in range(dim) for k in ("_new", "_old")] + ["P_new", "P_old"]


def _bar(k, ref=None, h=None, rhs_max=None):
    """1e-12 relative for every field but the pressure increment p~ (P_new), which gets 1e-11: it is
    the iterate of a singular Neumann Poisson solve whose coarsest-level pseudo-inverse is computed
    independently on each side, and the operator's conditioning (about (2/(pi h))^2) magnifies the
    per-cycle rounding differences (1.4e-12 seen)."""
    return 1e-11 if k == "P_new" else 1e-12


@pytest.mark.parametrize("shape", [(32, 32), (64, 128), (16, 16, 16), (32, 32, 32)])
def test_projection_step_matches_oracle_fp64(cuda_lib, shape):
    fas = cuda_lib
    dim = len(shape)
    ns, prm, h = _ns_pair(fas, shape, 0, dt=2e-3)
    ref = ns_state(shape, 531)
    gpu = {k: _t(v) for k, v in ref.items()}
    names = _fields_dim(dim)
    for step in range(3):
        infos, dmax = fas.ns_projection_step(ns, gpu)
        infos_ref, div_ref, rhs_ref = st.projection_step(ref, shape, h, prm)
        got = [infos[a] for a in range(dim)] + [infos[3]]
        assert [i.cycles for i in got] == [i.cycles for i in infos_ref], "step %d" % step
        assert all(i.converged for i in got)
        for k in names:
            assert _rel(_n(gpu[k]), ref[k]) <= _bar(k, ref, h, rhs_ref), (step, k)
        assert dmax <= 1e-9 * max(div_ref, 1.0) + 1e-9


@pytest.mark.parametrize("shape", [(64, 64), (32, 32, 32)])
def test_projection_step_mixed_matches_oracle(cuda_lib, shape):
    """Mixed-precision solves inside the step: every field within 1e-10 relative max-norm of the
    oracle's float64 step. Every solve on both sides is taken to 1e-12 relative residual, so that the
    comparison measures the mixed-precision solver rather than where two iterations that both meet a
    1e-10 residual happened to stop."""
    fas = cuda_lib
    dim = len(shape)
    ns, prm, h = _ns_pair(fas, shape, 1, dt=2e-3, tol=1e-12)
    ref = ns_state(shape, 541)
    gpu = {k: _t(v) for k, v in ref.items()}
    for step in range(2):
        infos, dmax = fas.ns_projection_step(ns, gpu)
        st.projection_step(ref, shape, h, prm)
        assert all(infos[a].converged for a in range(dim)) and infos[3].converged
        for k in _fields_dim(dim):
            assert _rel(_n(gpu[k]), ref[k]) <= 1e-10, (step, k, _rel(_n(gpu[k]), ref[k]))


def test_projection_step_2d_cavity_from_rest(cuda_lib):
    """The lid drags the top row of x-velocity forward; the step keeps the wall slots at 0."""
    fas = cuda_lib
    w = ns_cavity(n=64, dim=2, nsteps=5)
    ns, prm, h = _ns_pair(fas, w["shape"], 0, Re=w["Re"], dt=w["dt"], lid=w["lid"])
    ref = {k: v.copy() for k, v in w["fields"].items()}
    gpu = {k: _t(v) for k, v in w["fields"].items()}
    for _ in range(w["nsteps"]):
        fas.ns_projection_step(ns, gpu)
        st.projection_step(ref, w["shape"], h, prm)
    U = _n(gpu["U_old"])
    assert U[-1].mean() > 0 and np.all(U[:, -1] == 0) and np.all(_n(gpu["V_old"])[-1] == 0)
    for k in _fields_dim(2):
        assert _rel(_n(gpu[k]), ref[k]) <= 1e-12, k


@pytest.mark.parametrize("precision", [0, 1])
def test_projection_step_cavity_256_cube_properties(cuda_lib, precision):
    """Two steps of the 256^3 lid-driven cavity (Re 100, dt 1e-3). After the second step (from a
    state with flow), checked with oracle functions on the returned fields:
      - each viscous residual f_c - A c~ (f_c from the oracle's source) is within tolerance;
      - the pressure residual and max |div u^{n+1}| agree: div u^{n+1} = -(r_p) exactly up to rounding;
      - u^{n+1} = c~ - dt grad p~ and p^{n+1} = p^n + p~."""
    fas = cuda_lib
    w = ns_cavity(n=256, dim=3, nsteps=2)
    shape, h, dt = w["shape"], w["h"], w["dt"]
    ns, prm, _ = _ns_pair(fas, shape, precision, Re=w["Re"], dt=dt, lid=w["lid"])
    gpu = {k: _t(v) for k, v in w["fields"].items()}
    del w["fields"]
    infos, dmax = fas.ns_projection_step(ns, gpu)
    assert all(i.converged for i in infos[:3]) and infos[3].converged
    before = {k: _n(gpu[k]) for k in ("U_old", "V_old", "W_old", "P_old")}
    infos, dmax = fas.ns_projection_step(ns, gpu)
    assert all(i.converged for i in infos[:3]) and infos[3].converged
    vel_n = [before[nm + "_old"] for nm in NS_NAMES]
    beta = dt / w["Re"]
    for comp, nm in enumerate(NS_NAMES):
        op = st.FaceOperator(shape, h, 1.0, beta, comp)
        f = vel_n[comp] - dt * st.convection(vel_n, comp, h, w["lid"]) - dt * st.pressure_gradient(
            before["P_old"], comp, h)
        f = f + st.lid_rhs(shape, comp, beta, h, w["lid"])
        f[st.frozen_slice(op)] = 0.0
        ct = _n(gpu[nm + "_new"])
        r = st.residual_face(op, ct, f)
        fn = cc.norm2(f)
        assert cc.norm2(r) <= 1e-10 * fn * (1 + 1e-3), nm
        assert abs(cc.norm2(r) - infos[comp].res) <= 1e-3 * infos[comp].res + 1e-14 * fn, nm
        # projection identity
        expect = ct - dt * st.pressure_gradient(_n(gpu["P_new"]), comp, h)
        assert _rel(_n(gpu[nm + "_old"]), expect) <= 1e-14, nm
        del f, r, ct, expect
    vel_t = [_n(gpu[nm + "_new"]) for nm in NS_NAMES]
    rhs = -st.divergence(vel_t, h)
    pop = cc.Operator(shape, h, 0.0, dt, 1.0)
    pn = _n(gpu["P_new"])
    rp = (rhs - rhs.mean()) - cc.apply_A(pop, pn)
    assert cc.norm2(rp) <= 1e-10 * cc.norm2(rhs) * (1 + 1e-3)
    div = st.divergence([_n(gpu[nm + "_old"]) for nm in NS_NAMES], h)
    assert abs(float(np.max(np.abs(div))) - dmax) <= 1e-12 * max(dmax, 1.0)
    assert dmax <= float(np.max(np.abs(rp))) + abs(float(rhs.mean())) + 1e-9
    assert np.array_equal(_n(gpu["P_old"]), before["P_old"] + pn)


# ---------------------------------------------------------------------------------------------
# body force and the paper's asymptotic-in-time convergence test (Sec. 4.4.3)
# ---------------------------------------------------------------------------------------------

def test_forced_projection_step_matches_oracle(cuda_lib):
    from workloads import mms_field, ns_mms
    fas = cuda_lib
    w = ns_mms(64, 10.0)
    shape, h, dt = w["shape"], w["h"], 0.05
    ns, prm, _ = _ns_pair(fas, shape, 0, Re=10.0, dt=dt, lid=(0.0, 0.0, 0.0))
    ref = ns_state(shape, 551, amplitude=0.2)
    gpu = {k: _t(v) for k, v in ref.items()}
    for step in range(3):
        t1 = (step + 1) * dt
        F = [mms_field(w["force"][0], t1, 0), mms_field(w["force"][1], t1, 1)]
        fas.ns_projection_step(ns, gpu, force=[_t(F[0]), _t(F[1])])
        st.projection_step(ref, shape, h, prm, force=F)
        for k in _fields_dim(2):
            assert _rel(_n(gpu[k]), ref[k]) <= 1e-12, (step, k)


def test_paper_first_order_convergence_table(cuda_lib):
    """Table first-convergence-test (Sec. 4.4.3) on the GPU at 1024^2 (the paper: 4096^2; the spatial
    error left at 1024^2 is below 0.5 % of every entry): u, v, p errors at t = 1 for dt = 1/10 ... 1/80
    within 1.5 % of the printed values, and their ratios (first order) within 3 %."""
    import json
    import os

    import torch
    from workloads import ns_mms
    fas = cuda_lib
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ns_first_order_mms.json")))
    n = 1024
    w = ns_mms(n, 10.0)
    shape, h = w["shape"], w["h"]

    def dev_terms(terms):
        return [(fn, torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda()) for fn, Y, X in terms]

    def field(terms, t, comp=None):
        out = sum(float(fn(t)) * torch.outer(Y, X) for fn, Y, X in terms)
        if comp == 0:
            out[:, -1] = 0.0
        elif comp == 1:
            out[-1, :] = 0.0
        return out.contiguous()

    fu, fv = dev_terms(w["force"][0]), dev_terms(w["force"][1])
    eu, ev, ep = dev_terms(w["exact"][0]), dev_terms(w["exact"][1]), dev_terms(w["exact"]["p"])
    errs = []
    for nsteps in g["dt_inverse"][:4]:
        dt = 1.0 / nsteps
        sp = fas.fas_default_params()
        sp.tol, sp.kmax, sp.coarsest = 1e-9, 20, 4
        pp = fas.fas_default_params()
        pp.tol, pp.kmax, pp.coarsest, pp.coarse_exact = 1e-9, 60, 4, 1
        ns = fas.ns_create(shape, h, 10.0, dt, lid=(0.0, 0.0, 0.0), solver=sp, pressure=pp)
        flds = {k: torch.zeros(shape, dtype=torch.float64, device="cuda") for k in _fields_dim(2)}
        for k in range(nsteps):
            t1 = (k + 1) * dt
            infos, _ = fas.ns_projection_step(ns, flds, want_div=False, force=[field(fu, t1, 0), field(fv, t1, 1)])
            assert infos[0].converged and infos[1].converged and infos[3].converged
        l2 = lambda a, b: float(torch.sqrt(h * h * torch.sum((a - b) ** 2)))  # noqa: E731
        errs.append((l2(flds["U_old"], field(eu, 1.0, 0)), l2(flds["V_old"], field(ev, 1.0, 1)),
                     l2(flds["P_old"], field(ep, 1.0))))
        fas.ns_destroy(ns)
    for row, e in enumerate(errs):
        for k, key in enumerate(("err_u", "err_v", "err_p")):
            assert abs(e[k] - g[key][row]) <= 0.015 * g[key][row], (key, row, e[k], g[key][row])
    for row in range(1, len(errs)):
        for k, key in enumerate(("err_u", "err_v", "err_p")):
            mine = errs[row - 1][k] / errs[row][k]
            printed = g[key][row - 1] / g[key][row]
            assert abs(mine / printed - 1.0) <= 0.03, (key, row, mine, printed)



# ---------------------------------------------------------------------------------------------
# second-order scheme (Sec. 4.3)
# ---------------------------------------------------------------------------------------------

def _state2(shape, seed):
    """c^n in *_new, a different c^{n-1} in *_old (second-order slot convention)."""
    a = ns_state(shape, seed)
    b = ns_state(shape, seed + 1, amplitude=0.4)
    dim = len(shape)
    out = {}
    for k in range(dim):
        out[NS_NAMES[k] + "_new"] = a[NS_NAMES[k] + "_old"]
        out[NS_NAMES[k] + "_old"] = b[NS_NAMES[k] + "_old"]
    out["P_old"] = a["P_old"]
    out["P_new"] = np.zeros(shape)
    return out


@pytest.mark.parametrize("shape", [(32, 32), (64, 128), (16, 16, 16), (32, 32, 32)])
def test_second_order_step_matches_oracle_fp64(cuda_lib, shape):
    fas = cuda_lib
    dim = len(shape)
    ns, prm, h = _ns_pair(fas, shape, 0, dt=2e-3, order=2)
    ref = _state2(shape, 561)
    gpu = {k: _t(v) for k, v in ref.items()}
    for step in range(3):
        infos, dmax = fas.ns_projection_step(ns, gpu)
        infos_ref, div_ref, rhs_ref = st.projection_step2(ref, shape, h, prm)
        got = [infos[a] for a in range(dim)] + [infos[3]]
        assert [i.cycles for i in got] == [i.cycles for i in infos_ref], "step %d" % step
        for k in _fields_dim(dim):
            assert _rel(_n(gpu[k]), ref[k]) <= _bar(k, ref, h, rhs_ref), (step, k, _bar(k, ref, h, rhs_ref))
        assert dmax <= 1e-9 * max(div_ref, 1.0) + 1e-9


@pytest.mark.parametrize("shape", [(64, 64), (16, 32, 32)])
def test_second_order_step_mixed_matches_oracle(cuda_lib, shape):
    """Second-order step with mixed-precision solves: every field within 1e-10 relative max-norm of
    the oracle's float64 step, every solve on both sides taken to 1e-12 relative residual."""
    fas = cuda_lib
    dim = len(shape)
    ns, prm, h = _ns_pair(fas, shape, 1, dt=2e-3, order=2, tol=1e-12)
    ref = _state2(shape, 571)
    gpu = {k: _t(v) for k, v in ref.items()}
    for step in range(2):
        infos, _ = fas.ns_projection_step(ns, gpu)
        st.projection_step2(ref, shape, h, prm)
        assert all(infos[a].converged for a in range(dim)) and infos[3].converged
        for k in _fields_dim(dim):
            assert _rel(_n(gpu[k]), ref[k]) <= 1e-10, (step, k, _rel(_n(gpu[k]), ref[k]))


def test_order_rejected(cuda_lib):
    fas = cuda_lib
    with pytest.raises(fas.FasError) as e:
        fas.ns_create((32, 32), 1.0 / 32, 100.0, 1e-3, order=3)
    assert e.value.status == fas.FAS_EUNSUPPORTED


def test_paper_second_order_convergence_table(cuda_lib):
    """Table second-convergence-test (Sec. 4.4.3) on the GPU at 1024^2 with the step-averaged body
    force: u, v, p errors at t = 1 for dt = 1/10, 1/20, 1/40 within 2.5 % of the printed values (the
    garbled u and p entries at 1/20 read as the values their printed orders imply); u, v errors fall
    by about 4 per halving of dt."""
    import json
    import os

    import torch
    from workloads import ns_mms
    fas = cuda_lib
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ns_second_order_mms.json")))
    n = 1024
    w = ns_mms(n, 10.0)
    shape, h = w["shape"], w["h"]

    def dev_terms(terms):
        return [(fn, torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda()) for fn, Y, X in terms]

    def field(terms, t, comp=None):
        out = sum(float(fn(t)) * torch.outer(Y, X) for fn, Y, X in terms)
        if comp == 0:
            out[:, -1] = 0.0
        elif comp == 1:
            out[-1, :] = 0.0
        return out.contiguous()

    fu, fv = dev_terms(w["force"][0]), dev_terms(w["force"][1])
    eu, ev, ep = dev_terms(w["exact"][0]), dev_terms(w["exact"][1]), dev_terms(w["exact"]["p"])
    errs = []
    for nsteps in g["dt_inverse"][:3]:
        dt = 1.0 / nsteps
        sp = fas.fas_default_params()
        sp.tol, sp.kmax, sp.coarsest = 1e-9, 20, 4
        pp = fas.fas_default_params()
        pp.tol, pp.kmax, pp.coarsest, pp.coarse_exact = 1e-9, 60, 4, 1
        ns = fas.ns_create(shape, h, 10.0, dt, lid=(0.0, 0.0, 0.0), order=2, solver=sp, pressure=pp)
        flds = {k: torch.zeros(shape, dtype=torch.float64, device="cuda") for k in _fields_dim(2)}
        for k in range(nsteps):
            a, b = k * dt, (k + 1) * dt
            F = [0.5 * (field(fu, a, 0) + field(fu, b, 0)), 0.5 * (field(fv, a, 1) + field(fv, b, 1))]
            infos, _ = fas.ns_projection_step(ns, flds, want_div=False, force=F)
            assert infos[0].converged and infos[1].converged and infos[3].converged
        l2 = lambda x, y: float(torch.sqrt(h * h * torch.sum((x - y) ** 2)))  # noqa: E731
        errs.append((l2(flds["U_new"], field(eu, 1.0, 0)), l2(flds["V_new"], field(ev, 1.0, 1)),
                     l2(flds["P_old"], field(ep, 1.0))))
        fas.ns_destroy(ns)
    for row, e in enumerate(errs):
        for k, key in enumerate(("err_u_read", "err_v", "err_p_read")):
            assert abs(e[k] - g[key][row]) <= 0.025 * g[key][row], (key, row, e[k], g[key][row])
    for row in range(1, len(errs)):
        for k in (0, 1):
            assert 3.6 < errs[row - 1][k] / errs[row][k] < 4.6, (row, k, errs)


@pytest.mark.parametrize("shape,steps,order", [((512, 512), 2, 1), ((64, 64, 64), 2, 1), ((128, 128, 128), 1, 1),
                                               ((64, 64, 64), 2, 2)])
def test_projection_steps_larger_grids_match_oracle(cuda_lib, shape, steps, order):
    """Projection steps on larger grids than the other parity tests (up to 128^3, where the oracle
    still runs a step in seconds): every field within 1e-12 relative max-norm of the oracle's (the
    pressure increment 1e-11), equal cycle counts, float64 solves."""
    fas = cuda_lib
    dim = len(shape)
    ns, prm, h = _ns_pair(fas, shape, 0, dt=2e-3, order=order)
    ref = ns_state(shape, 591) if order == 1 else _state2(shape, 592)
    gpu = {k: _t(v) for k, v in ref.items()}
    step_fn = st.projection_step if order == 1 else st.projection_step2
    for step in range(steps):
        infos, _ = fas.ns_projection_step(ns, gpu)
        infos_ref, _, rhs_ref = step_fn(ref, shape, h, prm)
        got = [infos[a] for a in range(dim)] + [infos[3]]
        assert [i.cycles for i in got] == [i.cycles for i in infos_ref], "step %d" % step
        for k in _fields_dim(dim):
            assert _rel(_n(gpu[k]), ref[k]) <= _bar(k), (step, k, _rel(_n(gpu[k]), ref[k]))
