"""The float64 work done with integer operations (bits64.cuh) is exact.

- The integer float32 <-> float64 conversions equal the hardware conversions bit for bit on special
  values, ties and millions of random patterns (fas_selftest_conversions).
- The refinement residual r32 = (float)(f - A u) of the mixed solve (fas_residual_ir): where the
  stencil qualifies, the kernel computes S = sum_nb u_nb - M u exactly and then
  r = RN(c RN(S) + RN(f - alpha u)) rounded to float32; that value is reproduced here in exact rational
  arithmetic (fractions.Fraction), so every such cell must match bit for bit. The other cells use the
  float64 point equation and are compared with the oracle's float64 residual.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cell_centred as cc
from oracle import staggered as st
from workloads import noisy_cos_mode, random_field, uniform, zero_wall_slot

pytestmark = pytest.mark.gpu
N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_conversions_match_hardware(cuda_lib):
    fas = cuda_lib
    assert fas.fas_selftest_conversions(1 << 22, seed=7) == 0
    assert fas.fas_selftest_conversions(0) == 0  # the special values alone


def _exp_field(x):
    return int((np.float64(x).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def _mult(bc, fax, dim):
    """Multiplicity of each of the 2*dim faces for a boundary cell (x_lo, x_hi, y_lo, ...)."""
    out = []
    for face in range(2 * dim):
        if fax is not None and face // 2 == fax:
            out.append(1)
        else:
            out.append(2 if bc[face] == D_ else 0)
    return out


def _expected_exact(u, f, idx, alpha, c, mult):
    """The exact-path value for cell idx (physical order i, j[, l]) or None when the cell takes the
    float64 path (the kernel's criteria)."""
    dim = u.ndim
    shape_phys = list(reversed(u.shape))
    vals_nb = []
    M = 0
    for a in range(dim):
        for side, off in ((0, -1), (1, +1)):
            k = list(idx)
            k[a] += off
            if 0 <= k[a] < shape_phys[a]:
                vals_nb.append(float(u[tuple(reversed(k))]))
                M += 1
            else:
                M += mult[2 * a + side]
    uc = float(u[tuple(reversed(idx))])
    # exact zeros take no part in the exponent range (the 3D kernel treats them as exact values)
    es = [_exp_field(v) for v in [uc] + vals_nb if v != 0.0]
    if es and (any(e == 0 or e == 0x7FF for e in es) or max(es) - min(es) > 5):
        return None
    S = sum(Fraction(v) for v in vals_nb) - M * Fraction(uc)
    Sd = float(S)
    if S != 0 and (abs(Sd) < 2.2250738585072014e-308 or not np.isfinite(Sd)):
        return None
    T = float(Fraction(float(f[tuple(reversed(idx))])) - Fraction(alpha) * Fraction(uc))
    r = float(Fraction(c) * Fraction(Sd) + Fraction(T))
    return np.float32(r)


CASES = [
    # shape, field, bc, alpha, beta, face axis, least fraction of sampled cells on the exact path.
    # 2D cell grids with nx a multiple of 128 run the strip kernel, which decides per warp row (three
    # rows of 130 values): fields crossing zero or random fields take the float64 path there.
    ((256, 256), "positive", (N_,) * 4, 1.0, 1e-3, None, 0.95),
    ((256, 512), "smooth", (D_, N_, N_, D_), 1.0, 1e-3, None, 0.0),
    ((128, 256), "random", (D_, N_, N_, D_), 1.0, 5e-2, None, 0.0),
    ((128, 128), "positive", (D_,) * 4, 1.0, 1e-2, None, 0.95),
    ((64, 64), "zeros", (N_,) * 4, 0.0, 1.0, None, 0.0),
    ((64, 32), "smooth", (N_, D_, D_, N_), 1.0, 1e-3, None, 0.6),
    ((32, 32, 32), "smooth", (D_, N_, N_, N_, D_, D_), 1.0, 1e-3, None, 0.8),
    ((16, 32, 16), "random", (N_,) * 6, 0.7, 2e-2, None, 0.5),
    ((64, 128), "random", (D_,) * 4, 1.0, 1e-3, 1, 0.5),
    ((16, 16, 32), "smooth", (D_,) * 6, 1.0, 1e-4, 0, 0.8),
    # 3D strip kernel: nx a multiple of 128, ny a multiple of 8 (cells and every face axis)
    ((16, 32, 128), "positive", (D_, N_, N_, N_, D_, D_), 1.0, 1e-3, None, 0.95),
    ((8, 16, 256), "smooth", (N_,) * 6, 1.0, 1e-3, None, 0.0),
    ((16, 16, 128), "positive", (D_,) * 6, 1.0, 1e-3, 0, 0.9),
    ((16, 16, 128), "positive", (D_,) * 6, 1.0, 1e-3, 1, 0.9),
    ((16, 16, 128), "positive", (D_,) * 6, 1.0, 1e-3, 2, 0.9),
    ((8, 8, 128), "zeros", (N_,) * 6, 0.0, 1.0, None, 0.0),
]


@pytest.mark.parametrize("shape,kind,bc,alpha,beta,fax,cover", CASES)
def test_refinement_residual_exact(cuda_lib, shape, kind, bc, alpha, beta, fax, cover):
    import torch
    fas = cuda_lib
    dim = len(shape)
    h = 1.0 / shape[-1]
    if kind in ("smooth", "positive"):
        u = noisy_cos_mode(shape, 601) + (1.5 if kind == "positive" else 0.0)
    else:
        u = random_field(shape, 602, -1, 1)
    if kind == "zeros":
        u.ravel()[::7] = 0.0
    f = u + 1e-3 * random_field(shape, 603, -1, 1)
    kw = {}
    if fax is not None:
        kw["location"] = fas.FAS_FACE_X + fax
        u = zero_wall_slot(u, fax)
    p = fas.make_params(shape, h, alpha=alpha, beta=beta, bc=bc, **kw)
    ctx = fas.fas_create(p)
    r32 = torch.empty(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    nrm = fas.fas_residual_ir(ctx, _t(u), _t(f), r32)
    got = r32.cpu().numpy().reshape(shape)
    assert abs(nrm - float(np.linalg.norm(got.astype(np.float64)))) <= 1e-5 * nrm
    # the oracle's float64 residual for every cell
    if fax is None:
        r64 = cc.residual(cc.Operator(shape, h, alpha, beta, 1.0, bc), u, f)
    else:
        r64 = st.residual_face(st.FaceOperator(shape, h, alpha, beta, fax), u, f)
    c = (beta * 1.0) / (h * h)
    mult = _mult(bc, fax, dim)
    # sample cells: random ones plus every cell of the first and last rows (boundary classes)
    ncell = int(np.prod(shape))
    picks = (uniform(604, 1, 1500) * ncell).astype(np.int64)
    rows = np.concatenate([np.arange(shape[-1]), ncell - 1 - np.arange(shape[-1])])
    cells = np.unique(np.concatenate([picks, rows]))
    n_exact, n_cells = 0, 0
    for lin in cells:
        nidx = np.unravel_index(int(lin), shape)
        idx = tuple(reversed([int(v) for v in nidx]))  # physical i, j[, l]
        if fax is not None and idx[fax] == shape[dim - 1 - fax] - 1:
            assert got[nidx] == 0.0
            continue
        n_cells += 1
        exp = _expected_exact(u, f, idx, alpha, c, mult)
        if exp is not None and got[nidx].view(np.uint32) == exp.view(np.uint32):
            n_exact += 1
            continue
        # the float64 point equation
        ref = r64[nidx]
        scale = abs(float(f[nidx])) + (abs(alpha) + 12 * c) * abs(float(u[nidx])) + 1e-300
        assert abs(float(got[nidx]) - ref) <= 2.0 ** -23 * abs(ref) + 1e-13 * scale, idx
    assert n_exact >= cover * n_cells, (n_exact, n_cells)


def test_refinement_residual_is_reproducible(cuda_lib):
    """The 2D strip kernel hands its segments to whichever warp is free: r32 must not depend on that
    assignment (bit for bit); the norm sums per-block partials whose float32 accumulation order
    does, so only its last bits may vary."""
    import torch
    fas = cuda_lib
    shape = (1024, 1024)
    u = noisy_cos_mode(shape, 611)  # crosses zero: some segments take the float64 path
    f = u + 1e-3 * random_field(shape, 612, -1, 1)
    ctx = fas.fas_create(fas.make_params(shape, 1.0 / 1024, alpha=1.0, beta=1e-4, precision=fas.FAS_MIXED))
    ut, ft = _t(u), _t(f)
    r32 = torch.empty(u.size, dtype=torch.float32, device="cuda")
    first = fas.fas_residual_ir(ctx, ut, ft, r32)
    r_first = r32.clone()
    ref = float(np.linalg.norm(r_first.cpu().numpy().astype(np.float64)))
    assert abs(first - ref) <= 1e-6 * ref
    for _ in range(6):
        nrm = fas.fas_residual_ir(ctx, ut, ft, r32)
        assert abs(nrm - first) <= 1e-9 * first
        assert torch.equal(r32, r_first)


def test_bounded_wait_runs_out_and_context_stays_usable(cuda_lib):
    """The 3D refinement residual waits for its tile copies with a deadline. With one copy withheld
    (the test hook), the call returns FAS_ETIMEOUT after the deadline instead of waiting forever; the
    next call on the same context gives the same residual as before, bit for bit, and a solve on the
    context converges."""
    import torch
    fas = cuda_lib
    shape = (32, 64, 128)
    u = noisy_cos_mode(shape, 621) + 1.5
    f = u + 1e-3 * random_field(shape, 622, -1, 1)
    ctx = fas.fas_create(fas.make_params(shape, 1.0 / 128, alpha=1.0, beta=1e-3, precision=fas.FAS_MIXED, kmax=60))
    ut, ft = _t(u), _t(f)
    r32 = torch.empty(u.size, dtype=torch.float32, device="cuda")
    n0 = fas.fas_residual_ir(ctx, ut, ft, r32)
    r_ref = r32.clone()
    fas.fas_debug_bounded_wait(20_000_000, withhold_next=1)  # 20 ms
    try:
        with pytest.raises(fas.FasError) as e:
            fas.fas_residual_ir(ctx, ut, ft, r32)
        assert e.value.status == fas.FAS_ETIMEOUT
    finally:
        fas.fas_debug_bounded_wait(1_000_000_000, withhold_next=0)
    n1 = fas.fas_residual_ir(ctx, ut, ft, r32)
    assert torch.equal(r32, r_ref) and abs(n1 - n0) <= 1e-9 * n0
    x = _t(np.zeros(shape))
    assert fas.fas_solve(ctx, x, ft).converged


def test_bounded_wait_of_the_fused_sweep(cuda_lib):
    """The same for the sweep-fused 3D smoother (forced on a small level with path 2): a withheld tile
    copy makes the V-cycle return FAS_ETIMEOUT after the deadline; the next V-cycle on the same context
    from the same start gives the result of an undisturbed context bit for bit."""
    fas = cuda_lib
    shape = (32, 64, 128)
    params = fas.make_params(shape, 1.0 / 128, alpha=1.0, beta=2e-3, precision=fas.FAS_MIXED, path=2, use_graph=0)
    u0 = random_field(shape, 631)
    f = _t(random_field(shape, 632, -1, 1))
    ref = _t(u0)
    fas.fas_vcycle(fas.fas_create(params), ref, f)
    ctx = fas.fas_create(params)
    fas.fas_debug_bounded_wait(20_000_000, withhold_next=2)
    try:
        with pytest.raises(fas.FasError) as e:
            fas.fas_vcycle(ctx, _t(u0), f)
        assert e.value.status == fas.FAS_ETIMEOUT
    finally:
        fas.fas_debug_bounded_wait(1_000_000_000, withhold_next=0)
    u = _t(u0)
    fas.fas_vcycle(ctx, u, f)
    np.testing.assert_array_equal(u.cpu().numpy(), ref.cpu().numpy())
