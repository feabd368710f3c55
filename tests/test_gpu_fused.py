"""The sweep-fused float32 kernels compute exactly what the per-operation kernels compute.

Both paths evaluate every point with the same expression in the same order, so mixed-precision
refinement steps through either path must give bit-identical float64 iterates. The per-operation
path is itself pinned to the oracle (test_gpu_parity.py)."""
import numpy as np
import pytest

from oracle import cell_centred as cc
from workloads import noisy_cos_mode, random_field

pytestmark = pytest.mark.gpu
N_, D_ = cc.NEUMANN, cc.DIRICHLET


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("shape", [(256, 256), (128, 512), (1024, 1024), (64, 2048), (2048, 256)])
@pytest.mark.parametrize("bc", [(N_,) * 4, (D_,) * 4, (D_, N_, N_, D_)])
@pytest.mark.parametrize("nu,inner", [(2, 1), (1, 1), (2, 2)])
def test_fused_equals_per_operation(cuda_lib, shape, bc, nu, inner):
    fas = cuda_lib
    h = 1.0 / shape[-1]
    u0 = random_field(shape, 301)
    f = noisy_cos_mode(shape, 302)
    outs = []
    for path in (0, 2, 1):  # default, fused on every level the kernels handle, per-operation
        ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=2e-3, bc=bc, coarsest=4, precision=1,
                                             path=path, nu1=nu, nu2=nu, inner_cycles=inner))
        u = _t(u0)
        for _ in range(4):
            fas.fas_vcycle(ctx, u, _t(f))
        outs.append(u.cpu().numpy())
        fas.fas_destroy(ctx)
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[1], outs[2])


@pytest.mark.parametrize("seg", [8, 16, 64, 256])
def test_fused_segment_sizes(cuda_lib, seg):
    fas = cuda_lib
    shape = (512, 512)
    u0 = random_field(shape, 311)
    f = random_field(shape, 312, -1, 1)
    outs = []
    for path, sg in ((2, seg), (1, 0)):
        ctx = fas.fas_create(fas.make_params(shape, 1.0 / 512, beta=1e-3, precision=1, path=path, seg_rows=sg))
        u = _t(u0)
        for _ in range(3):
            fas.fas_vcycle(ctx, u, _t(f))
        outs.append(u.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_profiler_reports_fused_kernels(cuda_lib):
    fas = cuda_lib
    shape = (1024, 1024)
    ctx = fas.fas_create(fas.make_params(shape, 1.0 / 1024, beta=1e-3, precision=1))
    fas.fas_prof_enable(ctx, True)
    u = _t(np.zeros(shape))
    info = fas.fas_solve(ctx, u, _t(noisy_cos_mode(shape, 321)))
    recs = fas.fas_prof_read(ctx)
    fams = {(r["family"], r["level"]) for r in recs}
    # one inner cycle: the level-0 post-smoothing also adds to the float64 solution (timed as "update")
    assert ("smooth", 0) in fams and ("update", 0) in fams and ("prolong", 1) in fams
    assert ("ir", 0) in fams and ("coarse", 3) in fams
    sm0 = [r for r in recs if r["family"] == "smooth" and r["level"] == 0][0]
    assert sm0["launches"] == info.cycles and sm0["ms"] > 0


def _fused3d_vcycles(fas, shape, bc, nu, path, cycles=3):
    h = 1.0 / shape[-1]
    u0 = random_field(shape, 321)
    f = noisy_cos_mode(shape, 322)
    ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=2e-3, bc=bc, coarsest=4, precision=1,
                                         path=path, nu1=nu, nu2=nu))
    u = _t(u0)
    ft = _t(f)
    for _ in range(cycles):
        fas.fas_vcycle(ctx, u, ft)
    fas.fas_destroy(ctx)
    return u.cpu().numpy()


@pytest.mark.parametrize("bc", [(N_,) * 6, (D_, N_, N_, D_, N_, D_)])
@pytest.mark.parametrize("nu", [2, 3])
def test_fused_3d_sweep_full_size_level(cuda_lib, bc, nu):
    """At a size the fused 3D sweep is used for (256 x 512 x 512, level 0): V-cycles equal the
    per-operation path's bit for bit."""
    fas = cuda_lib
    shape = (256, 512, 512)
    a = _fused3d_vcycles(fas, shape, bc, nu, 0, cycles=2)
    b = _fused3d_vcycles(fas, shape, bc, nu, 1, cycles=2)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("shape", [(16, 32, 128), (32, 64, 256), (8, 16, 128), (64, 128, 256), (32, 16, 512)])
@pytest.mark.parametrize("bc", [(N_,) * 6, (D_,) * 6, (D_, N_, N_, D_, N_, D_)])
@pytest.mark.parametrize("nu", [1, 2, 3])
def test_fused_3d_sweep_equals_per_operation(cuda_lib, shape, bc, nu):
    """The sweep-fused 3D float32 smoothing (both colour phases in one pass, pairs of sweeps ping-pong
    between two buffers; path 2 uses it on levels below the size where it pays) gives the
    per-operation colour launches' mixed-precision iterates bit for bit: strips of 128 columns, row
    groups that do not divide ny, short plane segments, every boundary kind, an odd sweep count (its
    last sweep runs per colour phase)."""
    fas = cuda_lib
    np.testing.assert_array_equal(_fused3d_vcycles(fas, shape, bc, nu, 2), _fused3d_vcycles(fas, shape, bc, nu, 1))
