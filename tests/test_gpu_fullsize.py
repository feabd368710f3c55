"""The benchmarked workloads at their full sizes, in the benchmark's launch configuration, against the
plain definition of what they converge to.

With homogeneous Neumann faces and a constant diffusivity the cell-centred operator I - dt Lap_h is
diagonalised by the type-II cosine transform, with eigenvalues 1 + dt (4/h^2) sum_axes sin^2(pi k / 2N):
one backward-Euler step is exactly u^{n+1} = IDCT(DCT(u^n + dt f) / lambda). Each GPU step stops at a
residual r_k with ||r_k||_2 <= 1e-10 ||b_k||_2; the step's own error is A^-1 r_k, and since A is
symmetric with eigenvalues >= 1 (||A^-1||_2 <= 1) neither that error nor those of earlier steps grows,
so after k steps ||u_gpu - u_exact||_2 <= sum_k ||r_k||_2 (the final residuals the solver reports).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _exact_steps(u0, fsrc, dt, h, nsteps):
    fft = pytest.importorskip("scipy.fft")
    shape = u0.shape
    lam = 1.0
    for ax, n in enumerate(shape):
        l1 = 4.0 / (h * h) * np.sin(np.arange(n) * np.pi / (2 * n)) ** 2
        sh = [1] * len(shape)
        sh[ax] = n
        lam = lam + dt * l1.reshape(sh)
    u = u0.copy()
    for _ in range(nsteps):
        b = u + dt * fsrc if fsrc is not None else u
        u = fft.idctn(fft.dctn(b, type=2, norm="ortho", workers=-1) / lam, type=2, norm="ortho", workers=-1)
    return u


def _check(got, ref, infos):
    """The error bound above, with 2% slack for the float32 rounding of the residual the norm is taken
    of and the transform's own rounding (~1e-16 ||u|| log n)."""
    err = float(np.linalg.norm(got - ref))
    bound = 1.02 * sum(i.res for i in infos) + 1e-13 * float(np.linalg.norm(ref))
    assert err <= bound, (err, bound)
    # and the per-step residuals are themselves within the tolerance
    assert all(i.converged and i.rel <= 1e-10 for i in infos), [i.as_dict() for i in infos]


def test_heat2d_8192_mixed_against_exact_stepping(cuda_lib):
    """The 8192^2 benchmark workload (Neumann, dt 1e-4, 16-Gaussian source), mixed precision with
    two float32 cycles per refinement step and one CUDA graph per solve (the bench's configuration),
    two backward-Euler steps."""
    import torch
    from workloads import heat2d_large
    fas = cuda_lib
    w = heat2d_large(n=8192, nsteps=2)
    shape, h, dt, nsteps = w["shape"], w["h"], w["dt"], w["nsteps"]
    ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=dt, coarsest=4, precision=fas.FAS_MIXED,
                                         inner_cycles=2, use_graph=1))
    u = torch.from_numpy(w["u0"]).cuda()
    infos = fas.fas_heat_run(ctx, u, torch.from_numpy(w["fsrc"]).cuda(), dt, nsteps)
    got = u.cpu().numpy()
    _check(got, _exact_steps(w["u0"], w["fsrc"], dt, h, nsteps), infos)


def test_heat3d_512_mixed_against_exact_stepping(cuda_lib):
    """The 512^3 workload (Neumann, dt 1e-4, no source), mixed precision, one backward-Euler step."""
    import torch
    from workloads import heat3d
    fas = cuda_lib
    w = heat3d(n=512, nsteps=1)
    shape, h, dt = w["shape"], w["h"], w["dt"]
    ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=dt, coarsest=4, precision=fas.FAS_MIXED))
    u = torch.from_numpy(w["u0"]).cuda()
    infos = fas.fas_heat_run(ctx, u, None, dt, 1)
    got = u.cpu().numpy()
    del u
    _check(got, _exact_steps(w["u0"], None, dt, h, 1), infos)
