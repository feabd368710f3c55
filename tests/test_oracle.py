"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test ties an oracle function to something other than itself: closed-form eigenpairs of the
discrete operator, the defining property of a Gauss-Seidel point update, a literal point-by-point
red-black loop, exact transfer identities, dense direct and fast-transform solves, closed-form
eigenmode decay of backward Euler, and the errors the paper prints in Tables err_2D / err_3D.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import cell_centred as cc
from tests.mms import exact_and_source, l2_error
from workloads import random_field

N_, D_, P_ = cc.NEUMANN, cc.DIRICHLET, cc.PERIODIC
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_error_tables.json")


def _mode_1d(kind_lo, kind_hi, n, k):
    """Eigenvector and eigenvalue of the 1D cell-centred -d^2/dx^2 with ghost relations
    (Neumann ghost = cell, Dirichlet ghost = -cell) on n cells of width h = 1/n."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    if kind_lo == N_ and kind_hi == N_:
        theta = k * math.pi  # cosine modes, k = 0..n-1
        v = np.cos(theta * x)
    elif kind_lo == D_ and kind_hi == D_:
        theta = (k + 1) * math.pi  # sine modes, k = 0..n-1
        v = np.sin(theta * x)
    elif kind_lo == D_ and kind_hi == N_:
        theta = (k + 0.5) * math.pi
        v = np.sin(theta * x)
    else:  # Neumann low, Dirichlet high
        theta = (k + 0.5) * math.pi
        v = np.cos(theta * x)
    lam = 4.0 / (h * h) * math.sin(theta * h / 2.0) ** 2
    return v, lam


@pytest.mark.parametrize("bc", [(N_, N_, N_, N_), (D_, D_, D_, D_), (D_, N_, D_, N_), (N_, D_, D_, N_)])
def test_operator_2d_closed_form_eigenpairs(bc):
    """Sec. 2.2 operator with the ghost relations of Eqs. boundry1-2: tensor products of the 1D
    cosine / sine modes are eigenvectors with eigenvalue alpha + beta (lam_x + lam_y)."""
    nx, ny = 16, 8
    h = 1.0 / nx
    alpha, beta = 0.7, 1.3e-3
    op = cc.Operator((ny, nx), h, alpha, beta, 1.0, bc)
    rng_pairs = [(0, 0), (1, 3), (5, 2), (15, 7), (8, 0)]
    for kx, ky in rng_pairs:
        vx, lx = _mode_1d(bc[0], bc[1], nx, kx)
        # y axis has ny cells but the same h: rescale the 1D mode to h = 1/nx
        y = (np.arange(ny) + 0.5) * h
        if bc[2] == N_ and bc[3] == N_:
            th = ky * math.pi / (ny * h)
            vy = np.cos(th * y)
        elif bc[2] == D_ and bc[3] == D_:
            th = (ky + 1) * math.pi / (ny * h)
            vy = np.sin(th * y)
        elif bc[2] == D_ and bc[3] == N_:
            th = (ky + 0.5) * math.pi / (ny * h)
            vy = np.sin(th * y)
        else:
            th = (ky + 0.5) * math.pi / (ny * h)
            vy = np.cos(th * y)
        ly = 4.0 / (h * h) * math.sin(th * h / 2.0) ** 2
        v = vy[:, None] * vx[None, :]
        Av = cc.apply_A(op, v)
        lam = alpha + beta * (lx + ly)
        np.testing.assert_allclose(Av, lam * v, atol=1e-12 * lam)


def test_operator_3d_closed_form_eigenpairs():
    n = 8
    h = 1.0 / n
    op = cc.Operator((n, n, n), h, 1.0, 2e-3, 1.0, (D_, N_, N_, N_, D_, D_))
    for kx, ky, kz in [(0, 0, 0), (1, 2, 3), (7, 7, 7)]:
        vx, lx = _mode_1d(D_, N_, n, kx)
        vy, ly = _mode_1d(N_, N_, n, ky)
        vz, lz = _mode_1d(D_, D_, n, kz)
        v = vz[:, None, None] * vy[None, :, None] * vx[None, None, :]
        lam = 1.0 + 2e-3 * (lx + ly + lz)
        np.testing.assert_allclose(cc.apply_A(op, v), lam * v, atol=1e-12 * lam)


def test_operator_variable_kappa_linear_field():
    """With u = x along x and kappa = kappa(x), the difference across every interior face is h, so
    face i+1/2 carries kappa_f h with kappa_f the mean of its two cells (reading G8), while the
    Neumann ghosts make the two boundary faces carry nothing. Then
    A u = alpha u - beta / h^2 (F_{i+1/2} - F_{i-1/2}) in closed form."""
    nx, ny = 12, 4
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    kap1 = 1.0 + 0.5 * np.sin(3.0 * x) + x * x
    kappa = np.tile(kap1, (ny, 1))
    u = np.tile(x, (ny, 1))
    alpha, beta = 0.3, 0.01
    op = cc.Operator((ny, nx), h, alpha, beta, kappa, (N_,) * 4)
    Au = cc.apply_A(op, u)
    kf = 0.5 * (kap1[:-1] + kap1[1:])  # interior faces i+1/2
    flux = np.concatenate([[0.0], kf * h, [0.0]])  # kappa_f (u_{i+1}-u_i); Neumann faces zero
    expect = alpha * x - beta / h ** 2 * (flux[1:] - flux[:-1])
    np.testing.assert_allclose(Au, np.tile(expect, (ny, 1)), rtol=1e-13, atol=1e-13)


def test_operator_symmetric_and_conservative():
    """The assembled matrix is symmetric for every boundary mix and a variable kappa, and with all
    Neumann faces the diffusive part sums to zero (no flux leaves the box)."""
    shape = (4, 8)
    h = 1.0 / 8
    kappa = 1.0 + random_field(shape, 11)
    for bc in [(N_,) * 4, (D_, N_, N_, D_), (D_,) * 4]:
        op = cc.Operator(shape, h, 0.5, 0.02, kappa, bc)
        M = cc.dense_matrix(op)
        np.testing.assert_allclose(M, M.T, atol=1e-12)
    op = cc.Operator(shape, h, 0.0, 1.0, kappa, (N_,) * 4)
    u = random_field(shape, 12)
    assert abs(np.sum(cc.apply_A(op, u))) < 1e-10


# ------------------------------------------------------------------------------------------
# the smoother
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("bc_kind", ["neumann", "dirichlet", "mixed", "periodic", "periodic_x"])
@pytest.mark.parametrize("var_kappa", [False, True])
def test_each_set_update_zeroes_its_residual(dim, bc_kind, var_kappa):
    """Defining property of a Gauss-Seidel update (Eqs. FCGS-1..4): right after a parity set is
    updated, the residual f - A u of the ghost-defined operator vanishes on that set. This pins the
    folded boundary handling (reading G2) to the ghost relations (reading G1)."""
    shape = (8, 8) if dim == 2 else (4, 8, 4)
    h = 1.0 / 8
    bc = {"neumann": (N_,) * (2 * dim), "dirichlet": (D_,) * (2 * dim),
          "mixed": (D_, N_, N_, D_, D_, N_)[: 2 * dim], "periodic": (P_,) * (2 * dim),
          "periodic_x": (P_, P_, D_, N_, N_, D_)[: 2 * dim]}[bc_kind]
    kappa = (0.5 + random_field(shape, 3)) if var_kappa else 1.7
    op = cc.Operator(shape, h, 0.9, 0.05, kappa, bc)
    u = random_field(shape, 4)
    f = random_field(shape, 5, -1.0, 1.0)
    coef = cc.smoother_coefficients(op)
    sets = cc.SETS_2D if dim == 2 else cc.SETS_3D
    for parities in sets:
        cc.xmcgs_sweep(op, u, f, coef, sets=[parities])
        _, cell = cc._set_slices(op, parities)
        r = cc.residual(op, u, f)
        scale = np.max(np.abs(f)) + np.max(np.abs(cc.apply_A(op, u)))
        assert np.max(np.abs(r[cell])) < 1e-13 * scale


def _rbgs_literal(op, u, f, colours=(1, 0)):
    """Point-by-point red-black Gauss-Seidel (Appendix A): all points with i+j(+l) odd, then all
    with i+j(+l) even (or the colours in the order given), each solved exactly for its own value
    with its neighbours' current values. Written independently of the oracle: scalar loops, ghost
    relation solved per point."""
    dim = op.dim
    h2 = op.h * op.h
    n = op.shape
    kap = np.broadcast_to(np.asarray(op.kappa, dtype=float), n)
    for colour in colours:
        for idx in np.ndindex(*n):
            ijl = [c + 1 for c in idx[::-1]]  # 1-based (i, j, l)
            if sum(ijl) % 2 != colour:
                continue
            diag = op.alpha * h2
            acc = h2 * f[idx]
            for ax in range(dim):
                lo, hi = op.axis_bc(ax)
                for s, kind in ((-1, lo), (+1, hi)):
                    nb = list(idx)
                    nb[ax] += s
                    if kind == P_:
                        nb[ax] %= n[ax]  # the wrapped neighbour
                    if 0 <= nb[ax] < n[ax]:
                        kf = 0.5 * (kap[idx] + kap[tuple(nb)])
                        diag += op.beta * kf
                        acc += op.beta * kf * u[tuple(nb)]
                    elif kind == D_:
                        diag += 2.0 * op.beta * kap[idx]
            u[idx] = acc / diag


@pytest.mark.parametrize("dim", [2, 3])
def test_xmcgs_equals_red_black_loop(dim):
    """X-MCGS with the paper's set order equals red-black Gauss-Seidel (odd colour first), since
    sets 1,2 (and 3,4; in 3D 1-4 and 5-8) never neighbour each other."""
    shape = (8, 8) if dim == 2 else (4, 4, 8)
    op = cc.Operator(shape, 1.0 / 8, 1.0, 0.1, 0.5 + random_field(shape, 7),
                     (D_, N_, N_, D_, N_, D_)[: 2 * dim])
    u0 = random_field(shape, 8)
    f = random_field(shape, 9, -1.0, 1.0)
    a = u0.copy()
    cc.smooth(op, a, f, 2)
    b = u0.copy()
    _rbgs_literal(op, b, f)
    _rbgs_literal(op, b, f)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)
    # the order of the colours matters: even-first gives a different iterate
    c = u0.copy()
    sets = cc.SETS_2D if dim == 2 else cc.SETS_3D
    half = len(sets) // 2
    cc.xmcgs_sweep(op, c, f, sets=sets[half:] + sets[:half])
    d = u0.copy()
    cc.xmcgs_sweep(op, d, f)
    assert np.max(np.abs(c - d)) > 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_xmcgs_equals_red_black_loop(dim):
    """Reading A17: on periodic axes the wrapped cells are ordinary neighbours; X-MCGS still equals
    the literal red-black loop (n even keeps the colouring consistent across the wrap)."""
    shape = (8, 8) if dim == 2 else (4, 4, 8)
    op = cc.Operator(shape, 1.0 / 8, 1.0, 0.1, 0.5 + random_field(shape, 27),
                     (P_, P_, D_, N_, P_, P_)[: 2 * dim])
    u0 = random_field(shape, 28)
    f = random_field(shape, 29, -1.0, 1.0)
    a = u0.copy()
    cc.smooth(op, a, f, 2)
    b = u0.copy()
    _rbgs_literal(op, b, f)
    _rbgs_literal(op, b, f)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_operator_fourier_eigenpairs(dim):
    """On an all-periodic grid with constant kappa, cos(2 pi k . x + phi) at the cell centres is an
    eigenvector of A with eigenvalue alpha + beta (4 kappa / h^2) sum_a sin^2(pi k_a h)."""
    n = 16
    h = 1.0 / n
    shape = (n,) * dim
    op = cc.Operator(shape, h, 0.7, 0.02, 1.3, (P_,) * (2 * dim))
    grids = np.meshgrid(*[(np.arange(n) + 0.5) * h] * dim, indexing="ij")  # numpy axis order
    for k in ((1, 0, 2), (3, 5, 1), (8, 2, 7)):
        k = k[:dim]
        phase = 2.0 * np.pi * sum(kk * g for kk, g in zip(k, grids)) + 0.3
        u = np.cos(phase)
        lam = op.alpha + op.beta * 4.0 * 1.3 / h ** 2 * sum(np.sin(np.pi * kk * h) ** 2 for kk in k)
        np.testing.assert_allclose(cc.apply_A(op, u), lam * u, rtol=0, atol=1e-11 * lam)


@pytest.mark.parametrize("alpha", [1.0, 0.0])
def test_periodic_solve_matches_fourier_solution(alpha):
    """The FAS solve on an all-periodic grid equals the exact solution by the discrete Fourier
    transform (alpha = 0: the singular problem, zero-mean right-hand side and solution, G7)."""
    n = 128
    h = 1.0 / n
    beta = 1e-3 if alpha else 1.0
    op = cc.Operator((n, n), h, alpha, beta, 1.0, (P_,) * 4)
    f = random_field((n, n), 31, -1.0, 1.0)
    if alpha == 0.0:
        f -= f.mean()
    lam1 = 4.0 / h ** 2 * np.sin(np.pi * np.arange(n) / n) ** 2
    lam = alpha + beta * (lam1[:, None] + lam1[None, :])
    fh = np.fft.fft2(f)
    if alpha == 0.0:
        lam[0, 0] = 1.0
        fh[0, 0] = 0.0
    ref = np.real(np.fft.ifft2(fh / lam))
    u = np.zeros((n, n))
    info = cc.solve(cc.build_levels(op, 4), u, f, cc.Params(tol=1e-13, kmax=60, coarsest=4, coarse_exact=True))
    assert info.converged
    assert np.max(np.abs(u - ref)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetric_ordering_equals_forward_backward_loops(dim):
    """The "1234-4321" ordering of Sec. 2.3 (a forward sweep, then the sets in reverse order) equals
    red-black Gauss-Seidel with the odd colour first, then with the even colour first; a third sweep
    is forward again."""
    shape = (8, 8) if dim == 2 else (4, 4, 8)
    op = cc.Operator(shape, 1.0 / 8, 1.0, 0.1, 0.5 + random_field(shape, 17),
                     (D_, N_, N_, D_, N_, D_)[: 2 * dim])
    u0 = random_field(shape, 18)
    f = random_field(shape, 19, -1.0, 1.0)
    a = u0.copy()
    cc.smooth(op, a, f, 3, ordering="1234-4321")
    b = u0.copy()
    for colours in ((1, 0), (0, 1), (1, 0)):
        _rbgs_literal(op, b, f, colours)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)
    # and it is not the forward ordering
    c = u0.copy()
    cc.smooth(op, c, f, 3)
    assert np.max(np.abs(a - c)) > 1e-6


def test_forward_ordering_converges_faster_than_symmetric():
    """Sec. 2.3 (smoother comparison figure): on the asymptotic test problem of Sec. 3.1.2 (exact
    solution substituted into the PDE, zero start, s = 2, res < 1e-9, coarsest 4^2) the X-shape with
    the 1234-1234 ordering needs the fewest V-cycles; the symmetric 1234-4321 ordering needs more.
    The paper prints the counts only in a figure, so only the order of the two is checked."""
    n = 256
    p, f = exact_and_source(n, 2)
    op = cc.Operator((n, n), 1.0 / n, 1.0, 1.0, 1.0, (D_,) * 4)
    cycles = {}
    for ordering in ("1234-1234", "1234-4321"):
        u = np.zeros((n, n))
        info = cc.solve(cc.build_levels(op, 4), u, f,
                        cc.Params(tol=1e-9, tol_mode="absolute", kmax=100, coarsest=4, ordering=ordering))
        assert info.converged
        cycles[ordering] = info.cycles
    assert cycles["1234-1234"] < cycles["1234-4321"]


def test_smoother_fixed_point_is_direct_solution():
    shape = (8, 16)
    op = cc.Operator(shape, 1.0 / 16, 1.0, 0.01, 1.0 + random_field(shape, 21), (D_, N_, D_, N_))
    f = random_field(shape, 22, -1, 1)
    u = np.zeros(shape)
    cc.smooth(op, u, f, 400)
    exact = np.linalg.solve(cc.dense_matrix(op), f.ravel()).reshape(shape)
    np.testing.assert_allclose(u, exact, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------
# transfers
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(8, 16), (4, 8, 8)])
def test_restriction_prolongation_identities(shape):
    """Appendix C: R averages 2^d children, P injects. Exact identities: R P y = y,
    <R x, y> 2^d = <x, P y>, constants preserved both ways."""
    d = len(shape)
    x = random_field(shape, 31, -1, 1)
    yc = random_field(tuple(n // 2 for n in shape), 32, -1, 1)
    np.testing.assert_allclose(cc.restrict(cc.prolong(yc)), yc, rtol=0, atol=1e-15)
    lhs = np.sum(cc.restrict(x) * yc) * 2 ** d
    rhs = np.sum(x * cc.prolong(yc))
    assert abs(lhs - rhs) < 1e-12
    np.testing.assert_array_equal(cc.restrict(np.full(shape, 3.25)), 3.25)
    np.testing.assert_array_equal(cc.prolong(np.full(yc.shape, -2.5)), -2.5)
    # children of coarse cell (0, 0[, 0]) are the 2^d cells with all 0-based indices in {0, 1}
    first = x[tuple(slice(0, 2) for _ in shape)]
    assert abs(cc.restrict(x)[(0,) * d] - first.mean()) < 1e-15


# ------------------------------------------------------------------------------------------
# the V-cycle and its converged result
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 8), (2, 16), (3, 8)])
@pytest.mark.parametrize("bc_kind", ["neumann", "dirichlet", "mixed"])
@pytest.mark.parametrize("var_kappa", [False, True])
def test_vcycle_converges_to_dense_solution(dim, n, bc_kind, var_kappa):
    shape = (n,) * dim
    bc = {"neumann": (N_,) * (2 * dim), "dirichlet": (D_,) * (2 * dim),
          "mixed": (D_, N_, N_, D_, N_, N_)[: 2 * dim]}[bc_kind]
    kappa = 1.0 + 0.5 * np.tanh(random_field(shape, 41, -2, 2)) if var_kappa else 1.0
    op = cc.Operator(shape, 1.0 / n, 1.0, 1e-2, kappa, bc)
    f = random_field(shape, 42, -1, 1)
    prm = cc.Params(tol=1e-14, kmax=60, coarsest=2)
    u = np.zeros(shape)
    info = cc.solve(cc.build_levels(op, 2), u, f, prm)
    exact = np.linalg.solve(cc.dense_matrix(op), f.ravel()).reshape(shape)
    assert np.max(np.abs(u - exact)) <= 1e-12 * np.max(np.abs(exact))
    assert info.converged


def test_vcycle_exact_coarsest_and_coarsest_sizes():
    shape = (16, 32)
    op = cc.Operator(shape, 1.0 / 32, 1.0, 0.05, 1.0, (N_,) * 4)
    f = random_field(shape, 51, -1, 1)
    exact = np.linalg.solve(cc.dense_matrix(op), f.ravel()).reshape(shape)
    for coarsest, exact_c in [(2, False), (4, False), (4, True), (8, True)]:
        prm = cc.Params(tol=1e-13, kmax=60, coarsest=coarsest, coarse_exact=exact_c)
        u = np.zeros(shape)
        cc.solve(cc.build_levels(op, coarsest), u, f, prm)
        np.testing.assert_allclose(u, exact, rtol=0, atol=1e-11 * np.max(np.abs(exact)))


@pytest.mark.parametrize("shape,coarsest,exact_c", [((2, 2), 2, True), ((4, 4), 2, False), ((2, 16), 2, True),
                                                    ((4, 256), 4, True), ((2, 2, 2), 2, True), ((4, 4, 4), 2, False),
                                                    ((2, 4, 8), 2, True)])
def test_smallest_and_thinnest_grids_match_dense_solution(shape, coarsest, exact_c):
    """One-level grids (the shortest axis already at the coarsest size) and two-level ones, with the
    mixed Dirichlet/Neumann faces of the GPU edge-case tests: the oracle's solve equals the dense
    solution of A u = f."""
    bc = (D_, N_, N_, D_, N_, D_)[: 2 * len(shape)]
    op = cc.Operator(shape, 1.0 / shape[-1], 1.0, 1e-2, 1.0, bc)
    f = random_field(shape, 281, -1, 1)
    u = np.zeros(shape)
    info = cc.solve(cc.build_levels(op, coarsest), u, f,
                    cc.Params(tol=1e-13, kmax=200, coarsest=coarsest, coarse_exact=exact_c))
    exact = np.linalg.solve(cc.dense_matrix(op), f.ravel()).reshape(shape)
    assert info.converged
    assert np.max(np.abs(u - exact)) <= 1e-12 * np.max(np.abs(exact))


def test_zero_rhs_keeps_zero_and_decays_a_guess():
    """f = 0: from u = 0 the solve stays at 0 exactly; from a random guess it converges to the unique
    solution 0 (alpha > 0), its residual 1e10 times below the initial one."""
    shape = (32, 32)
    op = cc.Operator(shape, 1.0 / 32, 1.0, 1e-3, 1.0, (N_,) * 4)
    zero = np.zeros(shape)
    u = np.zeros(shape)
    info = cc.solve(cc.build_levels(op, 4), u, zero, cc.Params(tol=1e-10, kmax=30, coarsest=4))
    assert info.converged and not np.any(u)
    u0 = random_field(shape, 271, -1, 1)
    u = u0.copy()
    info = cc.solve(cc.build_levels(op, 4), u, zero, cc.Params(tol=1e-10, kmax=30, coarsest=4))
    assert info.converged
    assert cc.norm2(cc.residual(op, u, zero)) <= 1e-10 * cc.norm2(cc.residual(op, u0, zero))


def test_singular_neumann_poisson_matches_cosine_transform():
    """Reading G7: alpha = 0 with all-Neumann faces; mean-zero solution of -beta Lap u = f - mean f.
    The cosine transform (DCT-II) diagonalises the operator with eigenvalues beta (lam_x + lam_y)."""
    scipy_fft = pytest.importorskip("scipy.fft")
    n = 32
    shape = (n, n)
    op = cc.Operator(shape, 1.0 / n, 0.0, 1.0, 1.0, (N_,) * 4)
    f = random_field(shape, 61, -1, 1)
    prm = cc.Params(tol=1e-12, kmax=200, coarsest=4, coarse_exact=True)
    u = np.zeros(shape)
    info = cc.solve(cc.build_levels(op, 4), u, f, prm)
    assert info.converged
    h = 1.0 / n
    lam1 = 4.0 / h ** 2 * np.sin(np.arange(n) * np.pi * h / 2) ** 2
    lam = lam1[:, None] + lam1[None, :]
    F = scipy_fft.dctn(f - f.mean(), type=2, norm="ortho")
    lam[0, 0] = 1.0
    U = F / lam
    U[0, 0] = 0.0
    ref = scipy_fft.idctn(U, type=2, norm="ortho")
    np.testing.assert_allclose(u, ref, atol=1e-10 * np.max(np.abs(ref)))
    assert abs(u.mean()) < 1e-14


def test_heat_solve_matches_cosine_transform_large():
    """Converged heat/Helmholtz solve at 256^2 (Neumann, kappa 1) against the exact DCT solve."""
    scipy_fft = pytest.importorskip("scipy.fft")
    n = 256
    shape = (n, n)
    dt = 1e-3
    op = cc.heat_operator(shape, 1.0 / n, dt)
    f = random_field(shape, 71, -1, 1)
    prm = cc.Params(tol=1e-12, kmax=40, coarsest=4)
    u = np.zeros(shape)
    cc.solve(cc.build_levels(op, 4), u, f, prm)
    h = 1.0 / n
    lam1 = 4.0 / h ** 2 * np.sin(np.arange(n) * np.pi * h / 2) ** 2
    lam = 1.0 + dt * (lam1[:, None] + lam1[None, :])
    ref = scipy_fft.idctn(scipy_fft.dctn(f, type=2, norm="ortho") / lam, type=2, norm="ortho")
    np.testing.assert_allclose(u, ref, atol=1e-11 * np.max(np.abs(ref)))


def test_dirichlet_values_folded_into_rhs():
    """Reading G10: with every face Dirichlet of the same value g and f = alpha g, the constant field
    g solves the problem (each ghost 2g - g = g carries no flux)."""
    shape = (16, 16)
    g = 0.75
    op = cc.Operator(shape, 1.0 / 16, 0.4, 0.02, 1.0 + random_field(shape, 81), (D_,) * 4)
    f = cc.fold_dirichlet_rhs(op, np.full(shape, 0.4 * g), [g] * 4)
    u = np.zeros(shape)
    cc.solve(cc.build_levels(op, 2), u, f, cc.Params(tol=1e-14, kmax=80, coarsest=2))
    np.testing.assert_allclose(u, g, rtol=1e-12)


def test_heat_eigenmode_decay_closed_form():
    """Backward Euler on u0 = cos(pi x) cos(pi y) (an exact Neumann eigenvector): after n steps
    u^n = (1 + dt lam)^(-n) u0 with lam = 2 (4/h^2) sin^2(pi h / 2)."""
    n = 64
    shape = (n, n)
    h, dt, steps = 1.0 / n, 1e-3, 10
    x = (np.arange(n) + 0.5) * h
    u0 = np.cos(np.pi * x)[:, None] * np.cos(np.pi * x)[None, :]
    op = cc.heat_operator(shape, h, dt)
    u, infos = cc.heat_run(op, u0, None, dt, steps, cc.Params(tol=1e-13, kmax=40, coarsest=4))
    lam = 2 * 4.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    np.testing.assert_allclose(u, (1 + dt * lam) ** (-steps) * u0, atol=1e-12)
    assert all(i.converged for i in infos)


def test_paper_error_table_2d_and_order():
    """Table err_2D (Sec. 3.1.2): error 2.58e-6 at 1024^2 (all faces homogeneous Dirichlet, reading
    G1), and second order between smaller grids."""
    gold = json.load(open(GOLDEN))
    errs = {}
    for n in (256, 512, 1024):
        p, f = exact_and_source(n, 2)
        op = cc.Operator((n, n), 1.0 / n, 1.0, 1.0, 1.0, (D_,) * 4)
        prm = cc.Params(tol=1e-9, tol_mode="absolute", kmax=20, coarsest=2)
        u = np.zeros((n, n))
        info = cc.solve(cc.build_levels(op, 2), u, f, prm)
        assert info.converged
        errs[n] = l2_error(u, p, n, 2)
    assert float("%.3g" % errs[1024]) == gold["err_2d"]["1024"]
    for a, b in ((256, 512), (512, 1024)):
        assert abs(math.log2(errs[a] / errs[b]) - 2.0) < 0.02


def test_paper_error_table_3d():
    """Table err_3D (Sec. 3.1.2): 1.74e-3 at 32^3 and 4.33e-4 at 64^3, order 2.01."""
    gold = json.load(open(GOLDEN))
    errs = {}
    for n in (32, 64):
        p, f = exact_and_source(n, 3)
        op = cc.Operator((n,) * 3, 1.0 / n, 1.0, 1.0, 1.0, (D_,) * 6)
        prm = cc.Params(tol=1e-9, tol_mode="absolute", kmax=20, coarsest=2)
        u = np.zeros((n,) * 3)
        info = cc.solve(cc.build_levels(op, 2), u, f, prm)
        assert info.converged
        errs[n] = l2_error(u, p, n, 3)
        assert float("%.3g" % errs[n]) == gold["err_3d"][str(n)]
    assert abs(math.log2(errs[32] / errs[64]) - gold["order_3d"]["64"]) < 0.01


def test_vcycle_contraction_nearly_h_independent():
    """Sec. 3.1.1: residual decay at nearly the same rate on every grid (f = L_h p_exact, random
    [0,1] start). The absolute rate is not printed (figure only), so only its spread is checked."""
    rhos = []
    for n in (32, 64, 128, 256):
        p, _ = exact_and_source(n, 2)
        op = cc.Operator((n, n), 1.0 / n, 1.0, 1.0, 1.0, (D_,) * 4)
        f = cc.apply_A(op, p)
        u = random_field((n, n), 91)
        info = cc.solve(cc.build_levels(op, 2), u, f, cc.Params(tol=1e-300, kmax=6, coarsest=2))
        rhos.append(info.rho)
    assert max(rhos) < 0.2
    assert max(rhos) - min(rhos) < 0.06


def test_mixed_precision_matches_fp64_solution():
    n = 128
    shape = (n, n)
    op = cc.heat_operator(shape, 1.0 / n, 1e-3)
    levels = cc.build_levels(op, 4)
    f = random_field(shape, 101, -1, 1)
    prm = cc.Params(tol=1e-10, kmax=40, coarsest=4)
    u64 = np.zeros(shape)
    cc.solve(levels, u64, f, cc.Params(tol=1e-14, kmax=40, coarsest=4))
    um = np.zeros(shape)
    info = cc.solve_mixed(levels, cc.as_float32(levels), um, f, prm)
    assert info.converged and info.rel <= 1e-10
    assert np.max(np.abs(um - u64)) <= 1e-10 * np.max(np.abs(u64))
