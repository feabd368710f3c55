"""FP64 oracle of the cell-centred matrix-free FAS multigrid (test infrastructure only).

Follows the paper section by section:
  * grid and ghost layer ............ Sec. 2.1 (cell centres x_i = (i - 1/2) h, one ghost layer)
  * discrete operator L_h ........... Sec. 2.2, Eq. PDE_discret with the ghost relations of
                                      Eqs. boundry1-2, generalised to A u = alpha u - beta div(kappa grad u)
  * residual and its L2 norm ........ Sec. 2.2, Eq. residual
  * FAS two-grid solver ............. Algorithm 1 (TMGSolver), with the recursion of the remark that
                                      follows it (coarse steps replaced by a recursive call)
  * X-MCGS smoother ................. Sec. 2.3, Eqs. FCGS-1..FCGS-4 (2D, four parity sets in order
                                      1,2,3,4); Appendix B (3D, eight parity sets in order 1..8);
                                      the symmetric "1234-4321" ordering of the smoother comparison
                                      in Sec. 2.3 (forward and backward sweeps alternating)
  * restriction / prolongation ...... Appendix C (four-point average, piecewise-constant injection;
                                      3D analogues with eight children)
  * heat stepping ................... Sec. 1 (backward Euler, new step overwrites the old)

Readings where the paper is silent, garbled or self-contradictory:
  G1  Boundary ghosts: homogeneous Dirichlet is ghost = -adjacent cell (Eq. boundry1, first half);
      homogeneous Neumann is ghost = adjacent cell (Eq. boundry1, second half). Each face of the
      box carries one of the two kinds, chosen by the caller.
  G2  The smoother folds the ghost relation into the point equation: the Gauss-Seidel update solves
      the point's equation exactly with its ghost tied to it (Neumann drops the face, Dirichlet
      doubles the face's diagonal share). Listing-free reading of Eqs. FCGS-1..4 at boundary cells.
  G3  Every cell is updated once per sweep (the 3D set ranges 2:2:M_1-1 read as 2:2:M_1).
  G4b The "1234-4321" ordering (Sec. 2.3): within a smoothing step of s sweeps the odd-numbered
      sweeps visit the sets forward and the even-numbered ones backward, on every level.
  G5  Stopping test relative to ||f||_2 by default; the paper's absolute h-weighted norm on request.
  G6  Coarsest level: the paper's s smoothing sweeps by default, a dense direct solve on request.
  G7  Singular all-Neumann problems (alpha = 0): the right-hand side is projected to zero mean and
      the mean of the iterate removed after each cycle; the dense coarsest solve is least-squares.
  G8  Variable diffusivity: face kappa is the mean of the two cells; a boundary face takes its
      cell's kappa; coarse levels use the four- (eight-) cell average of kappa.
  A17 Periodic axes (for the grain-growth example of Sec. 3.3.1): the grid wraps around; the face
      between the last and the first cell is an interior face (mean kappa), every cell has all its
      neighbours, and with n even the red-black colouring stays consistent across the wrap.
  G10 Inhomogeneous Dirichlet values are moved into the right-hand side once (fold_dirichlet_rhs);
      the solver's operator is linear on every level.

Array convention: numpy shape (ny, nx) or (nz, ny, nx), x fastest; the paper's index i runs along x,
j along y, l along z. Boundary-condition kinds are given per physical face in the order
(x_lo, x_hi, y_lo, y_hi[, z_lo, z_hi]).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

NEUMANN = 0
DIRICHLET = 1
PERIODIC = 2  # both faces of an axis: the grid wraps around (reading A17)


@dataclass
class Operator:
    """A u = alpha u - beta div_h(kappa grad_h u) on a uniform cell-centred grid of spacing h."""

    shape: tuple
    h: float
    alpha: float = 1.0
    beta: float = 1.0
    kappa: object = 1.0  # scalar or a cell field of `shape`
    bc: tuple = None  # kinds per physical face (x_lo, x_hi, y_lo, y_hi[, z_lo, z_hi])
    dtype: object = np.float64

    def __post_init__(self):
        self.shape = tuple(int(n) for n in self.shape)
        if self.bc is None:
            self.bc = (NEUMANN,) * (2 * len(self.shape))
        self.bc = tuple(int(b) for b in self.bc)
        assert len(self.bc) == 2 * self.dim
        for a in range(self.dim):
            if PERIODIC in self.bc[2 * a:2 * a + 2]:
                assert self.bc[2 * a] == self.bc[2 * a + 1] == PERIODIC, "periodic faces come in pairs"

    @property
    def dim(self):
        return len(self.shape)

    def axis_bc(self, ax):
        """(lo, hi) kinds of numpy axis `ax` (numpy axis ax is physical axis dim-1-ax)."""
        a = self.dim - 1 - ax
        return self.bc[2 * a], self.bc[2 * a + 1]

    @property
    def singular(self):
        return self.alpha == 0.0 and all(b != DIRICHLET for b in self.bc)


@dataclass
class Params:
    """User parameters of Algorithm 1 (s, kMax, tol) plus the readings' switches."""

    nu1: int = 2
    nu2: int = 2
    nu_coarse: int = None  # sweeps on the coarsest level; the paper uses s (= nu1)
    kmax: int = 20
    tol: float = 1e-10
    tol_mode: str = "relative"  # or "absolute" (paper's h-weighted norm, Eq. residual)
    coarsest: int = 4  # cells along the shortest axis of the coarsest level
    coarse_exact: bool = False
    ordering: str = "1234-1234"  # or "1234-4321": each smoothing step alternates forward/backward sweeps

    def sweeps_coarse(self):
        return self.nu1 if self.nu_coarse is None else self.nu_coarse


# ---------------------------------------------------------------------------------------------
# diffusivity on faces (reading G8)
# ---------------------------------------------------------------------------------------------

def _take(a, idx, ax):
    sl = [slice(None)] * a.ndim
    sl[ax] = idx
    return a[tuple(sl)]


def face_kappa(op: Operator, ax: int) -> np.ndarray:
    """kappa on the n+1 faces normal to numpy axis `ax`: interior faces take the mean of their two
    cells, the two boundary faces take the kappa of their cell; on a periodic axis the two boundary
    faces are one face, between the last and the first cell, and take their mean."""
    shape = list(op.shape)
    if np.isscalar(op.kappa):
        shape[ax] += 1
        return np.full(shape, op.kappa, dtype=op.dtype)
    k = np.asarray(op.kappa, dtype=op.dtype)
    inner = 0.5 * (_take(k, slice(0, -1), ax) + _take(k, slice(1, None), ax))
    lo = _take(k, slice(0, 1), ax)
    hi = _take(k, slice(-1, None), ax)
    if op.axis_bc(ax)[0] == PERIODIC:
        lo = hi = 0.5 * (hi + lo)
    return np.concatenate([lo, inner, hi], axis=ax)


# ---------------------------------------------------------------------------------------------
# the operator and the residual (Sec. 2.2)
# ---------------------------------------------------------------------------------------------

def apply_A(op: Operator, u: np.ndarray) -> np.ndarray:
    """A u with the ghost layer of Sec. 2.1 filled from the boundary relations (reading G1):
    Neumann ghost = adjacent cell, Dirichlet ghost = -adjacent cell. Fluxes kappa_f (u_R - u_L)
    live on faces; (A u)_c = alpha u_c - beta / h^2 * (sum of outgoing flux differences)."""
    u = np.asarray(u, dtype=op.dtype)
    out = op.alpha * u
    scale = op.beta / (op.h * op.h)
    for ax in range(op.dim):
        lo_kind, hi_kind = op.axis_bc(ax)
        first = _take(u, slice(0, 1), ax)
        last = _take(u, slice(-1, None), ax)
        if lo_kind == PERIODIC:  # the neighbours across the boundary are the wrapped cells
            ghost_lo, ghost_hi = last, first
        else:
            ghost_lo = first if lo_kind == NEUMANN else -first
            ghost_hi = last if hi_kind == NEUMANN else -last
        ext = np.concatenate([ghost_lo, u, ghost_hi], axis=ax)
        flux = face_kappa(op, ax) * np.diff(ext, axis=ax)
        out = out - scale * np.diff(flux, axis=ax)
    return out


def residual(op: Operator, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Point-wise residual r = f - L_h(u) (Sec. 2.2)."""
    return np.asarray(f, dtype=op.dtype) - apply_A(op, u)


def norm2(r: np.ndarray) -> float:
    return float(np.sqrt(np.sum(np.asarray(r, dtype=np.float64) ** 2)))


def paper_res(op: Operator, r: np.ndarray) -> float:
    """res = ||r||_{L2(Omega)} = h^{d/2} (sum r^2)^{1/2} (Eq. residual, written for 2D as h (...))."""
    return op.h ** (op.dim / 2.0) * norm2(r)


def fold_dirichlet_rhs(op: Operator, f: np.ndarray, values) -> np.ndarray:
    """Reading G10: with ghost = 2 g - u on a Dirichlet face of value g, the constant part
    2 beta kappa_f g / h^2 of the boundary cell's equation moves to the right-hand side.
    `values` lists g per physical face (ignored on Neumann faces)."""
    f = np.array(f, dtype=op.dtype, copy=True)
    scale = 2.0 * op.beta / (op.h * op.h)
    for ax in range(op.dim):
        a = op.dim - 1 - ax
        kf = face_kappa(op, ax)
        for side, idx, fidx in ((0, 0, 0), (1, -1, -1)):
            if op.bc[2 * a + side] != DIRICHLET:
                continue
            g = values[2 * a + side]
            sl = [slice(None)] * op.dim
            sl[ax] = idx
            fsl = [slice(None)] * op.dim
            fsl[ax] = fidx
            f[tuple(sl)] += scale * kf[tuple(fsl)] * g
    return f


# ---------------------------------------------------------------------------------------------
# X-MCGS smoother (Sec. 2.3 and Appendix B)
# ---------------------------------------------------------------------------------------------

# Parity sets as (parity of i, parity of j[, parity of l]) with 1 = odd, 0 = even, in update order.
SETS_2D = ((1, 0), (0, 1), (0, 0), (1, 1))  # Eqs. FCGS-1..FCGS-4
SETS_3D = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1),  # Appendix B, sets 1-4 (i+j+l odd)
           (1, 0, 1), (0, 1, 1), (0, 0, 0), (1, 1, 0))  # sets 5-8 (i+j+l even)


@dataclass
class SmootherCoefficients:
    """Folded point equation (reading G2): for cell c,
         D_c u_c = h^2 f_c + beta * sum over interior faces of kappa_f u_nb,
       D_c = alpha h^2 + beta * sum_f d_f with d_f = kappa_f (interior face), 0 (Neumann face),
       2 kappa_f (Dirichlet face). weights[(ax, s)] is kappa_f towards neighbour s = -1/+1 along
       numpy axis ax, zero across a boundary face."""

    D: np.ndarray
    weights: dict = field(default_factory=dict)


def smoother_coefficients(op: Operator) -> SmootherCoefficients:
    D = np.full(op.shape, op.alpha * op.h * op.h, dtype=op.dtype)
    weights = {}
    for ax in range(op.dim):
        kf = face_kappa(op, ax)
        n = op.shape[ax]
        lo_kind, hi_kind = op.axis_bc(ax)
        k_lo = _take(kf, slice(0, n), ax).copy()  # face below each cell
        k_hi = _take(kf, slice(1, n + 1), ax).copy()  # face above each cell
        w_lo = k_lo.copy()
        w_hi = k_hi.copy()
        d_lo = k_lo.copy()
        d_hi = k_hi.copy()
        # boundary faces carry no neighbour; their diagonal share follows the ghost relation
        # (a periodic boundary face is an interior face whose neighbour is the wrapped cell)
        sl0 = [slice(None)] * op.dim
        sl0[ax] = 0
        sl1 = [slice(None)] * op.dim
        sl1[ax] = n - 1
        if lo_kind != PERIODIC:
            w_lo[tuple(sl0)] = 0.0
            w_hi[tuple(sl1)] = 0.0
            d_lo[tuple(sl0)] = 0.0 if lo_kind == NEUMANN else 2.0 * k_lo[tuple(sl0)]
            d_hi[tuple(sl1)] = 0.0 if hi_kind == NEUMANN else 2.0 * k_hi[tuple(sl1)]
        D = D + op.beta * (d_lo + d_hi)
        weights[(ax, -1)] = w_lo
        weights[(ax, +1)] = w_hi
    return SmootherCoefficients(D=D, weights=weights)


def _set_slices(op: Operator, parities):
    """Slices of the cells of one parity set, in numpy axis order. parities are given for
    (i, j[, l]) = (x, y[, z]); odd 1-based index means even 0-based index."""
    offs = [0 if p == 1 else 1 for p in parities]  # physical order x, y, z
    offs = offs[::-1]  # numpy order
    cell = tuple(slice(o, n, 2) for o, n in zip(offs, op.shape))
    return offs, cell


def _wrap_ghosts(pad: np.ndarray, ax: int, n: int) -> None:
    """Copy the first and last interior slabs of `pad` along axis `ax` into the opposite ghosts."""
    dst = [slice(None)] * pad.ndim
    src = [slice(None)] * pad.ndim
    dst[ax], src[ax] = 0, n
    pad[tuple(dst)] = pad[tuple(src)]
    dst[ax], src[ax] = n + 1, 1
    pad[tuple(dst)] = pad[tuple(src)]


def xmcgs_sweep(op: Operator, u: np.ndarray, f: np.ndarray,
                coef: SmootherCoefficients | None = None, sets=None) -> None:
    """One X-MCGS sweep in place: the parity sets updated one after another in the paper's order,
    every point of a set from the current values of its neighbours (Eqs. FCGS-1..4; for
    alpha = beta = kappa = 1 an interior update is (sum of 4 neighbours + h^2 f) / (4 + h^2))."""
    if coef is None:
        coef = smoother_coefficients(op)
    if sets is None:
        sets = SETS_2D if op.dim == 2 else SETS_3D
    h2 = op.h * op.h
    f = np.asarray(f, dtype=op.dtype)
    pad = np.zeros(tuple(n + 2 for n in op.shape), dtype=op.dtype)
    inner = tuple(slice(1, n + 1) for n in op.shape)
    pad[inner] = u
    periodic = [ax for ax in range(op.dim) if op.axis_bc(ax)[0] == PERIODIC]
    for parities in sets:
        for ax in periodic:  # ghost layers hold the current values of the wrapped cells
            _wrap_ghosts(pad, ax, op.shape[ax])
        offs, cell = _set_slices(op, parities)
        nbsum = np.zeros(pad[tuple(slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape))].shape,
                         dtype=op.dtype)
        for ax in range(op.dim):
            for s in (-1, +1):
                sl = [slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape)]
                sl[ax] = slice(offs[ax] + 1 + s, op.shape[ax] + 1 + s, 2)
                nbsum = nbsum + coef.weights[(ax, s)][cell] * pad[tuple(sl)]
        target = tuple(slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape))
        pad[target] = (h2 * f[cell] + op.beta * nbsum) / coef.D[cell]
    u[...] = pad[inner]


def smooth(op: Operator, u: np.ndarray, f: np.ndarray, sweeps: int,
           coef: SmootherCoefficients | None = None, ordering: str = "1234-1234") -> None:
    """S applied `sweeps` times (the inner loops m = 1..s of Algorithm 1). ordering "1234-1234":
    every sweep visits the sets in the paper's order; "1234-4321" (Sec. 2.3, the symmetric variant
    compared with it): the second, fourth, ... sweep visits them in reverse order."""
    if ordering not in ("1234-1234", "1234-4321"):
        raise ValueError("ordering must be '1234-1234' or '1234-4321'")
    if coef is None:
        coef = smoother_coefficients(op)
    forward = SETS_2D if op.dim == 2 else SETS_3D
    for m in range(sweeps):
        backward = ordering == "1234-4321" and m % 2 == 1
        xmcgs_sweep(op, u, f, coef, sets=forward[::-1] if backward else forward)


# ---------------------------------------------------------------------------------------------
# transfers (Appendix C)
# ---------------------------------------------------------------------------------------------

def restrict(u: np.ndarray) -> np.ndarray:
    """R: each coarse cell is the average of its 2^d children (four-point average in 2D)."""
    d = u.ndim
    acc = None
    for corner in np.ndindex(*(2,) * d):
        child = u[tuple(slice(c, None, 2) for c in corner)]
        acc = child.copy() if acc is None else acc + child
    return acc / (2 ** d)


def prolong(uc: np.ndarray) -> np.ndarray:
    """P: piecewise-constant injection, every child takes its parent's value."""
    out = uc
    for ax in range(uc.ndim):
        out = np.repeat(out, 2, axis=ax)
    return out


# ---------------------------------------------------------------------------------------------
# level hierarchy and the FAS V-cycle (Algorithm 1 + recursion remark)
# ---------------------------------------------------------------------------------------------

def coarsen(op: Operator) -> Operator:
    """Operator of the next coarser grid: half the cells per axis, h0 = 2 h1 (Sec. 2.1); same
    alpha, beta and boundary kinds; kappa averaged over children (reading G8)."""
    kappa = op.kappa if np.isscalar(op.kappa) else restrict(np.asarray(op.kappa, dtype=op.dtype))
    return replace(op, shape=tuple(n // 2 for n in op.shape), h=2.0 * op.h, kappa=kappa)


def build_levels(op: Operator, coarsest: int = 4) -> list:
    """Finest first; coarsen while the shortest axis is longer than `coarsest`."""
    if any(n % 2 or n < 1 for n in op.shape) and min(op.shape) > coarsest:
        raise ValueError("grid sizes must be powers of two")
    levels = [op]
    while min(levels[-1].shape) > coarsest:
        levels.append(coarsen(levels[-1]))
    return levels


def dense_matrix(op: Operator) -> np.ndarray:
    """Matrix of A assembled by applying A to unit vectors (only for the tiny coarsest level)."""
    n = int(np.prod(op.shape))
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = apply_A(replace(op, dtype=np.float64), e.reshape(op.shape)).ravel()
    return M


def coarsest_solve(op: Operator, u: np.ndarray, f: np.ndarray, params: Params) -> None:
    """Coarsest level (reading G6): s X-MCGS sweeps (the paper's remark replacing the direct
    solve), or an exact dense solve (least-squares / minimum norm when singular, reading G7)."""
    if not params.coarse_exact:
        smooth(op, u, f, params.sweeps_coarse(), ordering=params.ordering)
        return
    M = dense_matrix(op)
    rhs = np.asarray(f, dtype=np.float64).ravel()
    if op.singular:
        sol = np.linalg.lstsq(M, rhs - rhs.mean(), rcond=None)[0]
    else:
        sol = np.linalg.solve(M, rhs)
    u[...] = sol.reshape(op.shape).astype(op.dtype)


def vcycle(levels: list, u: np.ndarray, f: np.ndarray, params: Params, level: int = 0) -> None:
    """One FAS V-cycle in place on `u` (Algorithm 1, one pass of its k loop, with the coarse-grid
    steps replaced by a recursive call as in the remark after Algorithm 1)."""
    op = levels[level]
    if level == len(levels) - 1:
        coarsest_solve(op, u, f, params)
        return
    coef = smoother_coefficients(op)
    smooth(op, u, f, params.nu1, coef, params.ordering)  # fine-grid pre-smoothing
    r1 = residual(op, u, f)  # fine-grid point-wise residual
    u0 = restrict(u)  # coarse-grid approximation p0 = R(p1)
    r0 = restrict(r1)  # r0 = R(r1)
    u0_start = u0.copy()
    f0 = r0 + apply_A(levels[level + 1], u0)  # coarse source term (tau correction)
    vcycle(levels, u0, f0, params, level + 1)  # coarse problem, recursively
    c0 = u0 - u0_start  # coarse-grid correction
    u += prolong(c0)  # fine-grid correction
    smooth(op, u, f, params.nu2, coef, params.ordering)  # fine-grid post-smoothing


@dataclass
class SolveInfo:
    cycles: int = 0
    res0: float = 0.0
    res: float = 0.0
    rel: float = 0.0
    converged: bool = False
    history: list = field(default_factory=list)

    @property
    def rho(self):
        """Mean contraction factor (res_k / res_0)^(1/k)."""
        if self.cycles == 0 or self.res0 == 0.0:
            return 0.0
        return (self.res / self.res0) ** (1.0 / self.cycles)


def _stop_value(op: Operator, r: np.ndarray, params: Params) -> float:
    return paper_res(op, r) if params.tol_mode == "absolute" else norm2(r)


def solve(levels: list, u: np.ndarray, f: np.ndarray, params: Params) -> SolveInfo:
    """Algorithm 1's outer loop: V-cycles k = 1..kMax, each followed by the residual test
    (reading G5: relative to ||f||_2 unless the paper's absolute mode is chosen)."""
    op = levels[0]
    f = np.asarray(f, dtype=op.dtype)
    if op.singular:
        f = f - f.mean()
    info = SolveInfo()
    r = residual(op, u, f)
    info.res0 = _stop_value(op, r, params)
    info.history.append(info.res0)
    if params.tol_mode == "absolute":
        ref = 1.0
    else:
        fn = norm2(f)
        ref = fn if fn > 0.0 else info.res0
    for _ in range(params.kmax):
        vcycle(levels, u, f, params)
        if op.singular:
            u -= u.mean()
        info.cycles += 1
        r = residual(op, u, f)
        info.res = _stop_value(op, r, params)
        info.history.append(info.res)
        info.rel = info.res / ref if ref > 0 else 0.0
        if info.res <= params.tol * ref:
            info.converged = True
            break
    return info


def solve_mixed(levels64: list, levels32: list, u: np.ndarray, f: np.ndarray,
                params: Params, inner_cycles: int = 1) -> SolveInfo:
    """Mixed-precision iterative refinement (not in the paper): the residual r = f - A u and the
    update u += e in float64, the correction e from `inner_cycles` float32 V-cycles on A e = r
    started from e = 0 (all smoothing, transfers and coarse levels in float32)."""
    op = levels64[0]
    f = np.asarray(f, dtype=np.float64)
    info = SolveInfo()
    r = residual(op, u, f)
    info.res0 = norm2(r)
    info.history.append(info.res0)
    fn = norm2(f)
    ref = fn if fn > 0.0 else info.res0
    for _ in range(params.kmax):
        r32 = r.astype(np.float32)
        e = np.zeros(op.shape, dtype=np.float32)
        for _ in range(inner_cycles):
            vcycle(levels32, e, r32, params)
        u += e.astype(np.float64)
        info.cycles += 1
        r = residual(op, u, f)
        info.res = norm2(r)
        info.history.append(info.res)
        info.rel = info.res / ref if ref > 0 else 0.0
        if info.res <= params.tol * ref:
            info.converged = True
            break
    return info


def as_float32(levels: list) -> list:
    return [replace(op, dtype=np.float32,
                    kappa=op.kappa if np.isscalar(op.kappa)
                    else np.asarray(op.kappa, dtype=np.float32)) for op in levels]


# ---------------------------------------------------------------------------------------------
# backward-Euler heat stepping
# ---------------------------------------------------------------------------------------------

def heat_operator(shape, h, dt, kappa=1.0, bc=None) -> Operator:
    """(I - dt div(kappa grad)) u^{n+1} = u^n + dt f: alpha = 1, beta = dt."""
    return Operator(shape=shape, h=h, alpha=1.0, beta=dt, kappa=kappa, bc=bc)


def heat_run(op: Operator, u0: np.ndarray, fsrc, dt: float, nsteps: int, params: Params,
             mixed: bool = False):
    """Backward-Euler steps; each solve starts from u^n and overwrites it with u^{n+1}."""
    levels = build_levels(op, params.coarsest)
    levels32 = as_float32(levels) if mixed else None
    u = np.array(u0, dtype=np.float64, copy=True)
    infos = []
    for _ in range(nsteps):
        b = u.copy() if fsrc is None else u + dt * np.asarray(fsrc, dtype=np.float64)
        if mixed:
            infos.append(solve_mixed(levels, levels32, u, b, params))
        else:
            infos.append(solve(levels, u, b, params))
    return u, infos


# ---------------------------------------------------------------------------------------------
# adjoint of backward-Euler heat stepping (not in the paper)
# ---------------------------------------------------------------------------------------------

def kappa_gradient(op: Operator, u: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """-(d(mu^T A u) / d kappa) per cell for A u = alpha u - beta div(kappa grad u) with face kappa
    the mean of its two cells (reading G8): an interior face between cells c and nb contributes
    -(beta/h^2) (u_nb - u_c)(mu_nb - mu_c), half to each cell; a Dirichlet face (ghost -u_c, face
    kappa = kappa_c) contributes -(2 beta/h^2) mu_c u_c to its cell; Neumann faces carry no flux."""
    g = np.zeros(op.shape)
    scale = op.beta / (op.h * op.h)
    for ax in range(op.dim):
        n = op.shape[ax]
        du = np.diff(u, axis=ax)
        dmu = np.diff(mu, axis=ax)
        face = -scale * du * dmu  # dL/d kappa_f of each interior face
        lo = [slice(None)] * op.dim
        lo[ax] = slice(0, n - 1)
        hi = [slice(None)] * op.dim
        hi[ax] = slice(1, n)
        g[tuple(lo)] += 0.5 * face
        g[tuple(hi)] += 0.5 * face
        lo_kind, hi_kind = op.axis_bc(ax)
        for kind, idx in ((lo_kind, 0), (hi_kind, n - 1)):
            if kind == DIRICHLET:
                sl = [slice(None)] * op.dim
                sl[ax] = idx
                g[tuple(sl)] -= 2.0 * scale * mu[tuple(sl)] * u[tuple(sl)]
    return g


def adjoint_heat(op: Operator, u0: np.ndarray, fsrc, dt: float, nsteps: int, dL_duT: np.ndarray,
                 params: Params):
    """Gradients of a loss L(u^N) of the backward-Euler run (A u^{n+1} = u^n + dt f, A symmetric)
    with respect to u^0, f and kappa, given dL/du^N:
        lambda^N = dL/du^N;  for n = N-1..0:  mu = A^{-1} lambda^{n+1},
        dL/df += dt mu,  dL/dkappa += kappa_gradient(u^{n+1}, mu),  lambda^n = mu;
        dL/du^0 = lambda^0.
    Every state of the forward run is kept (no checkpointing: small problems only)."""
    levels = build_levels(op, params.coarsest)
    f = np.zeros(op.shape) if fsrc is None else np.asarray(fsrc, dtype=np.float64)
    states = [np.array(u0, dtype=np.float64, copy=True)]
    u = states[0].copy()
    for _ in range(nsteps):
        b = u + dt * f
        solve(levels, u, b, params)
        states.append(u.copy())
    lam = np.array(dL_duT, dtype=np.float64, copy=True)
    g_f = np.zeros(op.shape)
    g_k = np.zeros(op.shape)
    for n in range(nsteps - 1, -1, -1):
        mu = lam.copy()  # initial guess
        solve(levels, mu, lam, params)
        g_f += dt * mu
        g_k += kappa_gradient(op, states[n + 1], mu)
        lam = mu
    return states[-1], lam, g_f, g_k
