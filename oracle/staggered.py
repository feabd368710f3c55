"""FP64 oracle of the staggered (MAC) grid parts (test infrastructure only).

Follows the paper:
  * face-centred unknowns and their boundary treatment ... Sec. 4.1 (u on east-west faces, v on
    north-south faces, w on bottom-top faces; boundary faces held fixed, tangential walls by ghosts)
  * X-MCGS on face grids ................................ Sec. 4.1 (sets by the parity of the face
    index and the cell indices, updated as in Eqs. FCGS-1..4)
  * face restriction / prolongation ..................... Appendix D (reading G9 below)
  * first-order projection scheme ....................... Sec. 4.2, Scheme first-1..4, in the
    memory-efficient order of the 8-field table (u^{n+1} into U_old, tilde-u in U_new, ...)
  * convection by third-order WENO ...................... Sec. 4.2 (reading G11 below)

Storage of a face field of component a (physical axis a; numpy axis dim-1-a): the array has the
cell-field shape; along its own axis, slot s holds face s+1 (faces 1..n-1 are the unknowns) and slot
n-1 holds the far wall face n, whose normal velocity is 0 and is never changed; face 0 (the near wall)
is not stored and is 0.

Readings:
  G9  Appendix D's restriction is printed with the roles of i and j transposed. Read: weights
      (1, 2, 1)/4 across the three fine faces 2i-1/2, 2i+1/2, 2i+3/2 of the normal direction times
      (1, 1)/2 over the two fine cells of each tangential direction. Prolongation as printed: a fine
      face coincident with a coarse face takes the tangential 3/4-1/4 interpolation, a face between
      two coarse faces the average of its two neighbours; coarse ghosts follow the (homogeneous)
      boundary condition.
  G10 Wall velocities (the lid) are folded into the right-hand side once: every level solves the
      homogeneous problem.
  G11 WENO3 convection: Jiang-Shu third order with two substencils, ideal weights 1/3 and 2/3,
      epsilon 1e-6, for the derivative of the advected component in each direction, upwinded by the
      sign of the advecting velocity at the point; advecting components are interpolated to the
      point by averaging their 2 (2D) or 4 (3D) surrounding faces. Values beyond a wall: the normal
      component is reflected oddly about the wall face, a tangential component by ghost = 2 g - inside
      (g the wall's tangential velocity). The convection term alone is not pinned by a printed
      formula (the paper prints none): its own tests are exactness on linear fields and zero
      convection of a uniform flow. The projection steps that contain it are pinned by the paper's
      first- and second-order convergence tables for the manufactured solution (Sec. 4.4.3), which
      this oracle reproduces within 1-2 % (tests/golden/ns_*_order_mms.json).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import cell_centred as cc

EPS_WENO = 1e-6


@dataclass
class FaceOperator:
    """A u = alpha u - beta Lap_h u for the face component of physical axis `axis` with all walls
    Dirichlet (normal component 0 on its own walls; tangential walls by ghost = -inside after the
    wall values are folded into the right-hand side)."""

    shape: tuple
    h: float
    alpha: float
    beta: float
    axis: int  # physical axis of the component (0 x, 1 y, 2 z)
    dtype: object = np.float64

    @property
    def dim(self):
        return len(self.shape)

    @property
    def fax(self):
        """numpy axis of the component's own (normal) direction."""
        return self.dim - 1 - self.axis


def frozen_slice(op: FaceOperator):
    sl = [slice(None)] * op.dim
    sl[op.fax] = op.shape[op.fax] - 1
    return tuple(sl)


def apply_A_face(op: FaceOperator, u: np.ndarray) -> np.ndarray:
    """A u at the interior faces; 0 on the frozen wall slot."""
    u = np.asarray(u, dtype=op.dtype)
    out = op.alpha * u
    scale = op.beta / (op.h * op.h)
    for ax in range(op.dim):
        n = op.shape[ax]
        if ax == op.fax:
            zero = np.zeros_like(cc._take(u, slice(0, 1), ax))
            ext = np.concatenate([zero, u], axis=ax)  # faces 0..n (slot n-1 = face n = 0)
            lap = cc._take(ext, slice(0, n - 1), ax) - 2.0 * cc._take(ext, slice(1, n), ax) + \
                cc._take(ext, slice(2, n + 1), ax)
            pad = np.zeros_like(cc._take(u, slice(0, 1), ax))
            out = out - scale * np.concatenate([lap, pad], axis=ax)
        else:
            first = cc._take(u, slice(0, 1), ax)
            last = cc._take(u, slice(-1, None), ax)
            ext = np.concatenate([-first, u, -last], axis=ax)
            out = out - scale * np.diff(ext, n=2, axis=ax)
    out[frozen_slice(op)] = 0.0
    return out


def residual_face(op: FaceOperator, u, f):
    r = np.asarray(f, dtype=op.dtype) - apply_A_face(op, u)
    r[frozen_slice(op)] = 0.0
    return r


def _sets(dim):
    return cc.SETS_2D if dim == 2 else cc.SETS_3D


def xmcgs_sweep_face(op: FaceOperator, u: np.ndarray, f: np.ndarray) -> None:
    """One X-MCGS sweep on the face grid: the parity sets (face index i along the component's axis,
    1-based cell indices along the others) in the paper's order; the wall slot is never updated.
    Point update: (h^2 f + beta * sum of neighbour values) / (alpha h^2 + beta * sum of weights),
    weight 1 per neighbour along the normal axis (a wall face counts with value 0) and per interior
    tangential neighbour, 2 per tangential wall (ghost = -inside)."""
    h2 = op.h * op.h
    f = np.asarray(f, dtype=op.dtype)
    pad = np.zeros(tuple(n + 2 for n in op.shape), dtype=op.dtype)
    inner = tuple(slice(1, n + 1) for n in op.shape)
    pad[inner] = u
    # diagonal
    D = np.full(op.shape, op.alpha * h2)
    for ax in range(op.dim):
        n = op.shape[ax]
        if ax == op.fax:
            D = D + 2.0 * op.beta
        else:
            w = np.full(op.shape, 2.0)  # two interior neighbours
            for idx in (0, n - 1):
                sl = [slice(None)] * op.dim
                sl[ax] = idx
                w[tuple(sl)] += 1.0  # wall side: ghost -inside adds 2, neighbour removed 1
            D = D + op.beta * w
    for parities in _sets(op.dim):
        # slot s along the face axis is face s+1: its 1-based index parity is that of s+1, the same
        # rule as for 1-based cell indices of 0-based position s
        offs, cell = cc._set_slices(op, parities)
        nb = np.zeros(pad[tuple(slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape))].shape)
        for ax in range(op.dim):
            for s in (-1, +1):
                sl = [slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape)]
                sl[ax] = slice(offs[ax] + 1 + s, op.shape[ax] + 1 + s, 2)
                nb = nb + pad[tuple(sl)]
        target = tuple(slice(o + 1, n + 1, 2) for o, n in zip(offs, op.shape))
        new = (h2 * f[cell] + op.beta * nb) / D[cell]
        # keep the wall slot
        fr = [slice(None)] * op.dim
        fslots = np.arange(offs[op.fax], op.shape[op.fax], 2)
        keep = fslots == op.shape[op.fax] - 1
        if keep.any():
            fr[op.fax] = np.where(keep)[0]
            new[tuple(fr)] = 0.0
        pad[target] = new
    u[...] = pad[inner]


def restrict_face(op: FaceOperator, v: np.ndarray) -> np.ndarray:
    """Appendix D restriction (reading G9): coarse slot S (face S+1) = sum over the fine faces
    2S+1, 2S+2, 2S+3 (slots 2S, 2S+1, 2S+2) with weights 1/4, 1/2, 1/4, times the average of the two
    fine cells along every tangential axis. The coarse wall slot is 0."""
    fa = op.fax
    nf = op.shape[fa]
    nc = nf // 2
    # tangential averages first
    t = v
    for ax in range(op.dim):
        if ax != fa:
            t = 0.5 * (cc._take(t, slice(0, None, 2), ax) + cc._take(t, slice(1, None, 2), ax))
    out = np.zeros(tuple(n // 2 for n in op.shape))
    a = cc._take(t, slice(0, nf - 2, 2), fa)  # slots 2S, S = 0..nc-2
    b = cc._take(t, slice(1, nf - 1, 2), fa)  # 2S+1
    c = cc._take(t, slice(2, nf, 2), fa)  # 2S+2
    sl = [slice(None)] * op.dim
    sl[fa] = slice(0, nc - 1)
    out[tuple(sl)] = 0.25 * a + 0.5 * b + 0.25 * c
    return out


def prolong_face(op: FaceOperator, cvals: np.ndarray) -> np.ndarray:
    """Appendix D prolongation of a coarse correction: along every tangential axis the fine cell
    2J takes (3 c_J + c_{J-1})/4 and 2J+1 takes (3 c_J + c_{J+1})/4, with coarse ghosts -c at walls;
    along the normal axis a fine face coincident with a coarse face takes that value, a fine face
    between two coarse faces the average of the two (wall faces 0)."""
    fa = op.fax
    t = np.asarray(cvals, dtype=np.float64)
    for ax in range(op.dim):
        if ax == fa:
            continue
        n = t.shape[ax]
        first = cc._take(t, slice(0, 1), ax)
        last = cc._take(t, slice(-1, None), ax)
        ext = np.concatenate([-first, t, -last], axis=ax)
        lo = 0.75 * cc._take(ext, slice(1, n + 1), ax) + 0.25 * cc._take(ext, slice(0, n), ax)
        hi = 0.75 * cc._take(ext, slice(1, n + 1), ax) + 0.25 * cc._take(ext, slice(2, n + 2), ax)
        shp = list(t.shape)
        shp[ax] = 2 * n
        out = np.empty(shp)
        s0 = [slice(None)] * t.ndim
        s0[ax] = slice(0, None, 2)
        s1 = [slice(None)] * t.ndim
        s1[ax] = slice(1, None, 2)
        out[tuple(s0)] = lo
        out[tuple(s1)] = hi
        t = out
    nc = t.shape[fa]
    shp = list(t.shape)
    shp[fa] = 2 * nc
    out = np.zeros(shp)
    # coarse slot S (face S+1) coincides with fine face 2S+2 = fine slot 2S+1
    so = [slice(None)] * t.ndim
    so[fa] = slice(1, 2 * nc - 2, 2)
    out[tuple(so)] = cc._take(t, slice(0, nc - 1), fa)
    # fine slot 2S (face 2S+1) between coarse faces S and S+1 (slots S-1 and S; face 0 is 0)
    zero = np.zeros_like(cc._take(t, slice(0, 1), fa))
    ext = np.concatenate([zero, cc._take(t, slice(0, nc - 1), fa)], axis=fa)  # faces 0..nc-1
    se = [slice(None)] * t.ndim
    se[fa] = slice(0, 2 * nc - 2, 2)
    right = np.concatenate([cc._take(t, slice(0, nc - 1), fa)], axis=fa)
    out[tuple(se)] = 0.5 * (cc._take(ext, slice(0, nc - 1), fa) + right)
    # fine slot 2nc-2 (face 2nc-1) between coarse face nc-1 (slot nc-2) and the wall face nc
    sl2 = [slice(None)] * t.ndim
    sl2[fa] = 2 * nc - 2
    sl3 = [slice(None)] * t.ndim
    sl3[fa] = nc - 2
    out[tuple(sl2)] = 0.5 * t[tuple(sl3)]
    return out


def build_levels_face(op: FaceOperator, coarsest: int = 4):
    levels = [op]
    while min(levels[-1].shape) > coarsest:
        o = levels[-1]
        levels.append(replace(o, shape=tuple(n // 2 for n in o.shape), h=2.0 * o.h))
    return levels


def vcycle_face(levels, u, f, params: cc.Params, level: int = 0) -> None:
    """Algorithm 1 with recursion on the face grid (same steps as cell_centred.vcycle)."""
    op = levels[level]
    if level == len(levels) - 1:
        for _ in range(params.sweeps_coarse()):
            xmcgs_sweep_face(op, u, f)
        return
    for _ in range(params.nu1):
        xmcgs_sweep_face(op, u, f)
    r1 = residual_face(op, u, f)
    u0 = restrict_face(op, u)
    r0 = restrict_face(op, r1)
    u0_start = u0.copy()
    f0 = r0 + apply_A_face(levels[level + 1], u0)
    vcycle_face(levels, u0, f0, params, level + 1)
    u += prolong_face(op, u0 - u0_start)
    u[frozen_slice(op)] = 0.0
    for _ in range(params.nu2):
        xmcgs_sweep_face(op, u, f)


def solve_face(levels, u, f, params: cc.Params) -> cc.SolveInfo:
    op = levels[0]
    info = cc.SolveInfo()
    info.res0 = cc.norm2(residual_face(op, u, f))
    fn = cc.norm2(f)
    ref = fn if fn > 0 else info.res0
    for _ in range(params.kmax):
        vcycle_face(levels, u, f, params)
        info.cycles += 1
        info.res = cc.norm2(residual_face(op, u, f))
        info.rel = info.res / ref if ref > 0 else 0.0
        if info.res <= params.tol * ref:
            info.converged = True
            break
    return info


def dense_matrix_face(op: FaceOperator) -> np.ndarray:
    n = int(np.prod(op.shape))
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = apply_A_face(op, e.reshape(op.shape)).ravel()
    return M


# ---------------------------------------------------------------------------------------------
# projection scheme (Sec. 4.2)
# ---------------------------------------------------------------------------------------------



def faces_ext(phi: np.ndarray, fax: int) -> np.ndarray:
    """Face values 0..n along fax as an array of length n+1 on that axis (walls 0)."""
    zero = np.zeros_like(cc._take(phi, slice(0, 1), fax))
    return np.concatenate([zero, phi], axis=fax)


def divergence(vel, h):
    """div u at cells: sum over axes of (face k+1 - face k)/h, wall faces 0."""
    dim = len(vel)
    out = 0.0
    for a in range(dim):
        fax = dim - 1 - a
        ext = faces_ext(vel[a], fax)
        out = out + np.diff(ext, axis=fax) / h
    return out


def _ext_values(phi, ax, n_ghost, normal, g_lo, g_hi):
    """phi extended by n_ghost values on both ends of numpy axis ax. Normal direction (the
    component's own axis, faces): array of faces 0..n with odd reflection beyond the walls
    (face -k = -face k). Tangential (cells): ghost = 2 g - inside, mirrored."""
    if normal:
        core = faces_ext(phi, ax)  # faces 0..n, length n+1
        n = core.shape[ax] - 1
        lo = [-cc._take(core, slice(k, k + 1), ax) for k in range(n_ghost, 0, -1)]
        hi = [-cc._take(core, slice(n - k, n - k + 1), ax) for k in range(1, n_ghost + 1)]
        return np.concatenate(lo + [core] + hi, axis=ax), 1  # offset of face 0 is n_ghost
    n = phi.shape[ax]
    lo = [2.0 * g_lo - cc._take(phi, slice(k - 1, k), ax) for k in range(n_ghost, 0, -1)]
    hi = [2.0 * g_hi - cc._take(phi, slice(n - k, n - k + 1), ax) for k in range(1, n_ghost + 1)]
    return np.concatenate(lo + [phi] + hi, axis=ax), 0


def weno3_derivatives(phi, ax, h, normal, g_lo, g_hi):
    """Upwind-biased WENO3 derivatives of phi along numpy axis ax at the unknown points (faces 1..n-1
    along the normal axis, all cells along a tangential one): returns (d_minus, d_plus), the
    left-biased and right-biased approximations (reading G11)."""
    ext, _ = _ext_values(phi, ax, 3, normal, g_lo, g_hi)
    # positions of the unknowns inside ext
    n = phi.shape[ax]
    if normal:
        start, count = 3 + 1, n - 1  # face 1 is at 3 + 1
    else:
        start, count = 3, n

    def val(shift):
        return cc._take(ext, slice(start + shift, start + shift + count), ax)

    v1 = (val(-1) - val(-2)) / h
    v2 = (val(0) - val(-1)) / h
    v3 = (val(1) - val(0)) / h
    v4 = (val(2) - val(1)) / h

    def weno(a, b, c):  # a, b, c: the three first differences, upwind side first
        p0 = 0.5 * (3.0 * b - a)
        p1 = 0.5 * (b + c)
        b0 = (b - a) ** 2
        b1 = (c - b) ** 2
        a0 = (1.0 / 3.0) / (EPS_WENO + b0) ** 2
        a1 = (2.0 / 3.0) / (EPS_WENO + b1) ** 2
        return (a0 * p0 + a1 * p1) / (a0 + a1)

    dm = weno(v1, v2, v3)
    dp = weno(v4, v3, v2)
    return dm, dp


def advecting_velocity(vel, comp, a):
    """Component a of the velocity at the unknown points of component comp (a != comp): average of
    the surrounding a-faces: cells k-1, k along comp's axis, faces j, j+1 along a."""
    dim = len(vel)
    fc = dim - 1 - comp
    fa = dim - 1 - a
    ph = faces_ext(vel[a], fa)  # faces 0..n along fa
    n_fa = vel[a].shape[fa]
    s = 0.5 * (cc._take(ph, slice(0, n_fa), fa) + cc._take(ph, slice(1, n_fa + 1), fa))  # cell centres along fa
    nfc = s.shape[fc]
    t = 0.5 * (cc._take(s, slice(0, nfc - 1), fc) + cc._take(s, slice(1, nfc), fc))  # faces 1..n-1 along fc
    pad = np.zeros_like(cc._take(t, slice(0, 1), fc))
    return np.concatenate([t, pad], axis=fc)


def convection(vel, comp, h, lid):
    """(u . grad) of component comp at its unknowns (WENO3, upwinded by the advecting velocity)."""
    return convection_of(vel[comp], vel, comp, h, lid)


def convection_of(phi, advect, comp, h, lid):
    """(a . grad) phi for the face field phi of component comp: WENO3 derivatives of phi, upwinded by
    the advecting velocity, whose component a is interpolated from advect[a] (a != comp) or is phi
    itself (a == comp)."""
    dim = phi.ndim
    fc = dim - 1 - comp
    out = np.zeros(phi.shape)
    for a in range(dim):
        ax = dim - 1 - a
        normal = a == comp
        # wall tangential values of comp on the two walls normal to axis a
        g_lo = 0.0
        g_hi = lid[comp] if (a == dim - 1) else 0.0  # the lid is the top wall of the last axis
        dm, dp = weno3_derivatives(phi, ax, h, normal, g_lo, g_hi)
        if normal:
            adv = phi
            pad = np.zeros_like(cc._take(phi, slice(0, 1), ax))
            dm = np.concatenate([dm, pad], axis=ax)
            dp = np.concatenate([dp, pad], axis=ax)
        else:
            adv = advecting_velocity(advect, comp, a)
        out = out + np.where(adv > 0.0, adv * dm, adv * dp)
    out[tuple(slice(None) if k != fc else phi.shape[fc] - 1 for k in range(dim))] = 0.0
    return out


def pressure_gradient(p, comp, h):
    """(p_k - p_{k-1})/h at faces k = 1..n-1 of component comp, 0 on the wall slot."""
    dim = p.ndim
    fc = dim - 1 - comp
    g = np.diff(p, axis=fc) / h
    pad = np.zeros_like(cc._take(p, slice(0, 1), fc))
    return np.concatenate([g, pad], axis=fc)


def lid_rhs(shape, comp, beta, h, lid):
    """Reading G10: the tangential wall velocity g of the lid (top wall of the last axis) enters the
    cells next to it as 2 beta g / h^2."""
    out = np.zeros(shape)
    dim = len(shape)
    if comp == dim - 1 or lid[comp] == 0.0:
        return out
    sl = [slice(None)] * dim
    sl[0] = shape[0] - 1  # numpy axis 0 = last physical axis
    out[tuple(sl)] = 2.0 * beta * lid[comp] / (h * h)
    fc = dim - 1 - comp
    out[tuple(slice(None) if k != fc else shape[fc] - 1 for k in range(dim))] = 0.0
    return out


@dataclass
class NSParams:
    Re: float = 100.0
    dt: float = 1e-3
    lid: tuple = (1.0, 0.0, 0.0)
    solver: cc.Params = None
    pressure: cc.Params = None


def projection_step(fields: dict, shape, h, prm: NSParams, force=None):
    """Scheme first-1..4 in the order of the 8-field memory-efficient table:
        f_c = c^n - dt (u^n . grad c^n)_WENO3 - dt (grad p^n)_c          (source, into a solver temporary)
        (I - dt/Re Lap) tilde-c = f_c, from c^n, into C_new              (viscous solves)
        dt Lap tilde-p = div tilde-u, i.e. -dt Lap tilde-p = -div tilde-u (pressure, Neumann, mean 0) into P_new
        c^{n+1} = tilde-c - dt (grad tilde-p)_c into C_old; p^{n+1} = p^n + tilde-p into P_old.
    fields: U_new, U_old, V_new, V_old, [W_new, W_old,] P_new, P_old (numpy arrays, updated in place).
    force (optional): per component, the body force at t^{n+1} on its faces; it enters the viscous
    right-hand side as + dt F (backward Euler on the forced momentum equation).
    Returns the solve infos and max |div u^{n+1}|."""
    dim = len(shape)
    names = ["U", "V", "W"][:dim]
    dt = prm.dt
    beta = dt / prm.Re
    sol = prm.solver or cc.Params(tol=1e-10, kmax=40, coarsest=4)
    psol = prm.pressure or cc.Params(tol=1e-10, kmax=60, coarsest=4, coarse_exact=True)
    vel_n = [fields[nm + "_old"] for nm in names]
    p_n = fields["P_old"]
    infos = []
    for comp, nm in enumerate(names):
        f = vel_n[comp] - dt * convection(vel_n, comp, h, prm.lid) - dt * pressure_gradient(p_n, comp, h)
        if force is not None and force[comp] is not None:
            f = f + dt * np.asarray(force[comp], dtype=np.float64)
        op = FaceOperator(shape, h, 1.0, beta, comp)
        f = f + lid_rhs(shape, comp, beta, h, prm.lid)
        f[frozen_slice(op)] = 0.0
        fields[nm + "_new"][...] = vel_n[comp]
        infos.append(solve_face(build_levels_face(op, sol.coarsest), fields[nm + "_new"], f, sol))
    vel_t = [fields[nm + "_new"] for nm in names]
    rhs = -divergence(vel_t, h)
    pop = cc.Operator(shape, h, 0.0, dt, 1.0)
    fields["P_new"][...] = 0.0
    infos.append(cc.solve(cc.build_levels(pop, psol.coarsest), fields["P_new"], rhs, psol))
    for comp, nm in enumerate(names):
        fields[nm + "_old"][...] = vel_t[comp] - dt * pressure_gradient(fields["P_new"], comp, h)
    fields["P_old"] += fields["P_new"]
    div = divergence([fields[nm + "_old"] for nm in names], h)
    return infos, float(np.max(np.abs(div))), float(np.max(np.abs(rhs)))


def projection_step2(fields: dict, shape, h, prm: NSParams, force=None):
    """Scheme second-1..4 (Sec. 4.3) in the order of the memory-efficient 8-field table of the
    second-order scheme. On entry C_new holds c^n and C_old holds c^{n-1} (both c^0 at the first step);
    for each component c in turn:
        f_c = c^n - dt (a . grad) cbar + (dt / 2Re) Lap c^n - dt (grad p^n)_c (+ dt F_c)   cbar = (3c^n - c^{n-1})/2
              advecting a: (a^n + a~^{n+1})/2 for the components already solved in this step,
              (3a^n - a^{n-1})/2 for the others (cbar itself along c)
        C_old <- C_new (the lagged update), then (I - dt/2Re Lap) c~ = f_c from c^n into C_new;
    then -dt Lap p~ = -div u~ into P_new, c^{n+1} = c~ - dt (grad p~)_c in C_new, P_old += P_new.
    The lid enters once for the implicit and once for the explicit half of the viscous term, 2 beta g /
    h^2 each with beta = dt / 2Re. force: per component, the body force at t^{n+1/2} (reading)."""
    dim = len(shape)
    names = ["U", "V", "W"][:dim]
    dt = prm.dt
    beta = dt / (2.0 * prm.Re)
    sol = prm.solver or cc.Params(tol=1e-10, kmax=40, coarsest=4)
    psol = prm.pressure or cc.Params(tol=1e-10, kmax=60, coarsest=4, coarse_exact=True)
    p_n = fields["P_old"]
    infos = []
    for comp, nm in enumerate(names):
        cur = [fields[m + "_new"] for m in names]
        old = [fields[m + "_old"] for m in names]
        cbar = 0.5 * (3.0 * cur[comp] - old[comp])
        advect = []
        for a in range(dim):
            if a < comp:
                advect.append(0.5 * (old[a] + cur[a]))  # a^n (lagged into C_old) and a~^{n+1}
            else:
                advect.append(0.5 * (3.0 * cur[a] - old[a]))
        op = FaceOperator(shape, h, 1.0, beta, comp)
        lap = -apply_A_face(FaceOperator(shape, h, 0.0, 1.0, comp), cur[comp])
        f = cur[comp] - dt * convection_of(cbar, advect, comp, h, prm.lid) + beta * lap \
            - dt * pressure_gradient(p_n, comp, h)
        if force is not None and force[comp] is not None:
            f = f + dt * np.asarray(force[comp], dtype=np.float64)
        f = f + 2.0 * lid_rhs(shape, comp, beta, h, prm.lid)
        f[frozen_slice(op)] = 0.0
        fields[nm + "_old"][...] = cur[comp]
        infos.append(solve_face(build_levels_face(op, sol.coarsest), fields[nm + "_new"], f, sol))
    vel_t = [fields[nm + "_new"] for nm in names]
    rhs = -divergence(vel_t, h)
    pop = cc.Operator(shape, h, 0.0, dt, 1.0)
    fields["P_new"][...] = 0.0
    infos.append(cc.solve(cc.build_levels(pop, psol.coarsest), fields["P_new"], rhs, psol))
    for comp, nm in enumerate(names):
        fields[nm + "_new"][...] = vel_t[comp] - dt * pressure_gradient(fields["P_new"], comp, h)
    fields["P_old"] += fields["P_new"]
    div = divergence([fields[nm + "_new"] for nm in names], h)
    return infos, float(np.max(np.abs(div))), float(np.max(np.abs(rhs)))
