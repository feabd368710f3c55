"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module holds no arithmetic of the multigrid method itself: it only draws random numbers and
evaluates the closed-form fields (cosine modes, Gaussian bumps, smoothed noise) that the paper's
workloads are shaped like. Both sides of every parity test receive the identical float64 arrays
produced here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter mode: element k of a stream with key K is
mix64(K + (k + 1) * GAMMA). The 53 high bits of each 64-bit output give a uniform double in [0, 1).
The generator is written out here from its published definition so that results do not depend on
the numpy version installed on a machine.

Array convention everywhere in this project: C order with x fastest, so a 2D field has numpy shape
(ny, nx) and is indexed [j, i]; a 3D field has shape (nz, ny, nx) and is indexed [l, j, i]. Cell
centres are x_i = (i + 1/2) h for 0-based i (the paper's x_i = (i - 1/2) h with 1-based i).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags: one independent stream per (seed, purpose)
TAG_NOISE = 1
TAG_SOURCE = 2
TAG_KAPPA = 3
TAG_TARGET = 4
TAG_SIZES = 5
TAG_COEF = 6
TAG_NORMAL = 7
TAG_INIT = 8
TAG_VEL = 9  # 9, 10, 11: velocity components x, y, z
TAG_PRES = 12
TAG_GRAIN = 13


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> np.uint64:
    """64-bit key of the stream (seed, tag), scrambled so that nearby seeds give unrelated keys."""
    with np.errstate(over="ignore"):
        base = np.array([(int(seed) * 256 + int(tag)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix64(base + GAMMA)[0]


def uniform(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` uniform doubles in [0, 1) from stream (seed, tag), starting at element `offset`."""
    key = stream_key(seed, tag)
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + k * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, tag: int, count: int) -> np.ndarray:
    """`count` standard normal doubles by the Box-Muller transform of pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, tag, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:count]


def cell_centres(n: int, h: float | None = None) -> np.ndarray:
    """Cell-centre coordinates (i + 1/2) h, i = 0..n-1, on [0, n h]; h defaults to 1/n."""
    if h is None:
        h = 1.0 / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _grids(shape, h):
    axes = [cell_centres(n, h) for n in shape]  # numpy axis order (z, y, x)
    return np.meshgrid(*axes, indexing="ij")


def cos_mode(shape, h=None) -> np.ndarray:
    """prod over axes of cos(pi * x_axis): the slowest Neumann eigenmode on [0,1]^d."""
    if h is None:
        h = 1.0 / shape[-1]
    grids = _grids(shape, h)
    out = np.ones(shape)
    for g in grids:
        out *= np.cos(math.pi * g)
    return out


def noisy_cos_mode(shape, seed: int, amplitude: float = 1e-2) -> np.ndarray:
    """cos-mode initial field plus `amplitude` * U(-1, 1) noise (heat workloads)."""
    n = int(np.prod(shape))
    noise = 2.0 * uniform(seed, TAG_NOISE, n) - 1.0
    return cos_mode(shape) + amplitude * noise.reshape(shape)


def gaussian_sum(shape, seed: int, tag: int, count: int, sigma: float,
                 amp_lo: float = -1.0, amp_hi: float = 1.0) -> np.ndarray:
    """sum_k a_k exp(-|x - c_k|^2 / (2 sigma^2)), centres c_k ~ U(0,1)^d, a_k ~ U(amp_lo, amp_hi)."""
    d = len(shape)
    draws = uniform(seed, tag, count * (d + 1))
    centres = draws[: count * d].reshape(count, d)  # columns in physical order x, y, (z)
    amps = amp_lo + (amp_hi - amp_lo) * draws[count * d:]
    h = 1.0 / shape[-1]
    axes_phys = [cell_centres(n, h) for n in reversed(shape)]  # x, y, (z)
    out = np.zeros(shape)
    for k in range(count):
        # separable evaluation: product over axes of 1D Gaussians
        factors = [np.exp(-((axes_phys[a] - centres[k, a]) ** 2) / (2.0 * sigma * sigma))
                   for a in range(d)]
        term = factors[0]
        for a in range(1, d):
            term = np.multiply.outer(factors[a], term)  # builds (.., y, x) order
        out += amps[k] * term
    return out


# ---------------------------------------------------------------------------------------------
# workload recipes (the shapes and value distributions of the paper's heat / Helmholtz problems)
# ---------------------------------------------------------------------------------------------

def heat2d_small(n: int = 128, seed: int = 0):
    """128^2 heat: Neumann, kappa 1, dt 1e-3, 10 steps, u0 = cos mode + 1e-2 noise, no source."""
    shape = (n, n)
    return dict(shape=shape, h=1.0 / n, dt=1e-3, nsteps=10, kappa=1.0,
                u0=noisy_cos_mode(shape, seed), fsrc=None)


def heat2d_large(n: int = 8192, seed: int = 1, nsteps: int = 20):
    """8192^2 heat: Neumann, kappa 1, dt 1e-4, 20 steps, u0 = cos mode + noise,
    source = 16 Gaussians (sigma 0.02, centres U(0,1)^2, amplitudes U(-1,1))."""
    shape = (n, n)
    return dict(shape=shape, h=1.0 / n, dt=1e-4, nsteps=nsteps, kappa=1.0,
                u0=noisy_cos_mode(shape, seed),
                fsrc=gaussian_sum(shape, seed, TAG_SOURCE, 16, 0.02))


def heat3d(n: int = 512, seed: int = 2, nsteps: int = 10):
    """512^3 heat, 7-point: Neumann, kappa 1, dt 1e-4, 10 steps, u0 = 3D cos mode + noise."""
    shape = (n, n, n)
    return dict(shape=shape, h=1.0 / n, dt=1e-4, nsteps=nsteps, kappa=1.0,
                u0=noisy_cos_mode(shape, seed), fsrc=None)


def smoothed_normal(shape, seed: int, passes: int = 3) -> np.ndarray:
    """N(0,1) field smoothed by `passes` damped-Jacobi averages f <- f/2 + (1/8) sum_4 nbrs with
    mirrored (zero-flux) edges. Input preparation only; not the solver's smoother."""
    f = normal(seed, TAG_NORMAL, int(np.prod(shape))).reshape(shape)
    for _ in range(passes):
        p = np.pad(f, 1, mode="edge")
        nb = p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:]
        f = 0.5 * f + 0.125 * nb
    return f


def batched_helmholtz(count: int = 96, seed: int = 3, sizes=(64, 128, 256, 512, 1024, 2048)):
    """Independent 2D problems (I - dt kappa Lap) u = f: n uniform over `sizes`, kappa ~ U(0.5, 2),
    dt uniform over {1e-4, 1e-3}, Neumann, f = N(0,1) smoothed by 3 Jacobi passes."""
    draws = uniform(seed, TAG_SIZES, 3 * count)
    problems = []
    for p in range(count):
        n = sizes[min(int(draws[3 * p] * len(sizes)), len(sizes) - 1)]
        kappa = 0.5 + 1.5 * draws[3 * p + 1]
        dt = 1e-4 if draws[3 * p + 2] < 0.5 else 1e-3
        problems.append(dict(n=n, kappa=float(kappa), dt=dt, seed=seed * 1000 + p))
    return problems


def batched_problem_rhs(problem) -> np.ndarray:
    n = problem["n"]
    return smoothed_normal((n, n), problem["seed"])


def adjoint_heat(n: int = 1024, nsteps: int = 50):
    """1024^2 heat with varying diffusivity kappa = 1 + 0.5 tanh(sum of 8 Gaussians, sigma 0.1,
    amplitudes U(-2,2)); u0 cos mode + noise; source 16 Gaussians (sigma 0.05); target 4 Gaussians
    (sigma 0.15). Loss ||u_T - u_target||^2."""
    shape = (n, n)
    g = gaussian_sum(shape, 4, TAG_KAPPA, 8, 0.1, -2.0, 2.0)
    return dict(shape=shape, h=1.0 / n, dt=1e-3, nsteps=nsteps,
                kappa=1.0 + 0.5 * np.tanh(g),
                u0=noisy_cos_mode(shape, 4),
                fsrc=gaussian_sum(shape, 5, TAG_SOURCE, 16, 0.05),
                target=gaussian_sum(shape, 6, TAG_TARGET, 4, 0.15))


def random_field(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform U(lo, hi) field (random initial guesses and random test operands)."""
    return lo + (hi - lo) * uniform(seed, TAG_INIT, int(np.prod(shape))).reshape(shape)


# ---------------------------------------------------------------------------------------------
# staggered (MAC) grid states: component a of the velocity on the faces normal to physical axis a,
# stored in the cell-field shape with slot s = face s+1 along that axis and the far wall face (always
# 0) in the last slot
# ---------------------------------------------------------------------------------------------

NS_NAMES = ("U", "V", "W")


def zero_wall_slot(v: np.ndarray, comp: int) -> np.ndarray:
    """Set the stored far-wall slot of a face field of component comp to 0 (layout only)."""
    dim = v.ndim
    sl = [slice(None)] * dim
    sl[dim - 1 - comp] = v.shape[dim - 1 - comp] - 1
    v[tuple(sl)] = 0.0
    return v


def ns_state(shape, seed: int, amplitude: float = 0.5) -> dict:
    """Eight fields of a synthetic flow state: each velocity component a sum of 6 Gaussians (sigma
    0.15, amplitudes U(-1,1)) times `amplitude`, zero on its wall slot; pressure 0.1 x 4 Gaussians
    (sigma 0.2); the *_new work fields zero. Flow in every direction, for parity tests."""
    dim = len(shape)
    out = {}
    for a in range(dim):
        v = amplitude * gaussian_sum(shape, seed, TAG_VEL + a, 6, 0.15)
        out[NS_NAMES[a] + "_old"] = zero_wall_slot(v, a)
        out[NS_NAMES[a] + "_new"] = np.zeros(shape)
    out["P_old"] = 0.1 * gaussian_sum(shape, seed, TAG_PRES, 4, 0.2)
    out["P_new"] = np.zeros(shape)
    return out


def ns_cavity(n: int = 256, dim: int = 3, nsteps: int = 20):
    """Lid-driven cavity on [0,1]^dim: n cells per axis, Re 100, dt 1e-3, the top wall of the last
    axis moving with velocity 1 along x, fluid at rest at t = 0."""
    shape = (n,) * dim
    fields = {NS_NAMES[a] + k: np.zeros(shape) for a in range(dim) for k in ("_old", "_new")}
    fields["P_old"] = np.zeros(shape)
    fields["P_new"] = np.zeros(shape)
    return dict(shape=shape, h=1.0 / n, Re=100.0, dt=1e-3, nsteps=nsteps, lid=(1.0, 0.0, 0.0), fields=fields)


# ---------------------------------------------------------------------------------------------
# the manufactured Navier-Stokes solution of the paper's asymptotic-in-time test (Sec. 4.4.3)
# ---------------------------------------------------------------------------------------------

def _sin2(t):
    return np.sin(t) ** 2


def ns_mms(n: int, Re: float = 10.0) -> dict:
    """On [0,1]^2 with n x n cells: p = sin t (sin(pi y) - 2/pi), u = sin t sin^2(pi x) sin(2 pi y),
    v = -sin t sin(2 pi x) sin^2(pi y), divergence free and 0 on the walls; the body force is
    F = u_t + (u . grad) u + grad p - (1/Re) Lap u of that solution. Every field is a sum of terms
    c(t) * outer(Y(y), X(x)) evaluated at its own points: u on x-faces (x = (i+1) h, y = (j+1/2) h),
    v on y-faces, p at cell centres. Returns 'exact' and 'force' term lists per component (0 = u,
    1 = v, 'p' = pressure)."""
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h  # cell centres
    f = (np.arange(n) + 1.0) * h  # faces 1..n (slot s = face s+1)
    pi = np.pi
    s1, s2, cs = np.sin, _sin2, np.cos
    one = np.ones(n)
    exact = {
        0: [(s1, np.sin(2 * pi * c), np.sin(pi * f) ** 2)],
        1: [(s1, -np.sin(pi * f) ** 2, np.sin(2 * pi * c))],
        "p": [(s1, np.sin(pi * c) - 2.0 / pi, one)],
    }
    # u at (x = f, y = c)
    xu, yu = f, c
    force_u = [
        (cs, np.sin(2 * pi * yu), np.sin(pi * xu) ** 2),                                        # u_t
        (s2, np.sin(2 * pi * yu) ** 2, pi * np.sin(2 * pi * xu) * np.sin(pi * xu) ** 2),       # u u_x
        (s2, 2 * pi * np.sin(pi * yu) ** 2 * np.cos(2 * pi * yu),
         -np.sin(2 * pi * xu) * np.sin(pi * xu) ** 2),                                         # v u_y
        (s1, np.sin(2 * pi * yu), -2 * pi ** 2 * np.cos(2 * pi * xu) / Re),                    # -u_xx/Re
        (s1, np.sin(2 * pi * yu), 4 * pi ** 2 * np.sin(pi * xu) ** 2 / Re),                    # -u_yy/Re
    ]
    # v at (x = c, y = f)
    xv, yv = c, f
    force_v = [
        (cs, np.sin(pi * yv) ** 2, -np.sin(2 * pi * xv)),                                      # v_t
        (s2, np.sin(2 * pi * yv) * np.sin(pi * yv) ** 2,
         -2 * pi * np.sin(pi * xv) ** 2 * np.cos(2 * pi * xv)),                                # u v_x
        (s2, np.sin(pi * yv) ** 2 * np.sin(2 * pi * yv), pi * np.sin(2 * pi * xv) ** 2),       # v v_y
        (s1, pi * np.cos(pi * yv), np.ones(n)),                                                # p_y
        (s1, np.sin(pi * yv) ** 2, -4 * pi ** 2 * np.sin(2 * pi * xv) / Re),                   # -v_xx/Re
        (s1, np.cos(2 * pi * yv), 2 * pi ** 2 * np.sin(2 * pi * xv) / Re),                     # -v_yy/Re
    ]
    return dict(shape=(n, n), h=h, Re=Re, exact=exact, force={0: force_u, 1: force_v})


def mms_field(terms, t: float, comp=None) -> np.ndarray:
    """Sum of c(t) outer(Y, X) over the terms (numpy order (y, x)); a velocity component's far wall
    slot is set to 0 (its wall value)."""
    out = None
    for fn, Y, X in terms:
        term = float(fn(t)) * np.multiply.outer(Y, X)
        out = term if out is None else out + term
    if comp is not None:
        zero_wall_slot(out, comp)
    return out


def grain_growth_fields(q: int, shape, seed: int = 5) -> np.ndarray:
    """Grain growth (Sec. 3.3.1): q order parameters on a periodic grid, U(-0.001, 0.001) per cell
    (the paper's disordered, liquid-like start); shape (q,) + grid shape."""
    n = int(np.prod(shape))
    return (uniform(seed, TAG_GRAIN, q * n) * 0.002 - 0.001).reshape((q,) + tuple(shape))


def grain_growth(n: int = 512, q: int = 1189, seed: int = 5):
    """The paper's 2D grain-growth run: 512^2 cells, h = 2 (domain [0, 1024]^2), dt = 0.25, q up to
    1189 order parameters, periodic in every direction."""
    shape = (n, n)
    return dict(shape=shape, q=q, h=2.0, dt=0.25, etas=grain_growth_fields(q, shape, seed))
