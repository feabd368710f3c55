"""Python binding of libfasmg.so, the GB300 matrix-free FAS multigrid library.

Argument marshalling only: every step of the solver runs in the library's CUDA kernels. The functions
carry the C-ABI names of include/fas.h and take torch CUDA tensors (float64, contiguous, C order with
x fastest) for device fields. There is no CPU fallback: if the library has not been built, load()
raises.

    import paper_2510_11152_gb300 as fas
    p = fas.fas_default_params(); p.dim = 2; p.n[:2] = (1024, 1024); p.h = 1 / 1024
    ctx = fas.fas_create(p)
    info = fas.fas_solve(ctx, u, f)
    fas.fas_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB as LIB_PATH

__all__ = [
    "FasError", "fas_params", "fas_info", "load", "fas_default_params", "fas_create", "fas_destroy",
    "fas_num_levels", "fas_vcycle", "fas_solve", "fas_heat_run", "fas_heat_run_host", "fas_residual",
    "fas_smooth", "fas_restrict", "fas_prolong_add", "fas_last_error", "fas_launch_count", "Solver",
    "fas_prof_enable", "fas_prof_read", "make_params", "fas_vcycle_small_static", "fas_solve_batched",
    "fas_autotune", "fas_heat_adjoint", "fas_fold_dirichlet", "solve", "HeatSolve", "fas_probe_fp64_rate",
    "gg_model", "gg_create", "gg_step", "gg_rhs", "gg_destroy", "fas_debug_bounded_wait",
]

FAS_OK, FAS_EINVAL, FAS_ENOMEM, FAS_ENOTCONV, FAS_ENONFINITE, FAS_ETIMEOUT, FAS_ECUDA, FAS_EUNSUPPORTED = range(8)
STATUS_NAMES = ["FAS_OK", "FAS_EINVAL", "FAS_ENOMEM", "FAS_ENOTCONV", "FAS_ENONFINITE", "FAS_ETIMEOUT",
                "FAS_ECUDA", "FAS_EUNSUPPORTED"]
FAS_BC_NEUMANN, FAS_BC_DIRICHLET, FAS_BC_PERIODIC = 0, 1, 2
FAS_FP64, FAS_MIXED = 0, 1
FAS_ORDER_FORWARD, FAS_ORDER_SYMMETRIC = 0, 1  # X-MCGS 1234-1234 / 1234-4321 (Sec. 2.3)
FAS_CELL, FAS_FACE_X, FAS_FACE_Y, FAS_FACE_Z = 0, 1, 2, 3


class fas_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("kappa", ctypes.c_void_p),
        ("kappa_const", ctypes.c_double), ("bc", ctypes.c_int * 6), ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int), ("nu_coarse", ctypes.c_int), ("kmax", ctypes.c_int),
        ("coarsest", ctypes.c_int), ("coarse_exact", ctypes.c_int), ("tol", ctypes.c_double),
        ("tol_relative", ctypes.c_int), ("precision", ctypes.c_int), ("inner_cycles", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("path", ctypes.c_int), ("seg_rows", ctypes.c_int),
        ("location", ctypes.c_int), ("ordering", ctypes.c_int),
    ]


class fas_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("converged", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("rel", ctypes.c_double), ("rho", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fas_tune_result(ctypes.Structure):
    _fields_ = [("inner_cycles", ctypes.c_int), ("seg_rows", ctypes.c_int), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gg_model(ctypes.Structure):
    """Model constants of the grain-growth step (Sec. 3.3.1): L, alpha, beta, gamma, kappa."""
    _fields_ = [("L", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("kappa", ctypes.c_double)]


class FasError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = fas_last_error() if _lib is not None else ""
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES[status] if 0 <= status < 8 else status, msg))


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def load(path: str | None = None):
    """Load libfasmg.so (built by paper_2510_11152_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libfasmg.so not built (%s); run paper_2510_11152_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    sig = {
        "fas_default_params": (None, [ctypes.POINTER(fas_params)]),
        "fas_create": (_I, [ctypes.POINTER(fas_params), _P, ctypes.POINTER(_P)]),
        "fas_destroy": (_I, [_P]),
        "fas_num_levels": (_I, [_P]),
        "fas_vcycle": (_I, [_P, _P, _P, ctypes.POINTER(fas_info)]),
        "fas_solve": (_I, [_P, _P, _P, ctypes.POINTER(fas_info)]),
        "fas_heat_run": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(fas_info)]),
        "fas_heat_run_host": (_I, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(fas_info)]),
        "fas_residual": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(_D)]),
        "fas_smooth": (_I, [_P, _I, _P, _P, _I]),
        "fas_restrict": (_I, [_P, _I, _P, _P]),
        "fas_prolong_add": (_I, [_P, _I, _P, _P]),
        "fas_last_error": (ctypes.c_char_p, []),
        "fas_launch_count": (ctypes.c_longlong, [_P, _I]),
        "fas_prof_enable": (_I, [_P, _I]),
        "fas_vcycle_small_static": (_I, [ctypes.POINTER(fas_params), _P, _P, _I, ctypes.POINTER(_D), _P]),
        "fas_solve_batched": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                   ctypes.POINTER(fas_info), _P]),
        "fas_autotune": (_I, [_P, _P, _P, ctypes.POINTER(fas_tune_result)]),
        "fas_heat_adjoint": (_I, [_P, _P, _P, _D, _I, _P, _P, _P, _P, _P, _I]),
        "fas_prof_read": (_I, [_P, ctypes.c_void_p, _I, ctypes.POINTER(_I)]),
        "fas_residual_ir": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D)]),
        "fas_fold_dirichlet": (_I, [_P, _P, ctypes.POINTER(_D)]),
        "fas_selftest_conversions": (_I, [ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)]),
        "fas_probe_fp64_rate": (_I, [ctypes.POINTER(_D)]),
        "fas_debug_bounded_wait": (_I, [ctypes.c_longlong, _I]),
        "ns_create": (_I, [_I, ctypes.POINTER(_I), _D, _D, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(fas_params),
                           ctypes.POINTER(fas_params), _P, ctypes.POINTER(_P)]),
        "ns_projection_step": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(fas_info),
                                    ctypes.POINTER(_D)]),
        "ns_launch_count": (ctypes.c_longlong, [_P, _I]),
        "gg_create": (_I, [_I, ctypes.POINTER(_I), _D, _D, _I, ctypes.POINTER(gg_model), ctypes.POINTER(fas_params),
                           _I, _P, ctypes.POINTER(_P)]),
        "gg_step": (_I, [_P, _P, ctypes.POINTER(fas_info)]),
        "gg_rhs": (_I, [_P, _P, _P]),
        "gg_destroy": (_I, [_P]),
        "ns_destroy": (_I, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status != FAS_OK:
        raise FasError(status, where)


def _dev(t, what, numel=None):
    """Device pointer of a float64 contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be contiguous float64" % what)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (what, t.numel(), numel))
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def fas_last_error() -> str:
    return load().fas_last_error().decode()


def fas_default_params() -> fas_params:
    p = fas_params()
    load().fas_default_params(ctypes.byref(p))
    return p


class _Ctx:
    """Owns a fas_ctx* together with the parameters and the tensors it must keep alive."""

    def __init__(self, handle, params, keep):
        self.handle = handle
        self.params = params
        self.keep = keep

    @property
    def cells(self):
        p = self.params
        return p.n[0] * p.n[1] * (p.n[2] if p.dim == 3 else 1)

    def level_cells(self, level):
        p = self.params
        c = (p.n[0] >> level) * (p.n[1] >> level)
        return c * ((p.n[2] >> level) if p.dim == 3 else 1)

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.fas_destroy(self.handle)
            self.handle = None


def fas_create(params: fas_params, stream=None, kappa=None) -> _Ctx:
    """fas_create; `kappa` (optional float64 CUDA tensor) sets params.kappa."""
    lib = load()
    if kappa is not None:
        params.kappa = _dev(kappa, "kappa")
    out = _P()
    _check(lib.fas_create(ctypes.byref(params), _stream_handle(stream), ctypes.byref(out)), "fas_create")
    return _Ctx(out, params, [kappa])


def fas_destroy(ctx: _Ctx) -> None:
    if ctx.handle:
        _check(load().fas_destroy(ctx.handle), "fas_destroy")
        ctx.handle = None


def fas_num_levels(ctx: _Ctx) -> int:
    return load().fas_num_levels(ctx.handle)


def _info_call(fn, ctx, where, *args, allow_notconv=False):
    info = fas_info()
    st = fn(ctx.handle, *args, ctypes.byref(info))
    if not (allow_notconv and st == FAS_ENOTCONV):
        _check(st, where)
    return info


def fas_vcycle(ctx: _Ctx, u, f) -> fas_info:
    n = ctx.cells
    return _info_call(load().fas_vcycle, ctx, "fas_vcycle", _dev(u, "u", n), _dev(f, "f", n))


def fas_solve(ctx: _Ctx, u, f, allow_notconv=False) -> fas_info:
    n = ctx.cells
    return _info_call(load().fas_solve, ctx, "fas_solve", _dev(u, "u", n), _dev(f, "f", n),
                      allow_notconv=allow_notconv)


def fas_heat_run(ctx: _Ctx, u, fsrc, dt: float, nsteps: int):
    n = ctx.cells
    infos = (fas_info * max(nsteps, 1))()
    st = load().fas_heat_run(ctx.handle, _dev(u, "u", n), _dev(fsrc, "fsrc", n), float(dt), int(nsteps), infos)
    _check(st, "fas_heat_run")
    return [infos[k] for k in range(nsteps)]


def fas_heat_run_host(ctx: _Ctx, u0_host, uT_host, fsrc_host, dt: float, nsteps: int):
    """Host float64 arrays (numpy, C-contiguous; pinned memory copies fastest). uT_host may be u0_host."""
    import numpy as np
    n = ctx.cells
    for a, what in ((u0_host, "u0_host"), (uT_host, "uT_host"), (fsrc_host, "fsrc_host")):
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n):
            raise TypeError("%s must be a C-contiguous float64 array of %d elements" % (what, n))
    infos = (fas_info * max(nsteps, 1))()
    fptr = None if fsrc_host is None else fsrc_host.ctypes.data
    st = load().fas_heat_run_host(ctx.handle, u0_host.ctypes.data, uT_host.ctypes.data, fptr, float(dt),
                                  int(nsteps), infos)
    _check(st, "fas_heat_run_host")
    return [infos[k] for k in range(nsteps)]


def fas_fold_dirichlet(ctx: _Ctx, f, values) -> None:
    """f += 2 beta kappa g / h^2 next to every Dirichlet face with value g (values: 6 floats, x_lo ..
    z_hi; Neumann entries ignored)."""
    vals = (_D * 6)(*[float(v) for v in list(values) + [0.0] * (6 - len(values))])
    _check(load().fas_fold_dirichlet(ctx.handle, _dev(f, "f", ctx.cells), vals), "fas_fold_dirichlet")


def fas_residual(ctx: _Ctx, level: int, u, f, out=None) -> float:
    n = ctx.level_cells(level)
    norm = _D()
    _check(load().fas_residual(ctx.handle, level, _dev(u, "u", n), _dev(f, "f", n), _dev(out, "out", n),
                               ctypes.byref(norm)), "fas_residual")
    return norm.value


def fas_residual_ir(ctx: _Ctx, u, f, r32) -> float:
    """The mixed solve's refinement residual r32 = (float)(f - A u) on level 0 (float32 CUDA tensor)."""
    import torch
    n = ctx.cells
    if not isinstance(r32, torch.Tensor) or r32.dtype != torch.float32 or not r32.is_cuda or r32.numel() != n \
            or not r32.is_contiguous():
        raise TypeError("r32 must be a contiguous float32 CUDA tensor of %d elements" % n)
    nrm = _D(0.0)
    _check(load().fas_residual_ir(ctx.handle, _dev(u, "u", n), _dev(f, "f", n), r32.data_ptr(), ctypes.byref(nrm)),
           "fas_residual_ir")
    return nrm.value


def fas_selftest_conversions(count: int, seed: int = 1) -> int:
    """Mismatches between the integer float32<->float64 conversions and the hardware ones."""
    out = ctypes.c_longlong(0)
    _check(load().fas_selftest_conversions(int(count), int(seed), ctypes.byref(out)), "fas_selftest_conversions")
    return out.value


def fas_probe_fp64_rate() -> float:
    """Measured float64 FMA throughput of the current device in TFLOP/s (an FMA counts as two)."""
    out = ctypes.c_double(0.0)
    _check(load().fas_probe_fp64_rate(ctypes.byref(out)), "fas_probe_fp64_rate")
    return out.value


def fas_debug_bounded_wait(limit_ns: int, withhold_next: int = 0) -> None:
    """Deadline of the kernels' bounded waits, and the test hook that withholds one copy of the next
    launch of the 3D refinement residual (withhold_next 1) or of the fused 3D sweep (2); its waits then
    run out and the call reports FAS_ETIMEOUT."""
    _check(load().fas_debug_bounded_wait(int(limit_ns), int(withhold_next)), "fas_debug_bounded_wait")


def fas_smooth(ctx: _Ctx, level: int, u, f, sweeps: int) -> None:
    n = ctx.level_cells(level)
    _check(load().fas_smooth(ctx.handle, level, _dev(u, "u", n), _dev(f, "f", n), int(sweeps)), "fas_smooth")


def fas_restrict(ctx: _Ctx, level: int, u, uc) -> None:
    _check(load().fas_restrict(ctx.handle, level, _dev(u, "u", ctx.level_cells(level)),
                               _dev(uc, "uc", ctx.level_cells(level + 1))), "fas_restrict")


def fas_prolong_add(ctx: _Ctx, level: int, u, c) -> None:
    _check(load().fas_prolong_add(ctx.handle, level, _dev(u, "u", ctx.level_cells(level)),
                                  _dev(c, "c", ctx.level_cells(level + 1))), "fas_prolong_add")


def fas_vcycle_small_static(params: fas_params, u, f, ncycles: int, stream=None, want_res: bool = True):
    """ncycles V-cycles on a small grid with no device allocation (see include/fas.h); returns
    ||f - A u||_2 after the last cycle (None when want_res is False: the call does not wait)."""
    n = params.n[0] * params.n[1] * (params.n[2] if params.dim == 3 else 1)
    res = _D()
    st = load().fas_vcycle_small_static(ctypes.byref(params), _dev(u, "u", n), _dev(f, "f", n), int(ncycles),
                                        ctypes.byref(res) if want_res else None, _stream_handle(stream))
    _check(st, "fas_vcycle_small_static")
    return res.value if want_res else None


def fas_solve_batched(ctxs, us, fs, stream=None, allow_notconv=False):
    """Solve independent problems (one context each) in one graph launch; returns their fas_info."""
    n = len(ctxs)
    if not (len(us) == len(fs) == n) or n == 0:
        raise ValueError("need equal, non-empty lists of contexts, u and f")
    harr = (_P * n)(*[c.handle for c in ctxs])
    uarr = (_P * n)(*[_dev(u, "u", c.cells) for c, u in zip(ctxs, us)])
    farr = (_P * n)(*[_dev(f, "f", c.cells) for c, f in zip(ctxs, fs)])
    infos = (fas_info * n)()
    st = load().fas_solve_batched(harr, n, uarr, farr, infos, _stream_handle(stream))
    if not (allow_notconv and st == FAS_ENOTCONV):
        _check(st, "fas_solve_batched")
    return [infos[k] for k in range(n)]


def fas_heat_adjoint(ctx: _Ctx, u0, fsrc, dt: float, nsteps: int, dL_duT, uT=None, g_u0=None, g_f=None,
                     g_kappa=None, ckpt_every: int = 10) -> None:
    """Gradients of a loss of the final heat state (see include/fas.h); outputs written in place."""
    n = ctx.cells
    _check(load().fas_heat_adjoint(ctx.handle, _dev(u0, "u0", n), _dev(fsrc, "fsrc", n), float(dt), int(nsteps),
                                   _dev(dL_duT, "dL_duT", n), _dev(uT, "uT", n), _dev(g_u0, "g_u0", n),
                                   _dev(g_f, "g_f", n), _dev(g_kappa, "g_kappa", n), int(ckpt_every)),
           "fas_heat_adjoint")


def fas_autotune(ctx: _Ctx, u_scratch, f) -> dict:
    """Choose the context's launch parameters by timing whole solves (cached per size class)."""
    out = fas_tune_result()
    _check(load().fas_autotune(ctx.handle, _dev(u_scratch, "u_scratch", ctx.cells), _dev(f, "f", ctx.cells),
                               ctypes.byref(out)), "fas_autotune")
    ctx.params.inner_cycles = out.inner_cycles
    ctx.params.seg_rows = out.seg_rows
    return out.as_dict()


def fas_launch_count(ctx: _Ctx, reset: bool = False) -> int:
    return load().fas_launch_count(ctx.handle, 1 if reset else 0)


class _NsCtx:
    """Owns an ns_ctx* (projection step on the MAC grid) and its grid shape (numpy order)."""

    def __init__(self, handle, shape):
        self.handle = handle
        self.shape = tuple(shape)
        self.cells = 1
        for v in shape:
            self.cells *= int(v)

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.ns_destroy(self.handle)
            self.handle = None


NS_FIELDS = ("U_new", "U_old", "V_new", "V_old", "W_new", "W_old", "P_new", "P_old")


def ns_create(shape, h: float, Re: float, dt: float, lid=(1.0, 0.0, 0.0), order: int = 1, solver=None,
              pressure=None, stream=None) -> _NsCtx:
    """ns_create for a numpy-order shape ((ny, nx) or (nz, ny, nx)); solver / pressure are fas_params
    (None: the library's defaults)."""
    lib = load()
    dim = len(shape)
    phys = list(reversed([int(v) for v in shape])) + [1] * (3 - dim)
    n = (_I * 3)(*phys)
    lid3 = (_D * 3)(*(list(lid) + [0.0] * 3)[:3])
    out = _P()
    sp = ctypes.byref(solver) if solver is not None else None
    pp = ctypes.byref(pressure) if pressure is not None else None
    _check(lib.ns_create(dim, n, float(h), float(Re), float(dt), int(order), lid3, sp, pp, _stream_handle(stream),
                         ctypes.byref(out)), "ns_create")
    return _NsCtx(out, shape)


def ns_projection_step(ns: _NsCtx, fields: dict, want_div: bool = True, allow_notconv: bool = False, force=None):
    """One projection step on the eight resident fields (dict of float64 CUDA tensors named as in
    NS_FIELDS; W_* absent in 2D); force: optional list of per-component body-force tensors at t^{n+1}.
    Returns (infos[4], max |div u^{n+1}| or None)."""
    n = ns.cells
    ptrs = (_P * 8)(*[_dev(fields.get(k), k, n) for k in NS_FIELDS])
    fptr = None
    if force is not None:
        fl = list(force) + [None] * (3 - len(force))
        fptr = (_P * 3)(*[_dev(t, "force", n) for t in fl[:3]])
    infos = (fas_info * 4)()
    dmax = _D(0.0)
    st = load().ns_projection_step(ns.handle, ptrs, fptr, infos, ctypes.byref(dmax) if want_div else None)
    if not (allow_notconv and st == FAS_ENOTCONV):
        _check(st, "ns_projection_step")
    return [infos[k] for k in range(4)], (dmax.value if want_div else None)


def ns_launch_count(ns: _NsCtx, reset: bool = False) -> int:
    return int(load().ns_launch_count(ns.handle, 1 if reset else 0))


def ns_destroy(ns: _NsCtx) -> None:
    if ns.handle:
        _check(load().ns_destroy(ns.handle), "ns_destroy")
        ns.handle = None


class _GgCtx:
    """Owns a gg_ctx* (grain-growth step), its grid shape (numpy order) and q."""

    def __init__(self, handle, shape, q):
        self.handle = handle
        self.shape = tuple(shape)
        self.q = int(q)
        self.cells = 1
        for v in shape:
            self.cells *= int(v)

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.gg_destroy(self.handle)
            self.handle = None


def gg_create(shape, h: float, dt: float, q: int, model=None, solver=None, batch: int = 0, stream=None) -> _GgCtx:
    """gg_create for a numpy-order periodic grid shape; model: gg_model or a dict of its fields (None:
    the paper's constants); solver: fas_params (None: the library's defaults)."""
    lib = load()
    dim = len(shape)
    phys = list(reversed([int(v) for v in shape])) + [1] * (3 - dim)
    n = (_I * 3)(*phys)
    if isinstance(model, dict):
        model = gg_model(**model)
    out = _P()
    _check(lib.gg_create(dim, n, float(h), float(dt), int(q), ctypes.byref(model) if model is not None else None,
                         ctypes.byref(solver) if solver is not None else None, int(batch), _stream_handle(stream),
                         ctypes.byref(out)), "gg_create")
    return _GgCtx(out, shape, q)


def gg_step(gg: _GgCtx, eta, allow_notconv: bool = False):
    """One grain-growth step in place on eta (float64 CUDA tensor of shape (q,) + grid); returns the
    q solver reports."""
    infos = (fas_info * gg.q)()
    st = load().gg_step(gg.handle, _dev(eta, "eta", gg.q * gg.cells), infos)
    if not (allow_notconv and st == FAS_ENOTCONV):
        _check(st, "gg_step")
    return [infos[k] for k in range(gg.q)]


def gg_rhs(gg: _GgCtx, eta, rhs) -> None:
    """The q right-hand sides of the step from eta (both float64 CUDA tensors of shape (q,) + grid)."""
    n = gg.q * gg.cells
    _check(load().gg_rhs(gg.handle, _dev(eta, "eta", n), _dev(rhs, "rhs", n)), "gg_rhs")


def gg_destroy(gg: _GgCtx) -> None:
    if gg.handle:
        _check(load().gg_destroy(gg.handle), "gg_destroy")
        gg.handle = None


class fas_prof_record(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("level", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("units", ctypes.c_double)]


FAMILIES = ["smooth", "residual", "restrict", "tau", "prolong", "coarse", "ir", "norm", "other", "update"]


def fas_prof_enable(ctx: _Ctx, on: bool = True) -> None:
    _check(load().fas_prof_enable(ctx.handle, 1 if on else 0), "fas_prof_enable")


def fas_prof_read(ctx: _Ctx):
    """Aggregated kernel timings: list of dicts (family, level, launches, ms, units)."""
    cap = 256
    buf = (fas_prof_record * cap)()
    cnt = _I()
    _check(load().fas_prof_read(ctx.handle, buf, cap, ctypes.byref(cnt)), "fas_prof_read")
    out = []
    for k in range(min(cnt.value, cap)):
        r = buf[k]
        out.append(dict(family=FAMILIES[r.family] if 0 <= r.family < len(FAMILIES) else r.family,
                        level=r.level, launches=r.launches, ms=r.ms, units=r.units))
    return out


def make_params(shape, h, alpha=1.0, beta=1.0, kappa_const=1.0, bc=None, **kw) -> fas_params:
    """fas_params for a numpy-order shape ((ny, nx) or (nz, ny, nx)); keyword overrides by field."""
    p = fas_default_params()
    dim = len(shape)
    p.dim = dim
    phys = list(reversed(shape)) + [1] * (3 - dim)
    for a in range(3):
        p.n[a] = int(phys[a])
    p.h = float(h)
    p.alpha = float(alpha)
    p.beta = float(beta)
    p.kappa_const = float(kappa_const)
    if bc is not None:
        for k, v in enumerate(bc):
            p.bc[k] = int(v)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError("fas_params has no field %s" % k)
        setattr(p, k, v)
    return p


def solve(u, f, h, kappa=None, stream=None, allow_notconv=False, **params) -> fas_info:
    """One call: A u = f (A u = alpha u - beta div(kappa grad u)) on the grid of u's shape, solved in
    place from u's current values to the tolerance; params are fas_params fields (alpha, beta, bc,
    precision, tol, ...). Creates and frees a context; keep a Solver for repeated solves."""
    ctx = fas_create(make_params(tuple(u.shape), h, **params), stream=stream, kappa=kappa)
    try:
        return fas_solve(ctx, u, f, allow_notconv=allow_notconv)
    finally:
        fas_destroy(ctx)


def __getattr__(name):
    if name == "HeatSolve":  # the autograd Function, imported on first use
        from .autograd import HeatSolve
        return HeatSolve
    raise AttributeError("module %r has no attribute %r" % (__name__, name))


class Solver:
    """Convenience owner of a context: Solver(shape, h, ...).solve(u, f)."""

    def __init__(self, shape, h, kappa=None, stream=None, **kw):
        self.shape = tuple(shape)
        self.ctx = fas_create(make_params(self.shape, h, **kw), stream=stream, kappa=kappa)

    def vcycle(self, u, f):
        return fas_vcycle(self.ctx, u, f)

    def solve(self, u, f, allow_notconv=False):
        return fas_solve(self.ctx, u, f, allow_notconv=allow_notconv)

    def heat_run(self, u, fsrc, dt, nsteps):
        return fas_heat_run(self.ctx, u, fsrc, dt, nsteps)

    @property
    def levels(self):
        return fas_num_levels(self.ctx)

    def close(self):
        fas_destroy(self.ctx)
