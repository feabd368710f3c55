"""torch.autograd.Function over the library's heat run and its hand-written adjoint.

    uT = HeatSolve.apply(u0, fsrc, kappa, h, dt, nsteps)   # float64 CUDA tensors (ny, nx) / (nz, ny, nx)
    loss = ((uT - target) ** 2).sum(); loss.backward()      # gradients for u0, fsrc and kappa

Forward runs fas_heat_run; backward runs fas_heat_adjoint, which recomputes the forward states from
checkpoints kept every `ckpt_every` steps. Both are kernels of libfasmg.so; this module only passes
tensors across.
"""
from __future__ import annotations

import torch

from . import fas_create, fas_heat_adjoint, fas_heat_run, make_params


class HeatSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, fsrc, kappa, h, dt, nsteps, ckpt_every=10, options=None):
        opts = dict(options or {})
        params = make_params(tuple(u0.shape), h, alpha=1.0, beta=dt, **opts)
        fctx = fas_create(params, kappa=kappa.detach().contiguous())
        uT = u0.detach().clone().contiguous()
        f = None if fsrc is None else fsrc.detach().contiguous()
        fas_heat_run(fctx, uT, f, dt, nsteps)
        ctx.fctx = fctx
        ctx.meta = (dt, nsteps, ckpt_every)
        ctx.has_f = fsrc is not None
        ctx.save_for_backward(u0, fsrc if fsrc is not None else u0, kappa)
        return uT

    @staticmethod
    def backward(ctx, grad_uT):
        u0, fsrc, kappa = ctx.saved_tensors
        dt, nsteps, ckpt_every = ctx.meta
        g_u0 = torch.empty_like(u0)
        g_f = torch.empty_like(u0)
        g_k = torch.empty_like(kappa)
        fas_heat_adjoint(ctx.fctx, u0.detach().contiguous(), fsrc.detach().contiguous() if ctx.has_f else None,
                         dt, nsteps, grad_uT.detach().contiguous(), None, g_u0, g_f, g_k, ckpt_every)
        return g_u0, (g_f if ctx.has_f else None), g_k, None, None, None, None, None
