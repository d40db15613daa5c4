"""Differentiable operations of the library.

``tridiag_solve(a, b, c, d, dims, solve_dim)``
returns x = A^{-1} d along one mesh axis and back-propagates through the
library's adjoint kernel (trid_solve_batch_adjoint): g_d = A^{-T} g_x and
g_a_i = -g_d_i x_{i-1}, g_b_i = -g_d_i x_i, g_c_i = -g_d_i x_{i+1}.  Entries that
are not part of A (a on each system's first row, c on its last) get zero
gradient.  Both directions run in the CUDA library; torch only supplies
memory, the stream and the autograd graph.

``adi2d(u0, kappa, dims, lam, nsteps, every)`` runs the 2D ADI heat step with
a diffusivity field (adi2v_forward) and back-propagates to u0 and kappa with
adi2v_backward: the forward keeps u every ``every`` steps, the backward
recomputes each segment from its checkpoint and runs it in reverse with the
adjoint solves.
"""
from __future__ import annotations

import torch

from . import trid


class TridSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, c, d, dims, solve_dim):
        x = d.detach().clone()
        trid.solve(a.detach(), b.detach(), c.detach(), x, dims, solve_dim)
        ctx.save_for_backward(a, b, c, x)
        ctx.dims = tuple(int(v) for v in dims)
        ctx.solve_dim = int(solve_dim)
        return x

    @staticmethod
    def backward(ctx, gx):
        a, b, c, x = ctx.saved_tensors
        need = ctx.needs_input_grad
        ga, gb, gc, gd = trid.adjoint(a.detach(), b.detach(), c.detach(), x,
                                      gx.contiguous(), ctx.dims, ctx.solve_dim,
                                      need_coef_grads=any(need[:3]))
        return (ga if need[0] else None, gb if need[1] else None, gc if need[2] else None,
                gd if need[3] else None, None, None)


def tridiag_solve(a, b, c, d, dims, solve_dim: int):
    """x = A^{-1} d along ``solve_dim`` of the column-major mesh ``dims``."""
    return TridSolve.apply(a, b, c, d, dims, solve_dim)


class DiffADI2D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kappa, dims, lam, nsteps, every):
        u0c = u0.detach().contiguous()
        kc = kappa.detach().contiguous()
        uT, ckpt = trid.adi2v_forward(u0c, kc, dims, lam, nsteps, every)
        ctx.save_for_backward(kc)
        ctx.ckpt = ckpt
        ctx.args = (tuple(int(v) for v in dims), float(lam), int(nsteps), int(every))
        return uT

    @staticmethod
    def backward(ctx, g_uT):
        (kc,) = ctx.saved_tensors
        dims, lam, nsteps, every = ctx.args
        g_u0, g_k, _ = trid.adi2v_backward(g_uT.contiguous(), kc, dims, lam, nsteps, every,
                                           ctx.ckpt)
        need = ctx.needs_input_grad
        return (g_u0 if need[0] else None, g_k if need[1] else None, None, None, None, None)


def adi2d(u0, kappa, dims, lam: float, nsteps: int, every: int = 10):
    """u after ``nsteps`` 2D ADI steps with diffusivity field ``kappa``."""
    return DiffADI2D.apply(u0, kappa, dims, lam, nsteps, every)
