"""Differentiable batched solve: ``tridiag_solve(a, b, c, d, dims, solve_dim)``
returns x = A^{-1} d along one mesh axis and back-propagates through the
library's adjoint kernel (trid_solve_batch_adjoint): g_d = A^{-T} g_x and
g_a_i = -g_d_i x_{i-1}, g_b_i = -g_d_i x_i, g_c_i = -g_d_i x_{i+1}.  Entries that
are not part of A (a on each system's first row, c on its last) get zero
gradient.  Both directions run in the CUDA library; torch only supplies
memory, the stream and the autograd graph.
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
