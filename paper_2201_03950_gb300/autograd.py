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
adjoint solves.  On a CUDA device both directions are captured once per
(dims, lam, nsteps, every, dtype, device) into CUDA graphs and replayed: a
call copies its inputs into the graphs' buffers, replays, and returns copies
of the outputs (the checkpoints included, so interleaved forward and backward
calls stay independent).  ``graphs=False`` runs the library calls directly.
"""
from __future__ import annotations

from collections import OrderedDict

import torch

from . import trid

_GRAPH_CACHE: "OrderedDict[tuple, _ADIGraphs]" = OrderedDict()
_GRAPH_CACHE_MAX = 2


class _ADIGraphs:
    """Forward and backward of adi2d captured for one problem shape."""

    def __init__(self, dims, lam, nsteps, every, dtype, device):
        n = dims[0] * dims[1]
        self.u0 = torch.zeros(n, dtype=dtype, device=device)
        self.k = torch.ones(n, dtype=dtype, device=device)
        self.g = torch.zeros(n, dtype=dtype, device=device)
        self.ck_in = torch.empty(trid.adi2v_checkpoint_bytes(dims, nsteps, every, dtype),
                                 dtype=torch.uint8, device=device)
        self.ws = torch.empty(trid.adi2v_workspace_bytes(dims, nsteps, every, dtype),
                              dtype=torch.uint8, device=device)
        args = (dims, lam, nsteps, every)
        # one direct call first: the library's per-device set-up is not capturable
        uT, ck = trid.adi2v_forward(self.u0, self.k, *args, workspace=self.ws)
        trid.adi2v_backward(self.g, self.k, *args, ck, workspace=self.ws)
        torch.cuda.current_stream().synchronize()
        self.fwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.fwd):
            self.uT, self.ck = trid.adi2v_forward(self.u0, self.k, *args, workspace=self.ws,
                                                  stream=torch.cuda.current_stream())
        self.bwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.bwd):
            self.gu, self.gk, _ = trid.adi2v_backward(self.g, self.k, *args, self.ck_in,
                                                      workspace=self.ws,
                                                      stream=torch.cuda.current_stream())

    def forward(self, u0, kappa):
        self.u0.copy_(u0.reshape(-1))
        self.k.copy_(kappa.reshape(-1))
        self.fwd.replay()
        return self.uT.clone().view_as(u0), self.ck.clone()

    def backward(self, g_uT, kappa, ckpt):
        self.g.copy_(g_uT.reshape(-1))
        self.k.copy_(kappa.reshape(-1))
        self.ck_in.copy_(ckpt)
        self.bwd.replay()
        return self.gu.clone(), self.gk.clone()


def _graphs_for(dims, lam, nsteps, every, dtype, device):
    key = (dims, lam, nsteps, every, dtype, device)
    g = _GRAPH_CACHE.get(key)
    if g is None:
        g = _ADIGraphs(dims, lam, nsteps, every, dtype, device)
        _GRAPH_CACHE[key] = g
        while len(_GRAPH_CACHE) > _GRAPH_CACHE_MAX:
            _GRAPH_CACHE.popitem(last=False)
    else:
        _GRAPH_CACHE.move_to_end(key)
    return g


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
    def forward(ctx, u0, kappa, dims, lam, nsteps, every, graphs=True):
        u0c = u0.detach().contiguous()
        kc = kappa.detach().contiguous()
        args = (tuple(int(v) for v in dims), float(lam), int(nsteps), int(every))
        gr = None
        if graphs and u0c.is_cuda and args[2] > 0:
            gr = _graphs_for(*args, u0c.dtype, u0c.device)
            uT, ckpt = gr.forward(u0c, kc)
        else:
            uT, ckpt = trid.adi2v_forward(u0c, kc, *args)
        ctx.save_for_backward(kc)
        ctx.ckpt = ckpt
        ctx.graphs = gr
        ctx.args = args
        return uT

    @staticmethod
    def backward(ctx, g_uT):
        (kc,) = ctx.saved_tensors
        dims, lam, nsteps, every = ctx.args
        g = g_uT.contiguous()
        if ctx.graphs is not None:
            g_u0, g_k = ctx.graphs.backward(g, kc, ctx.ckpt)
            g_u0, g_k = g_u0.view_as(g), g_k.view_as(g)
        else:
            g_u0, g_k, _ = trid.adi2v_backward(g, kc, dims, lam, nsteps, every, ctx.ckpt)
        need = ctx.needs_input_grad
        return (g_u0 if need[0] else None, g_k if need[1] else None, None, None, None, None, None)


def adi2d(u0, kappa, dims, lam: float, nsteps: int, every: int = 10, graphs: bool = True):
    """u after ``nsteps`` 2D ADI steps with diffusivity field ``kappa``."""
    return DiffADI2D.apply(u0, kappa, dims, lam, nsteps, every, graphs)
