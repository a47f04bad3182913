"""torch.autograd.Function for W^K(b): K unrolled iterations as a function of the
pinned positions b, differentiated by the library's hand-written adjoint.

Argument marshalling only; the forward pass is ffa_forward_unrolled and the
backward pass is ffa_backward_unrolled.
"""
from __future__ import annotations

import torch


class UnrolledSolve(torch.autograd.Function):
    """W^K = Phi^K(b): set the pins to b, init from W0, run K iterations."""

    @staticmethod
    def forward(ctx, b, solver, W0, K: int, ckpt_every: int):
        b = b.detach().to(torch.float64).contiguous()
        solver.set_handles(b)
        solver.init(W0)
        solver.forward_unrolled(K, ckpt_every)
        W = torch.empty((solver.n, solver.d), dtype=torch.float64, device=b.device)
        solver.W(W)
        ctx.solver = solver
        ctx.b_shape = tuple(b.shape)
        ctx.b_device = b.device
        return W

    @staticmethod
    def backward(ctx, gW):
        gb = torch.empty(ctx.b_shape, dtype=torch.float64, device=ctx.b_device)
        ctx.solver.backward_unrolled(gW.detach().to(torch.float64).contiguous(), gb)
        return gb, None, None, None, None


def unrolled_solve(b, solver, W0, K: int, ckpt_every: int = 20):
    return UnrolledSolve.apply(b, solver, W0, K, ckpt_every)
