"""torch.autograd.Function wrappers around the library's forward and adjoint sweeps.

``UnrolledSweeps.apply(w, alpha, x0, ctx)`` runs K checkpointed sweeps of the NAG
form of Table 1 (at = alpha) in the library and returns x_K; its backward calls the
library's adjoint sweep (A symmetric, so the same stencil runs in reverse) and
returns dL/dw, dL/dalpha and dL/dx0. ``LogResidualLoss.apply(x, ctx)`` is the log
form of eq. 15 with its gradient from the library. Both take padded buffers (the
layout of include/richm.h) and [batch][m] coefficient tensors.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import richm


@dataclass
class SweepContext:
    op: richm.Operator
    b: torch.Tensor          # padded right-hand side
    dtype: int = richm.F32
    m: int = 16
    K: int = 64
    every: int = 8
    precond: int = 0
    relax: float = 1.0       # SSOR relaxation factor (precond 2)


class UnrolledSweeps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, alpha, x0, sc: SweepContext):
        op = sc.op
        ck = torch.empty(op.checkpoint_elems(sc.K, sc.every), dtype=richm.TORCH_DTYPE[sc.dtype], device="cuda")
        xK = op.zeros(sc.dtype)
        w = w.contiguous()
        alpha = alpha.contiguous()
        op.forward_checkpointed(sc.dtype, x0.contiguous(), sc.b, w, alpha, None, sc.m, sc.K, sc.every, sc.precond,
                                ck, xK, relax=sc.relax)
        ctx.save_for_backward(w, alpha, ck)
        ctx.sc = sc
        return xK

    @staticmethod
    def backward(ctx, gK):
        w, alpha, ck = ctx.saved_tensors
        sc = ctx.sc
        gw = torch.zeros_like(w)
        ga = torch.zeros_like(alpha)
        gx0 = sc.op.zeros(sc.dtype)
        sc.op.sweeps_adjoint(sc.dtype, ck, sc.every, sc.b, gK.contiguous(), w, alpha, None, sc.m, sc.K, sc.precond,
                             gw, ga, None, gx0, relax=sc.relax)
        return gw, ga, gx0, None


class LogResidualLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, sc: SweepContext):
        g = sc.op.zeros(sc.dtype)
        loss = sc.op.loss_log_residual(sc.dtype, x.contiguous(), sc.b, g)
        ctx.save_for_backward(g)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return g * gout.to(g.dtype), None
