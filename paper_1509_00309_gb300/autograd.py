"""torch.autograd.Function around the library's Newton–Schulz S^-1/2 and its hand-written
adjoint (clr_sqrt_inv / clr_sqrt_inv_backward).  Argument marshalling only: the forward and
backward passes run in the library's kernels."""
from __future__ import annotations

import torch

from .clr import Context


class ClrSqrtInv(torch.autograd.Function):
    """Z = S^-1/2 for a dense float64 CUDA tensor S, computed in CLR form with the given
    clusters; the backward pass runs the NS recurrences in reverse over the checkpointed
    iterates (alpha constant, truncation straight-through)."""

    @staticmethod
    def forward(fctx, s, ctx: Context, sizes, eps_lr: float, drop_norm: float):
        smat = ctx.from_dense(s.detach().contiguous(), sizes, eps_lr=eps_lr, drop_norm=drop_norm)
        z, stats, tape = ctx.sqrt_inv(smat, keep_tape=True)
        out = torch.empty_like(s)
        z.to_dense(out)
        fctx.clr = (ctx, smat, tape, list(sizes), eps_lr)
        fctx.stats = stats
        return out

    @staticmethod
    def backward(fctx, grad):
        ctx, smat, tape, sizes, eps_lr = fctx.clr
        zb = ctx.from_dense(grad.detach().contiguous(), sizes, eps_lr=eps_lr)
        sb = ctx.sqrt_inv_backward(tape, zb)
        out = torch.empty_like(grad)
        sb.to_dense(out)
        return out, None, None, None, None


def sqrt_inv(s, ctx: Context, sizes, eps_lr: float = 1e-8, drop_norm: float = 0.0):
    return ClrSqrtInv.apply(s, ctx, sizes, eps_lr, drop_norm)
