"""torch.autograd.Functions around the library's Newton–Schulz S^-1/2 and the CLR product,
with their hand-written adjoints (clr_sqrt_inv / clr_sqrt_inv_backward, clr_multiply /
clr_multiply_backward).  Argument marshalling only: the forward and backward passes run in the
library's kernels."""
from __future__ import annotations

import torch

from .clr import CLR_ENOCONV, ClrError, Context


class ClrSqrtInv(torch.autograd.Function):
    """Z = S^-1/2 for a dense float64 CUDA tensor S, computed in CLR form with the given
    clusters; the backward pass runs the NS recurrences in reverse over the checkpointed
    iterates (alpha constant, truncation straight-through)."""

    @staticmethod
    def forward(fctx, s, ctx: Context, sizes, eps_lr: float, drop_norm: float):
        smat = ctx.from_dense(s.detach().contiguous(), sizes, eps_lr=eps_lr, drop_norm=drop_norm)
        # the iteration must stop on its proxy ||X - I||; a residual held above the tolerance
        # by truncation at eps_lr is reported in the stats (fctx.stats) but does not stop the
        # forward pass
        z, stats, tape = ctx.sqrt_inv(smat, keep_tape=True, allow_noconv=True)
        if stats["status"] == CLR_ENOCONV and not stats["proxy_met"]:
            raise ClrError(CLR_ENOCONV, "Newton-Schulz did not reach ns_tol")
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


class ClrMultiply(torch.autograd.Function):
    """C = A B for dense float64 CUDA tensors A (row_sizes x inner_sizes clusters) and B
    (inner_sizes x col_sizes), held in CLR form built at eps_lr and multiplied by the library's
    CLR product (Section 4.1; the context's eps_lr and precision apply to the product).  The
    backward pass is the product's adjoint (clr_multiply_backward): Abar = Cbar B^T and
    Bbar = A^T Cbar as CLR products, the truncations treated as the identity."""

    @staticmethod
    def forward(fctx, a, b, ctx: Context, row_sizes, inner_sizes, col_sizes, eps_lr: float):
        am = ctx.from_dense(a.detach().contiguous(), row_sizes, inner_sizes, eps_lr=eps_lr)
        bm = ctx.from_dense(b.detach().contiguous(), inner_sizes, col_sizes, eps_lr=eps_lr)
        cm = ctx.zeros(row_sizes, col_sizes)
        ctx.multiply_into(am, bm, cm)
        out = torch.empty((a.shape[0], b.shape[1]), dtype=a.dtype, device=a.device)
        cm.to_dense(out)
        fctx.clr = (ctx, am, bm, list(row_sizes), list(col_sizes), eps_lr)
        return out

    @staticmethod
    def backward(fctx, grad):
        ctx, am, bm, rs, cs, eps_lr = fctx.clr
        gm = ctx.from_dense(grad.detach().contiguous(), rs, cs, eps_lr=eps_lr)
        need_a, need_b = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
        abar, bbar = ctx.multiply_backward(am, bm, gm, need_a=need_a, need_b=need_b)
        ga = gb = None
        if abar is not None:
            ga = torch.empty(abar.shape, dtype=grad.dtype, device=grad.device)
            abar.to_dense(ga)
        if bbar is not None:
            gb = torch.empty(bbar.shape, dtype=grad.dtype, device=grad.device)
            bbar.to_dense(gb)
        return ga, gb, None, None, None, None, None


def multiply(a, b, ctx: Context, row_sizes, inner_sizes=None, col_sizes=None,
             eps_lr: float = 1e-8):
    inner_sizes = row_sizes if inner_sizes is None else inner_sizes
    col_sizes = inner_sizes if col_sizes is None else col_sizes
    return ClrMultiply.apply(a, b, ctx, row_sizes, inner_sizes, col_sizes, eps_lr)
