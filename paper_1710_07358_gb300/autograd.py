"""torch.autograd.Function around the row reduction and its backward kernels.

``reduce(x, op, dim=-1)`` reduces along one dimension of a float32/float64 CUDA
tensor with op in {sum, max, min, prod}.  The forward runs pr_reduce_rows and
keeps what the backward needs (the first arg-extremum index for max/min; the
product of the non-zero elements, the zero count and the first zero's index for
prod); the backward runs pr_reduce_backward.  Gradient conventions:
  sum  -> grad_out broadcast;  max/min -> grad_out at the first arg-extremum;
  prod -> grad_out * prod_{j != i} x_j (zero-count aware, no division by zero).
"""
from __future__ import annotations

import torch

from . import pr


class RowReduce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x2d, op):
        if op in ("max", "min"):
            out, ai = pr.reduce_rows(x2d, op, argidx=True)
            ctx.save_for_backward(ai)
        elif op == "prod":
            out, ax = pr.reduce_rows(x2d, op, aux=True)
            ctx.save_for_backward(x2d, ax)
        elif op == "sum":
            out = pr.reduce_rows(x2d, op)
        else:
            raise ValueError("differentiable ops are sum, max, min and prod")
        ctx.op = op
        ctx.shape = x2d.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        op = ctx.op
        rows, cols = ctx.shape
        g = grad_out.contiguous()
        if op in ("max", "min"):
            (ai,) = ctx.saved_tensors
            gi = pr.reduce_backward(op, _Shape(rows, cols), g, argidx=ai)
        elif op == "prod":
            x2d, ax = ctx.saved_tensors
            gi = pr.reduce_backward(op, x2d, g, aux=ax)
        else:
            gi = pr.reduce_backward(op, _Shape(rows, cols), g)
        return gi, None


class _Shape:
    """Stands in for x where the backward needs only its shape."""

    def __init__(self, rows, cols):
        self.shape = (rows, cols)

    def data_ptr(self):
        return 0


def reduce(x: torch.Tensor, op: str, dim: int = -1) -> torch.Tensor:
    """Differentiable reduction of x along `dim` (float32 / float64 CUDA tensors)."""
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("differentiable reductions support float32 and float64")
    dim = dim % x.dim()
    xm = x.movedim(dim, -1)
    lead = xm.shape[:-1]
    x2d = xm.reshape(-1, xm.shape[-1]).contiguous()
    out = RowReduce.apply(x2d, op)
    return out.reshape(lead)
