"""torch.autograd.Function around the row reduction and its backward kernels.

``reduce(x, op, dim=-1)`` reduces along one dimension of a float32/float64 CUDA
tensor with op in {sum, max, min, prod}.  The forward runs pr_reduce_axis on the
tensor as it lies in memory ([outer, n, inner] around the reduced dimension; the
last dimension is pr_reduce_rows) and keeps what the backward needs (the first
arg-extremum index for max/min; the product of the non-zero elements, the zero
count and the first zero's index for prod); the backward runs
pr_reduce_axis_backward.  Gradient conventions:
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

    def __init__(self, *shape):
        self.shape = tuple(shape)

    def data_ptr(self):
        return 0


class AxisReduce(torch.autograd.Function):
    """Reduction of one dimension of a contiguous tensor, in place in memory."""

    @staticmethod
    def forward(ctx, x, op, dim):
        if op in ("max", "min"):
            out, ai = pr.reduce_axis(x, op, dim, argidx=True)
            ctx.save_for_backward(ai)
        elif op == "prod":
            out, ax = pr.reduce_axis(x, op, dim, aux=True)
            ctx.save_for_backward(x, ax)
        elif op == "sum":
            out = pr.reduce_axis(x, op, dim)
        else:
            raise ValueError("differentiable ops are sum, max, min and prod")
        ctx.op = op
        ctx.dim = dim
        ctx.shape = tuple(x.shape)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        op = ctx.op
        g = grad_out.contiguous()
        if op in ("max", "min"):
            (ai,) = ctx.saved_tensors
            gi = pr.reduce_axis_backward(op, _Shape(*ctx.shape), ctx.dim, g, argidx=ai)
        elif op == "prod":
            x, ax = ctx.saved_tensors
            gi = pr.reduce_axis_backward(op, x, ctx.dim, g, aux=ax)
        else:
            gi = pr.reduce_axis_backward(op, _Shape(*ctx.shape), ctx.dim, g)
        return gi, None, None


def reduce(x: torch.Tensor, op: str, dim: int = -1) -> torch.Tensor:
    """Differentiable reduction of x along `dim` (float32 / float64 CUDA tensors)."""
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("differentiable reductions support float32 and float64")
    if x.dim() == 0:
        raise ValueError("reduce needs at least one dimension")
    dim = dim % x.dim()
    return AxisReduce.apply(x.contiguous(), op, dim)
