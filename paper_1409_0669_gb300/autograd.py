"""Differentiable forms of the products, as torch.autograd.Functions whose
forward and backward both run in this library's kernels.

  y = gemv(A, x)          dA = dy x^T (dense_outer), dx = A^T dy (the
                          column-major GEMV kernel on A's row-major storage)
  y = spmv(csr, vals, x)  dvals = dy[row] * x[col] on the pattern
                          (csr_sampled_outer), dx = A^T dy as a CSR product on
                          the transpose, computed once per pattern by
                          csr_transpose (no atomics in the product)
  s = dot(x, y)           dx = ds * y, dy = ds * x (vec_scale_dev: ds stays
                          on the device)
"""
from __future__ import annotations

import torch

from . import (csr_sampled_outer, csr_spmv, csr_transpose, dense_gemv, dense_outer, vec_dot,
               vec_gather, vec_scale_dev)


class CsrPattern:
    """Row pointers and column indices of an m-by-n CSR matrix (int32, on the
    device), with its transpose computed on first use and kept."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, n_cols: int):
        self.row_ptr, self.col_idx, self.n_cols = row_ptr, col_idx, int(n_cols)
        self.m = row_ptr.numel() - 1
        self._t = None

    def transpose(self):
        if self._t is None:
            self._t = csr_transpose(self.row_ptr, self.col_idx, self.n_cols)
        return self._t


class _Gemv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, x):
        ctx.save_for_backward(A, x)
        return dense_gemv(A, x)

    @staticmethod
    def backward(ctx, dy):
        A, x = ctx.saved_tensors
        dy = dy.contiguous()
        dA = dx = None
        if ctx.needs_input_grad[0]:
            dA = dense_outer(dy, x)
        if ctx.needs_input_grad[1]:
            dx = dense_gemv(A.t(), dy)          # A^T dy: same storage, other layout
        return dA, dx


class _Spmv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, x, pattern: CsrPattern):
        ctx.pattern = pattern
        ctx.save_for_backward(vals, x)
        return csr_spmv(pattern.row_ptr, pattern.col_idx, vals, x, n_cols=pattern.n_cols)

    @staticmethod
    def backward(ctx, dy):
        vals, x = ctx.saved_tensors
        p = ctx.pattern
        dy = dy.contiguous()
        dvals = dx = None
        if ctx.needs_input_grad[0]:
            dvals = csr_sampled_outer(p.row_ptr, p.col_idx, dy, x)
        if ctx.needs_input_grad[1]:
            col_ptr, row_idx, perm = p.transpose()
            vals_t = vec_gather(vals, perm)
            dx = csr_spmv(col_ptr, row_idx, vals_t, dy, n_cols=p.m)
        return dvals, dx, None


class _Dot(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y):
        ctx.save_for_backward(x, y)
        return vec_dot(x, y).reshape(())

    @staticmethod
    def backward(ctx, ds):
        x, y = ctx.saved_tensors
        ds = ds.reshape(1).contiguous()
        if ds.dtype != (torch.float64 if x.dtype == torch.float64 else torch.float32):
            ds = ds.to(torch.float64 if x.dtype == torch.float64 else torch.float32)
        dx = vec_scale_dev(y, ds) if ctx.needs_input_grad[0] else None
        dy = vec_scale_dev(x, ds) if ctx.needs_input_grad[1] else None
        return dx, dy


def gemv(A: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """y = A x (A row-major 2-D), differentiable in A and x."""
    return _Gemv.apply(A, x)


def spmv(pattern: CsrPattern, vals: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """y = A x for the CSR matrix (pattern, vals), differentiable in vals and x."""
    return _Spmv.apply(vals, x, pattern)


def dot(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """s = <x, y> as a 0-d tensor (float32 for FP32/BF16/FP16, float64 for FP64),
    differentiable in x and y."""
    return _Dot.apply(x, y)
