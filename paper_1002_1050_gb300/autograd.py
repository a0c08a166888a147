"""torch.autograd wrappers of the library's forward and adjoint kernels.

conv_sum(a, b, beta)  -> C, differentiable in a, b (complex128) and beta (float64);
d_table(beta, ...)    -> d, differentiable in beta.
Both backward passes call the library's adjoint kernels (chains recomputed on the GPU,
no table stored); PyTorch only supplies memory, streams and the autograd graph.
"""
from __future__ import annotations

import torch

from . import wigner as W


class WignerConvSum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, beta, form="fp64"):
        C = W.wigner_conv_sum(beta.contiguous(), a.contiguous(), b.contiguous(), form=form)
        ctx.save_for_backward(a, b, beta, C)
        return C

    @staticmethod
    def backward(ctx, grad_c):
        a, b, beta, C = ctx.saved_tensors
        need_a, need_b, need_beta = ctx.needs_input_grad[:3]
        ga, gb, gbeta = W.wigner_conv_sum_backward(beta.contiguous(), a.contiguous(), b.contiguous(),
                                                   C if need_beta else None, grad_c.contiguous(),
                                                   need_a=need_a, need_b=need_b, need_beta=need_beta)
        return ga, gb, gbeta, None


class WignerDTable(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, l_max, mb_max, ms_max, form="fp64"):
        d = W.wigner_d_table(beta.contiguous(), l_max, mb_max, ms_max, form=form)
        ctx.save_for_backward(beta)
        ctx.orders = (l_max, mb_max, ms_max)
        return d

    @staticmethod
    def backward(ctx, grad_d):
        (beta,) = ctx.saved_tensors
        l_max, mb_max, ms_max = ctx.orders
        g = W.wigner_d_table_backward(beta.contiguous(), grad_d.contiguous(), l_max, mb_max, ms_max)
        return g, None, None, None, None


def conv_sum(a: torch.Tensor, b: torch.Tensor, beta: torch.Tensor, form: str = "fp64") -> torch.Tensor:
    """C[mb][ms][j] = sum_l conj(b[l][mb]) a[l][ms] d^l_{mb,ms}(beta_j), differentiable."""
    return WignerConvSum.apply(a, b, beta, form)


def d_table(beta: torch.Tensor, l_max: int, mb_max: int, ms_max: int, form: str = "fp64") -> torch.Tensor:
    """d[mb][ms][l][j], differentiable in beta."""
    return WignerDTable.apply(beta, l_max, mb_max, ms_max, form)
