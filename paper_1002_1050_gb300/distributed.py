"""Sharding the fused sum over GPUs (one process per GPU).

The chains of different angles are independent (Sec. 4.1: the paper gives each MPI
task a subset of the angles for this reason), so the forward pass shards the angle
list across ranks with no communication: each rank computes C for its own angles.
In the adjoint, grad_beta of a rank's angles is local, while grad_a and grad_b are
sums over all angles and need one sum-all-reduce across ranks.

`angle_shard` gives each rank a contiguous block of the angles (sizes differ by at most
one); `allreduce_sum_` sums tensors in place over the default process group (NCCL for
GPU tensors; any backend for host tensors).  `ShardedConvSum` is the autograd wrapper
whose backward performs that all-reduce, so every rank ends up with the gradient of
the whole-job loss with respect to the replicated a and b.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def angle_shard(n_beta: int, rank: int, world: int) -> slice:
    """Contiguous block of angle indices owned by `rank` of `world` ranks."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_beta, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def allreduce_sum_(*tensors):
    """In-place sum over all ranks of the default group (no-op when not distributed)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tensors
    for t in tensors:
        if t is None:
            continue
        if torch.is_complex(t):
            dist.all_reduce(torch.view_as_real(t), op=dist.ReduceOp.SUM)
        else:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors


class ShardedConvSum(torch.autograd.Function):
    """C_local = conv_sum(a, b, beta_local); backward all-reduces grad_a and grad_b."""

    @staticmethod
    def forward(ctx, a, b, beta_local, form="fp64"):
        from . import wigner as W

        C = W.wigner_conv_sum(beta_local.contiguous(), a.contiguous(), b.contiguous(), form=form)
        ctx.save_for_backward(a, b, beta_local, C)
        return C

    @staticmethod
    def backward(ctx, grad_c):
        from . import wigner as W

        a, b, beta, C = ctx.saved_tensors
        need_a, need_b, need_beta = ctx.needs_input_grad[:3]
        ga, gb, gbeta = W.wigner_conv_sum_backward(beta.contiguous(), a.contiguous(), b.contiguous(),
                                                   C if need_beta else None, grad_c.contiguous(),
                                                   need_a=need_a, need_b=need_b, need_beta=need_beta)
        allreduce_sum_(ga, gb)
        return ga, gb, gbeta, None
