"""Multi-shot gradients across ranks: one shot (source position) per rank, summed by one
collective.

The misfit of several shots is the sum of the shots' misfits (Eq. (3) with the data of
every source), so its gradient, and its Gauss-Newton Hessian-vector product, are the
sums of the per-shot ones.  Each rank solves its own shot at the same wave speed c (the
forward solve with its compressed history, the adjoint: all in the library) and one
all-reduce sums the gradient field and the misfit.  This module only schedules the
per-shot call and the collective (torch.distributed: NCCL between GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch
import torch.distributed as dist


def world(group=None) -> int:
    return dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1


def multishot_gradient(shot_gradient: Callable[[], Tuple[float, torch.Tensor]],
                       group: Optional[object] = None) -> Tuple[float, torch.Tensor]:
    """shot_gradient() -> (J_r, g_r) of this rank's shot.  Returns (sum_r J_r, sum_r g_r);
    the gradient tensor is summed in place (one all-reduce of the field, one of the
    misfit)."""
    J, g = shot_gradient()
    if world(group) > 1:
        Jt = torch.tensor([J], dtype=torch.float64, device=g.device)
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(Jt, op=dist.ReduceOp.SUM, group=group)
        J = float(Jt.item())
    return J, g


def multishot_hessvec(shot_hessvec: Callable[[], torch.Tensor],
                      group: Optional[object] = None) -> torch.Tensor:
    """shot_hessvec() -> H_r dc of this rank's shot; returns sum_r H_r dc (in place)."""
    h = shot_hessvec()
    if world(group) > 1:
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
    return h
