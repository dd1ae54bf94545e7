"""Slices split over ranks (Sec. III "Parallelism and complexity": the
sub-networks are independent subtasks, and one reduction of their partial
sums follows; the top-k runs on the reduced amplitudes).

One process per GPU.  Rank r contracts a contiguous share of the slice ids
into its own FP64 partial [G][2^l]; the partials are gathered on rank 0 in rank
order and added there in that order by ``tn_sum_partials`` (a fixed order, so
the sum does not depend on the collective's own reduction order); top-k and
XEB then run on rank 0 alone.  The collective is ``torch.distributed``'s
gather (NCCL between GPUs, gloo on CPU tensors); it moves one partial per
rank, G * 2^l * 16 bytes.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np


def partition(slice_ids: Sequence[int], rank: int, world: int) -> np.ndarray:
    """Rank `rank`'s contiguous share of `slice_ids`: shares differ in size by at
    most one and together hold every id once, in order."""
    ids = np.asarray(slice_ids, dtype=np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank or world size")
    lo = len(ids) * rank // world
    hi = len(ids) * (rank + 1) // world
    return ids[lo:hi]


def gather_partials(local, dist, world: int, rank: int):
    """Every rank's partial (a tensor of one shape on every rank) gathered on
    rank 0 as one tensor [world, *shape] in rank order; None on other ranks.
    With ``dist`` None (one process) the local partial alone."""
    import torch
    if dist is None or world == 1:
        return local.unsqueeze(0)
    # complex tensors travel as their real views (the backends reduce real types)
    x = torch.view_as_real(local.contiguous()) if local.is_complex() else local.contiguous()
    parts = torch.empty((world,) + tuple(x.shape), dtype=x.dtype, device=x.device) if rank == 0 else None
    dist.gather(x, gather_list=list(parts.unbind(0)) if rank == 0 else None, dst=0)
    if parts is None:
        return None
    return torch.view_as_complex(parts) if local.is_complex() else parts


def contract_partitioned(plan, slice_ids: Optional[Sequence[int]], dist, world: int, rank: int, out=None,
                         stream=None):
    """Sum over `slice_ids` (all slices when None) split over the ranks: rank 0
    returns the complex128 [G, 2^l] device tensor of the whole sum; other ranks
    return None.  Every rank must call it with the same slice ids."""
    import torch
    from . import binding as B
    if slice_ids is None:
        slice_ids = np.arange(plan.n_slices_total, dtype=np.int64)
    mine = partition(slice_ids, rank, world)
    local = plan.contract(mine, stream=stream)  # zeros when this rank's share is empty
    parts = gather_partials(local, dist, world, rank)
    if rank != 0:
        return None
    if out is None:
        out = torch.empty_like(local)
    s = stream if stream is not None else torch.cuda.current_stream()
    B.tn_sum_partials(parts.data_ptr(), parts.shape[0], local.numel(), out.data_ptr(), 0, s.cuda_stream)
    return out
