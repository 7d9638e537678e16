"""Shot sharding across ranks (one process per GPU).

The ESI normal equation is block-diagonal over shots (q and B belong to one shot), so each
rank takes a contiguous range of shots and solves, images and differentiates them with no
exchange on the data path.  The only exchange of the outer loop is the sum of the per-shot
model gradients (and misfits) over all shots; it is done here deterministically: every rank
gathers the others' partial sums and adds them in rank order, so the result does not depend
on the collective's reduction order.  The benchmark also uses the max of the ranks' times
and the sum of their cell updates.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def shot_range(ns_total: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous shots [lo, hi) of `rank`; the first ns_total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(ns_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def ordered_sum(t, dist=None):
    """Sum of `t` over ranks, added in rank order (bit-identical on every rank and for any
    collective algorithm).  Without a process group it is `t` itself."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t
    parts = [t.new_empty(t.shape) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t.contiguous())
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def sum_over_ranks(x: float, dist=None, device=None) -> float:
    """Sum of the ranks' values (work done by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t)


def reduce_objective(J: float, g, dist=None):
    """The outer loop's exchange: J and the model gradient `g` summed over the ranks in rank
    order.  For a torch tensor `g` (updated in place, dtype and device kept) the total J is
    returned; for a numpy array, (J_total, g_total)."""
    import torch
    is_np = not isinstance(g, torch.Tensor)
    gt = torch.from_numpy(np.ascontiguousarray(g)) if is_np else g
    t = torch.cat([torch.tensor([J], dtype=torch.float64, device=gt.device),
                   gt.reshape(-1).to(torch.float64)])
    tot = ordered_sum(t, dist)
    if is_np:
        return float(tot[0]), tot[1:].numpy().reshape(np.shape(g)).astype(np.asarray(g).dtype)
    gt.copy_(tot[1:].reshape(gt.shape).to(gt.dtype))
    return float(tot[0])
