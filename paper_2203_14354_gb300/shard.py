"""Running one photon job on several GPUs (one process per GPU).

Photons are independent and photon p's random stream depends only on
(seed, p), so a job of n photons splits into contiguous photon-id ranges,
one per rank, with no exchange while propagating; the per-rank tallies add
up to exactly the single-GPU result.  The only collective is one sum of the
integer (and adjoint FP64) tallies at the end."""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_range(n: int, rank: int, world: int, base: int = 0):
    """(photon_id_base, count) of `rank` for a job of n photons starting at base:
    contiguous ranges, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    lo = base + (n * rank) // world
    hi = base + (n * (rank + 1)) // world
    return lo, hi - lo


def reduce_tallies(out: dict, group=None, dst=None):
    """Sums every tally tensor of `out` over the ranks of `group` (in place):
    all ranks get the total, or only rank `dst` if given."""
    for k in sorted(out):
        t = out[k]
        if not torch.is_tensor(t):
            continue
        if dst is None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            dist.reduce(t, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return out


def propagate_sharded(tracker, n: int, seed: int = 0, base: int = 0, group=None, **kw):
    """One job of n photons (ids base .. base+n-1) over all ranks of `group`:
    each rank propagates its range with its own tracker, then the tallies are
    summed on every rank."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    lo, cnt = rank_range(n, rank, world, base)
    out = tracker.propagate(cnt, base=lo, seed=seed, **kw)
    if world > 1:
        reduce_tallies(out, group)
    return out
