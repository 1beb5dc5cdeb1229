"""Running one photon job on several GPUs (one process per GPU).

Photons are independent and photon p's random stream depends only on
(seed, p), so a job of n photons splits into contiguous photon-id ranges,
one per rank, with no exchange while propagating; the per-rank tallies add
up to exactly the single-GPU result.  The only collective is one sum of the
integer (and adjoint FP64) tallies at the end.

Batched events split the same way by event: contiguous event ranges with
about equal photon counts, each uploaded with its first event's id so that
every photon keeps its id ((event << 32) | i), and the per-event tallies
([E, P], [E, P, B+1], [E, P, K]) are assembled by one sum at the end."""
from __future__ import annotations

import bisect

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


def _world_rank(group):
    if dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def event_ranges(counts, world: int):
    """Contiguous event ranges [(lo, hi)] for `world` ranks with about equal
    photon counts: rank r starts at the first event whose photon prefix sum
    reaches r / world of the total (ranges may be empty when a few events
    hold most photons)."""
    if world < 1:
        raise ValueError(f"world {world}")
    pre = [0]
    for c in counts:
        if c < 0:
            raise ValueError("negative photon count")
        pre.append(pre[-1] + int(c))
    total = pre[-1]
    cuts = [0] + [min(len(counts), bisect.bisect_left(pre, (total * r + world - 1) // world)) for r in range(1, world)]
    cuts.append(len(counts))
    for r in range(1, world + 1):
        cuts[r] = max(cuts[r], cuts[r - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


class ShardedEvents:
    """Batched events of one job over all ranks of `group`: the tracker
    interface used by the calibration and EventLightCollection
    (upload_events, propagate_events; everything else is the tracker's),
    with each rank propagating its own event range and every rank receiving
    the whole job's per-event tallies, equal row for row to a single-GPU
    run."""

    def __init__(self, tracker, group=None):
        self.tracker = tracker
        self.group = group
        self.n_events = 0
        self.event_photons = 0
        self.range = (0, 0)

    def __getattr__(self, name):
        return getattr(self.tracker, name)

    def upload_events(self, events):
        world, rank = _world_rank(self.group)
        counts = [int(n) for _, n in events]
        lo, hi = event_ranges(counts, world)[rank]
        self.n_events, self.event_photons, self.range = len(events), sum(counts), (lo, hi)
        if hi > lo:
            self.tracker.upload_events(events[lo:hi], first_event=lo)

    def propagate_events(self, seed=0, n_tbins=256, hist=True, adjoint=False, **kw):
        """The whole job's tallies on every rank: lce, det [E, P], hist
        [E, P, n_tbins+1] if hist, adjoint [E, P, K] if adjoint, fates."""
        lo, hi = self.range
        world, _ = _world_rank(self.group)
        E, P = self.n_events, self.tracker.n_channels
        dev = self.tracker.device
        # the tracker's result layout (a rank with no events still joins the sum)
        full = dict(lce=torch.zeros((E, P), dtype=torch.int32, device=dev),
                    det=torch.zeros((E, P), dtype=torch.int32, device=dev),
                    fates=torch.zeros(self.tracker.n_fates, dtype=torch.int64, device=dev))
        if hist:
            full["hist"] = torch.zeros((E, P, n_tbins + 1), dtype=torch.int32, device=dev)
        if adjoint:
            full["adjoint"] = torch.zeros((E, P, self.tracker.n_tallies), dtype=torch.float64, device=dev)
        if hi > lo:
            part = self.tracker.propagate_events(seed=seed, n_tbins=n_tbins, hist=hist, adjoint=adjoint, **kw)
            for k, v in part.items():
                if k == "fates":
                    full[k] = full[k].to(v.dtype) + v
                else:
                    full[k] = full[k].to(v.dtype)
                    full[k][lo:hi] = v
        if world > 1:
            reduce_tallies(full, self.group)
        return full


def propagate_events_sharded(tracker, events, seed=0, group=None, **kw):
    """One batched-events job over all ranks of `group` (see ShardedEvents):
    returns the whole job's per-event tallies on every rank."""
    sh = ShardedEvents(tracker, group)
    sh.upload_events(events)
    return sh.propagate_events(seed=seed, **kw)
