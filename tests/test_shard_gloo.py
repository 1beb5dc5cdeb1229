"""Host logic of the multi-GPU path, run as world-size-2 gloo process groups
on the CPU: the photon-id ranges tile the job exactly, and the summed
per-rank tallies equal the tallies of the whole range computed at once (the
stand-in tracker tallies a deterministic function of each photon id, as the
real one does through its per-photon random stream).  Batched events shard
by event range: the ranges tile the event list with balanced photon counts,
and the assembled per-event tallies (counts, histograms, adjoint sums) equal
the single run's row for row."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2203_14354_gb300.shard import event_ranges, propagate_events_sharded, propagate_sharded, rank_range


def test_rank_ranges_tile_the_job():
    for n in (0, 1, 7, 1000, 10 ** 9 + 3):
        for world in (1, 2, 3, 8):
            ranges = [rank_range(n, r, world, base=5) for r in range(world)]
            assert ranges[0][0] == 5
            for (a, c), (b, _) in zip(ranges, ranges[1:]):
                assert a + c == b
            assert sum(c for _, c in ranges) == n
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        rank_range(10, 2, 2)


class _FakeTracker:
    """Tallies of photon ids [base, base+n): channel = hash(id, seed) mod P."""
    P = 13

    def propagate(self, n, base=0, seed=0, **kw):
        ids = torch.arange(base, base + n, dtype=torch.int64)
        ch = (ids * 2654435761 + seed * 97) % self.P
        lce = torch.bincount(ch, minlength=self.P).to(torch.int32)
        det = torch.bincount(ch[ids % 3 == 0], minlength=self.P).to(torch.int32)
        fates = torch.tensor([n, int((ids % 3 == 0).sum()), 0, 0, 0, 0, 0, 7 * n], dtype=torch.int64)
        adj = torch.zeros((self.P, 2), dtype=torch.float64)
        adj[:, 0] = lce.double() * 0.5
        return dict(lce=lce, det=det, fates=fates, adjoint=adj)


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = propagate_sharded(_FakeTracker(), n, seed=4, base=11)
    q.put((rank, {k: v.clone() for k, v in out.items()}))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world", [2])
def test_sharded_tallies_equal_single_run(world):
    n = 100_003
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = _FakeTracker().propagate(n, base=11, seed=4)
    for r in range(world):
        for k in want:
            assert torch.equal(got[r][k], want[k]), (r, k)


def test_event_ranges_tile_and_balance():
    rng = torch.Generator().manual_seed(3)
    for world in (1, 2, 3, 8):
        for E in (0, 1, 5, 300):
            counts = (torch.rand(E, generator=rng) * 1000).long().tolist()
            rs = event_ranges(counts, world)
            assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == E
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and a <= b
            total = sum(counts)
            if E >= 50 * world:   # many small events: each rank within one event of its share
                for a, b in rs:
                    assert abs(sum(counts[a:b]) - total / world) <= max(counts) + 1
    assert event_ranges([1, 1, 1, 100], 3) == [(0, 4), (4, 4), (4, 4)]
    with pytest.raises(ValueError):
        event_ranges([1, -1], 2)


class _FakeEventTracker:
    """Per-event tallies that depend only on each photon's id
    ((event id << 32) | i), as the real tracker's do."""
    P, K, B = 7, 4, 5
    n_fates = 10
    device = torch.device("cpu")
    n_channels = P
    n_tallies = K

    def upload_events(self, events, first_event=0):
        self.counts = [int(n) for _, n in events]
        self.first = first_event

    def propagate_events(self, seed=0, n_tbins=256, hist=True, adjoint=False, **kw):
        E = len(self.counts)
        out = dict(lce=torch.zeros((E, self.P), dtype=torch.int32), det=torch.zeros((E, self.P), dtype=torch.int32),
                   fates=torch.zeros(self.n_fates, dtype=torch.int64))
        if hist:
            out["hist"] = torch.zeros((E, self.P, n_tbins + 1), dtype=torch.int32)
        if adjoint:
            out["adjoint"] = torch.zeros((E, self.P, self.K), dtype=torch.float64)
        for e, n in enumerate(self.counts):
            ids = ((self.first + e) << 32) + torch.arange(n, dtype=torch.int64)
            h = (ids * 2654435761 + seed * 97) % 1000003
            ch = h % self.P
            out["lce"][e] = torch.bincount(ch, minlength=self.P).int()
            out["det"][e] = torch.bincount(ch[h % 3 == 0], minlength=self.P).int()
            if hist:
                out["hist"][e].view(-1).index_add_(0, ch * (n_tbins + 1) + h % (n_tbins + 1),
                                                   torch.ones(n, dtype=torch.int32))
            if adjoint:
                for k in range(self.K):
                    out["adjoint"][e, :, k].index_add_(0, ch, (h % (k + 5)).double() * 0.25)
            out["fates"][0] += n
            out["fates"][7] += int(h.sum() % 1000)
        return out


def _events(E=37, seed=5):
    gen = torch.Generator().manual_seed(seed)
    return [(None, int(x)) for x in (torch.rand(E, generator=gen) * 400).long()]


def _event_worker(rank, world, port, q, empty_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ev = _events()
    if empty_rank:   # the last event holds almost every photon: the second rank gets no event
        ev = ev[:1] + [(None, 100000)]
    out = propagate_events_sharded(_FakeEventTracker(), ev, seed=3, n_tbins=9, hist=True, adjoint=True)
    q.put((rank, {k: v.clone() for k, v in out.items()}))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("empty_rank", [False, True])
def test_sharded_events_equal_single_run(empty_rank):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_event_worker, args=(r, world, port, q, empty_rank)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ev = _events()
    if empty_rank:
        ev = ev[:1] + [(None, 100000)]
        assert event_ranges([n for _, n in ev], world)[1] == (2, 2)
    one = _FakeEventTracker()
    one.upload_events(ev)
    want = one.propagate_events(seed=3, n_tbins=9, hist=True, adjoint=True)
    for r in range(world):
        for k in want:
            assert got[r][k].dtype == want[k].dtype, (r, k)
            assert torch.equal(got[r][k], want[k]), (r, k)
