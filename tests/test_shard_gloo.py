"""Host logic of the multi-GPU path, run as world-size-2 gloo process groups
on the CPU: the photon-id ranges tile the job exactly, and the summed
per-rank tallies equal the tallies of the whole range computed at once (the
stand-in tracker tallies a deterministic function of each photon id, as the
real one does through its per-photon random stream)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2203_14354_gb300.shard import propagate_sharded, rank_range


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
