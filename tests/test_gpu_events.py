"""Batched events (lxo_upload_events / lxo_propagate_events) through the C
ABI: each event's tallies equal a single-source run of its photon ids
(e << 32) + i bit for bit; statistical parity with the oracle; a CUDA-graph
replay equals the eager launch; results do not depend on the launch shape."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from tests.paired import sign_test

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_events():
    from paper_2203_14354_gb300 import Tracker
    det = g.small_tpc()
    rng = np.random.default_rng(4)
    ev = []
    for k in range(40):
        x, y = rng.uniform(-60, 60, 2)
        z = rng.uniform(-95, -5)
        n = int(np.exp(rng.uniform(np.log(50), np.log(20000))))
        if k % 5 == 4:
            ev.append((g.Source(g.SRC_SEGMENT, g.GXE, center=(x, y, 0.5), p1=(x, y, 4.5)), n))
        elif k % 7 == 6:
            ev.append((g.Source(g.SRC_BALL, g.LXE, center=(x, y, z), radius=3.0), n))
        else:
            ev.append((g.Source(g.SRC_POINT, g.LXE, center=(x, y, z)), n))
    ev.append((g.Source(g.SRC_POINT, g.LXE, center=(0.0, 0.0, -50.0)), 0))  # an empty event
    trk = Tracker(det)
    trk.upload_events(ev)
    return det, trk, ev


def test_events_equal_single_source_runs(small_events):
    det, trk, ev = small_events
    out = trk.propagate_events(seed=9, n_tbins=64)
    assert int(out["fates"][:7].sum()) == sum(n for _, n in ev)
    fates_sum = torch.zeros_like(out["fates"])
    for e, (src, n) in enumerate(ev):
        one = trk.propagate(n, base=e << 32, seed=9, source=src, n_tbins=64)
        assert torch.equal(one["lce"], out["lce"][e]), e
        assert torch.equal(one["det"], out["det"][e]), e
        assert torch.equal(one["hist"], out["hist"][e]), e
        fates_sum += one["fates"]
    assert torch.equal(fates_sum, out["fates"])


def test_event_ranges_reproduce_the_single_launch(small_events):
    """Event-range sharding as one GPU runs it rank after rank (no
    collective): each range uploaded with its first event's id gives the
    single launch's rows bit for bit, and the fates sum to the single
    launch's; the FP64 adjoint sums agree to rounding (their atomic adds
    run in another order)."""
    from paper_2203_14354_gb300.shard import event_ranges
    det, trk, ev = small_events
    trk.set_adjoint([g.LXE], [0, 1])
    trk.upload_events(ev)
    want = trk.propagate_events(seed=13, n_tbins=32, adjoint=True)
    for world in (2, 3):
        got = {k: torch.zeros_like(v) for k, v in want.items()}
        for lo, hi in event_ranges([n for _, n in ev], world):
            if hi == lo:
                continue
            trk.upload_events(ev[lo:hi], first_event=lo)
            part = trk.propagate_events(seed=13, n_tbins=32, adjoint=True)
            for k, v in part.items():
                if k == "fates":
                    got[k] += v
                else:
                    got[k][lo:hi] = v
        for k in want:
            if k == "adjoint":
                assert torch.allclose(got[k], want[k], rtol=1e-12, atol=1e-9), world
            else:
                assert torch.equal(got[k], want[k]), (world, k)
    trk.set_adjoint([], [])
    trk.upload_events(ev)


def test_events_parity_with_oracle(small_events):
    """Per event, the light collected agrees with the oracle within 4 sigma
    of the two-sample Poisson difference, and the total within 2 %.  Paired:
    an event's photons are those of a single-source run with base e << 32
    (bit for bit, test above), so the oracle's per-photon outcomes are
    compared with the GPU's photon by photon; per (event, outcome) the
    discordant photons split evenly (sign test)."""
    det, trk, ev = small_events
    out = trk.propagate_events(seed=9, n_tbins=64)
    orc = O.Oracle(det)
    lce_o = np.zeros((len(ev), det.n_pmts))
    fg, dg, fo, do = [], [], [], []
    for e, (src, n) in enumerate(ev):
        if n:
            ref = orc.propagate(n, base=e << 32, seed=9, src=src, per_photon=True)
            lce_o[e] = ref["lce"]
            one = trk.propagate(n, base=e << 32, seed=9, source=src, per_photon=True, n_tbins=1)
            fg.append(one["fate"].cpu().numpy())
            dg.append(one["detail"].cpu().numpy().astype(np.int64) + (e << 20))
            fo.append(ref["fate"])
            do.append(ref["detail"].astype(np.int64) + (e << 20))
    lce_g = out["lce"].cpu().numpy()
    tot = lce_o.sum()
    assert abs(lce_g.sum() - tot) < 0.02 * tot
    for e, (_, n) in enumerate(ev):
        if n > 2000:
            a, b = lce_g[e].sum(), lce_o[e].sum()
            assert abs(a - b) <= 4 * np.sqrt(2 * max(b, 1)), e
    pt = sign_test(np.concatenate(fg), np.concatenate(dg), np.concatenate(fo), np.concatenate(do))
    print("PARITY events_small", pt)
    assert pt["same"] > 0.99, pt   # measured 0.9948


def test_events_cuda_graph_and_launch_shape(small_events):
    det, trk, ev = small_events
    ref = trk.propagate_events(seed=5, hist=False)
    out = trk.alloc_event_results(hist=False)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        trk.propagate_events(seed=5, out=out, hist=False, sync=False)  # warm-up outside the graph
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for v in out.values():
            v.zero_()
        trk.propagate_events(seed=5, out=out, hist=False, sync=False)
    for _ in range(3):
        graph.replay()
        torch.cuda.synchronize()
        for k in ("lce", "det", "fates"):
            assert torch.equal(out[k], ref[k]), k
    trk.sync()
    # both register budgets (up to 5 CTAs of 256 per SM: 48 registers; more: 32)
    for b, c, t in ((1, 16, 256), (3, 256, 256), (8, 64, 256), (2, 32, 128), (10, 64, 128), (16, 32, 128),
                    (0, 0, 0)):
        trk.set_launch(b, c, t)
        o = trk.propagate_events(seed=5, hist=False)
        for k in ("lce", "det", "fates"):
            assert torch.equal(o[k], ref[k]), (b, c, t, k)
    # the single-source kernel and the adjoint build too, in 128-thread CTAs
    # and in both register budgets
    one = trk.propagate(20000, seed=6, per_photon=True)
    trk.set_adjoint([g.LXE], [0])
    adj = trk.propagate(20000, seed=6, adjoint=True)
    for b, t in ((0, 128), (16, 128), (8, 256), (5, 256)):
        trk.set_launch(b, 0, t)
        for k, v in trk.propagate(20000, seed=6, per_photon=True).items():
            assert torch.equal(v, one[k]), (b, t, k)
        other = trk.propagate(20000, seed=6, adjoint=True)
        assert torch.equal(other["det"], adj["det"]), (b, t)
        assert torch.allclose(other["adjoint"], adj["adjoint"], rtol=1e-12, atol=1e-9), (b, t)
    trk.set_adjoint([], [])
    trk.set_launch(0, 0, 0)


def test_darwin_events_subset(tmp_path):
    from paper_2203_14354_gb300 import Tracker
    det = g.darwin()
    ev = g.darwin_events(seed=1)
    sub = ev[:48] + ev[4096:4100]
    trk = Tracker(det)
    trk.upload_events(sub)
    out = trk.propagate_events(seed=3, n_tbins=256)
    assert int(out["fates"][:7].sum()) == sum(n for _, n in sub)
    assert int(out["fates"][4]) + int(out["fates"][6]) <= 1e-4 * sum(n for _, n in sub) + 2
    for e in (0, 7, 48, 50):
        src, n = sub[e]
        one = trk.propagate(n, base=e << 32, seed=3, source=src, n_tbins=256)
        assert torch.equal(one["det"], out["det"][e]) and torch.equal(one["hist"], out["hist"][e])
    # S2 light in the gas reaches the top array far more than S1 light from deep in the LXe
    top = torch.from_numpy(det.pmt_array == 1).to(out["lce"].device)
    s2 = out["lce"][48:][:, top].sum() / out["lce"][48:].sum()
    s1 = out["lce"][:48][:, top].sum() / out["lce"][:48].sum().clamp(min=1)
    assert float(s2) > float(s1)


def test_darwin_events_full_size_sampled():
    """The full batched-events workload: 4096 S1 + 512 S2 events, 2.6e8
    photons, one launch. Sampled events (the largest among them) equal their
    single-source runs bit for bit; the photons of one S1 and one S2 event
    follow the oracle photon by photon."""
    from paper_2203_14354_gb300 import Tracker
    det = g.darwin()
    ev = g.darwin_events(seed=0)
    trk = Tracker(det)
    trk.upload_events(ev)
    out = trk.propagate_events(seed=4, n_tbins=64)
    total = sum(n for _, n in ev)
    assert int(out["fates"][:7].sum()) == total
    rng = np.random.default_rng(2)
    counts = np.array([n for _, n in ev])
    pick = list(rng.choice(len(ev), 20, replace=False)) + [int(np.argmax(counts[:4096])),
                                                         4096 + int(np.argmax(counts[4096:])),
                                                         int(np.argmin(counts)), len(ev) - 1]
    for e in pick:
        src, n = ev[e]
        one = trk.propagate(n, base=e << 32, seed=4, source=src, n_tbins=64)
        assert torch.equal(one["det"], out["det"][e]) and torch.equal(one["hist"], out["hist"][e]), e
    orc = O.Oracle(det)
    for e in (int(np.argmin(np.where(counts[:4096] > 2000, counts[:4096], 1 << 40))), 4096):
        src, n = ev[e]
        m = min(n, 3000)
        gp = trk.propagate(m, base=e << 32, seed=4, source=src, per_photon=True, n_tbins=1)
        ref = orc.propagate(m, base=e << 32, seed=4, src=src, per_photon=True, n_tbins=1)
        same = (gp["fate"].cpu().numpy() == ref["fate"]) & (gp["detail"].cpu().numpy() == ref["detail"])
        print("PARITY darwin_event", e, same.mean())
        assert same.mean() > 0.99, (e, same.mean())   # measured 0.994 - 0.996
