"""lxo_propagate_host_static: the propagation entry point for callers that
must not allocate device memory while they run (a host framework that hands
out all device memory from its own fixed pool, a data-acquisition loop that
cannot afford cudaMalloc failing or cudaFree waiting for the whole device).
Its scratch lives in a static device array inside the library.

The test calls it through the C ABI twice in a row and compares each result
with the allocating entry point lxo_propagate_host on the same photons: the
tallies are integers, so they must be identical (the tolerance of the parity
tests for integer work).  It also checks that tallies larger than the static
array are rejected, and that the entry point allocates no device memory:
after a first call has loaded everything it needs, many further calls leave
the device's free memory where it was.  This file is collected last on
purpose.

The entry point's own fault path (a device fault flag set by the kernel)
cannot be reached from here: every input that could set one is rejected on
the host first (channels, indices, sizes).  By reading: it reads and checks
the flags before any tally reaches the caller's arrays."""
import ctypes as C
import gc

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def host_buffers(trk, n_tbins):
    P = trk.n_channels
    return dict(lce=np.zeros(P, np.uint32), det=np.zeros(P, np.uint32),
                hist=np.zeros((P, n_tbins + 1), np.uint32), fates=np.zeros(trk.n_fates, np.uint64))


def call_static(trk, n, base, seed, n_tbins, out):
    from paper_2203_14354_gb300 import _capi as A
    from paper_2203_14354_gb300.tracker import make_source
    src = make_source(trk.det.source)
    rp = A.lxo_run_params(seed, 10000, n_tbins, 1.0, 0)
    r = A.lxo_results()
    r.lce, r.det, r.hist, r.fates = (out[k].ctypes.data for k in ("lce", "det", "hist", "fates"))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return A.lib().lxo_propagate_host_static(trk._ctx, C.byref(src), n, base, C.byref(rp), C.byref(r), stream)


def test_static_scratch_entry_matches_allocating_entry():
    from paper_2203_14354_gb300 import Tracker, geometry
    from paper_2203_14354_gb300 import _capi as A
    det = geometry.small_tpc()
    trk = Tracker(det)
    n, n_tbins = 40000, 1000
    for call, (base, seed) in enumerate([(0, 3), (40000, 4)]):
        want = trk.propagate_host(n, base=base, seed=seed, n_tbins=n_tbins)
        got = host_buffers(trk, n_tbins)
        assert call_static(trk, n, base, seed, n_tbins, got) == A.LXO_OK, call
        for k in ("lce", "det", "hist", "fates"):
            assert np.array_equal(got[k].astype(np.int64), want[k].astype(np.int64)), (call, k)
        assert int(got["fates"][:7].sum()) == n
    # results add to what the host arrays already hold: two halves of a run
    # accumulate to the whole run
    acc = host_buffers(trk, n_tbins)
    assert call_static(trk, n, 0, 3, n_tbins, acc) == A.LXO_OK
    assert call_static(trk, n, n, 3, n_tbins, acc) == A.LXO_OK
    both = trk.propagate_host(2 * n, base=0, seed=3, n_tbins=n_tbins)
    for k in ("lce", "det", "hist", "fates"):
        assert np.array_equal(acc[k].astype(np.int64), both[k].astype(np.int64)), k


def test_static_scratch_entry_rejects_oversized_tallies():
    from paper_2203_14354_gb300 import Tracker, geometry
    from paper_2203_14354_gb300 import _capi as A
    trk = Tracker(geometry.small_tpc())
    # 14 channels x (200000 + 1) bins x 4 B = 11.2 MB > the 8 MiB static array
    big = 200_000
    out = host_buffers(trk, big)
    assert call_static(trk, 1000, 0, 1, big, out) == A.LXO_ERR_ARG
    assert out["fates"].sum() == 0


def test_static_scratch_entry_allocates_no_device_memory():
    """A fresh context that never called the allocating entry point, a
    detector whose tallies need several MB (122 PMTs x 8001 time bins =
    3.9 MB, which lxo_propagate_host would allocate): after one warm-up call,
    further calls never lower the device's free memory.  (Memory freed by
    earlier tests' contexts may come back meanwhile, so free memory may rise,
    never fall.)"""
    from paper_2203_14354_gb300 import Tracker, geometry
    from paper_2203_14354_gb300 import _capi as A
    det = geometry.scaled_tpc()
    trk = Tracker(det)
    n_tbins = 8000
    out = host_buffers(trk, n_tbins)
    assert call_static(trk, 20000, 0, 1, n_tbins, out) == A.LXO_OK
    torch.cuda.synchronize()
    gc.collect()
    free0, _ = torch.cuda.mem_get_info()
    lowest = free0
    for k in range(20):
        assert call_static(trk, 20000, (k + 1) * 20000, 1, n_tbins, out) == A.LXO_OK, k
        lowest = min(lowest, torch.cuda.mem_get_info()[0])
    assert lowest >= free0, (free0, lowest)
    assert int(out["fates"][:7].sum()) == 21 * 20000
