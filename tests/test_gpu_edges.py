"""Edge cases of the C ABI on the GPU: photon ids above 2^32 (the high word
of the Philox counter) follow the oracle photon by photon; invalid arguments
are rejected with an error message, without a launch, and leave the context
usable; a run of one photon and a run that is not a multiple of the warp or
chunk size add up exactly to the runs they are split from."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from paper_2203_14354_gb300 import _capi as A
from paper_2203_14354_gb300._capi import LxoError
from tests.paired import sign_test

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    from paper_2203_14354_gb300 import Tracker
    det = g.small_tpc()
    return det, Tracker(det), O.Oracle(det)


@pytest.mark.parametrize("base", [(1 << 32) - 7, (1 << 40) + 12345, (1 << 62) + 99])
def test_large_photon_ids_follow_the_oracle(small, base):
    det, trk, orc = small
    n = 20_000
    gpu = trk.propagate(n, base=base, seed=17, per_photon=True)
    ref = orc.propagate(n, base=base, seed=17, per_photon=True)
    fate_g = gpu["fate"].cpu().numpy()
    det_g = gpu["detail"].cpu().numpy()
    pt = sign_test(fate_g, det_g, ref["fate"], ref["detail"])
    print("PARITY large_ids", base, pt)
    assert pt["same"] > 0.99, pt   # measured 0.9942 - 0.9949
    lg, lo = gpu["lce"].cpu().numpy().sum(), ref["lce"].sum()
    assert abs(int(lg) - int(lo)) <= 4 * np.sqrt(2.0 * lo)


def test_invalid_arguments_are_rejected(small):
    det, trk, orc = small
    ref = trk.propagate(5000, seed=3)
    bad_medium = g.Source(g.SRC_POINT, 99, center=(0.0, 0.0, -50.0))
    with pytest.raises(LxoError, match="medium"):
        trk.propagate(100, source=bad_medium)
    with pytest.raises(LxoError, match="time profile"):
        trk.propagate(100, source=g.Source(g.SRC_POINT, g.LXE, center=(0.0, 0.0, -50.0)).with_profile((1.5, 3.5, 24.0)))
    with pytest.raises(LxoError, match="polygon"):
        trk.propagate(100, source=g.Source(g.SRC_VOLUME_POLYGON, g.LXE, n_sides=2, radius=10.0, z_min=-50, z_max=-40))
    with pytest.raises(LxoError, match="surface"):
        trk.set_adjoint([], [99])
    with pytest.raises(LxoError):
        trk.upload_events([(g.Source(g.SRC_POINT, g.LXE).with_profile((0.5, -1.0, 24.0)), 10)])
    with pytest.raises(LxoError):
        trk.propagate(100, tbin_ns=0.0)
    # n_tbins + 1 must not wrap: bins are capped at LXO_MAX_TBINS
    for nb in (A.LXO_MAX_TBINS + 1, 0xFFFFFFFF):
        with pytest.raises(LxoError, match="n_tbins"):
            trk.propagate(100, n_tbins=nb, out=trk.alloc_results(4))
    # nothing ran, nothing broke: the same run gives the same tallies
    again = trk.propagate(5000, seed=3)
    for k in ("lce", "det", "hist", "fates"):
        assert torch.equal(ref[k], again[k]), k


def test_one_photon_and_ragged_splits(small):
    det, trk, orc = small
    n = 1_000_003
    whole = trk.propagate(n, seed=8)
    out = trk.alloc_results()
    for lo, cnt in ((0, 1), (1, 31), (32, 33), (65, 999_938)):
        trk.propagate(cnt, base=lo, seed=8, out=out)
    for k in ("lce", "det", "hist", "fates"):
        assert torch.equal(whole[k], out[k]), k
    one = trk.propagate(1, base=777, seed=8, per_photon=True)
    ref = orc.propagate(1, base=777, seed=8, per_photon=True)
    assert int(one["fates"][:7].sum()) == 1
    assert int(one["fate"][0]) == int(ref["fate"][0])
