"""The oracle's Philox4x32-10 (written from Salmon et al., SC'11) equals
cuRAND's device Philox4x32-10 word for word on random counters and keys --
a library implementation of the same published generator."""
import ctypes as C

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def test_oracle_philox_equals_curand():
    from tests.cuda import build as cb
    lib = C.CDLL(cb.build())
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] >>= 2        # cuRAND takes words 0-1 as a 64-bit offset x 4: keep it below 2^64
    ctr[: n // 4, :2] = 0  # include the counters the tracker uses (photon id low words, step, draw)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    out = np.zeros((n, 4), np.uint32)
    rc = lib.curand_philox_ref(ctr.ctypes.data_as(C.c_void_p), key.ctypes.data_as(C.c_void_p),
                               out.ctypes.data_as(C.c_void_p), n)
    assert rc == 0
    want = np.array([O.philox(ctr[i], key[i]) for i in range(n)], np.uint32)
    assert np.array_equal(out, want)
