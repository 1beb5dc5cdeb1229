"""The batched-event input generator: seeded, S1 counts log-uniform in
[1e2, 1e5] at points uniform in the active LXe, S2 counts log-uniform in
[1e5, 1e6] on vertical segments in the gas gap."""
import numpy as np
from scipy import stats

from paper_2203_14354_gb300 import geometry as g


def test_darwin_events_distributions():
    ev = g.darwin_events(seed=3)
    assert len(ev) == 4608
    s1, s2 = ev[:4096], ev[4096:]
    n1 = np.array([n for _, n in s1], float)
    n2 = np.array([n for _, n in s2], float)
    assert n1.min() >= 100 and n1.max() <= 1e5 and n2.min() >= 1e5 and n2.max() <= 1e6
    assert stats.kstest((np.log(n1) - np.log(1e2)) / (np.log(1e5) - np.log(1e2)), "uniform").pvalue > 1e-3
    assert stats.kstest((np.log(n2) - np.log(1e5)) / (np.log(1e6) - np.log(1e5)), "uniform").pvalue > 1e-3
    c = np.array([s.center for s, _ in s1])
    assert np.all(c[:, 2] >= -2597) and np.all(c[:, 2] <= -1)
    assert np.all(np.hypot(c[:, 0], c[:, 1]) <= 1300)
    assert all(s.kind == g.SRC_POINT and s.medium == g.LXE for s, _ in s1)
    for s, _ in s2:
        assert s.kind == g.SRC_SEGMENT and s.medium == g.GXE
        assert 2.0 < s.center[2] < s.p1[2] < 8.0 and s.center[:2] == s.p1[:2]
    assert [n for _, n in g.darwin_events(seed=3)] == [n for _, n in ev]
