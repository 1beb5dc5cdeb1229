"""The checked build (LXO_CHECK_BOUNDS: every BVH node, triangle record, cell
and tally row index compared with its array size inside the kernels) run on
the DARWIN-scale mesh: no index is ever out of range (no error bit set), and
its results equal the normal build's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2203_14354_gb300 import geometry as g, Tracker, _capi
det = g.darwin()
trk = Tracker(det)
out = trk.propagate(1_000_000, seed=3, n_tbins=256)
trk.upload_events(g.darwin_events(seed=5)[::97])
ev = trk.propagate_events(seed=6, n_tbins=64)
rng = np.random.default_rng(1)
org = torch.from_numpy(rng.uniform(-1250, 1250, (200_000, 3)).astype(np.float32)).cuda()
org[:, 2] = org[:, 2] - 1300.0
d = torch.nn.functional.normalize(torch.from_numpy(rng.normal(size=(200_000, 3)).astype(np.float32)), dim=1).cuda()
hit, t = trk.trace_rays(org, d)
trk.sync()  # raises on any device error bit
np.savez({path!r}, lce=out["lce"].cpu().numpy(), hist=out["hist"].cpu().numpy(), fates=out["fates"].cpu().numpy(),
         ev_det=ev["det"].cpu().numpy(), ev_hist=ev["hist"].cpu().numpy(), hit=hit.cpu().numpy(), t=t.cpu().numpy(),
         checked=np.array(_capi.checked()))
'''


def run(tmp_path, checked):
    path = str(tmp_path / ("checked.npz" if checked else "normal.npz"))
    env = dict(os.environ, LXO_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", RUN.format(root=ROOT, path=path)], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_checked_build_finds_no_bad_index_and_changes_nothing(tmp_path):
    a = run(tmp_path, checked=False)
    b = run(tmp_path, checked=True)
    assert not bool(a["checked"]) and bool(b["checked"])
    for k in ("lce", "hist", "fates", "ev_det", "ev_hist", "hit", "t"):
        assert np.array_equal(a[k], b[k]), k
