"""Design variants (Sec. 5) on the GPU against the oracle, on the DARWIN-scale
mesh without the wire meshes (and with the paper's five planes of parallel
wires on frames and PTFE cones on the windows) and with the paper's
best-guess optics: per-array
light collection agrees with the oracle, a single-phase detector collects
more light and one without a bottom array far less (the paper's signs:
+4.9 % abs. and 18 % against 43 %)."""
import numpy as np
import pytest

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from tests.paired import sign_test

pytestmark = pytest.mark.gpu

N = 200_000


def run_both(det, seed=4):
    from paper_2203_14354_gb300 import Tracker
    trk = Tracker(det)
    out = {k: v.cpu().numpy() for k, v in trk.propagate(N, seed=seed, per_photon=True).items()}
    trk.close()
    ref = O.Oracle(det).propagate(N, seed=seed, per_photon=True)
    pair = (out["fate"], out["detail"], ref["fate"], ref["detail"])
    return out["lce"].astype(np.float64), ref["lce"].astype(np.float64), pair


@pytest.fixture(scope="module")
def results():
    res = {}
    for name, kw in (("baseline", {}), ("single_phase", dict(single_phase=True)),
                     ("no_bottom_array", dict(bottom_array=False)),
                     ("paper_electrodes", dict(electrode_kind="wires", pmt_cones=6.0))):
        det = g.darwin(electrodes=(), **g.PAPER_OPTICS, **kw)
        res[name] = (det, *run_both(det))
    return res


@pytest.mark.parametrize("name", ["baseline", "single_phase", "no_bottom_array", "paper_electrodes"])
def test_variant_parity_with_oracle(results, name):
    """Per array within 4 sigma of the two-sample Poisson difference; paired
    per outcome (sign test of the discordant photons)."""
    det, a, b, pair = results[name]
    top = det.pmt_array == 1
    for sel in (top, ~top):
        if sel.any():
            x, y = a[sel].sum(), b[sel].sum()
            assert abs(x - y) <= 4 * np.sqrt(2 * max(y, 1.0)), (name, x, y)
    pt = sign_test(*pair)
    print("PARITY variant", name, pt)
    # measured 0.9957 - 0.9977; 0.974 with the paper's parallel wires, whose
    # many grazing wire edges let rounding decide more hits
    assert pt["same"] > (0.96 if name == "paper_electrodes" else 0.99), pt


def test_variant_directions(results):
    lce = {k: v[1].sum() / N for k, v in results.items()}
    assert lce["single_phase"] > lce["baseline"] + 0.02, lce
    assert lce["no_bottom_array"] < 0.6 * lce["baseline"], lce
