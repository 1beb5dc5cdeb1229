"""Host logic of the Python front end that needs no GPU: the tracker's
parameter updates (set_theta, used by finite differences, the autograd
Function and the calibration fit) go to the tracker's own tables, never to
the detector it was built from, so an oracle built from that detector
afterwards sees the original optics."""
import oracle as O
from paper_2203_14354_gb300 import geometry as g
from paper_2203_14354_gb300 import tracker as T


class _FakeLib:
    """Stands in for the C library: records the tables it is given."""

    def __init__(self):
        self.calls = []

    def lxo_set_materials(self, ctx, arr, n):
        self.calls.append(("materials", [(arr[i].abs_len_mm, arr[i].rayleigh_len_mm) for i in range(n)]))
        return 0

    def lxo_set_surfaces(self, ctx, arr, n):
        self.calls.append(("surfaces", [(arr[i].reflectivity, arr[i].transparency) for i in range(n)]))
        return 0


def _bare_tracker(det):
    trk = T.Tracker.__new__(T.Tracker)   # no GPU: only the table logic runs
    trk._L, trk._ctx = _FakeLib(), None
    trk.det = T.own_tables(det)
    trk.adj_mats, trk.adj_surfs = [g.LXE], [0, 1, 4]
    return trk


def test_set_theta_leaves_the_callers_detector_alone():
    det = g.scaled_tpc()
    before = [(m.abs_len_mm, m.rayleigh_len_mm) for m in det.materials]
    before_s = [(s.reflectivity, s.transparency) for s in det.surfaces]
    trk = _bare_tracker(det)
    theta0 = trk.theta().tolist()
    new = [30_000.0, 350.0, 0.97, 0.80, 0.5]
    trk.set_theta(new)
    # the tracker holds and uploads the new values ...
    assert trk.theta().tolist() == new
    kind, mats = trk._L.calls[0]
    assert kind == "materials" and mats[g.LXE][0] == 30_000.0 and abs(mats[g.LXE][1] - 350.0) < 1e-3
    # ... while the caller's detector keeps the old ones
    assert [(m.abs_len_mm, m.rayleigh_len_mm) for m in det.materials] == before
    assert [(s.reflectivity, s.transparency) for s in det.surfaces] == before_s
    assert theta0 != new
    # an oracle built from the detector now runs the original optics: the
    # same photons give the same tallies as an oracle of a fresh detector
    a = O.Oracle(det).propagate(3000, seed=2)
    b = O.Oracle(g.scaled_tpc()).propagate(3000, seed=2)
    assert (a["lce"] == b["lce"]).all() and (a["fates"] == b["fates"]).all()


def test_own_tables_shares_the_mesh_only():
    det = g.small_tpc()
    mine = T.own_tables(det)
    assert mine.verts is det.verts and mine.tris is det.tris
    assert all(a is not b for a, b in zip(mine.materials, det.materials))
    assert all(a is not b for a, b in zip(mine.surfaces, det.surfaces))
    assert mine.materials == det.materials and mine.surfaces == det.surfaces
