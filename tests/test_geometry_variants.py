"""Design variants of the DARWIN-scale detector (Sec. 5) as geometry and
surface switches, checked on the mesh without the electrode wire meshes
(the switches do not touch them): single phase has no gas and no liquid
surface, the variant without a bottom array has only the top channels and a
99 % PTFE floor, coatings change only the electrodes' surface entries, and
the best-guess optics follow Table 2."""
import numpy as np
import pytest

from paper_2203_14354_gb300 import geometry as g
from paper_2203_14354_gb300 import variants


@pytest.fixture(scope="module")
def base():
    return g.darwin(electrodes=())


def test_single_phase(base):
    d = g.darwin(electrodes=(), single_phase=True)
    assert not np.any(d.mat_inner == g.GXE) and not np.any(d.mat_outer == g.GXE)
    assert np.any(base.mat_outer == g.GXE)
    # the liquid surface is gone: no LXe/GXe boundary, and nothing else changed in size
    liquid = (base.mat_inner == g.LXE) & (base.mat_outer == g.GXE) & (base.surface == g.SURF_NONE)
    assert liquid.sum() > 0 and d.n_tris == base.n_tris - liquid.sum()
    assert d.surfaces[1].reflectivity == d.surfaces[0].reflectivity
    assert d.n_pmts == base.n_pmts


def test_no_bottom_array(base):
    d = g.darwin(electrodes=(), bottom_array=False)
    assert d.n_pmts == int((base.pmt_array == 1).sum()) and np.all(d.pmt_array == 1)
    ch = d.channel[d.channel >= 0]
    assert ch.min() == 0 and ch.max() == d.n_pmts - 1
    floor = d.surfaces.index(next(s for s in d.surfaces if s.name == "PTFE_bottom"))
    assert d.surfaces[floor].reflectivity == 0.99
    z = d.verts[d.tris].mean(1)[:, 2]
    at_floor = np.abs(z - (-2688.0)) < 1e-3
    assert at_floor.sum() > 0 and np.all(d.surface[at_floor] == floor)


def test_coatings_change_only_surfaces():
    opt = dict(k_seg=8, pitch_pmt=400.0, mesh_pitch=200.0)
    a = g.darwin(**opt)
    b = g.darwin(coated=("gate",), **opt)
    assert np.array_equal(a.tris, b.tris) and np.array_equal(a.surface, b.surface)
    names = [s.name for s in b.surfaces]
    assert "gate_AlMgF2" in names and "anode_SS" in names
    gate = b.surfaces[names.index("gate_AlMgF2")]
    assert gate.reflectivity == 0.90 and gate.spec_frac == pytest.approx(0.85 / 0.90)
    t = variants.coated_table(a.surfaces, ("gate", "anode", "cathode"))
    assert [s.name for s in t if s.name.endswith("_AlMgF2")] == ["gate_AlMgF2", "anode_AlMgF2", "cathode_AlMgF2"]
    assert [s.name for s in t][:4] == [s.name for s in a.surfaces][:4]


def test_paper_optics():
    d = g.darwin(electrodes=(), **g.PAPER_OPTICS)
    lxe, gxe = d.materials[g.LXE], d.materials[g.GXE]
    assert (lxe.abs_len_mm, lxe.rayleigh_len_mm) == (50_000.0, 360.0)
    assert (gxe.abs_len_mm, gxe.rayleigh_len_mm) == (500_000.0, 200_000.0)
    assert d.surfaces[0].reflectivity == 0.99 and d.surfaces[1].reflectivity == 0.80
    # specular/diffuse ratio 0.05 -> specular fraction 0.05 / 1.05
    assert d.surfaces[0].spec_frac / (1 - d.surfaces[0].spec_frac) == pytest.approx(0.05)


def _edge_uses(det):
    t = det.tris
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]).astype(np.int64), 1)
    return np.unique(e, axis=0, return_counts=True)[1]


@pytest.mark.parametrize("build", [g.small_tpc, g.scaled_tpc,
                                   lambda: g.darwin(electrodes=()),
                                   lambda: g.darwin(electrodes=(), single_phase=True),
                                   lambda: g.darwin(electrodes=(), bottom_array=False)])
def test_surfaces_have_no_open_edges(build):
    """Conforming meshes (no T-junctions): every edge belongs to two
    triangles, or three where a plate, a window rim or the liquid surface
    meets another surface; none is open, so no photon leaks through a gap."""
    uses = _edge_uses(build())
    assert uses.min() >= 2 and uses.max() <= 3


def test_pmt_cones_close_the_windows():
    """Conical PTFE reflectors on the windows: no open edge; the window rim
    is shared by four surfaces (plate, window face, window side, collar)."""
    d = g.darwin(electrodes=(), pmt_cones=6.0)
    uses = _edge_uses(d)
    assert uses.min() >= 2 and uses.max() <= 4
    base = g.darwin(electrodes=())
    # per window: an annulus of the front face turns into PTFE contact, plus cone and collar
    assert d.n_tris > base.n_tris
    z = d.verts[d.tris].mean(1)[:, 2]
    cone = (d.mat_outer == g.OPAQUE) & (d.surface == 0) & (z > -2688.0) & (z < -2682.0)
    assert cone.sum() == 889 * 4 * 32  # cone + collar, 2 x 32 triangles each, per bottom window


@pytest.fixture(scope="module")
def wires():
    return g.darwin(electrode_kind="wires", **g.PAPER_OPTICS)


def test_paper_wire_electrodes(wires):
    """Five planes of parallel 200 um wires (Sec. 2.1, Table 1): 5 mm pitch
    at z = 54, 12, 0 and 7.5 mm pitch at z = -2598, -2678, each prism 200 um
    wide, each plane with its frame surface."""
    d = wires
    names = [s.name for s in d.surfaces]
    for el in ("screen_top", "anode", "gate", "cathode", "screen_bottom"):
        assert f"{el}_SS" in names and f"{el}_frame" in names
    tv = d.verts[d.tris]
    zc = tv.mean(1)[:, 2]
    wire = d.mat_inner == g.OPAQUE
    for zz, pitch in ((54, 5.0), (12, 5.0), (0, 5.0), (-2598, 7.5), (-2678, 7.5)):
        m = wire & (np.abs(zc - zz) < 0.2)
        n_wires = m.sum() // 8
        assert abs(n_wires - 2 * (1290.0 * np.cos(np.pi / 24)) / pitch) < 4, (zz, n_wires)
        # every wire triangle lies within 100 um of its plane
        assert np.all(np.abs(tv[m][:, :, 2] - zz) <= 0.1 + 1e-4)
    # top frames carry PTFE, bottom ones steel
    assert d.surfaces[names.index("gate_frame")].reflectivity == d.surfaces[0].reflectivity
    assert d.surfaces[names.index("cathode_frame")].reflectivity == 0.30


def test_wire_layout_has_no_leaks_and_loss_table_closes(wires):
    import oracle as O
    from paper_2203_14354_gb300 import analysis
    n = 20_000
    r = O.Oracle(wires).propagate(n, seed=2)
    assert r["fates"][4] == 0 and r["fates"][6] == 0
    t = analysis.loss_table(wires, r["fates"], n)
    parts = (sum(v for k, v in t.items() if k in ("LXe", "GXe", "quartz", "opaque")) + t["electrodes"] + t["pmt_caps"]
             + t["ptfe"] + t["other_surfaces"] + t["escaped"] + t["truncated"])
    assert parts == pytest.approx(t["not_detected"], abs=1e-9)
    assert t["electrodes"] == pytest.approx(sum(t["electrode_parts"].values()))


def test_map_summary_reads_the_features():
    """The map summary finds the height where top and bottom arrays collect
    equally, the radial spread, the edge dips and the t90 profile, on
    synthetic maps with known values."""
    z = np.linspace(-2597.0, -1.0, 50)
    r2 = (np.arange(50) + 0.5) / 50 * 1280.0 ** 2
    top = np.tile(np.linspace(5.0, 40.0, 50)[:, None], (1, 50))
    bot = np.tile(np.linspace(35.0, 10.0, 50)[:, None], (1, 50))
    lce = top + bot
    lce[0, -1] -= 7.0  # a dip at the bottom edge
    t90 = np.tile(np.linspace(90.0, 150.0, 50)[:, None], (1, 50))
    s = variants.map_summary(dict(z=z, r2=r2, lce=lce, top=top, bottom=bot, t90=t90))
    # top = bottom where 5 + 35 f = 35 - 25 f, f = 0.5: mid-height
    assert s["z_equal_split"] == pytest.approx(-1299.0, abs=1e-6)
    assert s["radial_spread_mid_z"] == pytest.approx(0.0)
    assert s["bottom_edge_minus_bottom_centre"] == pytest.approx(-7.0)
    assert s["t90_near_bottom"] == pytest.approx(90.0) and s["t90_near_top"] == pytest.approx(150.0)


def test_scaled_tpc_has_61_plus_61_windows_in_five_hexagonal_rings():
    """The 50 cm TPC of the adjoint workload: 61 windows per array, the
    hexagonal rings 0..4 of the 80 mm lattice (ring k holds 6k sites)."""
    c = g.hex_lattice(80.0, 700.0)
    r = g.hex_ring(c, 80.0)
    assert [int((r == k).sum()) for k in range(6)] == [1, 6, 12, 18, 24, 30]
    # ring k sites lie between k * pitch * sqrt(3)/2 and k * pitch from the centre
    d = np.hypot(c[:, 0], c[:, 1])
    for k in range(1, 6):
        assert np.all(d[r == k] >= k * 80.0 * np.sqrt(3) / 2 - 1e-6) and np.all(d[r == k] <= k * 80.0 + 1e-6)
    det = g.scaled_tpc()
    assert det.n_pmts == 122 and np.bincount(det.pmt_array).tolist() == [61, 61]
    top = det.pmt_pos[det.pmt_array == 1][:, :2]
    assert np.allclose(np.sort(top, axis=0), np.sort(det.pmt_pos[det.pmt_array == 0][:, :2], axis=0))
    assert np.hypot(top[:, 0], top[:, 1]).max() == pytest.approx(320.0)


def test_grid_sources_fill_the_active_volume():
    """Calibration sources on the 10 cm 3-D grid: every source a grid node,
    inside the DARWIN-scale active volume (24-gon prism, z in [-2597, -1])
    at least 50 mm from each wall side, the cathode and the gate; 256 of
    about 12 000 nodes, seeded; the layout spans the volume in x, y and z."""
    import math
    det = g.Detector("src-only", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros(0, np.uint8),
                     np.zeros(0, np.uint8), np.zeros(0, np.uint16), np.zeros(0, np.int32), [], [],
                     np.zeros(0, np.int32), np.zeros((0, 3), np.float32),
                     g.Source(g.SRC_VOLUME_POLYGON, g.LXE, n_sides=24, radius=1300.0, z_min=-2597.0, z_max=-1.0))
    ev = g.grid_sources(det, 1_000_000)
    assert len(ev) == 256 and all(n == 1_000_000 and s.kind == g.SRC_POINT for s, n in ev)
    c = np.array([s.center for s, _ in ev])
    assert np.all(np.mod(c, 100.0) == 0.0)
    apothem = 1300.0 * math.cos(math.pi / 24)
    for k in range(24):
        a = 2 * math.pi * (k + 0.5) / 24
        assert np.all(c[:, 0] * math.cos(a) + c[:, 1] * math.sin(a) <= apothem - 50.0)
    assert c[:, 2].min() >= -2597.0 + 50.0 and c[:, 2].max() <= -1.0 - 50.0
    assert len(np.unique(c, axis=0)) == 256
    assert len(np.unique(c[:, 2])) >= 20 and np.ptp(c[:, 0]) >= 2000 and np.ptp(c[:, 1]) >= 2000
    every = g.grid_sources(det, 1, n_sources=10 ** 9)
    assert 11_000 < len(every) < 13_000
    assert [s.center for s, _ in g.grid_sources(det, 1, seed=0)] == [s.center for s, _ in ev]
    assert [s.center for s, _ in g.grid_sources(det, 1, seed=1)] != [s.center for s, _ in ev]
