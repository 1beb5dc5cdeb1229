"""Parity of the GPU closest-hit query (lxo_trace_rays, through the C ABI)
with the oracle: triangle ids bit-exact, hit distances within 1e-5 relative
(they are in fact bit-identical: both sides round the same float operations
in the same order)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g

pytestmark = pytest.mark.gpu
NO = 0xFFFFFFFF


@pytest.fixture(scope="module")
def Tracker():
    from paper_2203_14354_gb300 import Tracker
    return Tracker


def gpu_trace(trk, org, d, skip=None, tmax=None):
    dev = trk.device
    o = torch.from_numpy(np.ascontiguousarray(org, np.float32)).to(dev)
    dd = torch.from_numpy(np.ascontiguousarray(d, np.float32)).to(dev)
    sk = None if skip is None else torch.from_numpy(skip.astype(np.int64).astype(np.int32)).to(dev)
    tm = None if tmax is None else torch.from_numpy(np.ascontiguousarray(tmax, np.float32)).to(dev)
    hit, t = trk.trace_rays(o, dd, sk, tm)
    trk.sync()
    return hit.cpu().numpy().view(np.uint32), t.cpu().numpy()


def rays_for(det, n, seed, extent):
    rng = np.random.default_rng(seed)
    org = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # a third aimed exactly at vertices / edge midpoints, some axis-aligned
    tv = det.verts[det.tris].astype(np.float64)
    m = n // 3
    pick = rng.integers(0, det.n_tris, m)
    tgt = np.where(rng.uniform(size=(m, 1)) < 0.5, tv[pick, 0], 0.5 * (tv[pick, 0] + tv[pick, 1]))
    dd = tgt - org[:m]
    d[:m] = dd / np.linalg.norm(dd, axis=1, keepdims=True)
    k = n // 10
    ax = rng.integers(0, 3, k)
    d[m:m + k] = 0.0
    d[m + np.arange(k), ax] = rng.choice([-1.0, 1.0], k)
    return org, d.astype(np.float32)


def assert_same(h_g, t_g, h_o, t_o):
    assert np.array_equal(h_g, h_o), f"{(h_g != h_o).sum()} ids differ"
    hit = h_o != NO
    assert np.all(np.isinf(t_g[~hit]))
    np.testing.assert_allclose(t_g[hit], t_o[hit], rtol=1e-5, atol=0)
    assert np.array_equal(t_g[hit], t_o[hit])


@pytest.mark.parametrize("leaf", [1, 4, 8])
def test_trace_soup_bit_exact_vs_brute_force(Tracker, leaf):
    det = g.random_soup(3000, seed=3)
    trk = Tracker(det, leaf_size=leaf)
    orc = O.Oracle(det)
    org, d = rays_for(det, 6000, 1, 120.0)
    rng = np.random.default_rng(7)
    skip = rng.integers(0, det.n_tris, org.shape[0]).astype(np.uint32)
    skip[::2] = NO
    tmax = np.where(rng.uniform(size=org.shape[0]) < 0.3, rng.uniform(1, 200, org.shape[0]), np.inf).astype(np.float32)
    h_o, t_o = orc.trace(org, d, skip, tmax, brute=True)
    h_g, t_g = gpu_trace(trk, org, d, skip, tmax)
    assert_same(h_g, t_g, h_o, t_o)
    assert (h_o != NO).sum() > 1000


def test_trace_small_tpc_bit_exact(Tracker):
    det = g.small_tpc()
    trk = Tracker(det)
    orc = O.Oracle(det)
    org, d = rays_for(det, 20000, 2, 95.0)
    org[:, 2] = np.random.default_rng(3).uniform(-99, 4, org.shape[0])
    h_o, t_o = orc.trace(org, d, brute=True)
    h_g, t_g = gpu_trace(trk, org, d)
    assert_same(h_g, t_g, h_o, t_o)


def test_trace_watertight_sphere(Tracker):
    det = g.icosphere(50.0, subdiv=4)
    trk = Tracker(det)
    rng = np.random.default_rng(4)
    tv = det.verts[det.tris].astype(np.float64)
    targets = np.concatenate([det.verts.astype(np.float64), 0.5 * (tv[:, 0] + tv[:, 1])])
    org = rng.uniform(-10, 10, (targets.shape[0], 3))
    d = targets - org
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    h_g, t_g = gpu_trace(trk, org, d)
    assert np.all(h_g != NO)
    h_o, t_o = O.Oracle(det).trace(org.astype(np.float32), d.astype(np.float32), brute=True)
    assert_same(h_g, t_g, h_o, t_o)


def test_trace_single_triangle_and_empty_batch(Tracker):
    verts = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32)
    det = g.Detector("tri", verts, np.array([[0, 1, 2]], np.uint32), np.zeros(1, np.uint8), np.zeros(1, np.uint8),
                     np.full(1, g.SURF_NONE, np.uint16), np.full(1, -1, np.int32), [g.Material("m", 1.0)], [],
                     np.zeros(0, np.int32), np.zeros((0, 3), np.float32), g.Source(g.SRC_POINT))
    trk = Tracker(det)
    org, d = np.array([[0.2, 0.2, 0.0], [2, 2, 0]], np.float32), np.array([[0, 0, 1.0], [0, 0, 1.0]], np.float32)
    h, t = gpu_trace(trk, org, d)
    assert list(h) == [0, NO] and t[0] == pytest.approx(5.0, rel=1e-6)
    assert_same(h, t, *O.Oracle(det).trace(org, d, brute=True))
    h, t = gpu_trace(trk, np.zeros((0, 3)), np.zeros((0, 3)))
    assert h.size == 0


@pytest.fixture(scope="module")
def darwin():
    return g.darwin()


def test_trace_darwin_full_size_sampled(Tracker, darwin):
    """Full 1.8e7-triangle DARWIN mesh: rays from the active volume, from the
    gas gap and aimed at the wire meshes; GPU == oracle BVH (itself pinned to
    brute force), plus a few rays against brute force over every triangle."""
    det = darwin
    trk = Tracker(det)
    orc = O.Oracle(det)
    rng = np.random.default_rng(11)
    n = 60000
    r = 1280 * np.sqrt(rng.uniform(size=n))
    a = rng.uniform(0, 2 * np.pi, n)
    org = np.stack([r * np.cos(a), r * np.sin(a), rng.uniform(-2690, 60, n)], 1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # a third towards random points of the electrode planes (wire hits)
    m = n // 3
    tz = rng.choice([0.0, 8.0, -2598.0], m)
    tr = 1200 * np.sqrt(rng.uniform(size=m))
    ta = rng.uniform(0, 2 * np.pi, m)
    tgt = np.stack([tr * np.cos(ta), tr * np.sin(ta), tz + rng.uniform(-0.15, 0.15, m)], 1)
    dd = tgt - org[:m]
    d[:m] = dd / np.linalg.norm(dd, axis=1, keepdims=True)
    tmax = np.where(rng.uniform(size=n) < 0.5, rng.exponential(400.0, n), np.inf).astype(np.float32)
    org, d = org.astype(np.float32), d.astype(np.float32)
    h_o, t_o = orc.trace(org, d, tmax=tmax)
    h_g, t_g = gpu_trace(trk, org, d, tmax=tmax)
    assert_same(h_g, t_g, h_o, t_o)
    hit_surf = det.surface[h_o[h_o != NO]]
    assert np.isin([4, 5, 6], hit_surf).all()  # every wire mesh was hit
    k = 8
    h_b, t_b = orc.trace(org[:k], d[:k], tmax=tmax[:k], brute=True)
    assert_same(h_g[:k], t_g[:k], h_b, t_b)
