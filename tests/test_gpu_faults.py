"""Failure handling through the C ABI, with every fault made on the host (no
kernel is made to fault or hang): a corrupt mesh and non-finite or
out-of-range parameters are rejected before any launch; an open mesh leaks
photons, which end as ESCAPED in the expected number (the solid angle of
the missing face) on the GPU and in the oracle alike; zero-area triangles
added to a mesh change nothing; a step cap of one step truncates."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from paper_2203_14354_gb300._capi import LxoError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Tracker():
    from paper_2203_14354_gb300 import Tracker
    return Tracker


def open_box(half=50.0):
    """Unit-index medium inside a cube of black walls whose top face is missing."""
    det = g.reflector_box(reflectivity=0.0, half=half, z_bot=-half, z_top=half, mat_n=1.0)
    keep = ~((det.surface == 2) | (det.channel >= 0))        # drop the photocathode ceiling
    det = dataclasses.replace(det, tris=det.tris[keep], mat_inner=det.mat_inner[keep],
                              mat_outer=det.mat_outer[keep], surface=det.surface[keep],
                              channel=det.channel[keep])
    det.surface[det.surface == 1] = 0                          # the floor black too
    return det


def test_corrupt_mesh_and_bad_parameters_are_rejected(Tracker):
    det = g.small_tpc()
    bad = dataclasses.replace(det, tris=det.tris.copy())
    bad.tris[5, 1] = det.verts.shape[0] + 3
    with pytest.raises(LxoError, match="vertex index"):
        Tracker(bad)
    nan = dataclasses.replace(det, verts=det.verts.copy())
    nan.verts[7, 2] = np.nan
    with pytest.raises(LxoError, match="not finite"):
        Tracker(nan)
    trk = Tracker(det)
    mats = [dataclasses.replace(m) for m in det.materials]
    mats[0].abs_len_mm = float("nan")
    with pytest.raises(LxoError, match="material"):
        trk.set_materials(mats)
    surfs = [dataclasses.replace(sf) for sf in det.surfaces]
    surfs[0].reflectivity = 1.2
    with pytest.raises(LxoError, match="probability"):
        trk.set_surfaces(surfs)
    ref = trk.propagate(2000, seed=1)
    again = trk.propagate(2000, seed=1)  # the rejected tables left the context as it was
    assert torch.equal(ref["fates"], again["fates"])


def test_open_mesh_leaks_are_counted(Tracker):
    det = open_box()
    n = 300_000
    out = Tracker(det).propagate(n, seed=4)
    esc = int(out["fates"][4])
    # isotropic photons from the centre of a cube leave through one face in 1/6 of the cases
    assert abs(esc - n / 6) < 4 * np.sqrt(n * (1 / 6) * (5 / 6)), esc
    assert int(out["fates"][3]) + esc == n
    ref = O.Oracle(det).propagate(n, seed=4)
    assert int(ref["fates"][4]) == esc  # the same photons escape on both sides


def test_zero_area_triangles_change_nothing(Tracker):
    det = g.small_tpc()
    rng = np.random.default_rng(2)
    k = 200
    # degenerate triangles: three collinear vertices, and repeated vertices, inside the detector
    a = rng.uniform(-60, 60, (k, 3)).astype(np.float32)
    a[:, 2] = rng.uniform(-90, -10, k)
    b = a + np.float32(3.0)
    c = (a + b) / np.float32(2.0)
    extra = np.stack([a, b, c], 1)
    extra[: k // 2, 1] = extra[: k // 2, 0]
    nv = det.verts.shape[0]
    verts = np.concatenate([det.verts, extra.reshape(-1, 3)])
    tris = np.concatenate([det.tris, (nv + np.arange(3 * k)).reshape(k, 3).astype(det.tris.dtype)])
    fill = lambda x, v: np.concatenate([x, np.full(k, v, x.dtype)])
    deg = dataclasses.replace(det, verts=verts, tris=tris, mat_inner=fill(det.mat_inner, g.LXE),
                              mat_outer=fill(det.mat_outer, g.LXE), surface=fill(det.surface, g.SURF_NONE),
                              channel=fill(det.channel, -1))
    x = Tracker(det).propagate(100_000, seed=6, per_photon=True)
    y = Tracker(deg).propagate(100_000, seed=6, per_photon=True)
    for key in ("lce", "det", "hist", "fates", "fate", "steps", "time"):
        assert torch.equal(x[key], y[key]), key


def test_one_step_cap_truncates(Tracker):
    det = g.small_tpc()
    out = Tracker(det).propagate(50_000, seed=2, max_steps=1)
    f = out["fates"]
    assert int(f[7]) == 50_000  # every photon took exactly its one step
    assert int(f[5]) > 0 and int(f[:7].sum()) == 50_000
