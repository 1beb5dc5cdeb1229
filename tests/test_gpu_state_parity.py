"""Per-photon parity of the outgoing wave of every interaction (through the
C ABI): the GPU and the oracle propagate the same photons for 1, 2 and 3
interactions (max_steps), and the state each photon is left in -- position,
direction and polarisation -- is compared photon by photon.  Both sides
draw the same random numbers, so a photon takes the same branch on both
unless a uniform falls within rounding of a threshold; those few are
excluded by requiring the same fate, detail and step count.

The set-ups cover every branch that writes a direction or a polarisation:
Fresnel reflection and refraction below and above the critical angle
(Sec. 2.2, Sec. 3 worked examples), specular and Lambertian reflectors,
electrode wires, Rayleigh scattering and the photocathode, and the small
TPC's volume source mixing all of them.  The oracle's outgoing waves are
pinned to Maxwell's boundary conditions and to the perfect-conductor mirror
(tests/test_oracle_pins.py), so agreement here pins the kernel's."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from tests import closed_forms as CF

pytestmark = pytest.mark.gpu


def _rand_beam(n, z0, theta_deg, up=True, seed=5, spread=150.0, cone=0.0):
    """Beam at theta from the vertical (+- cone degrees of jitter), random
    azimuth of the tilt, random linear polarisation perpendicular to it."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3), np.float32)
    pos[:, :2] = rng.uniform(-spread, spread, (n, 2))
    pos[:, 2] = z0
    th = np.radians(theta_deg + rng.uniform(-cone, cone, n))
    ph = rng.uniform(0, 2 * np.pi, n)
    d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th) * (1 if up else -1)], 1)
    e = np.cross(d, rng.normal(size=(n, 3)))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    return pos, d.astype(np.float32), e.astype(np.float32)


CASES = {
    # name: (detector builder, beam builder or None for the detector's own source)
    "dielectric_below_critical": (g.layered_box, lambda n: _rand_beam(n, -50.0, 20.0, cone=15.0)),
    "dielectric_total_reflection": (g.layered_box, lambda n: _rand_beam(n, -50.0, 55.0, cone=15.0)),
    "quartz_window_oblique": (lambda: g.layered_box(with_gas=False),
                              lambda n: _rand_beam(n, -20.0, 60.0, cone=20.0)),
    "specular_mirror": (lambda: CF.mirror_floor_box(0.7),
                        lambda n: _rand_beam(n, -50.0, 40.0, up=False, cone=30.0)),
    "lambert_reflector": (lambda: g.reflector_box(0.9, 0.0),
                          lambda n: _rand_beam(n, 0.0, 30.0, up=False, cone=30.0)),
    "electrode_wires": (lambda: g.electrode_box(0.5, 0.8, 0.5), lambda n: _rand_beam(n, -50.0, 20.0, cone=20.0)),
    "rayleigh_bulk": (lambda: g.icosphere(100.0, subdiv=4, ray_len_mm=30.0, n_medium=1.69), None),
    "small_tpc": (g.small_tpc, None),
}


@pytest.fixture(scope="module")
def Tracker():
    from paper_2203_14354_gb300 import Tracker
    return Tracker


@pytest.mark.parametrize("case", list(CASES))
def test_outgoing_state_matches_oracle_per_photon(Tracker, case):
    make_det, make_beam = CASES[case]
    det = make_det()
    trk = Tracker(det)
    orc = O.Oracle(det)
    n = 20_000
    kw_g, kw_o = {}, {}
    if make_beam is not None:   # every beam starts in the LXe (material 0)
        beam = make_beam(n)
        kw_g = dict(source=g.Source(g.SRC_EXPLICIT, g.LXE),
                    explicit=tuple(torch.from_numpy(a).to(trk.device) for a in beam))
        kw_o = dict(src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=beam)
    for steps in (1, 2, 3):
        gpu = {k: v.cpu().numpy() for k, v in
               trk.propagate(n, seed=11, max_steps=steps, per_photon=True, **kw_g).items()}
        ref = orc.propagate(n, seed=11, max_steps=steps, per_photon=True, **kw_o)
        same = (gpu["fate"] == ref["fate"]) & (gpu["detail"] == ref["detail"]) & (gpu["steps"] == ref["steps"])
        assert same.mean() > 0.995, (case, steps, same.mean())
        sg, so = gpu["state"][same], ref["state"][same]
        scale = max(1.0, float(np.abs(so[:, :3]).max()))
        dpos = np.abs(sg[:, :3] - so[:, :3]).max(1) / scale
        ddir = np.abs(sg[:, 3:6] - so[:, 3:6]).max(1)
        dpol = np.abs(sg[:, 6:9] - so[:, 6:9]).max(1)
        # float32 photon state against the oracle's float64 physics, a few
        # steps deep: a handful of photons near a branch point differ more
        for name, d, tol in (("position", dpos, 2e-5), ("direction", ddir, 1e-4), ("polarisation", dpol, 1e-4)):
            assert np.mean(d < tol) > 0.999, (case, steps, name, np.quantile(d, [0.5, 0.999, 1.0]))
        # unit, transverse outgoing waves on the GPU
        norm_d = np.linalg.norm(sg[:, 3:6], axis=1)
        norm_e = np.linalg.norm(sg[:, 6:9], axis=1)
        assert np.all(np.abs(norm_d - 1) < 1e-5) and np.all(np.abs(norm_e - 1) < 1e-5)
        assert np.all(np.abs((sg[:, 3:6] * sg[:, 6:9]).sum(1)) < 1e-5)
