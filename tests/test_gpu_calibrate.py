"""Adjoint tallies of batched events (LXO_FLAG_ADJOINT in
lxo_propagate_events, Jacobian rows event * P + channel) and the gradient
calibration built on them: each event's sums equal a single-source adjoint run
of its photon ids, the sums agree with the oracle's, and Adam on the Poisson
deviance moves the four optical parameters from their defaults to the hidden
values that generated the target hit maps, within the statistical errors
the Fisher information gives."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import calibrate as cal
from paper_2203_14354_gb300 import geometry as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scaled():
    from paper_2203_14354_gb300 import Tracker
    det = g.scaled_tpc()
    for m in det.materials:  # float32 values on both sides
        m.abs_len_mm, m.rayleigh_len_mm = float(np.float32(m.abs_len_mm)), float(np.float32(m.rayleigh_len_mm))
    for sf in det.surfaces:
        sf.reflectivity, sf.transparency = float(np.float32(sf.reflectivity)), float(np.float32(sf.transparency))
    trk = Tracker(det)
    trk.set_adjoint([g.LXE], [0, 1, 4])
    return det, trk


def test_event_adjoint_equals_single_source_runs(scaled):
    det, trk = scaled
    ev = g.calibration_sources(20_000, n_x=3, n_z=3, spacing=120.0, z_center=-250.0)
    ev.append((g.Source(g.SRC_SEGMENT, g.GXE, center=(30.0, -40.0, 0.5), p1=(30.0, -40.0, 2.0)), 15_000))
    ev.append((g.Source(g.SRC_POINT, g.LXE, center=(0.0, 0.0, -100.0)), 0))
    trk.upload_events(ev)
    out = trk.propagate_events(seed=4, hist=False, adjoint=True)
    assert out["adjoint"].shape == (len(ev), trk.n_channels, trk.n_tallies)
    for e, (src, n) in enumerate(ev):
        one = trk.propagate(n, base=e << 32, seed=4, source=src, adjoint=True)
        assert torch.equal(one["det"], out["det"][e]), e
        # same photons, FP64 sums in another atomic order
        torch.testing.assert_close(out["adjoint"][e], one["adjoint"], rtol=1e-12, atol=1e-9)
    assert float(out["adjoint"][-1].abs().sum()) == 0.0
    # the Jacobian of the [E, P, K] sums has one row per (event, channel)
    J = trk.jacobian(out["adjoint"])
    assert J.shape == (len(ev), trk.n_channels, trk.n_params)
    for e in (0, 4, len(ev) - 2):
        torch.testing.assert_close(J[e], trk.jacobian(out["adjoint"][e]), rtol=1e-14, atol=0)
    gv = torch.rand(J.shape[:2], dtype=torch.float64, device=J.device)
    _, grad = trk.jacobian(out["adjoint"], gv)
    torch.testing.assert_close(grad, (J * gv[..., None]).sum((0, 1)), rtol=1e-10, atol=1e-9)


def test_event_adjoint_parity_with_oracle(scaled):
    det, trk = scaled
    ev = g.calibration_sources(60_000, n_x=2, n_z=2, spacing=200.0, z_center=-250.0)
    trk.upload_events(ev)
    out = trk.propagate_events(seed=8, hist=False, adjoint=True)
    orc = O.Oracle(det)
    orc.set_adjoint([g.LXE], [0, 1, 4])
    for e, (src, n) in enumerate(ev):
        ref = orc.propagate(n, base=e << 32, seed=8, src=src, adjoint=True)
        a = out["adjoint"][e].sum(0).cpu().numpy()
        b = ref["adjoint"].sum(0)
        np.testing.assert_allclose(a, b, rtol=0.04)
        Jg = trk.jacobian(out["adjoint"][e]).sum(0).cpu().numpy()
        Jo = orc.jacobian(ref["adjoint"]).sum(0)
        # the Rayleigh-length entry is a difference of two large terms whose
        # per-photon score l/L^2 - N/L has variance about E[N]/L^2 (N Poisson
        # given l): bound it by 4 standard deviations of the difference
        L_ray = det.materials[g.LXE].rayleigh_len_mm
        tol = 0.05 * np.abs(Jo)
        tol[1] = 4.0 * np.sqrt(2.0 * max(b[1], 1.0)) / L_ray
        assert np.all(np.abs(Jg - Jo) <= tol), (e, Jg, Jo, tol)


def test_calibration_recovers_hidden_parameters():
    """50 cm TPC, 64 point sources on a 5 cm grid, 2e5 photons each: start
    from the default optics, recover the hidden ones within 4.5 standard
    deviations of the fit's own covariance."""
    from paper_2203_14354_gb300 import Tracker
    det = g.scaled_tpc()
    trk = Tracker(det)
    trk.set_adjoint([g.LXE], [0, 1])
    theta0 = trk.theta().tolist()
    truth = [30_000.0, 350.0, 0.97, 0.80]
    ev = g.calibration_sources(200_000, n_x=8, n_z=8, spacing=50.0, z_center=-250.0)
    trk.upload_events(ev)
    target = cal.hit_maps(trk, truth, seed=7)
    c = cal.Calibration(trk, ev, target, model_scale=2)
    res = c.fit(theta0)
    rec = torch.tensor(res["theta"], dtype=torch.float64)
    sigma = c.covariance(rec, seed=98).diagonal().sqrt()
    pull = (rec - torch.tensor(truth, dtype=torch.float64)) / sigma
    assert torch.all(pull.abs() < 4.5), (rec, sigma, pull)
    start = (torch.tensor(theta0, dtype=torch.float64) - torch.tensor(truth, dtype=torch.float64)) / sigma
    assert float(pull.norm()) < 0.25 * float(start.norm()), (pull, start)
