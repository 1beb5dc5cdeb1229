"""GPU adjoint (LXO_FLAG_ADJOINT, lxo_adjoint_jacobian) through the C ABI:
closed-form derivatives, parity of the per-channel Jacobian with the oracle's
independent adjoint, agreement with central finite differences under common
random numbers, and the autograd Function's backward."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2203_14354_gb300 import tracker
    return tracker


def beam(n, z, up=True, seed=1, spread=10.0):
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 3), np.float32)
    p[:, 0] = rng.uniform(-spread, spread, n)
    p[:, 1] = rng.uniform(-spread, spread, n)
    p[:, 2] = z
    d = np.zeros((n, 3), np.float32)
    d[:, 2] = 1.0 if up else -1.0
    a = rng.uniform(0, 2 * np.pi, n)
    pol = np.stack([np.cos(a), np.sin(a), np.zeros(n)], 1).astype(np.float32)
    return tuple(torch.from_numpy(x).cuda() for x in (p, d, pol))


def test_gpu_adjoint_closed_forms(T):
    lam, R, n = 100.0, 100.0, 400_000
    trk = T.Tracker(g.icosphere(R, subdiv=5, abs_len_mm=lam))
    trk.set_adjoint([0], [])
    out = trk.propagate(n, adjoint=True)
    J = trk.jacobian(out["adjoint"]).cpu().numpy()
    want = n * R / lam ** 2 * math.exp(-R / lam)
    sig = R / lam ** 2 * math.sqrt(n * math.exp(-R / lam) * (1 - math.exp(-R / lam)))
    assert abs(J[0, 0] - want) < 4 * sig + 1e-3 * want
    # electrode transparency: d top / dT = N
    Tt, Rw = 0.9, 0.3
    trk = T.Tracker(g.electrode_box(Tt, Rw))
    trk.set_adjoint([], [2])
    out = trk.propagate(n, source=g.Source(g.SRC_EXPLICIT, 0), explicit=beam(n, -50.0), adjoint=True)
    J = trk.jacobian(out["adjoint"]).cpu().numpy()
    assert abs(J[1, 0] - n) < 4 * math.sqrt(n * Tt * (1 - Tt)) / Tt
    # mirror reflectivity: d top / dR = N
    Rm = 0.8
    trk = T.Tracker(g.reflector_box(Rm, 1.0))
    trk.set_adjoint([], [1])
    out = trk.propagate(n, source=g.Source(g.SRC_EXPLICIT, 0), explicit=beam(n, 0.0, up=False), adjoint=True)
    J = trk.jacobian(out["adjoint"]).cpu().numpy()
    assert abs(J[0, 0] - n) < 4 * math.sqrt(n * Rm * (1 - Rm)) / Rm


def scaled_spec():
    # theta = L_abs(LXe), L_ray(LXe), R(PTFE LXe), R(PTFE GXe), T(gate), T(anode), T(cathode)
    return [g.LXE], [0, 1, 4, 5, 6]


@pytest.fixture(scope="module")
def scaled(T):
    det = g.scaled_tpc()
    # the library holds parameters in float32: give the oracle the same values
    for m in det.materials:
        m.abs_len_mm, m.rayleigh_len_mm = float(np.float32(m.abs_len_mm)), float(np.float32(m.rayleigh_len_mm))
    for sf in det.surfaces:
        sf.reflectivity, sf.transparency = float(np.float32(sf.reflectivity)), float(np.float32(sf.transparency))
    trk = T.Tracker(det)
    mats, surfs = scaled_spec()
    trk.set_adjoint(mats, surfs)
    orc = O.Oracle(det)
    orc.set_adjoint(mats, surfs)
    return det, trk, orc


def pmt_rings(det):
    """Masks of the PMTs of one array on one hexagonal ring of the window
    lattice (pitch = nearest-neighbour distance), top array first."""
    pos = np.asarray(det.pmt_pos, np.float64)[:, :2]
    arr = np.asarray(det.pmt_array)
    one = pos[arr == 1]
    d = np.sqrt(((one[:, None] - one[None]) ** 2).sum(-1)) + np.eye(len(one)) * 1e30
    ring = g.hex_ring(pos, float(np.median(d.min(1))))
    return [(arr == a) & (ring == k) for a in (1, 0) for k in np.unique(ring[arr == a])]


def test_gpu_adjoint_matches_oracle(scaled):
    """GPU and oracle Jacobians of the same photon ids agree statistically:
    per aggregate (top, bottom, all) and per hexagonal ring of each array,
    and per parameter, the summed difference of 40 batches lies within 4
    batch-means standard errors (the photons are independent, so the batch
    differences are too; the same photons on both sides make the
    differences small); the aggregates also within 10 %."""
    det, trk, orc = scaled
    nb, m = 40, 5_000
    top = det.pmt_array == 1
    rings = pmt_rings(det)
    assert len(rings) == 10   # 61 + 61 PMTs: rings 0..4 of each array
    sels = (top, ~top, np.ones_like(top), *rings)
    d = np.zeros((len(sels), nb, trk.n_params))
    ref_tot = np.zeros((len(sels), trk.n_params))
    sums_g, sums_o = 0.0, 0.0
    for b in range(nb):
        out = trk.propagate(m, base=b * m, seed=3, adjoint=True)
        J_g = trk.jacobian(out["adjoint"]).cpu().numpy()
        ref = orc.propagate(m, base=b * m, seed=3, adjoint=True)
        J_o = orc.jacobian(ref["adjoint"])
        if b == 0:
            # the GPU Jacobian of the oracle's sums equals the oracle's Jacobian (same formula)
            J_go = trk.jacobian(torch.from_numpy(ref["adjoint"]).cuda()).cpu().numpy()
            np.testing.assert_allclose(J_go, J_o, rtol=1e-9, atol=1e-9)
        for k, sel in enumerate(sels):
            d[k, b] = J_g[sel].sum(0) - J_o[sel].sum(0)
            ref_tot[k] += J_o[sel].sum(0)
        sums_g = sums_g + out["adjoint"].cpu().numpy().sum(0)
        sums_o = sums_o + ref["adjoint"].sum(0)
    D = d.sum(1)
    se = np.sqrt(nb) * d.std(1, ddof=1)
    tiny = 1e-9 * np.abs(ref_tot).max()
    z = np.abs(D) / np.maximum(se, tiny)
    print("PARITY adjoint z per selection (rows: top, bottom, all, 10 rings):", np.round(z, 2).tolist())
    assert np.all(np.abs(D) <= 4 * se + tiny), (D, se)
    assert np.all(np.abs(D[:3]) <= 0.10 * np.abs(ref_tot[:3]) + tiny), (D[:3], ref_tot[:3])
    # the tallies themselves (path lengths, counts) agree per channel in sum
    np.testing.assert_allclose(sums_g, sums_o, rtol=0.03)


def test_gpu_adjoint_vs_central_fd_crn(scaled):
    """Central finite differences with common random numbers (same seed and
    photon ids at theta +- h): the total detected hits' derivative agrees
    with the adjoint within their batch-means errors."""
    det, trk, orc = scaled
    theta0 = trk.theta()
    n_b, B = 250_000, 8
    rel = {0: 0.02, 1: 0.02, 2: 0.002, 3: 0.01, 4: 0.01, 5: 0.01, 6: 0.01}
    adj = np.zeros((B, trk.n_params))
    fd = np.zeros((B, trk.n_params))
    trk.set_theta(theta0)
    for b in range(B):
        out = trk.propagate(n_b, base=b * n_b, seed=11, adjoint=True)
        adj[b] = trk.jacobian(out["adjoint"]).sum(0).cpu().numpy()
    for q, r in rel.items():
        h = r * float(theta0[q])
        for b in range(B):
            tot = []
            for sgn in (+1, -1):
                th = theta0.clone()
                th[q] += sgn * h
                trk.set_theta(th)
                out = trk.propagate(n_b, base=b * n_b, seed=11)
                tot.append(float(out["det"].sum().item()))
            fd[b, q] = (tot[0] - tot[1]) / (2 * h)
    trk.set_theta(theta0)
    a_m, a_s = adj.mean(0), adj.std(0, ddof=1) / math.sqrt(B)
    f_m, f_s = fd.mean(0), fd.std(0, ddof=1) / math.sqrt(B)
    z = np.abs(a_m - f_m) / np.sqrt(a_s ** 2 + f_s ** 2 + 1e-30)
    assert np.all(z < 4.5), (a_m, f_m, a_s, f_s, z)
    # where both estimates are sharp, they agree within 5 %
    sharp = (a_s < 0.02 * np.abs(a_m)) & (f_s < 0.02 * np.abs(f_m))
    assert np.all(np.abs(a_m[sharp] - f_m[sharp]) < 0.05 * np.abs(f_m[sharp]) + 4 * np.sqrt(a_s ** 2 + f_s ** 2)[sharp])


def test_light_collection_autograd(scaled, T):
    det, trk, orc = scaled
    theta = trk.theta().clone().requires_grad_(True)
    hits = T.LightCollection.apply(theta, trk, 100_000, 7)
    w = torch.linspace(0.0, 1.0, hits.numel(), dtype=torch.float64, device=hits.device)
    (hits * w).sum().backward()
    out = trk.propagate(100_000, seed=7, adjoint=True)
    J = trk.jacobian(out["adjoint"])
    want = (J * w[:, None]).sum(0).cpu()
    torch.testing.assert_close(theta.grad, want, rtol=1e-9, atol=1e-9)
    assert torch.equal(hits.cpu(), out["det"].double().cpu())


def test_adjoint_flag_does_not_change_the_forward(scaled):
    det, trk, orc = scaled
    a = trk.propagate(50_000, seed=2)
    b = trk.propagate(50_000, seed=2, adjoint=True)
    for k in ("lce", "det", "hist", "fates"):
        assert torch.equal(a[k], b[k]), k
