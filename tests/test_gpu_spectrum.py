"""Emission spectrum and dispersion on the GPU through the C ABI.

* Per-photon wavelengths equal the oracle's (same photon ids; float32
  against float64 Box-Muller).
* A spectrum without dispersion changes nothing.
* With dispersion, parity with the oracle on the small TPC uses the same
  criteria as the monochromatic path, and the photons do take other paths
  than at 175 nm.
* Closed forms: the dispersed E1 reflection series and the arrival time at
  c / n(lambda).
* Batched events with spectra equal single-source runs bit for bit.
* Bad spectra and dispersion are rejected before any launch, and the
  context stays usable afterwards."""
import math
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from paper_2203_14354_gb300._capi import LxoError
from tests.paired import sign_test
from tests.test_gpu_propagate import SAME_SMALL, beam, np_out, sig2, to_dev

pytestmark = pytest.mark.gpu

C_MM_NS = 299.792458


def dispersed(det, m=g.LXE, dn=-0.004, p=4.0):
    det.materials = list(det.materials)
    det.materials[m] = replace(det.materials[m], dn_dlambda_per_nm=dn, rayleigh_exp=p)
    return det


@pytest.fixture(scope="module")
def small():
    from paper_2203_14354_gb300 import Tracker
    det = g.small_tpc()
    return det, Tracker(det)


@pytest.fixture(scope="module")
def small_dispersed():
    from paper_2203_14354_gb300 import Tracker
    det = dispersed(g.small_tpc())
    det.source = det.source.with_spectrum(g.LXE_SPECTRUM)
    return det, Tracker(det), O.Oracle(det)


def test_wavelengths_match_oracle(small):
    det, trk = small
    orc = O.Oracle(det)
    n = 50_000
    src = det.source.with_spectrum(g.LXE_SPECTRUM)
    pos, d, pol, wl = trk.sample_source(n, base=991, seed=5, source=src, wavelength=True)
    ref = orc.sample_source(n, base=991, seed=5, src=src, wavelength=True)
    np.testing.assert_allclose(wl.cpu().numpy(), ref[4], rtol=0, atol=2e-3)
    # the spectrum leaves the rest of the first state bit-identical
    p0, d0, e0 = trk.sample_source(n, base=991, seed=5, source=det.source)
    assert torch.equal(pos, p0) and torch.equal(d, d0) and torch.equal(pol, e0)
    # one wavelength: exactly the mean (175 nm by default)
    assert torch.all(trk.sample_source(100, source=det.source, wavelength=True)[3] == 175.0)
    mono = replace(det.source, wl_mean_nm=160.0)
    assert torch.all(trk.sample_source(100, source=mono, wavelength=True)[3] == 160.0)


def test_spectrum_without_dispersion_changes_nothing(small):
    det, trk = small
    a = np_out(trk.propagate(100_000, seed=4, per_photon=True))
    b = np_out(trk.propagate(100_000, seed=4, per_photon=True, source=det.source.with_spectrum(g.LXE_SPECTRUM)))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_dispersion_parity_with_oracle(small_dispersed):
    det, trk, orc = small_dispersed
    n = 200_000
    gpu = np_out(trk.propagate(n, seed=0, per_photon=True))
    ref = orc.propagate(n, seed=0, per_photon=True)
    assert gpu["fates"][:7].sum() == n
    for key in ("lce", "det"):
        lg, lo = gpu[key].astype(np.int64), ref[key].astype(np.int64)
        for c in range(det.n_pmts):
            p = lo[c] / n
            assert abs(lg[c] - lo[c]) / n <= 4 * sig2(p, n, n) + 1e-9, (key, c, lg[c], lo[c])
        assert abs(lg.sum() - lo.sum()) / lo.sum() < 0.02
    pt = sign_test(gpu["fate"], gpu["detail"], ref["fate"], ref["detail"])
    print("PARITY dispersed_small_tpc", pt)
    assert pt["same"] > SAME_SMALL, pt
    same = (gpu["fate"] == ref["fate"]) & (gpu["detail"] == ref["detail"])
    both = same & (gpu["fate"] == 0)
    close = np.isclose(gpu["time"][both], ref["time"][both], rtol=1e-3, atol=1e-3)
    assert close.mean() > 0.995, close.mean()
    for k in range(7, gpu["fates"].size):
        a, b = int(gpu["fates"][k]), int(ref["fates"][k])
        if k == 7:
            assert abs(a - b) / b < 0.01
        else:
            p = b / n
            assert abs(a - b) / n <= 4 * sig2(p, n, n) + 1e-9, (k, a, b)
    # the dispersion is in effect: at 175 nm for every photon most photons take other paths
    from paper_2203_14354_gb300 import Tracker
    plain = np_out(Tracker(g.small_tpc()).propagate(n, seed=0, per_photon=True))
    unchanged = (plain["fate"] == gpu["fate"]) & (plain["steps"] == gpu["steps"]) & (plain["time"] == gpu["time"])
    assert unchanged.mean() < 0.5, unchanged.mean()


@pytest.mark.parametrize("wl", [160.0, 190.0])
def test_gpu_dispersed_reflection_series_e1(wl):
    from paper_2203_14354_gb300 import Tracker
    dn = -0.01
    trk = Tracker(dispersed(g.layered_box(), dn=dn, p=0.0))
    n = 200_000
    ex = to_dev(beam(n, (0, 0, -50), 0.0), trk.device)
    res = np_out(trk.propagate(n, source=g.Source(g.SRC_EXPLICIT, g.LXE, wl_mean_nm=wl), explicit=ex))
    n1 = 1.69 + dn * (wl - 175.0)
    r1 = ((n1 - 1.0) / (n1 + 1.0)) ** 2
    r2 = ((1.0 - 1.6) / 2.6) ** 2
    bottom = r1 + (1 - r1) ** 2 * r2 / (1 - r1 * r2)
    assert abs(res["lce"][0] / n - bottom) < 4 * math.sqrt(bottom * (1 - bottom) / n)


def test_gpu_dispersed_speed_and_rayleigh_length():
    from paper_2203_14354_gb300 import Tracker
    R, dn, wl, lam, p = 100.0, -0.004, 165.0, 80.0, 4.0
    det = dispersed(g.icosphere(R, subdiv=5, ray_len_mm=lam, n_medium=1.69), m=0, dn=dn, p=p)
    det.source = replace(det.source, wl_mean_nm=wl)
    n = 200_000
    res = np_out(Tracker(det).propagate(n, seed=6, per_photon=True))
    direct = res["steps"] == 1
    q = math.exp(-R / (lam * (wl / 175.0) ** p))
    assert abs(direct.mean() - q) < 4 * math.sqrt(q * (1 - q) / n) + 2e-4
    t_exp = R * (1.69 + dn * (wl - 175.0)) / C_MM_NS
    assert np.all(np.abs(res["time"][direct] - t_exp) < 1e-3 * t_exp)


def test_spectral_events_equal_single_source_runs(small_dispersed):
    det, trk, orc = small_dispersed
    ev = [(g.Source(g.SRC_POINT, g.LXE, center=(10.0 * k, -5.0, -20.0 - 10 * k)).with_spectrum(
        (170.0 + 2 * k, 5.0 + k)), 3000 + 500 * k) for k in range(6)]
    ev.append((g.Source(g.SRC_SEGMENT, g.GXE, center=(5.0, 5.0, 0.5), p1=(5.0, 5.0, 4.5)), 4000))
    trk.upload_events(ev)
    out = trk.propagate_events(seed=12, n_tbins=128)
    for e, (src, n) in enumerate(ev):
        one = trk.propagate(n, base=e << 32, seed=12, source=src, n_tbins=128)
        assert torch.equal(one["hist"], out["hist"][e]), e
        assert torch.equal(one["det"], out["det"][e]), e
        assert torch.equal(one["lce"], out["lce"][e]), e


def test_bad_spectra_and_dispersion_are_rejected(small):
    det, trk = small
    src = det.source.with_spectrum(g.LXE_SPECTRUM)
    with pytest.raises(LxoError, match="spectrum"):
        trk.propagate(1000, source=replace(src, wl_fwhm_nm=-1.0))
    with pytest.raises(LxoError, match="spectrum reaches"):
        trk.propagate(1000, source=g.Source(g.SRC_POINT, g.LXE, wl_mean_nm=5.0, wl_fwhm_nm=10.0))
    with pytest.raises(LxoError, match="dispersion"):
        trk.set_materials([replace(m, dn_dlambda_per_nm=float("nan")) for m in det.materials])
    # n(lambda) <= 0 within the spectrum: 1.69 - 0.1 * 25 < 0 at 200 nm
    bad = [replace(m, dn_dlambda_per_nm=-0.1) if i == g.LXE else m for i, m in enumerate(det.materials)]
    trk.set_materials(bad)
    try:
        with pytest.raises(LxoError, match="n <= 0"):
            trk.propagate(1000, source=src)
        point = g.Source(g.SRC_POINT, g.LXE, center=(0.0, 0.0, -50.0)).with_spectrum(g.LXE_SPECTRUM)
        trk.upload_events([(point, 100)])
        with pytest.raises(LxoError, match="n <= 0"):
            trk.propagate_events()
        # one wavelength at 175 nm stays valid
        trk.propagate(1000, source=det.source)
        # the adjoint has no tally for a wavelength-dependent Rayleigh length
        trk.set_materials([replace(m, rayleigh_exp=4.0) if i == g.LXE else m for i, m in enumerate(det.materials)])
        trk.set_adjoint(mats=[g.LXE])
        with pytest.raises(LxoError, match="rayleigh_exp"):
            trk.propagate(1000, adjoint=True)
    finally:
        trk.set_adjoint()
        trk.set_materials(det.materials)
    with pytest.raises(LxoError, match="spectrum"):
        trk.upload_events([(g.Source(g.SRC_POINT, g.LXE, wl_mean_nm=float("inf")), 10)])
    out = np_out(trk.propagate(10_000, seed=1, source=src))
    assert out["fates"][:7].sum() == 10_000
