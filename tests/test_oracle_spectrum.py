"""Pins of the oracle's emission spectrum and dispersion.

* The spectrum is a Gaussian with the LXe mean and FWHM (Sec. 2.2, Table 2).
  A KS test checks its shape. The definition of the full width at half
  maximum fixes P(|lambda - mean| < FWHM / 2) = erf(sqrt(ln 2)) = 0.761, which
  checks the FWHM-to-sigma conversion separately.
* With the Table 2 constants for every wavelength (no dispersion, the
  paper's setup), a spectrum changes no tally and no photon.
* A dispersed index moves the Sec. 3 worked examples as n(lambda) says: the
  normal-incidence reflection series (E1) and the LXe/GXe critical angle
  (E3).
* A scaled Rayleigh length gives an unscattered fraction of
  exp(-R / L(lambda)).
* The speed c / n(lambda) sets the arrival time of unscattered photons."""
import math
from dataclasses import replace

import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from tests.golden.load import paper_values
from tests.test_oracle_pins import _beam, binom_sigma

PV = paper_values()
N_LXE, N_GXE, N_Q = PV["n_lxe"], PV["n_gxe"], PV["n_quartz"]
C_MM_NS = 299.792458


@pytest.fixture(scope="module")
def orc():
    return O.Oracle(g.icosphere(100.0, subdiv=2))


def wavelengths(orc, src, n=40_000, seed=3):
    return orc.sample_source(n, seed=seed, src=src, wavelength=True)[4]


def with_material(det, m, **kw):
    det.materials = list(det.materials)
    det.materials[m] = replace(det.materials[m], **kw)
    return det


def test_no_spectrum_is_one_wavelength(orc):
    assert np.all(wavelengths(orc, g.Source(g.SRC_POINT, 0), 1000) == 175.0)
    assert np.all(wavelengths(orc, g.Source(g.SRC_POINT, 0, wl_mean_nm=160.0), 1000) == 160.0)


def test_lxe_spectrum_is_the_gaussian_of_its_mean_and_fwhm(orc):
    mean, fwhm = g.LXE_SPECTRUM
    wl = wavelengths(orc, g.Source(g.SRC_POINT, 0).with_spectrum(g.LXE_SPECTRUM))
    sigma = fwhm / (2 * math.sqrt(2 * math.log(2)))
    assert stats.kstest(wl, stats.norm(mean, sigma).cdf).pvalue > 1e-3
    # half maximum at mean +- FWHM/2: the Gaussian mass inside is erf(sqrt(ln 2))
    inside = np.mean(np.abs(wl - mean) < fwhm / 2)
    p = special.erf(math.sqrt(math.log(2)))
    assert abs(p - 0.7610) < 1e-4
    assert abs(inside - p) < 4 * binom_sigma(p, wl.size)
    assert abs(wl.mean() - mean) < 4 * sigma / math.sqrt(wl.size)


def test_spectrum_is_independent_of_the_rest_of_the_first_state(orc):
    src = g.Source(g.SRC_BALL, 0, center=(1.0, 2.0, 3.0), radius=20.0).with_profile(g.NR_PROFILE)
    a = orc.sample_source(20_000, seed=4, src=src, time=True)
    b = orc.sample_source(20_000, seed=4, src=src.with_spectrum(g.LXE_SPECTRUM), time=True, wavelength=True)
    for x, y in zip(a, b[:5]):
        assert np.array_equal(x, y)
    wl, t, d = b[5], b[4], b[1]
    lim = 4 / math.sqrt(wl.size)
    assert abs(np.corrcoef(wl, t)[0, 1]) < lim
    for a_ in range(3):
        assert abs(np.corrcoef(wl, d[:, a_])[0, 1]) < lim


def test_spectrum_without_dispersion_changes_no_step():
    """The paper's setup: optical constants at the mean wavelength for every
    photon, so a spectrum leaves every photon's fate, channel, steps and
    time unchanged."""
    det = g.small_tpc()
    o = O.Oracle(det)
    a = o.propagate(20_000, seed=7, per_photon=True)
    b = o.propagate(20_000, seed=7, per_photon=True, src=det.source.with_spectrum(g.LXE_SPECTRUM))
    for k in ("lce", "det", "hist", "fates", "fate", "detail", "steps", "time"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("wl", [160.0, 175.0, 190.0])
def test_dispersed_index_moves_the_reflection_series(wl):
    """Worked example E1 (Sec. 3) with n_LXe(lambda) = 1.69 - 0.01 (lambda - 175)."""
    dn = -0.01
    det = with_material(g.layered_box(), g.LXE, dn_dlambda_per_nm=dn)
    o = O.Oracle(det)
    n = 200_000
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE, wl_mean_nm=wl),
                      explicit=_beam(n, (0, 0, -50), 0.0))
    n1 = N_LXE + dn * (wl - 175.0)
    r1 = ((n1 - N_GXE) / (n1 + N_GXE)) ** 2
    r2 = ((N_GXE - N_Q) / (N_GXE + N_Q)) ** 2
    bottom = r1 + (1 - r1) ** 2 * r2 / (1 - r1 * r2)
    assert abs(res["lce"][0] / n - bottom) < 4 * binom_sigma(bottom, n)


def test_dispersed_index_moves_the_critical_angle():
    """E3: total internal reflection at the liquid surface above
    asin(1 / n_LXe(lambda)): 36.3 deg at 175 nm, 32.9 deg at 160 nm with
    dn/dlambda = -0.01 per nm, so a 34.5 deg beam reaches the top only at 175 nm."""
    det = with_material(g.layered_box(), g.LXE, dn_dlambda_per_nm=-0.01)
    o = O.Oracle(det)
    n = 20_000
    for wl, want_top in ((175.0, True), (160.0, False)):
        res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE, wl_mean_nm=wl),
                          explicit=_beam(n, (0, 0, -50), 34.5, spread=5))
        assert (res["lce"][1] > 0) == want_top, wl


@pytest.mark.parametrize("wl,p", [(150.0, 4.0), (175.0, 4.0), (150.0, 0.0), (200.0, 2.0)])
def test_rayleigh_length_scaling(wl, p):
    lam, R = 80.0, 100.0
    det = with_material(g.icosphere(R, subdiv=5, ray_len_mm=lam, n_medium=N_LXE), 0, rayleigh_exp=p)
    det.source = replace(det.source, wl_mean_nm=wl)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n, per_photon=True, seed=5)
    direct = res["steps"] == 1
    q = math.exp(-R / (lam * (wl / 175.0) ** p))
    assert abs(direct.mean() - q) < 4 * binom_sigma(q, n) + 2e-4


def test_dispersed_speed_sets_the_arrival_time():
    R, dn, wl = 100.0, -0.004, 165.0
    det = with_material(g.icosphere(R, subdiv=5, ray_len_mm=200.0, n_medium=N_LXE), 0, dn_dlambda_per_nm=dn)
    det.source = replace(det.source, wl_mean_nm=wl)
    res = O.Oracle(det).propagate(20_000, per_photon=True, seed=6)
    direct = res["steps"] == 1
    t_exp = R * (N_LXE + dn * (wl - 175.0)) / C_MM_NS
    assert direct.sum() > 1000
    assert np.all(np.abs(res["time"][direct] - t_exp) < 1e-3 * t_exp)
    # and not the 175 nm speed
    assert abs(t_exp - R * N_LXE / C_MM_NS) > 5e-3 * t_exp
