"""Pins of the CPU oracle against what the paper and the mathematics fix:
values printed in the paper's worked examples (Sec. 3), closed forms
(Fresnel equations, critical angle, Brewster angle, exponential survival,
escape from an absorbing sphere, geometric series of reflections), invariants
(energy conservation R + T = 1, Stokes relations, transversality), textbook
distributions (1 + cos^2 Rayleigh law, dipole sin^2 law, Lambert cosine law)
and brute force (BVH == all-triangle argmin).  Each is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2203_14354_gb300 import geometry as g
from tests import closed_forms as CF
from tests.golden.load import paper_values

PV = paper_values()
N_LXE, N_GXE, N_Q = PV["n_lxe"], PV["n_gxe"], PV["n_quartz"]


def binom_sigma(p, n):
    return math.sqrt(max(p * (1 - p), 1e-12) / n)


# ---------------------------------------------------------------- Philox ----
def test_uniform_mapping_range():
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert 0.0 < O.uniform(0x12345678) < 1.0


def test_philox_known_answers():
    """The published known-answer vectors of Philox4x32-10 (tests/golden),
    which fix every round constant and the order of the words."""
    from tests.golden.load import philox_kat
    rows = philox_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert [int(x) for x in O.philox(ctr, key)] == want


def test_draw_contract():
    """The oracle draws what the documented contract says, re-derived here
    from the pinned Philox and uniform mapping: key = (seed low, seed high),
    counter = (photon id low, high, step, draw); the source step is
    0xFFFFFFFF, its draw 0 gives cos(theta) = 2 u0 - 1 of an isotropic
    direction; the emission draw (draw 0xFFFFFFFF) picks the time-profile
    component from u0, the delay from u1 and the wavelength from u2, u3
    (Box-Muller); in step 0, draw 0's u0 sets the absorption distance
    -L ln u0.  Ids and seeds have non-zero high words."""
    seed = (3 << 32) | 11
    pids = [(7 << 32) | 5, (1 << 40) | 123, 42]

    def u(pid, step, draw):
        ctr = [pid & 0xFFFFFFFF, pid >> 32, step, draw]
        return [O.uniform(int(x)) for x in O.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])]

    det = g.icosphere(1000.0, subdiv=3, abs_len_mm=50.0, n_medium=N_LXE)
    o = O.Oracle(det)
    f, ts, tt = g.NR_PROFILE
    src = g.Source(g.SRC_POINT, 0).with_profile(g.NR_PROFILE).with_spectrum(g.LXE_SPECTRUM)
    sigma = g.LXE_SPECTRUM[1] / (2 * math.sqrt(2 * math.log(2)))
    for pid in pids:
        pos, d, pol, med, t, wl = o.sample_source(1, base=pid, seed=seed, src=src, time=True, wavelength=True)
        a = u(pid, 0xFFFFFFFF, 0)
        assert d[0, 2] == pytest.approx(2 * a[0] - 1, abs=1e-12)
        assert math.atan2(d[0, 1], d[0, 0]) % (2 * math.pi) == pytest.approx(2 * math.pi * a[1], abs=1e-9)
        e = u(pid, 0xFFFFFFFF, 0xFFFFFFFF)
        tau = ts if e[0] < f else tt
        assert t[0] == pytest.approx(-tau * math.log(e[1]), rel=1e-12)
        z = math.sqrt(-2 * math.log(e[2])) * math.cos(2 * math.pi * e[3])
        assert wl[0] == pytest.approx(g.LXE_SPECTRUM[0] + sigma * z, rel=1e-12)
        # step 0: absorbed at -L ln u0 (the sphere is 20 absorption lengths away)
        res = o.propagate(1, base=pid, seed=seed, src=g.Source(g.SRC_POINT, 0), per_photon=True)
        assert res["fate"][0] == O.BULK_ABS and res["steps"][0] == 1
        dist = -50.0 * math.log(u(pid, 0, 0)[0])
        assert res["time"][0] == pytest.approx(dist * N_LXE / 299.792458, rel=1e-6)


def test_philox_counter_sensitivity_and_uniformity():
    key = np.array([7, 11], np.uint32)
    outs = np.array([O.philox([i, 0, 0, 0], key) for i in range(4096)], np.uint64)
    # every counter word and key word changes the output
    base = O.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(O.philox(c, [5, 6]), base)
    assert not np.array_equal(O.philox([1, 2, 3, 4], [5, 7]), base)
    # no repeats among 16k words; chi^2 of the top 6 bits is flat
    flat = outs.ravel()
    assert len(np.unique(flat)) == flat.size
    hist = np.bincount((flat >> np.uint64(26)).astype(np.int64), minlength=64)
    assert stats.chisquare(hist).pvalue > 1e-4
    # bitwise balance: each of the 32 bits set about half of the time
    bits = ((flat[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).mean(0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / math.sqrt(flat.size))


# --------------------------------------------------------------- Fresnel ----
@pytest.mark.parametrize("n1,n2", [(N_LXE, N_GXE), (N_GXE, N_Q), (N_LXE, N_Q), (N_Q, N_LXE)])
def test_fresnel_normal_incidence_closed_form(n1, n2):
    f = O.fresnel(n1, n2, 1.0)
    r0 = (n1 - n2) / (n1 + n2)
    assert f["rs"] == pytest.approx(r0, abs=1e-15)
    assert f["rp"] == pytest.approx(-r0, abs=1e-15)  # p basis = s x k flips at normal incidence
    assert f["ts"] == pytest.approx(2 * n1 / (n1 + n2), abs=1e-15)


def test_fresnel_paper_values_e1():
    # Sec. 3: 6.5 % reflected at LXe/GXe, 4.6 % at GXe/quartz (normal incidence)
    r1 = O.fresnel(N_LXE, N_GXE, 1.0)["rs"] ** 2
    r2 = O.fresnel(N_GXE, N_Q, 1.0)["rs"] ** 2
    # the paper prints these to 0.1 % (truncated): 6.58 % -> "6.5 %", 4.66 % -> "4.6 %"
    assert 0.0 <= r1 - PV["e1_reflect_lxe_gxe"] < 0.001
    assert 0.0 <= (1 - r1) ** 2 * r2 - PV["e1_reflect_gxe_quartz"] < 0.001
    assert r1 == pytest.approx(0.065795, abs=1e-6)
    assert r2 == pytest.approx(0.053254, abs=1e-6)


@pytest.mark.parametrize("n1,n2", [(N_LXE, N_GXE), (N_GXE, N_Q), (N_LXE, N_Q), (N_Q, N_GXE)])
def test_fresnel_energy_conservation_and_stokes(n1, n2):
    for th in np.linspace(0.0, 89.0, 90):
        ci = math.cos(math.radians(th))
        f = O.fresnel(n1, n2, ci)
        if f["tir"]:
            continue
        ct = f["cos_t"]
        # Snell
        assert n1 * math.sqrt(1 - ci * ci) == pytest.approx(n2 * math.sqrt(1 - ct * ct), abs=1e-12)
        flux = n2 * ct / (n1 * ci)
        assert f["rs"] ** 2 + flux * f["ts"] ** 2 == pytest.approx(1.0, abs=1e-12)
        assert f["rp"] ** 2 + flux * f["tp"] ** 2 == pytest.approx(1.0, abs=1e-12)
        # Stokes relations: r' = -r, t t' = 1 - r^2 (reverse path n2 -> n1 at the refraction angle)
        b = O.fresnel(n2, n1, ct)
        assert b["rs"] == pytest.approx(-f["rs"], abs=1e-12)
        assert b["rp"] == pytest.approx(-f["rp"], abs=1e-12)
        assert f["ts"] * b["ts"] == pytest.approx(1 - f["rs"] ** 2, abs=1e-12)
        assert f["tp"] * b["tp"] == pytest.approx(1 - f["rp"] ** 2, abs=1e-12)


def test_brewster_and_critical_angles():
    # Brewster: tan(theta_B) = n2/n1 -> r_p = 0
    tb = math.atan(N_GXE / N_LXE)
    assert abs(O.fresnel(N_LXE, N_GXE, math.cos(tb))["rp"]) < 1e-12
    assert math.degrees(tb) == pytest.approx(30.61, abs=0.01)
    # critical angles: Sec. 3 (TIR at LXe/GXe at the expected angle; 75 deg on LXe/quartz reflects fully)
    for n1, n2, deg in [(N_LXE, N_GXE, 36.279), (N_LXE, N_Q, 71.217)]:
        tc = math.asin(n2 / n1)
        assert math.degrees(tc) == pytest.approx(deg, abs=1e-3)
        assert not O.fresnel(n1, n2, math.cos(tc - 1e-6))["tir"]
        assert O.fresnel(n1, n2, math.cos(tc + 1e-6))["tir"]
    assert O.fresnel(N_LXE, N_Q, math.cos(math.radians(75.0)))["tir"]


def _basis_case(theta_deg, pol_angle):
    th = math.radians(theta_deg)
    k = np.array([math.sin(th), 0.0, -math.cos(th)])
    N = np.array([0.0, 0.0, 1.0])
    s = np.cross(k, N)
    s /= np.linalg.norm(s)
    p = np.cross(s, k)
    eps = math.cos(pol_angle) * s + math.sin(pol_angle) * p
    return k, N, s, eps


def test_dielectric_geometry_and_polarisation():
    for th in (10.0, 25.0, 35.0, 50.0, 80.0):
        for pa in (0.0, 0.7, 1.5707963):
            k, N, s, eps = _basis_case(th, pa)
            for n1, n2 in [(N_LXE, N_GXE), (N_GXE, N_Q)]:
                for u in (1e-9, 1 - 1e-9):
                    refl, ko, eo, pr = O.dielectric(k, eps, N, n1, n2, u)
                    assert abs(np.linalg.norm(ko) - 1) < 1e-12 and abs(np.linalg.norm(eo) - 1) < 1e-12
                    assert abs(ko @ eo) < 1e-12
                    ci = -k @ N
                    if refl:
                        assert ko @ N == pytest.approx(ci, abs=1e-12)          # law of reflection
                        assert ko[0] == pytest.approx(k[0], abs=1e-12)
                    else:
                        st = n1 / n2 * math.sqrt(1 - ci * ci)
                        assert ko[0] == pytest.approx(st, abs=1e-12)            # Snell, in the plane
                        assert ko @ N < 0
                    # P(reflect) = cs^2 Rs + cp^2 Rp
                    f = O.fresnel(n1, n2, ci)
                    cs = eps @ s
                    want = 1.0 if f["tir"] else cs * cs * f["rs"] ** 2 + (1 - cs * cs) * f["rp"] ** 2
                    assert pr == pytest.approx(want, abs=1e-12)
                    assert refl == (u < want)


def test_brewster_reflection_is_s_polarised():
    tb = math.degrees(math.atan(N_GXE / N_LXE))
    k, N, s, eps = _basis_case(tb, 0.6)
    refl, ko, eo, pr = O.dielectric(k, eps, N, N_LXE, N_GXE, 1e-12)
    assert refl
    assert abs(abs(eo @ s) - 1.0) < 1e-9


def test_normal_incidence_keeps_photon():
    # Appendix item 1: plane of incidence undefined at normal incidence
    k = np.array([0.0, 0.0, -1.0])
    N = np.array([0.0, 0.0, 1.0])
    eps = np.array([1.0, 0.0, 0.0])
    refl, ko, eo, pr = O.dielectric(k, eps, N, N_LXE, N_GXE, 1e-9)
    assert refl and np.allclose(ko, [0, 0, 1]) and abs(abs(eo[0]) - 1) < 1e-12
    assert pr == pytest.approx(((N_LXE - N_GXE) / (N_LXE + N_GXE)) ** 2, abs=1e-12)
    refl, ko, eo, pr = O.dielectric(k, eps, N, N_LXE, N_GXE, 1 - 1e-9)
    assert not refl and np.allclose(ko, k) and abs(abs(eo[0]) - 1) < 1e-12


# ------------------------------------------------ outgoing polarisation -----
# The outgoing polarisation of a dielectric step is pinned by Maxwell's
# boundary conditions (Born & Wolf, Sec. 1.5.1), from which the Fresnel
# formulae themselves follow: across the interface the tangential components
# of E and of H = n k x E (non-magnetic media, units with c = mu = 1) are
# continuous.  The incident wave (k, eps) with unit amplitude, the reflected
# wave (k_r, e_r) and the transmitted wave (k_t, e_t) must therefore admit
# amplitudes a_r, a_t that satisfy four equations at once.  The oracle
# returns only normalised directions, so the test solves for a_r and a_t by
# least squares and requires a zero residual; a polarisation rotated within
# its plane (t_s and t_p swapped, r_s used for both components, a flipped p
# component) leaves a residual of order one.
def _tangential(v, N):
    return v - (v @ N) * N


def _maxwell_residual(k, eps, N, n1, n2, kr, er, kt, et):
    A = np.zeros((6, 2))
    b = np.zeros(6)
    A[:3, 0], A[:3, 1] = _tangential(er, N), -_tangential(et, N)
    b[:3] = -_tangential(eps, N)
    A[3:, 0] = n1 * _tangential(np.cross(kr, er), N)
    A[3:, 1] = -n2 * _tangential(np.cross(kt, et), N)
    b[3:] = -n1 * _tangential(np.cross(k, eps), N)
    amp, *_ = np.linalg.lstsq(A, b, rcond=None)
    return float(np.linalg.norm(A @ amp - b)), amp


def _both_branches(k, eps, N, n1, n2):
    r1, kr, er, pr = O.dielectric(k, eps, N, n1, n2, 0.0)
    r2, kt, et, _ = O.dielectric(k, eps, N, n1, n2, 1.0 - 1e-15)
    assert r1 and not r2
    return kr, er, kt, et, pr


@pytest.mark.parametrize("n1,n2", [(N_LXE, N_GXE), (N_GXE, N_Q), (N_LXE, N_Q), (N_Q, N_GXE), (N_GXE, N_LXE)])
def test_outgoing_polarisation_satisfies_maxwell_boundary_conditions(n1, n2):
    """Reflected and transmitted polarisations of the coherent reading
    (Sec. 2.2: Fresnel surfaces between LXe, GXe and quartz) at oblique
    incidence, for linear polarisations between pure s and pure p and
    interface normals in arbitrary orientation."""
    rng = np.random.default_rng(17)
    crit = math.degrees(math.asin(min(1.0, n2 / n1)))
    for th in (5.0, 20.0, 30.61, 45.0, 60.0, 80.0):
        if th >= crit - 0.5:
            continue
        for pa in (0.0, 0.4, 0.9, 1.3, math.pi / 2, 2.3):
            R = np.linalg.qr(rng.normal(size=(3, 3)))[0]   # random rotation of the whole set-up
            k, N, s, eps = (R @ v for v in _basis_case(th, pa))
            kr, er, kt, et, pr = _both_branches(k, eps, N, n1, n2)
            res, (ar, at) = _maxwell_residual(k, eps, N, n1, n2, kr, er, kt, et)
            assert res < 1e-9, (th, pa, res)
            # the amplitudes found carry the Fresnel energy balance:
            # reflectance + transmitted flux = 1, reflectance = P(reflect)
            ci, ct = -(k @ N), -(kt @ N)
            assert ar * ar == pytest.approx(pr, abs=1e-9)
            assert ar * ar + (n2 * ct) / (n1 * ci) * at * at == pytest.approx(1.0, abs=1e-9)


def test_transmitted_polarisation_angle_from_boundary_conditions():
    """The s / p mix of the refracted wave, tan(psi_t) = (t_p / t_s)
    tan(psi_i), and of the reflected wave, tan(psi_r) = (r_p / r_s)
    tan(psi_i) with p' = s x k', the amplitudes solved from the two boundary
    conditions of each polarisation (not from their closed forms), at the
    three interfaces of the detector (Sec. 2.2), away from Brewster's
    angle."""
    for n1, n2 in [(N_LXE, N_GXE), (N_GXE, N_Q), (N_LXE, N_Q)]:
        for th in (15.0, 34.0, 50.0, 70.0):
            c = CF.fresnel_bc(n1, n2, th)
            if c is None:
                continue
            k, N, s, eps = _basis_case(th, 0.7)
            kr, er, kt, et, _ = _both_branches(k, eps, N, n1, n2)
            psi_t = math.atan2(et @ np.cross(s, kt), et @ s)
            want = math.atan2(c["tp"] * math.sin(0.7), c["ts"] * math.cos(0.7))
            assert math.tan(psi_t) == pytest.approx(math.tan(want), rel=1e-9)
            want_r = c["rp"] * math.sin(0.7) / (c["rs"] * math.cos(0.7))
            assert (er @ np.cross(s, kr)) / (er @ s) == pytest.approx(want_r, rel=1e-9)


def test_total_internal_reflection_keeps_the_polarisation_magnitudes():
    """Under total internal reflection both amplitudes have modulus one
    (reading 1: the phases are dropped), so the s / p magnitudes of the
    polarisation are kept; and the reflected polarisation is continuous
    across the critical angle (its limit from below, where r_s, r_p -> 1),
    which fixes the sign of the p component."""
    for n1, n2 in [(N_LXE, N_GXE), (N_LXE, N_Q), (N_Q, N_GXE)]:
        crit = math.degrees(math.asin(n2 / n1))
        for th in (crit + 1.0, 0.5 * (crit + 90.0), 85.0):
            for pa in (0.3, 1.0, 2.0):
                k, N, s, eps = _basis_case(th, pa)
                refl, kr, er, pr = O.dielectric(k, eps, N, n1, n2, 1.0 - 1e-15)
                assert refl and pr == 1.0
                assert abs(er @ s) == pytest.approx(abs(math.cos(pa)), abs=1e-12)
                assert abs(er @ np.cross(s, kr)) == pytest.approx(abs(math.sin(pa)), abs=1e-12)
        for pa in (0.3, 1.0, 2.0):
            lo = _basis_case(crit - 1e-7, pa)
            hi = _basis_case(crit + 1e-7, pa)
            _, _, e_lo, _ = O.dielectric(lo[0], lo[3], lo[1], n1, n2, 0.0)
            _, _, e_hi, _ = O.dielectric(hi[0], hi[3], hi[1], n1, n2, 0.0)
            assert np.allclose(e_lo, e_hi, atol=2e-3), (n1, n2, pa, e_lo, e_hi)


def test_mirror_polarisation_is_the_perfect_conductor_field():
    """Specular reflection (Sec. 2.2, reflector surfaces): the law of
    reflection, and a polarisation whose tangential part is the negative of
    the incident one with the same modulus (the tangential E of a perfect
    conductor vanishes: E_i,t + E_r,t = 0 at unit reflected amplitude), and
    which is transverse to the reflected direction."""
    rng = np.random.default_rng(23)
    for _ in range(200):
        N = rng.normal(size=3)
        N /= np.linalg.norm(N)
        k = rng.normal(size=3)
        k -= (abs(k @ N) + 0.05) * N if k @ N > 0 else 0.0
        k /= np.linalg.norm(k)
        if k @ N > -0.02:
            continue
        eps = np.cross(k, rng.normal(size=3))
        eps /= np.linalg.norm(eps)
        kr, er = O.mirror(k, eps, N)
        assert kr @ N == pytest.approx(-(k @ N), abs=1e-12)
        assert np.allclose(_tangential(kr, N), _tangential(k, N), atol=1e-12)
        assert abs(er @ kr) < 1e-12 and abs(np.linalg.norm(er) - 1) < 1e-12
        assert np.allclose(_tangential(er, N), -_tangential(eps, N), atol=1e-9)


def test_two_interfaces_carry_the_refracted_polarisation():
    """An oblique beam, polarised half-way between s and p, crosses LXe ->
    GXe -> quartz (the layered set-up of the Sec. 3 worked examples, beam at
    34 deg, just below the LXe/GXe critical angle).  The s / p mix after the
    first refraction sets the reflectance of the quartz window (there R_s =
    0.36, R_p = 0.05), so the fraction reaching the top photocathode tests the
    transmitted polarisation end to end.  Expected value: the exact series
    of reflections between the window and the liquid surface, with the s
    fraction carried through each step by amplitudes from the boundary
    conditions."""
    o = O.Oracle(g.layered_box())
    n = 200_000
    psi = math.radians(45.0)
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=CF.oblique_beam(n, 34.0, psi, -50.0))
    assert res["fates"][O.ESCAPED] == 0 and res["fates"][O.GEOM_ERR] == 0
    top = CF.top_fraction(N_LXE, N_GXE, N_Q, 34.0, math.cos(psi) ** 2)
    frac = res["lce"][1] / n
    assert abs(frac - top) < 4 * binom_sigma(top, n), (frac, top)
    # with t_s and t_p exchanged the window's reflectance would move by > 0.05,
    # more than 40 sigma of this beam
    c1 = CF.fresnel_bc(N_LXE, N_GXE, 34.0)
    c2 = CF.fresnel_bc(N_GXE, N_Q, CF.refraction_angle(N_LXE, N_GXE, 34.0))
    f_ok = CF._after(0.5, c1["ts"], c1["tp"])
    f_swap = CF._after(0.5, c1["tp"], c1["ts"])
    assert abs(CF._reflectance(f_ok, c2) - CF._reflectance(f_swap, c2)) > 0.05


@pytest.mark.parametrize("psi_deg", [45.0, 70.0])
def test_mirror_then_brewster_surface(psi_deg):
    """A beam in the LXe heads down at Brewster's angle of the liquid
    surface (30.6 deg) onto a specular mirror of reflectivity 0.5, then up
    to the surface, where only its s component can reflect back towards the
    lossy mirror (R_p = 0, R_s = 0.23).  The top fraction therefore depends
    on the s / p mix that the mirror leaves (Sec. 2.2 reflector surfaces;
    Sec. 3 layered set-up).  Expected value: the exact series, the mirror
    keeping the s fraction."""
    th = math.degrees(math.atan(N_GXE / N_LXE))
    o = O.Oracle(CF.mirror_floor_box(0.5))
    n = 200_000
    psi = math.radians(psi_deg)
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE),
                      explicit=CF.oblique_beam(n, th, psi, -50.0, up=False))
    assert res["fates"][O.ESCAPED] == 0 and res["fates"][O.GEOM_ERR] == 0
    top = CF.top_fraction(N_LXE, N_GXE, N_Q, th, math.cos(psi) ** 2, first="mirror", mirror_floor=0.5)
    frac = res["lce"][1] / n
    assert abs(frac - top) < 4 * binom_sigma(top, n), (frac, top)


def test_final_state_output_is_the_photon_state():
    """The per-photon final state (the output through which the GPU's
    outgoing waves are compared with the oracle's) holds the photon where
    its last step left it: a beam sent up at 20 deg through the liquid
    surface of the layered set-up stops after one step on the surface,
    reflected by the law of reflection or refracted by Snell's law; after
    two steps the reflected photons sit on the bottom photocathode."""
    o = O.Oracle(g.layered_box())
    n = 2000
    beam = CF.oblique_beam(n, 20.0, 0.6, -50.0)
    r1 = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=beam, max_steps=1, per_photon=True)
    assert np.all(r1["fate"] == O.TRUNCATED) and np.all(r1["steps"] == 1)
    st = r1["state"].astype(np.float64)
    assert np.all(np.abs(st[:, 2]) < 1e-3)
    assert np.allclose(st[:, :2] - beam[0][:, :2], 50.0 * math.tan(math.radians(20.0)) * np.array([1, 0]), atol=1e-3)
    k = beam[1][0].astype(np.float64)
    refl = st[:, 5] < 0
    assert 0 < refl.sum() < n
    assert np.allclose(st[refl, 3:6], k * [1, 1, -1], atol=1e-6)
    assert np.allclose(st[~refl, 3], N_LXE / N_GXE * k[0], atol=1e-6)
    assert np.allclose(np.linalg.norm(st[:, 6:9], axis=1), 1, atol=1e-6)
    assert np.all(np.abs((st[:, 3:6] * st[:, 6:9]).sum(1)) < 1e-6)
    r2 = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=beam, max_steps=2, per_photon=True)
    down = r2["detail"] == 0
    assert np.array_equal(down & (r2["fate"] == O.DETECTED), refl)
    assert np.allclose(r2["state"][down, 2], -100.0, atol=1e-3)


# ------------------------------------------------------------- Rayleigh -----
def test_rayleigh_dipole_laws():
    rng = np.random.default_rng(5)
    n = 40000
    cos_th, cos_psi = np.empty(n), np.empty(n)
    for i in range(n):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        e = rng.normal(size=3)
        e -= (e @ k) * k
        e /= np.linalg.norm(e)
        ko, eo = O.rayleigh(k, e, pid=i, step=3, seed=9)
        assert abs(ko @ eo) < 1e-9 and abs(np.linalg.norm(eo) - 1) < 1e-9
        cos_th[i] = k @ ko
        cos_psi[i] = e @ ko
    # unpolarised marginal: density (3/8)(1 + c^2) on [-1, 1]; <c^2> = 2/5
    cdf_th = lambda c: (3 * (c + 1) + (c ** 3 + 1)) / 8
    assert stats.kstest(cos_th, cdf_th).pvalue > 1e-4
    assert np.mean(cos_th ** 2) == pytest.approx(0.4, abs=5 * 0.3 / math.sqrt(n))
    # relative to the polarisation: density (3/4)(1 - c^2) (dipole sin^2 law)
    cdf_psi = lambda c: (3 * (c + 1) - (c ** 3 + 1)) / 4
    assert stats.kstest(cos_psi, cdf_psi).pvalue > 1e-4
    assert np.mean(cos_psi ** 2) == pytest.approx(0.2, abs=5 * 0.25 / math.sqrt(n))


def test_lambert_cosine_law():
    N = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    n = 30000
    c = np.empty(n)
    for i in range(n):
        ko, eo = O.lambert(N, pid=i, step=1, seed=4)
        c[i] = ko @ N
        assert abs(ko @ eo) < 1e-9
    assert c.min() > 0
    assert stats.kstest(c, lambda x: np.clip(x, 0, 1) ** 2).pvalue > 1e-4


# ------------------------------------------------------------ intersection --
def test_intersection_axis_aligned_square_closed_form():
    # the square z = 10, |x|,|y| <= 5 as two triangles
    verts = np.array([[-5, -5, 10], [5, -5, 10], [5, 5, 10], [-5, 5, 10]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.uint32)
    z8 = np.zeros(2, np.uint8)
    det = g.Detector("sq", verts, tris, z8, z8.copy(), np.full(2, g.SURF_NONE, np.uint16), np.full(2, -1, np.int32),
                     [g.Material("m", 1.0)], [], np.zeros(0, np.int32), np.zeros((0, 3), np.float32),
                     g.Source(g.SRC_POINT))
    o = O.Oracle(det)
    rng = np.random.default_rng(0)
    n = 2000
    org = np.zeros((n, 3), np.float32)
    org[:, :2] = rng.uniform(-4, 4, (n, 2))
    dz = np.ones(n, np.float32)
    dirs = np.stack([rng.uniform(-0.1, 0.1, n), rng.uniform(-0.1, 0.1, n), dz], 1).astype(np.float32)
    hit, t = o.trace(org, dirs)
    land = org[:, :2] + 10 * dirs[:, :2]
    inside = np.all(np.abs(land) < 4.999, 1)
    assert np.all(hit[inside] != 0xFFFFFFFF)
    np.testing.assert_allclose(t[inside], 10.0, rtol=2e-7)
    # triangle choice matches which side of the diagonal y = x the ray lands on
    side = land[inside, 1] < land[inside, 0]
    assert np.array_equal(hit[inside] == 0, side)
    # rays pointing away miss; tmax clips; skip excludes
    hit2, _ = o.trace(org, -dirs)
    assert np.all(hit2 == 0xFFFFFFFF)
    hit3, _ = o.trace(org, dirs, tmax=np.full(n, 9.9, np.float32))
    assert np.all(hit3 == 0xFFFFFFFF)
    hit4, _ = o.trace(org[inside], dirs[inside], skip=hit[inside])
    assert np.all(hit4 == 0xFFFFFFFF)


def test_bvh_equals_brute_force_on_soup():
    det = g.random_soup(3000, seed=3)
    o = O.Oracle(det)
    rng = np.random.default_rng(1)
    n = 3000
    org = rng.uniform(-120, 120, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    # aim a third of the rays exactly at vertices and edge midpoints (ties, shared edges)
    tv = det.verts[det.tris]
    m = n // 3
    tgt = np.concatenate([tv[:m // 2, 0], (0.5 * (tv[m // 2:m, 0] + tv[m // 2:m, 1]))])
    dd = tgt - org[:m]
    d[:m] = (dd / np.linalg.norm(dd, axis=1, keepdims=True)).astype(np.float32)
    skip = rng.integers(0, det.n_tris, n).astype(np.uint32)
    skip[::2] = 0xFFFFFFFF
    tmax = np.where(rng.uniform(size=n) < 0.3, rng.uniform(1, 200, n), np.inf).astype(np.float32)
    hb, tb = o.trace(org, d, skip, tmax, brute=True)
    hv, tv2 = o.trace(org, d, skip, tmax, brute=False)
    assert np.array_equal(hb, hv)
    assert np.array_equal(tb, tv2)
    assert (hb != 0xFFFFFFFF).sum() > n // 4


def test_ties_go_to_the_smallest_index():
    """Exact ties: a soup whose first 400 triangles are repeated under ids
    1000..1399.  Every hit on a repeated triangle is a tie at the same t,
    and the smaller index wins, in the BVH as in the brute-force search."""
    from dataclasses import replace
    base = g.random_soup(1000, seed=5)
    extra = base.tris[:400]
    det = replace(base, tris=np.concatenate([base.tris, extra]),
                  mat_inner=np.concatenate([base.mat_inner, base.mat_inner[:400]]),
                  mat_outer=np.concatenate([base.mat_outer, base.mat_outer[:400]]),
                  surface=np.concatenate([base.surface, base.surface[:400]]),
                  channel=np.concatenate([base.channel, base.channel[:400]]))
    o = O.Oracle(det)
    rng = np.random.default_rng(6)
    n = 2000
    tv = det.verts[det.tris[:400]].astype(np.float64)
    k = rng.integers(0, 400, n)
    w = rng.dirichlet([1, 1, 1], n)
    tgt = np.einsum("nj,njk->nk", w, tv[k])
    org = (tgt + rng.normal(0, 60, (n, 3))).astype(np.float32)
    d = tgt - org
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    hb, tb = o.trace(org, d, None, None, brute=True)
    hv, tv2 = o.trace(org, d, None, None, brute=False)
    assert np.array_equal(hb, hv) and np.array_equal(tb, tv2)
    hit = hb != 0xFFFFFFFF
    assert np.sum(hit & (hb < 400)) > n // 2
    assert not np.any(hit & (hb >= 1000))


def test_watertight_closed_sphere():
    det = g.icosphere(50.0, subdiv=3)
    o = O.Oracle(det)
    tv = det.verts[det.tris].astype(np.float64)
    rng = np.random.default_rng(2)
    # from interior points, aim exactly at every vertex and at edge midpoints
    targets = np.concatenate([det.verts.astype(np.float64), 0.5 * (tv[:, 0] + tv[:, 1])])
    org = rng.uniform(-10, 10, (targets.shape[0], 3))
    d = targets - org
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    hit, t = o.trace(org.astype(np.float32), d.astype(np.float32))
    assert np.all(hit != 0xFFFFFFFF)


# ------------------------------------------------ full tracker: worked examples
def _beam(n, pos, theta_deg, seed=1, spread=10.0):
    rng = np.random.default_rng(seed)
    p = np.tile(np.asarray(pos, np.float32), (n, 1))
    p[:, 0] += rng.uniform(-spread, spread, n)
    p[:, 1] += rng.uniform(-spread, spread, n)
    th = math.radians(theta_deg)
    d = np.tile(np.array([math.sin(th), 0, math.cos(th)], np.float32), (n, 1))
    a = rng.uniform(0, 2 * np.pi, n)
    s = np.array([0, 1, 0], np.float32)
    pp = np.array([math.cos(th), 0, -math.sin(th)], np.float32)
    pol = (np.cos(a)[:, None] * s + np.sin(a)[:, None] * pp).astype(np.float32)
    return p, d, pol


def test_worked_example_e1_reflection_series():
    """Sec. 3 first check: 11.2 % bottom / 88.8 % top for photons sent straight up."""
    det = g.layered_box()
    o = O.Oracle(det)
    n = 200_000
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=_beam(n, (0, 0, -50), 0.0))
    r1 = ((N_LXE - N_GXE) / (N_LXE + N_GXE)) ** 2
    r2 = ((N_GXE - N_Q) / (N_GXE + N_Q)) ** 2
    bottom = r1 + (1 - r1) ** 2 * r2 / (1 - r1 * r2)
    frac = res["lce"] / n
    assert abs(frac[0] - bottom) < 4 * binom_sigma(bottom, n)
    assert abs(frac[1] - (1 - bottom)) < 4 * binom_sigma(bottom, n)
    assert round(frac[0], 3) == pytest.approx(PV["e1_bottom"], abs=0.0015)
    assert round(frac[1], 3) == pytest.approx(PV["e1_top"], abs=0.0015)
    assert res["fates"][O.ESCAPED] == 0 and res["fates"][O.GEOM_ERR] == 0


def test_total_internal_reflection_on_shared_edges():
    """Photons aimed exactly along the edges that the triangles of the liquid
    surface share (its fan's diagonals x = +-y) at 45 deg, above the LXe/GXe
    critical angle: every one is totally reflected back into the liquid and
    reaches the bottom photocathode.  None comes back through the
    neighbouring triangle of the edge, which a reflected photon left on the
    wrong side of the surface would (Sec. 3, Appendix item 2 on shared
    edges)."""
    det = g.layered_box()
    o = O.Oracle(det)
    n = 4000
    rng = np.random.default_rng(4)
    a = rng.uniform(-300, 300, n).astype(np.float32)
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    pos = np.stack([a, sgn * a, np.full(n, -50.0, np.float32)], 1).astype(np.float32)
    s = np.float32(math.sin(math.radians(45.0)) / math.sqrt(2.0))
    d = np.stack([np.full(n, s), sgn * s, np.full(n, np.float32(math.cos(math.radians(45.0))))], 1)
    d = d.astype(np.float32)
    e = np.cross(d, rng.normal(size=(n, 3)))
    pol = (e / np.linalg.norm(e, axis=1, keepdims=True)).astype(np.float32)
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=(pos, d, pol))
    assert res["fates"][O.GEOM_ERR] == 0 and res["fates"][O.ESCAPED] == 0
    assert res["lce"][0] == n and res["lce"][1] == 0


def test_worked_example_e2_total_internal_reflection():
    """Sec. 3 second check: 75 deg on the LXe/quartz window reflects 100 %."""
    det = g.layered_box(with_gas=False)
    o = O.Oracle(det)
    n = 50_000
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=_beam(n, (0, 0, -20), 75.0, spread=5))
    assert res["lce"][1] == 0
    assert PV["e2_tir_fraction_75deg"] == 1.0
    # just below the critical angle (71.2 deg) some photons enter the window
    res2 = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=_beam(n, (0, 0, -20), 70.0, spread=5))
    assert res2["lce"][1] > 0


def test_critical_angle_lxe_gxe_e3():
    det = g.layered_box()
    o = O.Oracle(det)
    n = 50_000
    for th, want_top in ((36.5, False), (36.0, True)):
        res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, g.LXE), explicit=_beam(n, (0, 0, -50), th, spread=5))
        assert (res["lce"][1] > 0) == want_top


# --------------------------------------------- full tracker: closed forms ----
def test_bulk_absorption_survival_exp():
    lam = 100.0
    det = g.icosphere(100.0, subdiv=5, abs_len_mm=lam)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n)
    p = math.exp(-100.0 / lam)
    assert abs(res["lce"][0] / n - p) < 4 * binom_sigma(p, n) + 2e-4
    assert res["fates"][O.BULK_ABS] + res["lce"].sum() == n


@pytest.mark.parametrize("tau", [1.0, 0.1])
def test_escape_from_absorbing_sphere(tau):
    R = 100.0
    det = g.icosphere(R, subdiv=5, abs_len_mm=R / tau)
    det.source = g.Source(g.SRC_BALL, 0, radius=R * 0.999)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n, seed=3)
    P = 3.0 / (8 * tau ** 3) * (2 * tau ** 2 - 1 + (1 + 2 * tau) * math.exp(-2 * tau))
    assert abs(res["lce"][0] / n - P) < 4 * binom_sigma(P, n) + 2e-3


def test_competing_absorption_and_rayleigh():
    """Absorption and Rayleigh scattering are independent exponential
    processes (their own uniforms of the step): a photon crosses R unscattered
    and unabsorbed with probability exp(-R/L_abs - R/L_ray), and its first
    interaction is an absorption with probability L_ray / (L_abs + L_ray)."""
    la, lr, R = 150.0, 100.0, 100.0
    det = g.icosphere(R, subdiv=5, abs_len_mm=la, ray_len_mm=lr, n_medium=N_LXE)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n, per_photon=True, seed=9)
    direct = (res["steps"] == 1) & (res["fate"] == O.DETECTED)
    p = math.exp(-R / la - R / lr)
    assert abs(direct.mean() - p) < 4 * binom_sigma(p, n) + 2e-4
    first_abs = (res["steps"] == 1) & (res["fate"] == O.BULK_ABS)
    q = (1 - p) * lr / (la + lr)
    assert abs(first_abs.mean() - q) < 4 * binom_sigma(q, n) + 2e-4


def test_rayleigh_mean_free_path_and_time():
    lam, R = 80.0, 100.0
    det = g.icosphere(R, subdiv=5, ray_len_mm=lam, n_medium=N_LXE)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n, per_photon=True, seed=5)
    direct = res["steps"] == 1
    p = math.exp(-R / lam)
    assert abs(direct.mean() - p) < 4 * binom_sigma(p, n) + 2e-4
    # unscattered photons arrive after R * n / c (within the tessellation depth)
    t_exp = R * N_LXE / 299.792458
    assert np.all(np.abs(res["time"][direct] - t_exp) < 1e-3 * t_exp)
    # without absorption every photon is eventually detected
    assert res["lce"][0] == n


def test_mirror_sphere_normal_incidence_series():
    """Radial photons hit a mirror sphere at normal incidence every 2R of
    path (Appendix item 1: such photons must be reflected, not dropped)."""
    lam, R = 300.0, 100.0
    det = g.icosphere(R, subdiv=6, surface_type=g.REFLECTOR, abs_len_mm=lam)
    det.surfaces[0] = g.Surface("mirror", g.REFLECTOR, reflectivity=1.0, spec_frac=1.0)
    o = O.Oracle(det)
    n = 50_000
    res = o.propagate(n, per_photon=True, seed=2)
    assert np.all(res["fate"] == O.BULK_ABS)
    q = math.exp(-R / lam)
    mean_steps = 1 + q / (1 - q * q)
    sd = np.std(res["steps"])
    assert abs(res["steps"].mean() - mean_steps) < 5 * sd / math.sqrt(n)


def test_reflector_absorption_geometric():
    R_ptfe = 0.8
    det = g.icosphere(100.0, subdiv=4, surface_type=g.REFLECTOR)
    det.surfaces[0] = g.Surface("ptfe", g.REFLECTOR, reflectivity=R_ptfe, spec_frac=0.0)
    o = O.Oracle(det)
    n = 50_000
    res = o.propagate(n, per_photon=True, seed=8)
    assert np.all(res["fate"] == O.SURF_ABS)
    mean = 1 / (1 - R_ptfe)
    sd = math.sqrt(R_ptfe) / (1 - R_ptfe)
    assert abs(res["steps"].mean() - mean) < 5 * sd / math.sqrt(n)


@pytest.mark.parametrize("kind", ["reflector", "electrode"])
def test_specular_share_of_reflections(kind):
    """Photons from the centre of a lossless reflecting sphere: a specular
    first reflection sends the photon back through the centre (second leg
    about 2R), a Lambertian one along a chord 2R cos(theta) with cos(theta) =
    sqrt(u), longer than 2R (1 - d) with probability 1 - (1 - d)^2 only.  The
    share of long second legs is the specular fraction f (+ that small
    Lambertian share); both the reflector and the wire reflection of an
    electrode follow it."""
    f, R, dl = 0.3, 100.0, 3e-3
    if kind == "reflector":
        det = g.icosphere(R, subdiv=5, surface_type=g.REFLECTOR)
        det.surfaces[0] = g.Surface("mirror", g.REFLECTOR, reflectivity=1.0, spec_frac=f)
    else:
        det = g.icosphere(R, subdiv=5, surface_type=g.ELECTRODE_T)
        det.surfaces[0] = g.Surface("wires", g.ELECTRODE_T, transparency=0.0, wire_reflectivity=1.0,
                                    wire_spec_frac=f)
    n = 100_000
    res = O.Oracle(det).propagate(n, per_photon=True, seed=12, max_steps=2)
    assert np.all(res["fate"] == O.TRUNCATED)
    leg2 = res["time"].astype(np.float64) * 299.792458 / det.materials[0].n - R
    long = np.mean(leg2 > 2 * R * (1 - dl))
    p = f + (1 - f) * (1 - (1 - dl) ** 2)
    assert abs(long - p) < 4 * binom_sigma(p, n) + 2e-3, (long, p)


def test_arrival_histogram_bins_the_photon_times():
    """The per-channel arrival histogram is the binning of the detected
    photons' own times: bin floor(t / width), the last bin for t beyond
    the range."""
    det = g.small_tpc()
    n, width, bins = 40_000, 0.25, 8
    res = O.Oracle(det).propagate(n, per_photon=True, seed=13, tbin_ns=width, n_tbins=bins)
    det_ph = res["fate"] == O.DETECTED
    ch, t = res["detail"][det_ph], res["time"][det_ph].astype(np.float64)
    b = np.minimum(np.floor(t / width), bins).astype(np.int64)
    want = np.zeros((det.n_pmts, bins + 1), np.int64)
    np.add.at(want, (ch, b), 1)
    assert np.array_equal(res["hist"].astype(np.int64), want)
    assert want[:, bins].sum() > 0 and want[:, :bins].sum() > 0


def test_electrode_transparency():
    T, Rw = 0.9, 0.3
    det = g.electrode_box(T, Rw)
    o = O.Oracle(det)
    n = 100_000
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, 0), explicit=_beam(n, (0, 0, -50), 0.0))
    assert abs(res["lce"][1] / n - T) < 4 * binom_sigma(T, n)
    absorbed = res["fates"][O.N_FIXED + 2 + 2]  # surface id 2 (electrode) after 2 materials
    pa = (1 - T) * (1 - Rw)
    assert abs(absorbed / n - pa) < 4 * binom_sigma(pa, n)


def test_quantum_efficiency_and_tallies_consistent():
    det = g.small_tpc()
    o = O.Oracle(det)
    n = 60_000
    res = o.propagate(n, per_photon=True, seed=11)
    f = res["fates"]
    assert f[:7].sum() == n
    assert f[7] == res["steps"].sum()
    assert res["lce"].sum() == f[O.DETECTED] + f[O.QE_FAIL]
    assert res["det"].sum() == f[O.DETECTED] == res["hist"].sum()
    qe = f[O.DETECTED] / res["lce"].sum()
    assert abs(qe - 0.3) < 4 * binom_sigma(0.3, res["lce"].sum())
    assert f[O.ESCAPED] == 0 and f[O.GEOM_ERR] == 0 and f[O.TRUNCATED] == 0
    # per-photon and aggregate agree
    det_ph = res["fate"] == O.DETECTED
    assert np.array_equal(np.bincount(res["detail"][det_ph], minlength=det.n_pmts), res["det"])


# ------------------------------------------------------------------ source --
def test_volume_source_uniform_isotropic():
    det = g.small_tpc()
    o = O.Oracle(det)
    n = 100_000
    pos, dirs, pol, med = o.sample_source(n, seed=1)
    r = np.hypot(pos[:, 0], pos[:, 1])
    assert r.max() <= 100.0 and pos[:, 2].min() >= -100 and pos[:, 2].max() <= 0
    # area fraction inside r < 50 of the 64-gon
    area64 = 0.5 * 64 * 100.0 ** 2 * math.sin(2 * math.pi / 64)
    p = math.pi * 50 ** 2 / area64
    assert abs((r < 50).mean() - p) < 4 * binom_sigma(p, n)
    assert stats.kstest((pos[:, 2] + 100) / 100, "uniform").pvalue > 1e-4
    assert stats.kstest((dirs[:, 2] + 1) / 2, "uniform").pvalue > 1e-4
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4
    assert np.max(np.abs((pol * dirs).sum(1))) < 1e-12
    assert np.all(med == g.LXE)


@pytest.mark.parametrize("n_sides, phase", [(6, 0.0), (6, 0.3), (24, 0.1)])
def test_polygon_source_fills_the_polygon_uniformly(n_sides, phase):
    """Positions of the polygon-prism source (the active volume of Sec. 3's
    uniform photon sources): every point lies inside the regular polygon
    whose vertices are R (cos, sin)(phase + 2 pi k / n), checked edge by edge
    with cross products; the density is uniform over its area, so the share
    inside the inscribed circle is pi a^2 / A with a = R cos(pi / n) and
    A = n R^2 sin(2 pi / n) / 2, and each of the n sectors between the centre
    and a side holds 1/n of the points; z is uniform."""
    det = g.small_tpc()
    R, n = 100.0, 60_000
    src = g.Source(g.SRC_VOLUME_POLYGON, g.LXE, n_sides=n_sides, radius=R, phase=phase, z_min=-90.0, z_max=-10.0)
    pos = O.Oracle(det).sample_source(n, seed=3, src=src)[0]
    ang = phase + 2 * np.pi * np.arange(n_sides + 1) / n_sides
    v = R * np.stack([np.cos(ang), np.sin(ang)], 1)
    for k in range(n_sides):
        e = v[k + 1] - v[k]
        side = e[0] * (pos[:, 1] - v[k][1]) - e[1] * (pos[:, 0] - v[k][0])
        assert side.min() >= -1e-9 * R * R, (k, side.min())
    a = R * math.cos(math.pi / n_sides)
    area = n_sides * R * R * math.sin(2 * math.pi / n_sides) / 2
    p_in = math.pi * a * a / area
    r = np.hypot(pos[:, 0], pos[:, 1])
    assert abs((r < a).mean() - p_in) < 4 * binom_sigma(p_in, n)
    sector = np.floor(np.mod(np.arctan2(pos[:, 1], pos[:, 0]) - phase, 2 * np.pi) / (2 * np.pi / n_sides))
    counts = np.bincount(sector.astype(int), minlength=n_sides)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert stats.kstest((pos[:, 2] + 90.0) / 80.0, "uniform").pvalue > 1e-4


def _check_uniform_polarisation(k, eps, n_bins=5):
    """A linear polarisation uniform in angle about the direction k has
    E[(eps.a)^2 | k] = (1 - (k.a)^2) / 2 for every fixed unit axis a (the
    mean of cos^2 over the angle); checked in bins of (k.a)^2 for the three
    axes, within 5 standard errors."""
    for a in range(3):
        c2, e2 = k[:, a] ** 2, eps[:, a] ** 2
        edges = np.quantile(c2, np.linspace(0, 1, n_bins + 1))
        for lo, hi in zip(edges[:-1], edges[1:]):
            m = (c2 >= lo) & (c2 <= hi)
            want = np.mean((1 - c2[m]) / 2)
            got = e2[m].mean()
            se = e2[m].std() / math.sqrt(m.sum())
            assert abs(got - want) < 5 * se + 1e-4, (a, lo, hi, got, want, se)
    # directions within 18 deg of a world axis: the polarisation's angle in
    # the plane perpendicular to that axis, taken modulo pi (a polarisation
    # is a line), is uniform
    for a in range(3):
        u, v = (a + 1) % 3, (a + 2) % 3
        for sgn in (1.0, -1.0):
            m = sgn * k[:, a] > 0.95
            if m.sum() < 500:
                continue
            ang = np.mod(np.arctan2(eps[m, v], eps[m, u]), np.pi) / np.pi
            assert stats.kstest(ang, "uniform").pvalue > 1e-4, (a, sgn)


def test_random_polarisation_is_uniform_about_the_direction():
    """Unpolarised light (Sec. 3: the sources emit random linear
    polarisation; Lambertian reflection depolarises): the source's and the
    Lambertian reflector's new polarisations are uniform in angle about
    their directions."""
    o = O.Oracle(g.small_tpc())
    n = 200_000
    pos, dirs, pol, med = o.sample_source(n, seed=3)
    _check_uniform_polarisation(dirs, pol)
    N = np.array([0.0, 0.0, 1.0])
    out = [O.lambert(N, pid=i, step=2, seed=8) for i in range(40_000)]
    _check_uniform_polarisation(np.array([x[0] for x in out]), np.array([x[1] for x in out]))


def test_generated_meshes_are_closed():
    for det in (g.small_tpc(), g.scaled_tpc(), g.layered_box(), g.icosphere(10, 2), g.electrode_box()):
        t = det.tris.astype(np.int64)
        e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), 1)
        _, cnt = np.unique(e, axis=0, return_counts=True)
        assert np.all(cnt >= 2), det.name
