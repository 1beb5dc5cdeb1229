"""Mutation tests of the oracle's pins.

Each entry plants one plausible mistake in a copy of oracle.c: a dropped
term, a wrong sign, a wrong index or a swapped operand. The copy is built
with the oracle's own flags, and the pins named beside the mistake are run
against it in a subprocess (ORACLE_LIB selects the library). At least one
of them must fail. The unmodified oracle passes every pin (the rest of the
suite), so a surviving mutant would mark a part of the oracle that no pin
fixes.

Two mistakes are left out because they change no result: both remove one of
two safeguards. Not skipping the last triangle hit changes nothing, because
the spawn offset already keeps a photon off that surface. Dropping the
1e-3 mm margin of the oracle's box test changes nothing, because its
double-precision slab test on exact float boxes never needed it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py::"
ADJ = "tests/test_oracle_adjoint.py::"
TIME = "tests/test_oracle_time_profile.py::"
SPEC = "tests/test_oracle_spectrum.py::"

# (name, text in oracle.c, planted replacement, pins that must catch it)
MUTANTS = [
    ("Philox multiplier off by two", "uint64_t p0 = (uint64_t)0xD2511F53u * c0;",
     "uint64_t p0 = (uint64_t)0xD2511F55u * c0;", [PINS + "test_philox_known_answers"]),
    ("Fresnel r_p numerator with the indices swapped", "out[1] = (n2 * cos_i - n1 * cos_t)",
     "out[1] = (n1 * cos_i - n2 * cos_t)", [PINS + "test_brewster_and_critical_angles"]),
    ("Fresnel t_s over the p denominator", "out[2] = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);",
     "out[2] = 2.0 * n1 * cos_i / (n2 * cos_i + n1 * cos_t);", [PINS + "test_fresnel_energy_conservation_and_stokes"]),
    ("refracted direction with the wrong sign of cos t", "k_out[a] = eta * k[a] + (eta * cos_i - cos_t) * N[a];",
     "k_out[a] = eta * k[a] + (eta * cos_i + cos_t) * N[a];", [PINS + "test_dielectric_geometry_and_polarisation"]),
    ("s and p reflectances swapped in P(reflect)",
     "double pr = tir ? 1.0 : cs * cs * f[0] * f[0] + cp * cp * f[1] * f[1];",
     "double pr = tir ? 1.0 : cs * cs * f[1] * f[1] + cp * cp * f[0] * f[0];",
     [PINS + "test_dielectric_geometry_and_polarisation", PINS + "test_brewster_reflection_is_s_polarised"]),
    ("Rayleigh cosine from the wrong root of the cubic", "(acos(1.0 - 2.0 * u[0]) + 4.0 * PI_D) / 3.0",
     "(acos(1.0 - 2.0 * u[0]) + 2.0 * PI_D) / 3.0", [PINS + "test_rayleigh_dipole_laws"]),
    ("Rayleigh cosine uniform instead of the dipole law",
     "double c = 2.0 * cos((acos(1.0 - 2.0 * u[0]) + 4.0 * PI_D) / 3.0);", "double c = 1.0 - 2.0 * u[0];",
     [PINS + "test_rayleigh_dipole_laws"]),
    ("Rayleigh polarisation not projected off the new direction",
     "for (int a = 0; a < 3; ++a) eps_out[a] = eps[a] - ce * k_out[a];",
     "for (int a = 0; a < 3; ++a) eps_out[a] = eps[a];", [PINS + "test_rayleigh_dipole_laws"]),
    ("Lambert cos theta uniform instead of sqrt(u)", "double c = sqrt(u[0]), sn", "double c = u[0], sn",
     [PINS + "test_lambert_cosine_law"]),
    ("absorption distance drawn from the Rayleigh uniform",
     "double d_abs = isinf(mat[1]) ? INFINITY : -mat[1] * log(u[0]);",
     "double d_abs = isinf(mat[1]) ? INFINITY : -mat[1] * log(u[1]);",
     [PINS + "test_competing_absorption_and_rayleigh"]),
    ("speed c n instead of c / n", "double vel = C_MM_PER_NS / index_at(mat, wl);",
     "double vel = C_MM_PER_NS * index_at(mat, wl);", [PINS + "test_rayleigh_mean_free_path_and_time"]),
    ("reflector absorbs the reflected share", "if (!(u[2] < sp[0])) { fate = ORC_SURF_ABS",
     "if (u[2] < sp[0]) { fate = ORC_SURF_ABS", [PINS + "test_reflector_absorption_geometric"]),
    ("electrode passes 1 - T", "if (u[2] < sp[3]) {", "if (u[2] < 1.0 - sp[3]) {",
     [PINS + "test_electrode_transparency"]),
    ("quantum efficiency inverted", "if (u[2] < sp[2]) { fate = ORC_DETECTED; }",
     "if (u[2] >= sp[2]) { fate = ORC_DETECTED; }", [PINS + "test_quantum_efficiency_and_tallies_consistent"]),
    ("mirror reflection with the wrong sign",
     "k_out[a] = k[a] + 2.0 * cos_i * N[a];\n        eps_out[a] = -eps[a] + 2.0 * pe * N[a];",
     "k_out[a] = k[a] - 2.0 * cos_i * N[a];\n        eps_out[a] = -eps[a] + 2.0 * pe * N[a];",
     [PINS + "test_mirror_sphere_normal_incidence_series"]),
    ("mirror polarisation not reflected", "eps_out[a] = -eps[a] + 2.0 * pe * N[a];", "eps_out[a] = eps[a];",
     [PINS + "test_mirror_polarisation_is_the_perfect_conductor_field", PINS + "test_mirror_then_brewster_surface"]),
    ("mirror polarisation: normal part dropped", "eps_out[a] = -eps[a] + 2.0 * pe * N[a];",
     "eps_out[a] = -eps[a] + pe * N[a];", [PINS + "test_mirror_polarisation_is_the_perfect_conductor_field"]),
    ("transmitted polarisation with t_s and t_p swapped",
     "eps_out[a] = cs * f[2] * s[a] + cp * f[3] * pt_v[a];", "eps_out[a] = cs * f[3] * s[a] + cp * f[2] * pt_v[a];",
     [PINS + "test_outgoing_polarisation_satisfies_maxwell_boundary_conditions",
      PINS + "test_two_interfaces_carry_the_refracted_polarisation"]),
    ("transmitted p basis from the incident direction", "cross3(s, k_out, pt_v);", "cross3(s, k, pt_v);",
     [PINS + "test_outgoing_polarisation_satisfies_maxwell_boundary_conditions"]),
    ("reflected polarisation with r_s for both components",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[1];",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[0];",
     [PINS + "test_outgoing_polarisation_satisfies_maxwell_boundary_conditions"]),
    ("reflected p component with the wrong sign",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[1];",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : -cp * f[1];",
     [PINS + "test_outgoing_polarisation_satisfies_maxwell_boundary_conditions"]),
    ("total internal reflection rotates the polarisation",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[1];",
     "double as = tir ? cp : cs * f[0], ap = tir ? cs : cp * f[1];",
     [PINS + "test_total_internal_reflection_keeps_the_polarisation_magnitudes"]),
    ("total internal reflection flips the p component",
     "double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[1];",
     "double as = tir ? cs : cs * f[0], ap = tir ? -cp : cp * f[1];",
     [PINS + "test_total_internal_reflection_keeps_the_polarisation_magnitudes"]),
    ("random polarisation at a fixed angle", "double ca = cos(alpha), sa = sin(alpha);",
     "double ca = 1.0, sa = 0.0 * alpha;",
     [PINS + "test_random_polarisation_is_uniform_about_the_direction"]),
    ("random polarisation angle over a quarter turn", "double ca = cos(alpha), sa = sin(alpha);",
     "double ca = cos(0.25 * alpha), sa = sin(0.25 * alpha);",
     [PINS + "test_random_polarisation_is_uniform_about_the_direction"]),
    ("volume source radius not square-rooted", "double r = R * sqrt(w[0]), a = TWO_PI * w[1];",
     "double r = R * w[0], a = TWO_PI * w[1];", [PINS + "test_volume_source_uniform_isotropic"]),
    ("source directions on a hemisphere", "draw4(seed, pid, SOURCE_STEP, 0, u);\n    double c = 2.0 * u[0] - 1.0",
     "draw4(seed, pid, SOURCE_STEP, 0, u);\n    double c = u[0]", [PINS + "test_volume_source_uniform_isotropic"]),
    ("refraction offset to the reflected side", "spawn_offset(pos, o_ray, th, Nf, refl ? 1.0 : -1.0);",
     "spawn_offset(pos, o_ray, th, Nf, refl ? -1.0 : 1.0);", [PINS + "test_total_internal_reflection_on_shared_edges"]),
    ("one-sided triangle test",
     "if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;",
     "if (U < 0.0f || V < 0.0f || W < 0.0f) return 0;",
     [PINS + "test_intersection_axis_aligned_square_closed_form", PINS + "test_watertight_closed_sphere"]),
    ("BVH ties broken to the largest triangle id",
     "uint32_t i = s->order[k];\n                float t;\n                if (i == skip) continue;\n"
     "                if (wray_hit(&r, &s->v[9ull * i], bt, &t)) {\n"
     "                    if (t < bt || (t == bt && (best == NO_HIT || i < best)))",
     "uint32_t i = s->order[k];\n                float t;\n                if (i == skip) continue;\n"
     "                if (wray_hit(&r, &s->v[9ull * i], bt, &t)) {\n"
     "                    if (t < bt || (t == bt && (best == NO_HIT || i > best)))",
     [PINS + "test_ties_go_to_the_smallest_index"]),
    ("singlet and triplet time constants swapped", "double tau = w[0] < p[14] ? p[15] : p[16];",
     "double tau = w[0] < p[14] ? p[16] : p[15];", [TIME + "test_nr_profile_mixture_cdf"]),
    ("spectrum FWHM taken as two sigma", "double sigma = p[18] / (2.0 * sqrt(2.0 * log(2.0)));",
     "double sigma = p[18] / 2.0;", [SPEC + "test_lxe_spectrum_is_the_gaussian_of_its_mean_and_fwhm"]),
    ("dispersion with the wrong sign", "return mat[0] + mat[3] * (wl - REF_WAVELENGTH_NM);",
     "return mat[0] - mat[3] * (wl - REF_WAVELENGTH_NM);", [SPEC + "test_dispersed_index_moves_the_reflection_series"]),
    ("Rayleigh-length scaling inverted", "pow(wl / REF_WAVELENGTH_NM, mat[4])", "pow(REF_WAVELENGTH_NM / wl, mat[4])",
     [SPEC + "test_rayleigh_length_scaling"]),
    ("absorption-length score over L instead of L^2", "j[2 * i] = isinf(La) ? 0.0 : t[2 * i] / (La * La);",
     "j[2 * i] = isinf(La) ? 0.0 : t[2 * i] / La;", [ADJ + "test_adjoint_exponential_survival"]),
    ("Rayleigh-length score with the wrong sign", "t[2 * i] / (Lr * Lr) - t[2 * i + 1] / Lr",
     "t[2 * i] / (Lr * Lr) + t[2 * i + 1] / Lr", [ADJ + "test_adjoint_rayleigh_length_zero_when_all_detected"]),
    ("electrode score with the wrong sign", "g = a / sp[3] - b / (1.0 - sp[3]);", "g = a / sp[3] + b / (1.0 - sp[3]);",
     [ADJ + "test_adjoint_electrode_transparency"]),
    ("reflector specular decision inverted", "reflect_specular = u[3] < sp[1];", "reflect_specular = u[3] >= sp[1];",
     [PINS + "test_specular_share_of_reflections[reflector]"]),
    ("electrode wire specular decision inverted", "reflect_specular = w[3] < sp[5];",
     "reflect_specular = w[3] >= sp[5];", [PINS + "test_specular_share_of_reflections[electrode]"]),
    ("arrival-time bin off by one", "double b = floor(time / tbin);", "double b = floor(time / tbin) + 1.0;",
     [PINS + "test_arrival_histogram_bins_the_photon_times"]),
    ("emission start time t0 dropped", "*t0 = p[13];", "*t0 = 0.0;", [TIME + "test_no_profile_starts_at_t0"]),
    ("light collection counts detected photons only",
     "if (fate == ORC_DETECTED || fate == ORC_QE_FAIL) ty->lce[detail] += 1;",
     "if (fate == ORC_DETECTED) ty->lce[detail] += 1;", [PINS + "test_quantum_efficiency_and_tallies_consistent"]),
    ("adjoint: path to a surface not tallied", "if (ms >= 0) tl[2 * ms] += (double)th;", "",
     [ADJ + "test_adjoint_exponential_survival"]),
    ("adjoint: Rayleigh scatters not counted", "if (ms >= 0) tl[2 * ms + 1] += 1.0;", "",
     [ADJ + "test_adjoint_rayleigh_length_zero_when_all_detected"]),
    ("adjoint: reflections not counted",
     "if (ss >= 0) tl[2 * na + 2 * ss] += 1.0;\n            reflect_specular = u[3] < sp[1];",
     "reflect_specular = u[3] < sp[1];", [ADJ + "test_adjoint_mirror_reflectivity"]),
    ("adjoint: electrode transmissions not counted",
     "if (ss >= 0) tl[2 * na + 2 * ss] += 1.0;\n                medium = to;", "medium = to;",
     [ADJ + "test_adjoint_electrode_transparency"]),
    ("adjoint: wire reflections not counted", "if (ss >= 0) tl[2 * na + 2 * ss + 1] += 1.0;", "",
     [ADJ + "test_adjoint_electrode_transparency"]),
    ("Philox Weyl constant off by one", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;",
     [PINS + "test_philox_known_answers"]),
    ("counter: photon id words swapped", "uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), step, draw};",
     "uint32_t ctr[4] = {(uint32_t)(pid >> 32), (uint32_t)pid, step, draw};", [PINS + "test_draw_contract"]),
    ("counter: step and draw swapped", "uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), step, draw};",
     "uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), draw, step};", [PINS + "test_draw_contract"]),
    ("key: seed words swapped", "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};", [PINS + "test_draw_contract"]),
    ("no spawn offset after a surface", "double eps = ldexp(m, -18);", "double eps = 0.0 * m;",
     [PINS + "test_total_internal_reflection_on_shared_edges"]),
    ("polygon source accepts the circumscribed circle", "double ap = R * cos(PI_D / n);", "double ap = R;",
     [PINS + "test_polygon_source_fills_the_polygon_uniformly"]),
    ("polygon source sides at the vertex angles", "double a = phase + TWO_PI * (k + 0.5) / n;",
     "double a = phase + TWO_PI * k / n;", [PINS + "test_polygon_source_fills_the_polygon_uniformly"]),
    ("slab test without ordering the two plane distances", "if (ta > tb) { double x = ta; ta = tb; tb = x; }", "",
     [PINS + "test_bvh_equals_brute_force_on_soup", PINS + "test_watertight_closed_sphere"]),
    ("uniform without the half-step offset", "return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);",
     "return ((double)(x >> 9)) * (1.0 / 8388608.0);", [PINS + "test_uniform_mapping_range"]),
    ("no special case at normal incidence",
     "if (norm3(s) < 1e-6) {\n        s[0] = eps[0]; s[1] = eps[1]; s[2] = eps[2];\n    } else {\n        normalize3(s);\n    }",
     "normalize3(s);", [PINS + "test_normal_incidence_keeps_photon", PINS + "test_worked_example_e1_reflection_series"]),
]


def _run_mutant(k, old, new, pins, tmp):
    """Build mutant k and run its pins against it; returns (exit code, output)."""
    from oracle import build
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    if src.count(old) != 1:
        return -1, "mutation site not unique"
    d = os.path.join(tmp, f"m{k}")
    os.makedirs(d)
    with open(os.path.join(d, "oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), os.path.join(d, "oracle.h"))
    lib = os.path.join(d, "liboracle_mutant.so")
    build.compile_library(os.path.join(d, "oracle.c"), lib)
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """All mutants built and run concurrently (each in its own process)."""
    import concurrent.futures as cf
    tmp = str(tmp_path_factory.mktemp("mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_run_mutant, k, old, new, pins, tmp) for k, (_, old, new, pins) in enumerate(MUTANTS)]
        return [f.result() for f in futs]


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(k, outcomes):
    name, _, _, pins = MUTANTS[k]
    code, out = outcomes[k]
    assert code != -1, f"mutation site of '{name}' not unique"
    assert code == 1, f"'{name}' survived {pins}:\n{out}"
