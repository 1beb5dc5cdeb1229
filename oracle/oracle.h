/*
 * CPU oracle of the optical-photon tracker: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, scalar C implementation of what the GPU path computes:
 * photons born in a source, propagated through a triangle mesh with bulk
 * absorption, dipole Rayleigh scattering, polarised Fresnel reflection /
 * refraction with total internal reflection, reflectivity-parameterised
 * surfaces, effective-transparency electrodes and photocathodes, ending in a
 * fate, a PMT channel and an arrival time (paper: Sec. 2.2, Sec. 3, Table 2,
 * Appendix items 1-3).  It shares no code with the CUDA library; only the
 * tests, the entry module's smoke() and the CPU-baseline leg of bench.py may
 * load it.
 *
 * Precision: physics in double; ray/triangle intersection in float32 (the
 * closest-hit triangle is an argmin decided in floating point, taken in the
 * kernel's precision so both sides decide it alike).
 *
 * Conventions (identical on both sides by definition, documented in the
 * library header): Philox4x32-10 counter layout and draw order, uniform
 * mapping, fate codes, tally layouts.
 */
#ifndef LXE_ORACLE_H
#define LXE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* fate codes */
enum { ORC_DETECTED = 0, ORC_QE_FAIL = 1, ORC_BULK_ABS = 2, ORC_SURF_ABS = 3,
       ORC_ESCAPED = 4, ORC_TRUNCATED = 5, ORC_GEOM_ERR = 6 };
/* surface types */
enum { ORC_ABSORBER = 0, ORC_REFLECTOR = 1, ORC_PHOTOCATHODE = 2, ORC_ELECTRODE_T = 3 };
/* source kinds */
enum { ORC_SRC_VOLUME_POLYGON = 0, ORC_SRC_POINT = 1, ORC_SRC_SEGMENT = 2, ORC_SRC_BALL = 3,
       ORC_SRC_EXPLICIT = 4 };

typedef struct orc_scene orc_scene;

/* Copies the mesh (float vertices [nv*3], uint32 triangles [nt*3], per-triangle
 * inner/outer material, surface id (0xFFFF = none), channel) and builds a
 * median-split BVH.  Returns NULL on bad input. */
orc_scene* orc_scene_new(const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                         const uint8_t* mat_inner, const uint8_t* mat_outer,
                         const uint16_t* surface, const int32_t* channel);
void orc_scene_free(orc_scene* s);
/* materials: [n*5] = {refractive index, absorption length mm, Rayleigh length mm (inf = none), all at
 * 175 nm; dn/dlambda per nm; Rayleigh-length exponent p}: a photon of wavelength wl sees the index
 * n + dn/dlambda (wl - 175) and the Rayleigh length L (wl / 175)^p */
int orc_set_materials(orc_scene* s, const double* m, int n);
/* surfaces: types[n]; params [n*6] = {R, spec_frac, qe, T, R_wire, wire_spec_frac} */
int orc_set_surfaces(orc_scene* s, const int* types, const double* p, int n);
int orc_set_channels(orc_scene* s, int n_channels);

/* closest hit for n rays; skip = UINT32_MAX for none; tmax may be NULL (= inf).
 * brute != 0 tests every triangle; otherwise the BVH.  hit = UINT32_MAX on miss. */
void orc_trace(const orc_scene* s, uint64_t n, const float* org, const float* dir,
               const uint32_t* skip, const float* tmax, uint32_t* hit, float* t, int brute);

/* source description packed as doubles:
 * [0] kind [1] medium [2] n_sides [3] radius [4] phase [5] z_min [6] z_max
 * [7..9] center [10..12] p1 [13] t0 [14] singlet fraction [15] singlet and
 * [16] triplet time constants (ns; both 0 = no emission delay) [17] mean
 * wavelength (nm; 0 = 175) and [18] FWHM of the Gaussian emission spectrum
 * (nm; 0 = one wavelength).
 * explicit_* used for ORC_SRC_EXPLICIT ([n*3] each). */
typedef struct {
    const double* src;
    const float* explicit_pos;
    const float* explicit_dir;
    const float* explicit_pol;
} orc_source;

/* source sampling only (first photon state), positions/dirs/pols [n*3];
 * medium [n], emission time [n] (ns) and wavelength [n] (nm) may be NULL */
void orc_sample_source(const orc_scene* s, const orc_source* src, uint64_t n, uint64_t base, uint64_t seed,
                       double* pos, double* dir, double* pol, int* medium, double* time, double* wavelength);

typedef struct {
    uint64_t* lce;        /* [P] photocathode arrivals */
    uint64_t* det;        /* [P] detected (after QE) */
    uint64_t* hist;       /* [P*(n_tbins+1)] detected arrival times */
    uint64_t* fates;      /* [8 + M + S]: per fate code (7), total steps, bulk per material, surface per id */
    uint32_t* ph_fate;    /* optional [n]: fate code */
    int32_t* ph_detail;   /* optional [n]: channel / material / surface / triangle */
    uint32_t* ph_steps;   /* optional [n] */
    float* ph_time;       /* optional [n]: time at the end (ns) */
    double* adjoint;      /* optional [P*K]: per-channel sums of the detected photons' tallies
                             (K = 2*n_mat + 2*n_surf of orc_set_adjoint) */
    float* ph_state;      /* optional [n*9]: position, direction, polarisation at the end */
} orc_results;

int orc_propagate(const orc_scene* s, const orc_source* src, uint64_t n, uint64_t base, uint64_t seed,
                  uint32_t max_steps, double tbin_ns, uint32_t n_tbins, orc_results* out, int n_threads);
/* returns -1 for bad arguments: no materials or channels, tbin_ns <= 0, n_tbins > 2^24 */

/* Score-function adjoint: per photon, tally the path length and the Rayleigh
 * count in each tracked material and, for each tracked surface, the number
 * of reflections (REFLECTOR) or of transmissions and wire reflections
 * (ELECTRODE_T); sums over detected photons per channel go to
 * orc_results.adjoint.  Tally k layout: material i -> 2i (length), 2i+1
 * (Rayleigh count); surface j -> 2n_mat+2j (reflections / transmissions),
 * 2n_mat+2j+1 (wire reflections). */
int orc_set_adjoint(orc_scene* s, const int* mats, int n_mats, const int* surfs, int n_surfs);
/* Jacobian d E[detected hits of channel c] / d theta_q from the tally sums
 * [P*K]: theta = (L_abs, L_ray) of each tracked material, then R (REFLECTOR)
 * or T (ELECTRODE_T) of each tracked surface; J [P * (2 n_mat + n_surf)]. */
void orc_jacobian(const orc_scene* s, const double* sums, double* J);

/* pieces exposed for the closed-form checks */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t x);
/* Fresnel amplitudes n1 -> n2 at cos(incidence): out = {rs, rp, ts, tp, cos_t, tir} */
void orc_fresnel(double n1, double n2, double cos_i, double out[6]);
/* one dielectric interaction: k, eps (unit), N facing the incident side; u decides.
 * out: k'[3], eps'[3]; returns 1 if reflected, 0 if refracted. */
int orc_dielectric(const double k[3], const double eps[3], const double N[3], double n1, double n2,
                   double u, double k_out[3], double eps_out[3], double* p_reflect);
/* specular reflection off a reflector: k' = k + 2 cos(i) N; eps' = -eps + 2 (eps.N) N made transverse
 * to k' and unit (N unit, on the incident side) */
void orc_mirror(const double k[3], const double eps[3], const double N[3], double k_out[3], double eps_out[3]);
/* samplers driven by the photon's Philox stream (photon id, step) */
void orc_rayleigh(const double k[3], const double eps[3], uint64_t pid, uint32_t step, uint64_t seed,
                  double k_out[3], double eps_out[3]);
void orc_lambert(const double N[3], uint64_t pid, uint32_t step, uint64_t seed, double k_out[3], double eps_out[3]);

#ifdef __cplusplus
}
#endif
#endif
