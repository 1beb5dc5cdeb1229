/*
 * lxo.h -- C ABI of the GB300 optical-photon tracker for liquid-xenon TPCs.
 *
 * The library propagates scintillation photons (175 nm, or a Gaussian
 * emission spectrum), one photon per GPU lane, through a triangle-mesh
 * detector to their fate, PMT channel and arrival time: exponential bulk absorption and Rayleigh scattering, polarised
 * Fresnel reflection / refraction with total internal reflection at
 * dielectric boundaries, reflectivity-parameterised surfaces (PTFE, stainless
 * steel), effective-transparency electrodes and photocathodes with a quantum
 * efficiency (arXiv:2203.14354, Sec. 2.1-2.2, Table 2, Sec. 3, Appendix).
 *
 * Conventions for every entry point:
 *  - Return 0 (LXO_OK) or a negative lxo_status; no exception crosses the
 *    ABI.  lxo_last_error(ctx) returns a message owned by the context, valid
 *    until the next call on that context.
 *  - "host" pointers are read during the call and stay owned by the caller.
 *    "device" pointers are CUDA device memory of the context's device, owned
 *    by the caller, and must stay valid until the work queued on `stream`
 *    completes.  Geometry, BVH and scratch memory are owned by the context.
 *  - Calls that take `stream` (a cudaStream_t; NULL = the legacy default
 *    stream) are asynchronous.  Faults detected inside a kernel (channel out
 *    of range, and in the bounds-checked build a traversal stack overflow or
 *    an index outside its array) set a device error word that lxo_sync()
 *    reads back and reports as LXO_ERR_DEVICE.
 *  - Result tallies ACCUMULATE: the caller zeroes them.  Photon p's random
 *    stream depends only on (seed, p), so splitting a run into several calls
 *    with disjoint photon_id_base ranges adds up to the same tallies.
 *
 * Units: mm, ns, nm (wavelength).  Speed of light 299.792458 mm/ns; a photon
 * moves at c/n of the medium it is in.
 *
 * Random numbers (identical in every implementation of this method): photon p
 * uses Philox4x32-10 (Salmon et al., SC'11) with key = (seed low 32 bits, seed
 * high 32 bits) and counter = (p low, p high, step, draw).  A 32-bit output x
 * maps to the uniform ((x >> 9) + 0.5) * 2^-23, never 0 or 1.  Source
 * sampling uses step = 0xFFFFFFFF.  In step s, draw 0 gives
 * u0 -> absorption distance -L_abs ln u0, u1 -> Rayleigh distance
 * -L_ray ln u1, u2 -> first surface decision, u3 -> second surface decision;
 * draw 1 gives new directions (Rayleigh scattering: u0 -> the cosine c of the
 * angle to the polarisation, c = 2 cos((acos(1 - 2 u0) + 4 pi) / 3), the
 * inverse CDF of the dipole law; u1 -> the azimuth about the polarisation).
 * The emission-time draw of a source with a scintillation time profile is
 * (step 0xFFFFFFFF, draw 0xFFFFFFFF): u0 < singlet_frac picks the singlet
 * component, and the delay is -tau ln u1 of the component picked.  The same
 * draw gives the wavelength of a source with a spectrum (Box-Muller):
 * z = sqrt(-2 ln u2) cos(2 pi u3).
 */
#ifndef LXO_H
#define LXO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lxo_status;
enum {
    LXO_OK = 0,
    LXO_ERR_ARG = -1,     /* invalid argument (message says which) */
    LXO_ERR_CUDA = -2,    /* a CUDA runtime call failed */
    LXO_ERR_STATE = -3,   /* call made in the wrong order (e.g. propagate before build_bvh) */
    LXO_ERR_DEVICE = -4,  /* a kernel reported a fault through the device error word */
    LXO_ERR_NOMEM = -5    /* host or device allocation failed */
};

typedef struct lxo_ctx lxo_ctx;

/* ---- tables (Table 2 of the paper; Sec. 2.2 surface models) ---------- */

/* Wavelength at which every material constant is quoted (Table 2 gives the
 * optical properties at 175 nm). */
#define LXO_REF_WAVELENGTH_NM 175.0f

/* Bulk optical medium.  abs_len_mm / rayleigh_len_mm: mean free paths of
 * absorption and Rayleigh scattering (Table 2); +inf (or <= 0) = none; NaN
 * is rejected.  n, abs_len_mm and rayleigh_len_mm hold at
 * LXO_REF_WAVELENGTH_NM.  The paper uses these mean-wavelength values for
 * every photon of its spectrum (Sec. 2.2), which is dn_dlambda_per_nm = 0 and
 * rayleigh_exp = 0.  Otherwise, for a photon of wavelength lambda (nm):
 *   n(lambda)            = n + dn_dlambda_per_nm * (lambda - LXO_REF_WAVELENGTH_NM)
 *   rayleigh_len(lambda) = rayleigh_len_mm * (lambda / LXO_REF_WAVELENGTH_NM)^rayleigh_exp
 * (rayleigh_exp = 4 is Rayleigh's lambda^-4 law); n(lambda) also sets the
 * speed c / n(lambda).  Both must be finite (LXO_ERR_ARG); a propagation whose
 * source spectrum reaches a wavelength with n(lambda) <= 0 fails with
 * LXO_ERR_ARG. */
typedef struct {
    float n;
    float abs_len_mm;
    float rayleigh_len_mm;
    float dn_dlambda_per_nm;
    float rayleigh_exp;
} lxo_material;

/* surface model types */
enum {
    LXO_SURF_ABSORBER = 0,      /* absorbs every photon (PMT cap, Sec. 2.1) */
    LXO_SURF_REFLECTOR = 1,     /* R_total independent of angle; of the reflected photons a fraction
                                   spec_frac is specular, the rest Lambertian (Sec. 2.2) */
    LXO_SURF_PHOTOCATHODE = 2,  /* photosensitive area: counts towards LCE; detected with probability qe */
    LXO_SURF_ELECTRODE_T = 3    /* thin electrode of effective transparency T (Geant4 model, Sec. 2.1):
                                   passes straight through with probability T, else hits a wire that
                                   reflects with wire_reflectivity (specular fraction wire_spec_frac) */
};

typedef struct {
    int32_t type;
    float reflectivity;       /* REFLECTOR: R_total */
    float spec_frac;          /* REFLECTOR: specular share of reflections, R_spec / (R_spec + R_diff) */
    float qe;                 /* PHOTOCATHODE */
    float transparency;       /* ELECTRODE_T */
    float wire_reflectivity;  /* ELECTRODE_T */
    float wire_spec_frac;     /* ELECTRODE_T */
} lxo_surface;

/* PMT table entry (metadata: array 0 = bottom, 1 = top; photocathode centre) */
typedef struct {
    int32_t channel;
    int32_t array;
    float center[3];
} lxo_pmt;

/* limits of the tables */
#define LXO_MAX_MATERIALS 16
#define LXO_MAX_SURFACES 48
#define LXO_SURF_NONE 0xFFFFu   /* bare dielectric boundary: Fresnel from the two indices */
#define LXO_NO_HIT 0xFFFFFFFFu

/* ---- sources (Sec. 3: uniform in the active volume, or point sources;
 *      isotropic, random linear polarisation, start time t0) ---------- */
enum {
    LXO_SRC_VOLUME_POLYGON = 0, /* uniform in an extruded regular polygon: n_sides (0 = circle),
                                   circumradius `radius`, vertex 0 at angle `phase`, z in [z_min, z_max] */
    LXO_SRC_POINT = 1,          /* at `center` */
    LXO_SRC_SEGMENT = 2,        /* uniform on the segment center -> p1 */
    LXO_SRC_BALL = 3,           /* uniform in the ball (center, radius) */
    LXO_SRC_EXPLICIT = 4        /* per-photon device arrays pos/dir/pol [n*3] (photon i = id - base) */
};

typedef struct {
    int32_t kind;
    int32_t medium;       /* material index the photons start in */
    int32_t n_sides;
    int32_t reserved;
    float radius, phase, z_min, z_max;
    float center[3];
    float p1[3];
    float t0;             /* ns */
    /* scintillation time profile (Sec. 2.2, Table 2: two exponential decay
     * components): emission at t0 + a delay drawn from the singlet component
     * (time constant tau_singlet_ns) with probability singlet_frac, else from
     * the triplet component (tau_triplet_ns).  Both constants 0: every photon
     * starts at t0.  A constant must be >= 0 and singlet_frac in [0, 1]. */
    float singlet_frac;
    float tau_singlet_ns;
    float tau_triplet_ns;
    /* emission spectrum (Sec. 2.2, Table 2: a Gaussian of mean 174.8 nm and
     * FWHM 10.2 nm for LXe): photon wavelength wl_mean_nm + sigma * z with
     * sigma = wl_fwhm_nm / (2 sqrt(2 ln 2)) and z a standard normal deviate
     * (|z| <= 5.8).  wl_mean_nm = 0 means LXO_REF_WAVELENGTH_NM; wl_fwhm_nm = 0
     * gives one wavelength.  Both must be finite and >= 0, and the spectrum
     * must stay above 0 nm.  It changes the path of a photon only through the
     * dispersion of lxo_material. */
    float wl_mean_nm;
    float wl_fwhm_nm;
    const float* pos;     /* EXPLICIT only, device [n*3] */
    const float* dir;     /* EXPLICIT only, device [n*3], unit */
    const float* pol;     /* EXPLICIT only, device [n*3], unit, made perpendicular to dir */
} lxo_source;

/* ---- run parameters and results --------------------------------------- */
typedef struct {
    uint64_t seed;
    uint32_t max_steps;   /* interactions per photon before it is cut as TRUNCATED (0 = 10000) */
    uint32_t n_tbins;     /* arrival-time bins per channel, <= LXO_MAX_TBINS; bin n_tbins is the overflow */
    float tbin_ns;        /* bin width (> 0) */
    uint32_t flags;       /* LXO_FLAG_* */
} lxo_run_params;

/* largest n_tbins (LXO_ERR_ARG above it) */
#define LXO_MAX_TBINS (1u << 24)

/* length of lxo_results.stats */
#define LXO_STATS_LEN 40u

/* run flags */
#define LXO_FLAG_STATS 1u    /* count traversal work into lxo_results.stats (a separate kernel build) */
#define LXO_FLAG_ADJOINT 2u  /* accumulate the adjoint tallies of detected photons into lxo_results.adjoint */

/* adjoint limits */
#define LXO_ADJ_MAX_MATERIALS 4
#define LXO_ADJ_MAX_SURFACES 8

/* fate codes (per photon) */
enum {
    LXO_FATE_DETECTED = 0,   /* reached a photocathode and passed the QE draw */
    LXO_FATE_QE_FAIL = 1,    /* reached a photocathode, not detected */
    LXO_FATE_BULK_ABS = 2,   /* absorbed in a medium */
    LXO_FATE_SURF_ABS = 3,   /* absorbed by a surface (reflector, cap, electrode wire) */
    LXO_FATE_ESCAPED = 4,    /* left the geometry (a leak: no surface ahead, no bulk process) */
    LXO_FATE_TRUNCATED = 5,  /* max_steps reached */
    LXO_FATE_GEOM_ERR = 6    /* inconsistent medium at a boundary or bad channel */
};
/* fates[] layout: [0..6] count per fate code, [7] total steps of all photons,
 * [8 + m] bulk absorptions in material m, [8 + M + s] absorptions on surface s
 * (M materials, S surfaces as set) -- the loss bookkeeping of Table 6. */
#define LXO_FATES_FIXED 8

typedef struct {
    uint32_t* lce;               /* device [P]: photocathode arrivals (light collection, Sec. 3) */
    uint32_t* det;               /* device [P]: detected after QE */
    uint32_t* hist;              /* device [P*(n_tbins+1)]: detected arrival-time histogram (row = channel) */
    unsigned long long* fates;   /* device [8+M+S] */
    uint32_t* ph_fate;           /* optional device [n]: fate code per photon */
    int32_t* ph_detail;          /* optional device [n]: channel (DETECTED, QE_FAIL), material (BULK_ABS),
                                    surface (SURF_ABS), triangle (GEOM_ERR); -1 (ESCAPED, TRUNCATED) */
    uint32_t* ph_steps;          /* optional device [n] */
    float* ph_time;              /* optional device [n]: time at the end, ns */
    double* adjoint;             /* device [P*K] with LXO_FLAG_ADJOINT: per channel, sums over detected
                                    photons of their tallies (layout of lxo_set_adjoint) */
    unsigned long long* stats;   /* device [LXO_STATS_LEN] with LXO_FLAG_STATS (accumulated): [0..3]
                                    photon steps, BVH nodes visited, leaves visited, triangles tested
                                    (lane counts); [4..6] warp iterations of the node loop, of the
                                    leaf loop and of the photon loop; [7..8] lane cycles in
                                    traversal, in steps; [9..17] steps in material 0 by nodes
                                    visited (bins of 8, last >= 64), [18] their leaves; [19..28]
                                    the same for other materials; [29..34] lane cycles in the node
                                    loop, the leaf loop, the traversal set-up, the step's draws, the
                                    interaction, and the refill (tallies, new photons) */
    float* ph_state;             /* optional device [n*9]: per photon, its state when it met its fate
                                    (or was cut by max_steps): position (mm), unit direction and unit
                                    polarisation, 3 floats each -- so the outgoing wave of every
                                    interaction can be checked photon by photon */
} lxo_results;

typedef struct {
    uint32_t n_tris, n_nodes, n_leaves, max_depth;
    uint64_t node_bytes, tri_bytes;
    double build_seconds, sah_cost;
} lxo_bvh_info;

typedef struct {
    uint32_t leaf_size;   /* max triangles per leaf, 1..8 (0 = 4) */
    uint32_t sah_bins;    /* bins per axis, 4..64 (0 = 16) */
    uint32_t n_threads;   /* host threads (0 = all cores) */
    uint32_t reserved;
} lxo_bvh_params;

/* ---- entry points ------------------------------------------------------ */

/* Creates a context on CUDA device `cuda_device` (allocates its scratch).
 * LXO_ERR_CUDA if no CUDA device is usable (no GPU: the library has no CPU
 * fallback), LXO_ERR_ARG for an index outside the devices. */
lxo_status lxo_create(lxo_ctx** out, int cuda_device);
void lxo_destroy(lxo_ctx* ctx);
const char* lxo_last_error(const lxo_ctx* ctx);

/* Detector mesh (Sec. 2.1: the detector as triangles, each boundary with the
 * materials on its two sides, a surface model and, for photocathodes, a PMT
 * channel).  Host arrays: verts [nv*3] mm; tris [nt*3] vertex indices;
 * mat_inner/mat_outer [nt] material on the side the geometric normal
 * (v1-v0)x(v2-v0) points away from / towards; surface [nt] surface index or
 * LXO_SURF_NONE; channel [nt] PMT channel of photocathode triangles, -1
 * elsewhere.  Copied; invalidates a previous BVH.  LXO_ERR_ARG for
 * 0 or >= 2^28 triangles, a vertex index >= nv or a non-finite vertex.
 * Zero-area triangles are accepted and never hit. */
lxo_status lxo_load_mesh(lxo_ctx* ctx, const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                         const uint8_t* mat_inner, const uint8_t* mat_outer, const uint16_t* surface,
                         const int32_t* channel);
/* Material table (Table 2).  Host array of 1 <= n <= LXO_MAX_MATERIALS.
 * LXO_ERR_ARG (table unchanged) if an index n is not > 0, a length is NaN or
 * a dispersion field is not finite.
 * A table change takes effect at the next propagation; it never rebuilds the
 * BVH. */
lxo_status lxo_set_materials(lxo_ctx* ctx, const lxo_material* m, uint32_t n);
/* Surface table (Sec. 2.2).  Host array of n <= LXO_MAX_SURFACES.
 * LXO_ERR_ARG (table unchanged) for an unknown type or a probability
 * (reflectivity, fractions, qe, transparency) outside [0, 1]. */
lxo_status lxo_set_surfaces(lxo_ctx* ctx, const lxo_surface* s, uint32_t n);
/* PMT table: n channels (the P of every per-channel tally). */
lxo_status lxo_set_pmts(lxo_ctx* ctx, const lxo_pmt* p, uint32_t n);

/* Builds the bounding-volume hierarchy on the host (binned SAH, all cores)
 * and uploads nodes and triangles to the device.  params may be NULL.
 * info (host, may be NULL) receives sizes and the build time.  LXO_ERR_ARG if
 * the forest is so deep that a traversal could overflow its fixed stack
 * (depth + 33 >= 96 entries; the kernels then need no overflow test). */
lxo_status lxo_build_bvh(lxo_ctx* ctx, const lxo_bvh_params* params, lxo_bvh_info* info);

/* Closest hit for n rays (device arrays): smallest t in (0, tmax] over all
 * triangles except skip[i] (LXO_NO_HIT = none), ties to the smallest
 * triangle index; float32 watertight test (Woop, Benthin & Wald, JCGT 2013).
 * org/dir [n*3]; skip, tmax may be NULL (none / +inf).  Writes hit [n]
 * (LXO_NO_HIT on miss) and t [n] (+inf on miss). */
lxo_status lxo_trace_rays(lxo_ctx* ctx, const float* org, const float* dir, const uint32_t* skip,
                          const float* tmax, uint32_t n, uint32_t* hit, float* t, void* stream);

/* The first state of photons base .. base+n-1 from a source: device arrays
 * pos, dir, pol [n*3] (float) and, if not NULL, the emission time [n] (ns;
 * t0 plus the delay of the source's scintillation time profile) and the
 * wavelength [n] (nm, drawn from the source's spectrum; a photon keeps it to
 * its fate). */
lxo_status lxo_sample_source(lxo_ctx* ctx, const lxo_source* src, uint64_t n, uint64_t photon_id_base,
                             uint64_t seed, float* pos, float* dir, float* pol, float* time, float* wavelength,
                             void* stream);

/* Propagates photons base .. base+n-1 to their fates and accumulates the
 * tallies into `out` (device buffers, caller-owned, zeroed by the caller).
 * Requires mesh, materials, surfaces, PMTs and BVH. */
lxo_status lxo_propagate(lxo_ctx* ctx, const lxo_source* src, uint64_t n, uint64_t photon_id_base,
                         const lxo_run_params* params, const lxo_results* out, void* stream);

/* The same with HOST result buffers (lce, det, hist, fates; the per-photon
 * arrays must be NULL): zeroes context-owned device tallies, propagates,
 * copies the tallies back and ADDS them to the host arrays.  Synchronous. */
lxo_status lxo_propagate_host(lxo_ctx* ctx, const lxo_source* src, uint64_t n, uint64_t photon_id_base,
                              const lxo_run_params* params, const lxo_results* host_out, void* stream);

/* ---- batched events ----------------------------------------------------
 * Many sources of uneven photon counts in one persistent launch (the
 * paper's LCE maps run ~2500 point sources, Sec. 4.1; S1 light from an
 * interaction point and S2 light along the electron path in the gas gap,
 * Sec. 1).  Event e's photon i has photon id (e << 32) | i (e = the event
 * id, see lxo_upload_events), so its random stream is that of a
 * single-source lxo_propagate with photon_id_base = e << 32, and each event
 * is reproducible on its own. */
typedef struct {
    int32_t kind;         /* LXO_SRC_POINT, LXO_SRC_SEGMENT or LXO_SRC_BALL */
    int32_t medium;
    float center[3];      /* point, segment start or ball centre */
    float p1[3];          /* segment end */
    float radius;         /* ball radius */
    float t0;             /* ns */
    float singlet_frac;   /* scintillation time profile, as in lxo_source */
    float tau_singlet_ns;
    float tau_triplet_ns;
    float wl_mean_nm;     /* emission spectrum, as in lxo_source */
    float wl_fwhm_nm;
    float reserved;
    uint64_t n_photons;   /* < 2^32 */
} lxo_event;

/* Copies the event table (host [n]) to the device (context-owned, replaces
 * the previous table).  Event e of the table has the event id
 * first_event + e (its photons have ids ((first_event + e) << 32) | i);
 * tallies still go to row e.  A job split into contiguous event ranges, one
 * per GPU, each uploaded with its first event's id, therefore reproduces the
 * single-GPU run's tallies row for row.  LXO_ERR_ARG if
 * first_event + n > 2^32.  Synchronous. */
lxo_status lxo_upload_events(lxo_ctx* ctx, const lxo_event* ev, uint32_t n, uint32_t first_event);

/* Propagates every photon of the uploaded events in one launch.  out (device,
 * caller-owned, accumulated): lce, det [E*P] (row = event), hist
 * [E*P*(n_tbins+1)] or NULL (no time histograms), fates [8+M+S] over all
 * events, and with LXO_FLAG_ADJOINT adjoint [E*P*K]; per-photon outputs and
 * stats must be NULL / off.  Uses only
 * device-resident tables, so it can be captured in a CUDA graph and replayed.
 * Asynchronous on `stream`. */
lxo_status lxo_propagate_events(lxo_ctx* ctx, const lxo_run_params* params, const lxo_results* out, void* stream);

/* Launch shape of the propagation kernels (found by an autotuner):
 * threads per block, 128 or 256 (0 = 256; each has its own kernel build
 * with the same registers per thread, and 256 is used for LXO_FLAG_STATS);
 * blocks_per_sm, counted in blocks of the chosen size: up to 5 (10 of 128)
 * selects the build with 48 registers per thread, 6..8 (12..16) the one
 * with 32; 0 = the occupancy limit of the 32-register build for the
 * forward and of the 48-register build for LXO_FLAG_ADJOINT; photon ids
 * taken per warp from the work queue, chunk in 1..4096 (0 = 64).  Results
 * do not depend on the shape. */
lxo_status lxo_set_launch(lxo_ctx* ctx, uint32_t blocks_per_sm, uint32_t chunk, uint32_t threads);

/* Adjoint (an extension of the paper's method: it has no gradients; the
 * quantities are its Table 2 parameters and the Sec. 2.1 electrode model).
 * The gradient of expected detected hits per channel with respect to
 *   theta = (L_abs, L_ray) of each material in `mats`, then R (REFLECTOR) or
 *           T (ELECTRODE_T) of each surface in `surfs`
 * is the score-function estimator: each photon tallies, in FP32,
 *   K = 2*n_mats + 2*n_surfs numbers -- for material i: path length (2i) and
 *   Rayleigh scatters (2i+1); for surface j: reflections or transmissions
 *   (2n_mats+2j) and wire reflections (2n_mats+2j+1) --
 * and on detection adds them (FP64) to lxo_results.adjoint[channel*K + k].
 * A detected path's log-probability has the derivatives
 *   d/dL_abs = l/L_abs^2, d/dL_ray = l/L_ray^2 - N/L_ray, d/dR = n/R,
 *   d/dT = n_T/T - n_W/(1-T),
 * so lxo_adjoint_jacobian turns the sums into J[channel][q] = dE[hits]/dtheta_q.
 * Host arrays; n_mats <= LXO_ADJ_MAX_MATERIALS, n_surfs <= LXO_ADJ_MAX_SURFACES;
 * surfaces must be REFLECTOR or ELECTRODE_T. */
lxo_status lxo_set_adjoint(lxo_ctx* ctx, const int32_t* mats, uint32_t n_mats, const int32_t* surfs,
                           uint32_t n_surfs);

/* J [R*Q] (device, Q = 2*n_mats + n_surfs) from tally sums [R*K] (device) at
 * the current material / surface values, R = n_rows (0 = P, one row per
 * channel; E*P for the sums of lxo_propagate_events, row = event*P +
 * channel); if g (device [R]) and grad (device [Q]) are not NULL, also
 * grad = J^T g (the vector-Jacobian product of a backward pass).
 * Asynchronous on `stream`. */
lxo_status lxo_adjoint_jacobian(lxo_ctx* ctx, const double* tally_sums, uint32_t n_rows, double* J, const double* g,
                                double* grad, void* stream);

/* Waits for `stream` and reports a device-side fault recorded since the last
 * lxo_sync (then clears it). */
lxo_status lxo_sync(lxo_ctx* ctx, void* stream);

/* Size of the library's static device scratch used by
 * lxo_propagate_host_static (held on every GPU that loads the library until
 * the process exits). */
#define LXO_STATIC_SCRATCH_BYTES (8u << 20)

/* lxo_propagate_host for callers that must not allocate device memory.
 * (This entry point has no counterpart in the paper: it is a deployment
 * variant.)  Some callers cannot call cudaMalloc once they are running: a
 * host framework that hands out all device memory from its own fixed pool,
 * or a data-acquisition loop that must never block, since cudaMalloc can
 * fail mid-run and cudaFree waits for the whole device.  lxo_propagate_host
 * allocates its device tallies on first use; this variant keeps them, with
 * the work-queue head and the error word, in one static device array of
 * LXO_STATIC_SCRATCH_BYTES inside the library, and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  - Same arguments and result as lxo_propagate_host: the tallies are ADDED
 *    to the caller's host arrays (lce, det [P], hist [P*(n_tbins+1)],
 *    fates [8+M+S]); per-photon outputs and LXO_FLAG_STATS are rejected.
 *  - Returns LXO_ERR_ARG if 256 + 8*(8+M+S) + 4*(2P + P*(n_tbins+1)) bytes
 *    exceed LXO_STATIC_SCRATCH_BYTES (the DARWIN-scale detector with 1000
 *    time bins needs 7.1 MB).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and may load the library's device code: make it
 *    before any stream capture.
 *  - Every call on a device shares the one array, and each call overwrites
 *    it; calls that overlap on the GPU (other streams or threads) race and
 *    corrupt each other's results.  Synchronous.
 *  - On success it allocates nothing, on the device or the host; the
 *    messages of its own argument checks are cut to the context string's
 *    current capacity.
 *  - A fault flagged by the kernel returns LXO_ERR_DEVICE (the flag word in
 *    the message, as lxo_sync reports it) and leaves the host arrays as they
 *    were. */
lxo_status lxo_propagate_host_static(lxo_ctx* ctx, const lxo_source* src, uint64_t n, uint64_t photon_id_base,
                                     const lxo_run_params* params, const lxo_results* host_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LXO_H */
