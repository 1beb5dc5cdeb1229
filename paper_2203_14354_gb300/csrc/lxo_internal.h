// Internal declarations shared by the C-ABI layer (lxo_api.cu), the kernels
// (lxo_kernels.cu) and the host BVH builder (bvh_build.cpp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lxo.h"

namespace lxo {

constexpr int kMaxFates = LXO_FATES_FIXED + LXO_MAX_MATERIALS + LXO_MAX_SURFACES;
constexpr int kMaxPolySides = 64;
constexpr int kStackSize = 96;          // traversal stack entries (>= BVH depth, enforced by the builder)
constexpr int kMaxDepth = 90;           // builder depth limit
constexpr uint32_t kSourceStep = 0xFFFFFFFFu;
constexpr int kMaxTries = 64;
constexpr int32_t kEmptyChild = INT32_MIN;  // empty layer cell or main tree

// device error bits: traversal stack overflow and an index out of its array
// (checked build only, LXO_CHECK_BOUNDS: the normal build's stack cannot
// overflow, lxo_build_bvh bounds the depth), PMT channel out of range
enum : int { kErrStack = 1, kErrChannel = 2, kErrBounds = 8 };

// Node: 64 bytes, boxes of both children (x, y, z slabs) + child references.
//   f[0] = (c0.lo.x, c0.hi.x, c1.lo.x, c1.hi.x)
//   f[1] = (c0.lo.y, c0.hi.y, c1.lo.y, c1.hi.y)
//   f[2] = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   f[3] = (ref0, ref1, -, -) as int bits
// ref >= 0: internal node index; ref < 0: leaf, ~ref = (first << 3) | (count - 1).
// Every node has two children (a one-leaf tree repeats its leaf); kEmptyChild
// marks an empty cell of a layer grid or an empty main tree.
// Triangle record: 48 bytes = 3 float4: (v0.xyz, v1.x), (v1.yz, v2.xy),
// (v2.z, id, attr, channel) -- id, attr and channel as int bits;
// attr = mat_inner | mat_outer << 8 | surface << 16.
// A planar cluster: a large set of triangles confined to a thin slab
// perpendicular to `axis` (an electrode wire mesh).  It gets its own tree: a
// kd top split on a 2-D grid of cells (in-plane axes u = axis+1, v = axis+2)
// over small per-cell sub-trees holding every triangle whose box overlaps the
// cell.  A ray crossing the slab starts at the sub-trees of the <= 4 cells its
// in-slab segment touches; other rays fall back to the cluster root.
constexpr int kMaxClusters = 8;
constexpr int kMaxCellsPerRay = 4;

struct ClusterHost {
    int axis;
    float slab_lo, slab_hi;     // along axis, widened by the box margin
    float u0, v0, inv_cell;     // grid origin and 1 / cell size
    int nu, nv;
    int32_t root;               // reference of the cluster tree root
    uint32_t cells_offset;      // first cell in BvhHost::cells
};

struct BvhHost {
    float4* nodes = nullptr;     // host copy [n_nodes * 4]
    float4* tris = nullptr;      // [n_records * 3]
    int32_t* cells = nullptr;    // [n_cells] sub-tree reference per cell (kEmptyChild if empty)
    uint32_t n_nodes = 0, n_records = 0, n_leaves = 0, max_depth = 0, n_cells = 0;
    int32_t main_root = kEmptyChild;  // root of the tree over the non-cluster triangles
    int n_clusters = 0;
    ClusterHost clusters[kMaxClusters];
    double sah_cost = 0.0, build_seconds = 0.0;
};

// Builds the forest from vertex triplets tri_v [nt*9].  cluster_of [nt]: -1
// for the main tree, else the planar cluster index (< n_clusters <=
// kMaxClusters); may be NULL.  expand: absolute widening of every box and
// slab (conservative traversal).  Returns 0 or -1 (err set).
int build_bvh(const float* tri_v, uint32_t nt, const int32_t* cluster_of, int n_clusters, uint32_t leaf_size,
              uint32_t bins, uint32_t n_threads, float expand, BvhHost* out, char* err, size_t err_len);
void free_bvh(BvhHost* b);

// Finds thin dense layers: along each axis, triangles at most 0.4 % of the
// scene extent thick, grouped while their extents overlap (3 mm tolerance),
// kept if a group holds >= 32768 triangles within 1 % of the scene extent.
// Writes cluster_of [nt] (-1 = main tree) and returns the number of layers
// (largest first, at most kMaxClusters).
int detect_layers(const float* tri_v, uint32_t nt, int32_t* cluster_of);

struct DevMaterial {
    float n;
    float n_over_c;   // ns per mm
    float abs_len;    // +inf = none
    float ray_len;    // +inf = none
    float dn;         // dn / dlambda per nm about the reference wavelength
    float dn_over_c;  // dn / c, ns per mm per nm
    float ray_exp;    // Rayleigh length scales as (lambda / reference)^ray_exp
};

// Gaussian emission spectrum: mean and standard deviation in nm (sigma 0 =
// one wavelength)
struct Spectrum {
    float mean, sigma;
};

struct DevSurface {
    int type;
    float R, spec, qe, T, Rw, wspec;
};

struct ClusterDev {
    int axis, nu, nv;
    int32_t root;
    float slab_lo, slab_hi, u0, v0, inv_cell, delta;
    const int32_t* cells;  // device [nu * nv], row v * nu + u
};

struct Scene {
    const float4* nodes;
    const float4* tris;    // records in leaf order
    uint32_t n_tris;
    uint32_t n_nodes, n_records;  // array sizes (checked by the LXO_CHECK_BOUNDS build)
    int32_t main_root;     // kEmptyChild if every triangle is in a cluster
    int n_clusters;
    ClusterDev clusters[kMaxClusters];
};

// Emission-time profile: delay -tau ln u, tau = tau_s with probability f_s,
// else tau_t; all zero = no delay.
struct TimeProfile {
    float f_s, tau_s, tau_t;
};

struct SourceDev {
    int kind, medium, n_sides;
    float radius, z_min, z_max, apothem, t0;
    TimeProfile prof;
    Spectrum spec;
    float phase_turns;    // polygon phase / (2 pi)
    float center[3], p1[3];
    float side_cos[kMaxPolySides], side_sin[kMaxPolySides];
    const float* pos;
    const float* dir;
    const float* pol;
};

struct EventDev {
    int kind, medium;
    float center[3], p1[3], radius, t0;
    TimeProfile prof;
    Spectrum spec;
};

struct PropParams {
    Scene sc;
    SourceDev src;
    DevMaterial mat[LXO_MAX_MATERIALS];
    DevSurface surf[LXO_MAX_SURFACES];
    int n_mat, n_surf, n_chan, n_fates;
    int spectral;                      // 1: some material has dispersion, photons carry a wavelength
    uint64_t n, base, seed;
    uint32_t max_steps, n_tbins, flags;
    float tbin;
    lxo_results out;
    int adj_k;                                   // tallies per photon (0 = no adjoint)
    signed char adj_mat_slot[LXO_MAX_MATERIALS]; // tracked material -> index, -1 if not
    signed char adj_surf_slot[LXO_MAX_SURFACES]; // tracked surface -> index, -1 if not
    int adj_n_mats;
    uint32_t n_events;                 // 0: single source
    uint32_t first_event;              // event id of events[0]: photon ids ((first_event + e) << 32) | i
    const EventDev* events;            // [n_events]
    const unsigned long long* ev_prefix;  // [n_events + 1] photon-count prefix sums
    uint32_t chunk;                    // photon ids per warp grab
    uint32_t blocks_per_sm;            // 0 = occupancy limit
    uint32_t block_threads;            // threads per CTA of the propagation kernel: 128 or 256 (0 = 256)
    unsigned long long* queue;   // scratch: work-queue head
    int* err;                    // scratch: device error word
};

// kernel launchers (lxo_kernels.cu)
cudaError_t launch_trace(const Scene& sc, const float* org, const float* dir, const uint32_t* skip,
                         const float* tmax, uint32_t n, uint32_t* hit, float* t, int* err, cudaStream_t st);
cudaError_t launch_sample_source(const PropParams& p, float* pos, float* dir, float* pol, float* time,
                                 float* wavelength, cudaStream_t st);
cudaError_t launch_propagate(const PropParams& p, int device, cudaStream_t st);

struct AdjCoef {   // per parameter q: J[c][q] = a * sums[c][ia] + b * sums[c][ib]
    int ia, ib;
    double a, b;
};
cudaError_t launch_adjoint_jacobian(const AdjCoef* coef_host, int Q, int K, int P, const double* sums, double* J,
                                    const double* g, double* grad, cudaStream_t st);

}  // namespace lxo
