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
constexpr int32_t kEmptyChild = INT32_MIN;  // child slot of a one-leaf root

// device error word bits
enum : int { kErrStack = 1, kErrChannel = 2, kErrTimeout = 4 };

// Node: 64 bytes, boxes of both children (x, y, z slabs) + child references.
//   f[0] = (c0.lo.x, c0.hi.x, c1.lo.x, c1.hi.x)
//   f[1] = (c0.lo.y, c0.hi.y, c1.lo.y, c1.hi.y)
//   f[2] = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   f[3] = (ref0, ref1, -, -) as int bits
// ref >= 0: internal node index; ref < 0: leaf, ~ref = (first << 3) | (count - 1);
// ref == kEmptyChild: no child.
// Triangle record: 48 bytes = 3 float4: (v0.xyz, v1.x), (v1.yz, v2.xy),
// (v2.z, id, attr, channel) -- id, attr and channel as int bits;
// attr = mat_inner | mat_outer << 8 | surface << 16.
struct BvhHost {
    float4* nodes = nullptr;     // host copy [n_nodes * 4]
    float4* tris = nullptr;      // [n_records * 3]
    uint32_t n_nodes = 0, n_records = 0, n_leaves = 0, max_depth = 0;
    double sah_cost = 0.0, build_seconds = 0.0;
};

// Builds the BVH from vertex triplets tri_v [nt*9].  expand: absolute
// widening of every box (conservative traversal).  Returns 0 or -1 (err set).
int build_bvh(const float* tri_v, uint32_t nt, uint32_t leaf_size, uint32_t bins, uint32_t n_threads,
              float expand, BvhHost* out, char* err, size_t err_len);
void free_bvh(BvhHost* b);

struct DevMaterial {
    float n;
    float n_over_c;   // ns per mm
    float abs_len;    // +inf = none
    float ray_len;    // +inf = none
};

struct DevSurface {
    int type;
    float R, spec, qe, T, Rw, wspec;
};

struct Scene {
    const float4* nodes;
    const float4* tris;    // records in leaf order
    uint32_t n_tris;
};

struct SourceDev {
    int kind, medium, n_sides;
    float radius, z_min, z_max, apothem, t0;
    float phase_turns;    // polygon phase / (2 pi)
    float center[3], p1[3];
    float side_cos[kMaxPolySides], side_sin[kMaxPolySides];
    const float* pos;
    const float* dir;
    const float* pol;
};

struct PropParams {
    Scene sc;
    SourceDev src;
    DevMaterial mat[LXO_MAX_MATERIALS];
    DevSurface surf[LXO_MAX_SURFACES];
    int n_mat, n_surf, n_chan, n_fates;
    uint64_t n, base, seed;
    uint32_t max_steps, n_tbins, flags;
    float tbin;
    lxo_results out;
    unsigned long long* queue;   // scratch: work-queue head
    int* err;                    // scratch: device error word
};

// kernel launchers (lxo_kernels.cu)
cudaError_t launch_trace(const Scene& sc, const float* org, const float* dir, const uint32_t* skip,
                         const float* tmax, uint32_t n, uint32_t* hit, float* t, int* err, cudaStream_t st);
cudaError_t launch_sample_source(const PropParams& p, float* pos, float* dir, float* pol, cudaStream_t st);
cudaError_t launch_propagate(const PropParams& p, int device, cudaStream_t st);

}  // namespace lxo
