// Device code of the photon tracker (sm_103a).
//
//  * k_trace:          one ray per lane, closest hit (the geometry query alone).
//  * k_sample_source:  first photon state from a source (one photon per lane).
//  * k_propagate:      persistent kernel; each lane carries one photon from its
//                      source to its fate (bulk absorption, Rayleigh, Fresnel /
//                      TIR, reflectors, electrodes, photocathode).  A lane whose
//                      photon died is refilled from a warp-local chunk of photon
//                      ids (warp ballot + prefix popcount), chunks come from a
//                      global atomic work queue: no lane idles while photons
//                      remain.  Fate tallies live in shared memory per CTA;
//                      per-channel counts and the time histogram use global
//                      atomics.  Template builds <kStats, kAdjoint, kSpectral>
//                      add traversal counters, the adjoint tallies, and a
//                      wavelength carried by each photon (dispersion); the
//                      default build <0,0,0> has none of them.
//
// Bit-exactness of the closest hit: the triangle test below performs the same
// IEEE float operations, in the same order, as a plain C implementation of
// the watertight test (Woop, Benthin & Wald, JCGT 2013); every operation is an
// explicit round-to-nearest intrinsic so the compiler cannot contract or
// reorder it.  Boxes are widened at build time and the box test uses a
// relative slack, so the traversal visits every box that holds a candidate.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lxo_internal.h"

namespace lxo {

#define FULL_MASK 0xFFFFFFFFu
// Checked build (a substitute for a memory checker): every BVH node,
// triangle record, cell and tally row index is compared with its array size
// before use; a bad one sets kErrBounds and ends the ray or skips the write,
// never an out-of-range access.  Compiled out by default.
#ifndef LXO_CHECK_BOUNDS
#define LXO_CHECK_BOUNDS 0
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct U4 {
    float u0, u1, u2, u3;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t x)
{
    // ((x >> 9) + 0.5) * 2^-23: exact in float, in [2^-24, 1 - 2^-24]
    return __fmul_rn(__uint2float_rn(x >> 9) + 0.5f, 1.1920928955078125e-07f);
}

__device__ __forceinline__ U4 draw4(uint64_t seed, uint64_t pid, uint32_t step, uint32_t draw)
{
    uint4 o = philox4x32_10(make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), step, draw),
                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return U4{u01(o.x), u01(o.y), u01(o.z), u01(o.w)};
}

// ---------------------------------------------------------------------------
// small float3 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return rsqrtf(dot(a, a)) * a; }

// orthonormal basis perpendicular to unit n (Duff et al., JCGT 6(1), 2017)
__device__ __forceinline__ void onb(float3 n, float3& t1, float3& t2)
{
    const float sgn = (n.z >= 0.0f) ? 1.0f : -1.0f;  // -0.0 counts as positive
    float a = -1.0f / (sgn + n.z);
    float b = n.x * n.y * a;
    t1 = f3(1.0f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    t2 = f3(b, sgn + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// watertight ray / triangle test (exact op order, see file header)
// ---------------------------------------------------------------------------
struct WRay {
    float ox, oy, oz;
    float Sx, Sy, Sz;
    int kx, ky, kz;
};

__device__ __forceinline__ float pick(int k, float x, float y, float z) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ WRay wray_setup(float3 o, float3 d)
{
    WRay r;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax >= ay) ? ((ax >= az) ? 0 : 2) : ((ay >= az) ? 1 : 2);
    int kx = kz + 1;
    if (kx == 3) kx = 0;
    int ky = kx + 1;
    if (ky == 3) ky = 0;
    float dkz = pick(kz, d.x, d.y, d.z);
    if (dkz < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.Sx = __fdiv_rn(pick(kx, d.x, d.y, d.z), dkz);
    r.Sy = __fdiv_rn(pick(ky, d.x, d.y, d.z), dkz);
    r.Sz = __fdiv_rn(1.0f, dkz);
    r.ox = o.x;
    r.oy = o.y;
    r.oz = o.z;
    return r;
}

// The edge functions again in double, for when one of them rounded to zero
// in float (Woop et al.'s fallback).  Out of line: it is rarely taken, and
// inline it costs the hot leaf loop registers.
__device__ __noinline__ void edges_fp64(float Ax, float Ay, float Bx, float By, float Cx, float Cy, float& U, float& V,
                                        float& W)
{
    U = __double2float_rn(__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx)));
    V = __double2float_rn(__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx)));
    W = __double2float_rn(__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax)));
}

__device__ __forceinline__ bool wray_hit(const WRay& r, float4 a, float4 b, float4 c, float tmax, float& t_out)
{
    // vertices v0 = a.xyz, v1 = (a.w, b.x, b.y), v2 = (b.z, b.w, c.x)
    const float A0 = __fsub_rn(a.x, r.ox), A1 = __fsub_rn(a.y, r.oy), A2 = __fsub_rn(a.z, r.oz);
    const float B0 = __fsub_rn(a.w, r.ox), B1 = __fsub_rn(b.x, r.oy), B2 = __fsub_rn(b.y, r.oz);
    const float C0 = __fsub_rn(b.z, r.ox), C1 = __fsub_rn(b.w, r.oy), C2 = __fsub_rn(c.x, r.oz);
    const float Akz = pick(r.kz, A0, A1, A2), Bkz = pick(r.kz, B0, B1, B2), Ckz = pick(r.kz, C0, C1, C2);
    const float Ax = __fsub_rn(pick(r.kx, A0, A1, A2), __fmul_rn(r.Sx, Akz));
    const float Ay = __fsub_rn(pick(r.ky, A0, A1, A2), __fmul_rn(r.Sy, Akz));
    const float Bx = __fsub_rn(pick(r.kx, B0, B1, B2), __fmul_rn(r.Sx, Bkz));
    const float By = __fsub_rn(pick(r.ky, B0, B1, B2), __fmul_rn(r.Sy, Bkz));
    const float Cx = __fsub_rn(pick(r.kx, C0, C1, C2), __fmul_rn(r.Sx, Ckz));
    const float Cy = __fsub_rn(pick(r.ky, C0, C1, C2), __fmul_rn(r.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) edges_fp64(Ax, Ay, Bx, By, Cx, Cy, U, V, W);
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return false;
    const float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
    const float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
    const float t = __fdiv_rn(T, det);
    if (!(t > 0.0f) || !(t <= tmax)) return false;
    t_out = t;
    return true;
}

// ---------------------------------------------------------------------------
// BVH traversal: closest hit with t in (0, tmax], skipping one triangle,
// ties to the smallest triangle id.
// ---------------------------------------------------------------------------
constexpr float kBoxSlack = 1.0f + 1.0f / 65536.0f;

struct Hit {
    uint32_t id;   // triangle id (LXO_NO_HIT on miss)
    uint32_t rec;  // record index in leaf order
    float t;
};

__device__ __forceinline__ float safe_inv(float d)
{
    return __frcp_rn(fabsf(d) < 1e-20f ? copysignf(1e-20f, d) : d);
}

// lane cycles by phase of the photon loop (counting build): node loop, leaf
// loop, traversal set-up (every entry, fresh or resumed), step draws,
// interaction, refill (tallies and new photons)
enum { kCycNode = 0, kCycLeaf, kCycBegin, kCycDraw, kCycFinish, kCycRefill, kCycPhases };

struct Counters {
    uint32_t nodes, leaves, tris;
    uint32_t node_iters, leaf_iters;   // warp iterations of the node / leaf loops (counted by one lane)
    unsigned long long trav_cycles;     // lane cycles inside the traversal
    unsigned long long cyc[kCycPhases];
};

__device__ __forceinline__ bool warp_leader()
{
    return (threadIdx.x & 31u) == (uint32_t)(__ffs(__activemask()) - 1);
}

// Leaf test of one leaf reference: every triangle of the leaf through the
// exact watertight test, keeping (t, id) minimal in that order.
template <bool kStats>
__device__ __forceinline__ void test_leaf(const Scene& sc, const WRay& wr, int ref, uint32_t skip, float& bt,
                                          uint32_t& best, uint32_t& best_rec, Counters& cnt, int* bounds_err)
{
    const uint32_t enc = ~(uint32_t)ref;
    const uint32_t first = enc >> 3, count = (enc & 7u) + 1u;
    if (LXO_CHECK_BOUNDS && (uint64_t)first + count > sc.n_records) {
        atomicOr(bounds_err, kErrBounds);
        return;
    }
    if (kStats) {
        cnt.leaves++;
        cnt.tris += count;
    }
    for (uint32_t k = 0; k < count; ++k) {
        const float4* tr = sc.tris + 3 * (size_t)(first + k);
        const float4 a = __ldg(tr + 0), b = __ldg(tr + 1), c = __ldg(tr + 2);
        const uint32_t id = __float_as_uint(c.y);
        if (id == skip) continue;
        float t;
        if (wray_hit(wr, a, b, c, bt, t)) {
            if (t < bt || (t == bt && (best == LXO_NO_HIT || id < best))) {
                bt = t;
                best = id;
                best_rec = first + k;
            }
        }
    }
}

constexpr int kDone = INT32_MIN + 1;  // stack sentinel; never a valid leaf reference (< 2^28 records)

// Traversal state of one ray (its stack lives in a separate local
// array of kStackSize entries).
struct TravState {
    WRay wr;
    float ix, iy, iz, oix, oiy, oiz;
    uint32_t skip;
    float bt;
    uint32_t best, best_rec;
    int node, leaf, sp;
};

// The per-ray constants of a query of ray (o, d) skipping triangle `skip`:
// the watertight test's shear and the slab test's inverse direction.
__device__ __forceinline__ void trav_setup(float3 o, float3 d, uint32_t skip, TravState& ts)
{
    ts.wr = wray_setup(o, d);
    ts.ix = safe_inv(d.x);
    ts.iy = safe_inv(d.y);
    ts.iz = safe_inv(d.z);
    ts.oix = o.x * ts.ix;
    ts.oiy = o.y * ts.iy;
    ts.oiz = o.z * ts.iz;
    ts.skip = skip;
}

// Enters the forest for a query with t in (0, tmax] (after trav_setup).
// Planar clusters: a ray crossing the slab within a few grid cells starts at
// those cells' sub-trees; any other ray meeting the slab at the cluster root.
__device__ __forceinline__ void trav_enter(const Scene& sc, float3 o, float3 d, float tmax, TravState& ts,
                                           int* stack)
{
    ts.bt = tmax;
    ts.best = LXO_NO_HIT;
    ts.best_rec = 0;
    stack[0] = kDone;
    int sp = 1;
    for (int c = 0; c < sc.n_clusters; ++c) {
        const ClusterDev& cl = sc.clusters[c];
        const float oa = pick(cl.axis, o.x, o.y, o.z), ia = pick(cl.axis, ts.ix, ts.iy, ts.iz);
        const float ta = (cl.slab_lo - oa) * ia, tb = (cl.slab_hi - oa) * ia;
        const float tin = fmaxf(fminf(ta, tb), 0.0f), tout = fminf(fmaxf(ta, tb), tmax * kBoxSlack);
        if (!(tin <= tout)) continue;
        if (tout < 1e30f) {
            const int bu = cl.axis == 2 ? 0 : cl.axis + 1;   // in-plane axes (axis+1, axis+2) mod 3
            const int bv = cl.axis == 0 ? 2 : cl.axis - 1;
            const float ou = pick(bu, o.x, o.y, o.z), du = pick(bu, d.x, d.y, d.z);
            const float ov = pick(bv, o.x, o.y, o.z), dv = pick(bv, d.x, d.y, d.z);
            const float u1 = ou + tin * du, u2 = ou + tout * du, v1 = ov + tin * dv, v2 = ov + tout * dv;
            const float fi0 = fmaxf(floorf((fminf(u1, u2) - cl.delta - cl.u0) * cl.inv_cell), 0.0f);
            const float fi1 = fminf(floorf((fmaxf(u1, u2) + cl.delta - cl.u0) * cl.inv_cell), (float)(cl.nu - 1));
            const float fj0 = fmaxf(floorf((fminf(v1, v2) - cl.delta - cl.v0) * cl.inv_cell), 0.0f);
            const float fj1 = fminf(floorf((fmaxf(v1, v2) + cl.delta - cl.v0) * cl.inv_cell), (float)(cl.nv - 1));
            if (!(fi0 <= fi1) || !(fj0 <= fj1)) continue;  // outside the cluster's grid
            if ((fi1 - fi0 + 1.0f) * (fj1 - fj0 + 1.0f) <= (float)kMaxCellsPerRay) {
                for (int j = (int)fj0; j <= (int)fj1; ++j)
                    for (int i = (int)fi0; i <= (int)fi1; ++i) {
                        if (LXO_CHECK_BOUNDS && (i < 0 || j < 0 || i >= cl.nu || j >= cl.nv)) continue;
                        const int r = __ldg(&cl.cells[(size_t)j * cl.nu + i]);
                        if (r != kEmptyChild) stack[sp++] = r;
                    }
                continue;
            }
        }
        stack[sp++] = cl.root;
    }
    ts.node = sc.main_root != kEmptyChild ? sc.main_root : stack[--sp];
    ts.leaf = 0;  // parked leaf (0 = none: reference 0 is an internal node, never a leaf)
    ts.sp = sp;
}

__device__ __forceinline__ void trav_begin(const Scene& sc, float3 o, float3 d, uint32_t skip, float tmax,
                                           TravState& ts, int* stack)
{
    trav_setup(o, d, skip, ts);
    trav_enter(sc, o, d, tmax, ts, stack);
}

// "While-while" traversal with postponed leaves (Aila & Laine, HPG 2009): a
// lane that reaches a leaf parks it and keeps descending until every active
// lane of the warp holds a leaf; then the warp tests leaves together.
// Runs the query to completion, or with kYield until the end of the first
// leaf phase after which some lane of the warp has finished its query: the
// lanes still tracing then leave with a resumable state (node >= 0, no
// parked leaf), so that the finished ones can take their next ray (dynamic
// ray fetch, after Aila & Laine).
template <bool kStats, bool kYield = false>
__device__ void trav_run(const Scene& sc, TravState& ts, int* stack, int* err, Counters& cnt)
{
    int node = ts.node, leaf = ts.leaf, sp = ts.sp;
    float bt = ts.bt;
    uint32_t best = ts.best, best_rec = ts.best_rec;
    long long tq = kStats ? clock64() : 0;
    while (true) {
        while (node >= 0) {
            if (kStats) {
                cnt.nodes++;
                if (warp_leader()) cnt.node_iters++;
            }
            if (LXO_CHECK_BOUNDS && (uint32_t)node >= sc.n_nodes) {
                atomicOr(err, kErrBounds);
                node = kDone;
                sp = 1;
                break;
            }
            const float4* nd = sc.nodes + 4 * (size_t)node;
            const float4 nx = __ldg(nd + 0), ny = __ldg(nd + 1), nz = __ldg(nd + 2);
            const int4 cr = __ldg(reinterpret_cast<const int4*>(nd + 3));
            const float lim = bt * kBoxSlack;
            const float ax0 = fmaf(nx.x, ts.ix, -ts.oix), ax1 = fmaf(nx.y, ts.ix, -ts.oix);
            const float ay0 = fmaf(ny.x, ts.iy, -ts.oiy), ay1 = fmaf(ny.y, ts.iy, -ts.oiy);
            const float az0 = fmaf(nz.x, ts.iz, -ts.oiz), az1 = fmaf(nz.y, ts.iz, -ts.oiz);
            const float bx0 = fmaf(nx.z, ts.ix, -ts.oix), bx1 = fmaf(nx.w, ts.ix, -ts.oix);
            const float by0 = fmaf(ny.z, ts.iy, -ts.oiy), by1 = fmaf(ny.w, ts.iy, -ts.oiy);
            const float bz0 = fmaf(nz.z, ts.iz, -ts.oiz), bz1 = fmaf(nz.w, ts.iz, -ts.oiz);
            const float an = fmaxf(fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)), fmaxf(fminf(az0, az1), 0.0f));
            const float af = fminf(fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)), fminf(fmaxf(az0, az1), lim));
            const float bn = fmaxf(fmaxf(fminf(bx0, bx1), fminf(by0, by1)), fmaxf(fminf(bz0, bz1), 0.0f));
            const float bf = fminf(fminf(fmaxf(bx0, bx1), fmaxf(by0, by1)), fminf(fmaxf(bz0, bz1), lim));
            const bool ha = an <= af;
            const bool hb = bn <= bf;   // every node has two children (see the builder)
            if (!ha && !hb) {
                node = stack[--sp];
            } else {
                const bool a_first = ha && (!hb || an <= bn);
                node = a_first ? cr.x : cr.y;
                if (ha && hb) {
                    // lxo_build_bvh rejects a forest whose depth plus the <= 33
                    // entries trav_begin pushes could reach kStackSize, so this
                    // cannot fire; only the checked build keeps the test (in the
                    // normal build the never-taken exit cost 5 % of the time)
                    if (LXO_CHECK_BOUNDS && sp >= kStackSize) {
                        atomicOr(err, kErrStack);
                        node = kDone;
                        sp = 1;
                        break;
                    }
                    stack[sp++] = a_first ? cr.y : cr.x;
                }
            }
            if (node < 0 && node != kDone && leaf == 0) {
                leaf = node;
                node = stack[--sp];
            }
            if (!__any_sync(__activemask(), leaf == 0)) break;
        }
        if (node < 0 && node != kDone && leaf == 0) {  // a leaf reference taken from the stack
            leaf = node;
            node = stack[--sp];
        }
        if (kStats) {
            const long long t1 = clock64();
            cnt.cyc[kCycNode] += (unsigned long long)(t1 - tq);
            tq = t1;
        }
        while (leaf != 0) {
            if (kStats && warp_leader()) cnt.leaf_iters++;
            test_leaf<kStats>(sc, ts.wr, leaf, ts.skip, bt, best, best_rec, cnt, err);
            leaf = 0;
            if (node < 0 && node != kDone) {
                leaf = node;
                node = stack[--sp];
            }
        }
        if (kStats) {
            const long long t1 = clock64();
            cnt.cyc[kCycLeaf] += (unsigned long long)(t1 - tq);
            tq = t1;
        }
        if (node == kDone) break;
        if (kYield && __activemask() != FULL_MASK) break;   // a lane finished (or was not tracing)
    }
    ts.node = node;
    ts.leaf = leaf;
    ts.sp = sp;
    ts.bt = bt;
    ts.best = best;
    ts.best_rec = best_rec;
}

__device__ __forceinline__ Hit trav_result(const TravState& ts)
{
    return Hit{ts.best, ts.best_rec, ts.best == LXO_NO_HIT ? INFINITY : ts.bt};
}

// State of a query between two entries to the traversal: node == kDone once
// it has finished (best, best_rec and bt then hold the hit).
struct TravResume {
    float bt;
    uint32_t best, best_rec;
    int node, sp;
};

// One entry to the traversal for the photon loop: a query whose state says
// kDone is new and enters the forest with t in (0, tmax]; any other resumes.
// The per-ray constants are recomputed at every entry from (o, d): the warp
// computes them anyway for its lanes that start a query, and they are not
// kept in registers while the warp does its interactions.
template <bool kStats>
__device__ void trav_step(const Scene& sc, float3 o, float3 d, uint32_t skip, float tmax, TravResume& tr,
                          int* stack, int* err, Counters& cnt)
{
    const long long t0 = kStats ? clock64() : 0;
    TravState ts;
    trav_setup(o, d, skip, ts);
    if (tr.node == kDone) {
        trav_enter(sc, o, d, tmax, ts, stack);
    } else {
        ts.bt = tr.bt;
        ts.best = tr.best;
        ts.best_rec = tr.best_rec;
        ts.node = tr.node;
        ts.leaf = 0;
        ts.sp = tr.sp;
    }
    if (kStats) cnt.cyc[kCycBegin] += (unsigned long long)(clock64() - t0);
    trav_run<kStats, true>(sc, ts, stack, err, cnt);
    if (kStats) cnt.trav_cycles += (unsigned long long)(clock64() - t0);
    tr.bt = ts.bt;
    tr.best = ts.best;
    tr.best_rec = ts.best_rec;
    tr.node = ts.node;
    tr.sp = ts.sp;
}

template <bool kStats>
__device__ Hit closest_hit(const Scene& sc, float3 o, float3 d, uint32_t skip, float tmax, int* err, Counters& cnt)
{
    TravState ts;
    int stack[kStackSize];
    const long long t0 = kStats ? clock64() : 0;
    trav_begin(sc, o, d, skip, tmax, ts, stack);
    if (kStats) cnt.cyc[kCycBegin] += (unsigned long long)(clock64() - t0);
    trav_run<kStats>(sc, ts, stack, err, cnt);
    return trav_result(ts);
}

__global__ void k_trace(const Scene sc, const float* __restrict__ org, const float* __restrict__ dir,
                        const uint32_t* __restrict__ skip, const float* __restrict__ tmax, uint32_t n,
                        uint32_t* __restrict__ hit, float* __restrict__ t, int* err)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 o = f3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
    const float3 d = f3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
    Counters cnt{};
    const Hit h = closest_hit<false>(sc, o, d, skip ? skip[i] : LXO_NO_HIT, tmax ? tmax[i] : INFINITY, err, cnt);
    hit[i] = h.id;
    t[i] = h.t;
}

// ---------------------------------------------------------------------------
// photon source
// ---------------------------------------------------------------------------
struct Photon {
    float3 pos, dir, pol;
    float time;
    float wl;             // wavelength, nm (set only when some material has dispersion)
    int medium;
    uint32_t last;
    uint32_t step;
    uint64_t pid;
};

__device__ __forceinline__ float3 random_pol(float3 k, float u)
{
    float3 e1, e2;
    onb(k, e1, e2);
    float s, c;
    sincospif(2.0f * u, &s, &c);
    return normalize(c * e1 + s * e2);
}

// Inside the regular polygon?  The point was drawn at azimuth 2 pi u inside
// the circumscribed circle, so only the side of its angular sector can bound
// it (the polygon is the union of the triangles centre-side).
__device__ __forceinline__ bool inside_poly(const SourceDev& s, float x, float y, float u_azimuth)
{
    if (s.n_sides <= 0) return true;
    float t = u_azimuth - s.phase_turns;
    t -= floorf(t);
    const int k = min((int)(t * (float)s.n_sides), s.n_sides - 1);
    return x * s.side_cos[k] + y * s.side_sin[k] <= s.apothem;
}

// Event of global photon index idx (binary search on the prefix sums) and
// the photon's first state: direction and polarisation as for any source,
// position from the event's point / segment / ball.
// Emission delay of the scintillation time profile (Sec. 2.2, Table 2): a
// mixture of two exponentials, from its own draw of the source step.
__device__ __forceinline__ float emission_delay(const PropParams& p, uint64_t pid, const TimeProfile& tp)
{
    if (tp.tau_s == 0.0f && tp.tau_t == 0.0f) return 0.0f;
    const U4 u = draw4(p.seed, pid, kSourceStep, 0xFFFFFFFFu);
    const float tau = u.u0 < tp.f_s ? tp.tau_s : tp.tau_t;
    return -tau * logf(u.u1);
}

// Wavelength from the Gaussian emission spectrum (Sec. 2.2, Table 2): the
// Box-Muller transform of the last two uniforms of the emission draw.
__device__ __forceinline__ float emission_wavelength(const PropParams& p, uint64_t pid, const Spectrum& sp)
{
    if (sp.sigma == 0.0f) return sp.mean;
    const U4 u = draw4(p.seed, pid, kSourceStep, 0xFFFFFFFFu);
    float s, c;
    sincospif(2.0f * u.u3, &s, &c);
    return fmaf(sp.sigma, sqrtf(-2.0f * logf(u.u2)) * c, sp.mean);
}

// Index and slowness (n / c) of a material at the photon's wavelength: the
// table values unless some material has dispersion (the kSpectral build of
// the propagation kernel, whose photons carry a wavelength).
template <bool kSpectral>
__device__ __forceinline__ float n_at(const DevMaterial& m, float wl)
{
    return kSpectral ? fmaf(m.dn, wl - LXO_REF_WAVELENGTH_NM, m.n) : m.n;
}

template <bool kSpectral>
__device__ __forceinline__ float n_over_c_at(const DevMaterial& m, float wl)
{
    return kSpectral ? fmaf(m.dn_over_c, wl - LXO_REF_WAVELENGTH_NM, m.n_over_c) : m.n_over_c;
}

__device__ Photon make_event_photon(const PropParams& p, uint64_t idx)
{
    uint32_t lo = 0, hi = p.n_events;  // find e with prefix[e] <= idx < prefix[e+1]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&p.ev_prefix[mid]) <= idx) lo = mid; else hi = mid;
    }
    const EventDev ev = p.events[lo];
    Photon ph;
    ph.pid = ((uint64_t)(p.first_event + lo) << 32) | (uint64_t)(idx - __ldg(&p.ev_prefix[lo]));
    ph.medium = ev.medium;
    ph.time = ev.t0 + emission_delay(p, ph.pid, ev.prof);
    ph.wl = p.spectral ? emission_wavelength(p, ph.pid, ev.spec) : 0.0f;
    ph.last = LXO_NO_HIT;
    ph.step = 0;
    const U4 u = draw4(p.seed, ph.pid, kSourceStep, 0);
    const float c = 2.0f * u.u0 - 1.0f, sn = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    float sp, cp;
    sincospif(2.0f * u.u1, &sp, &cp);
    ph.dir = f3(sn * cp, sn * sp, c);
    ph.pol = random_pol(ph.dir, u.u2);
    if (ev.kind == LXO_SRC_SEGMENT) {
        ph.pos = f3(ev.center[0] + u.u3 * (ev.p1[0] - ev.center[0]), ev.center[1] + u.u3 * (ev.p1[1] - ev.center[1]),
                    ev.center[2] + u.u3 * (ev.p1[2] - ev.center[2]));
    } else {
        ph.pos = f3(ev.center[0], ev.center[1], ev.center[2]);
        if (ev.kind == LXO_SRC_BALL) {
            for (int tr = 0; tr < kMaxTries; ++tr) {
                const U4 w = draw4(p.seed, ph.pid, kSourceStep, 1 + tr);
                const float x = ev.radius * (2.0f * w.u0 - 1.0f), y = ev.radius * (2.0f * w.u1 - 1.0f),
                            z = ev.radius * (2.0f * w.u2 - 1.0f);
                if (x * x + y * y + z * z <= ev.radius * ev.radius) {
                    ph.pos = f3(ev.center[0] + x, ev.center[1] + y, ev.center[2] + z);
                    break;
                }
            }
        }
    }
    return ph;
}

__device__ Photon make_photon(const PropParams& p, uint64_t idx)
{
    if (p.n_events) return make_event_photon(p, idx);
    const SourceDev& s = p.src;
    Photon ph;
    ph.pid = p.base + idx;
    ph.medium = s.medium;
    ph.time = s.t0 + emission_delay(p, ph.pid, s.prof);
    ph.wl = p.spectral ? emission_wavelength(p, ph.pid, s.spec) : 0.0f;
    ph.last = LXO_NO_HIT;
    ph.step = 0;
    if (s.kind == LXO_SRC_EXPLICIT) {
        ph.pos = f3(s.pos[3 * idx], s.pos[3 * idx + 1], s.pos[3 * idx + 2]);
        ph.dir = normalize(f3(s.dir[3 * idx], s.dir[3 * idx + 1], s.dir[3 * idx + 2]));
        float3 e = f3(s.pol[3 * idx], s.pol[3 * idx + 1], s.pol[3 * idx + 2]);
        ph.pol = normalize(e - dot(e, ph.dir) * ph.dir);
        return ph;
    }
    const U4 u = draw4(p.seed, ph.pid, kSourceStep, 0);
    const float c = 2.0f * u.u0 - 1.0f, sn = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    float sp, cp;
    sincospif(2.0f * u.u1, &sp, &cp);
    ph.dir = f3(sn * cp, sn * sp, c);
    ph.pol = random_pol(ph.dir, u.u2);
    if (s.kind == LXO_SRC_POINT) {
        ph.pos = f3(s.center[0], s.center[1], s.center[2]);
    } else if (s.kind == LXO_SRC_SEGMENT) {
        ph.pos = f3(s.center[0] + u.u3 * (s.p1[0] - s.center[0]), s.center[1] + u.u3 * (s.p1[1] - s.center[1]),
                    s.center[2] + u.u3 * (s.p1[2] - s.center[2]));
    } else if (s.kind == LXO_SRC_BALL) {
        ph.pos = f3(s.center[0], s.center[1], s.center[2]);
        for (int tr = 0; tr < kMaxTries; ++tr) {
            const U4 w = draw4(p.seed, ph.pid, kSourceStep, 1 + tr);
            const float x = s.radius * (2.0f * w.u0 - 1.0f), y = s.radius * (2.0f * w.u1 - 1.0f),
                        z = s.radius * (2.0f * w.u2 - 1.0f);
            if (x * x + y * y + z * z <= s.radius * s.radius) {
                ph.pos = f3(s.center[0] + x, s.center[1] + y, s.center[2] + z);
                break;
            }
        }
    } else {
        ph.pos = f3(0.0f, 0.0f, s.z_min + u.u3 * (s.z_max - s.z_min));
        for (int tr = 0; tr < kMaxTries; ++tr) {
            const U4 w = draw4(p.seed, ph.pid, kSourceStep, 1 + tr);
            float r = s.radius * sqrtf(w.u0), sa, ca;
            sincospif(2.0f * w.u1, &sa, &ca);
            if (inside_poly(s, r * ca, r * sa, w.u1)) {
                ph.pos.x = r * ca;
                ph.pos.y = r * sa;
                break;
            }
            r = s.radius * sqrtf(w.u2);
            sincospif(2.0f * w.u3, &sa, &ca);
            if (inside_poly(s, r * ca, r * sa, w.u3)) {
                ph.pos.x = r * ca;
                ph.pos.y = r * sa;
                break;
            }
        }
    }
    return ph;
}

// Out of line, for the photon loop that resumes queries: inline, its
// register demand spilled the traversal state that loop keeps across passes
// (1.5 % faster out of line; the loop of whole steps is faster with it
// inline).
__device__ __noinline__ Photon make_photon_outlined(const PropParams& p, uint64_t idx)
{
    return make_photon(p, idx);
}

__global__ void k_sample_source(const __grid_constant__ PropParams p, float* pos, float* dir, float* pol,
                                float* time, float* wavelength)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const Photon ph = make_photon(p, i);
    pos[3 * i] = ph.pos.x; pos[3 * i + 1] = ph.pos.y; pos[3 * i + 2] = ph.pos.z;
    dir[3 * i] = ph.dir.x; dir[3 * i + 1] = ph.dir.y; dir[3 * i + 2] = ph.dir.z;
    pol[3 * i] = ph.pol.x; pol[3 * i + 1] = ph.pol.y; pol[3 * i + 2] = ph.pol.z;
    if (time) time[i] = ph.time;
    if (wavelength) wavelength[i] = emission_wavelength(p, ph.pid, p.src.spec);
}

// ---------------------------------------------------------------------------
// interactions (Sec. 2.2; Appendix items 1 and 3)
// ---------------------------------------------------------------------------

// Rayleigh scattering, dipole law: density of the new direction k' is
// proportional to 1 - (k'.eps)^2; new polarisation = eps projected
// perpendicular to k'.  Sampled without a loop, in the frame whose pole is
// eps: c = cos(k', eps) from the inverse of its CDF, the cubic c^3 - 3c =
// 2 - 4 u0, c = 2 cos((acos(1 - 2 u0) + 4 pi) / 3); azimuth 2 pi u1 in
// onb(eps).  With w the unit azimuthal vector, k' = c eps + s w and the
// projection of eps perpendicular to k' is s (s eps - c w), s = sin.
__device__ __forceinline__ void rayleigh(Photon& ph, uint64_t seed)
{
    const U4 u = draw4(seed, ph.pid, ph.step, 1);
    const float a = acosf(1.0f - 2.0f * u.u0) * 0.318309886183790672f;   // in units of pi
    const float c = 2.0f * cospif((a + 4.0f) * (1.0f / 3.0f));
    const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    float sp, cp;
    sincospif(2.0f * u.u1, &sp, &cp);
    float3 e1, e2;
    onb(ph.pol, e1, e2);
    const float3 w = cp * e1 + sp * e2;
    const float3 eps = ph.pol;
    ph.dir = normalize(c * eps + s * w);
    ph.pol = normalize(s * eps - c * w);
}

// Lambertian reflection about the incident-side normal N (draw 1 of the step)
__device__ __forceinline__ void lambert(Photon& ph, float3 N, uint64_t seed)
{
    const U4 u = draw4(seed, ph.pid, ph.step, 1);
    const float c = sqrtf(u.u0), sn = sqrtf(fmaxf(0.0f, 1.0f - u.u0));
    float sp, cp;
    sincospif(2.0f * u.u1, &sp, &cp);
    float3 t1, t2;
    onb(N, t1, t2);
    ph.dir = normalize(c * N + sn * (cp * t1 + sp * t2));
    ph.pol = random_pol(ph.dir, u.u2);
}

__device__ __forceinline__ void mirror(Photon& ph, float3 N)
{
    const float ci = -dot(ph.dir, N);
    const float pe = dot(ph.pol, N);
    ph.dir = normalize(ph.dir + (2.0f * ci) * N);
    float3 e = (2.0f * pe) * N - ph.pol;
    e = e - dot(e, ph.dir) * ph.dir;
    ph.pol = normalize(e);
}

// Fresnel at a bare dielectric boundary n1 -> n2 with a linearly polarised
// photon: P(reflect) = cs^2 Rs + cp^2 Rp; outgoing polarisation is the
// coherent sum of the s and p amplitudes (p basis = s x k of each wave;
// magnitudes only under total internal reflection).  Normal incidence:
// s = eps (Appendix item 1).  Returns true if reflected.
__device__ __forceinline__ bool dielectric(Photon& ph, float3 N, float n1, float n2, float u)
{
    const float3 k = ph.dir;
    const float ci = fminf(1.0f, -dot(k, N));
    float3 s = cross(k, N);
    const float sl2 = dot(s, s);
    s = (sl2 < 1e-12f) ? ph.pol : rsqrtf(sl2) * s;
    const float3 pin = cross(s, k);
    const float cs = dot(ph.pol, s), cpv = dot(ph.pol, pin);
    const float eta = n1 / n2;
    const float st2 = eta * eta * (1.0f - ci * ci);
    float rs = 1.0f, rp = 1.0f, ts = 0.0f, tp = 0.0f, ct = 0.0f, pr = 1.0f;
    const bool tir = st2 >= 1.0f;
    if (!tir) {
        ct = sqrtf(1.0f - st2);
        const float a = n1 * ci, b = n2 * ct, c2 = n2 * ci, d2 = n1 * ct;
        // one fast reciprocal per denominator (2 ulp; the physics is float32
        // and statistical, unlike the exact intersection)
        const float i1 = __fdividef(1.0f, a + b), i2 = __fdividef(1.0f, c2 + d2);
        rs = (a - b) * i1;
        rp = (c2 - d2) * i2;
        ts = 2.0f * a * i1;
        tp = 2.0f * a * i2;
        pr = cs * cs * rs * rs + cpv * cpv * rp * rp;
    }
    if (u < pr) {
        const float3 kr = normalize(k + (2.0f * ci) * N);
        const float3 pr_v = cross(s, kr);
        const float as = tir ? cs : cs * rs, ap = tir ? cpv : cpv * rp;
        ph.dir = kr;
        ph.pol = normalize(as * s + ap * pr_v);
        return true;
    }
    const float3 kt = normalize(eta * k + (eta * ci - ct) * N);
    const float3 pt_v = cross(s, kt);
    ph.dir = kt;
    ph.pol = normalize((cs * ts) * s + (cpv * tp) * pt_v);
    return false;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) { return fmaxf(a, fmaxf(b, c)); }

// move off the surface just hit by a margin above the rounding of the hit point
__device__ __forceinline__ void spawn_offset(Photon& ph, float3 o_ray, float t_hit, float3 N, float side)
{
    float m = fmaxf(fmaxf(1.0f, t_hit), fmaxf(fmax3(fabsf(ph.pos.x), fabsf(ph.pos.y), fabsf(ph.pos.z)),
                                              fmax3(fabsf(o_ray.x), fabsf(o_ray.y), fabsf(o_ray.z))));
    const float eps = m * 3.814697265625e-06f;  // 2^-18
    ph.pos = ph.pos + (side * eps) * N;
}

// one interaction; returns -1 if the photon lives on, else its fate code
// (detail set to channel / material / surface / triangle)
// First half of a step: the step's uniforms and the absorption / Rayleigh
// distances in the current medium.
struct StepDraw {
    float d_abs, d_ray, u2, u3;
};

template <bool kSpectral>
__device__ __forceinline__ StepDraw begin_step(const PropParams& p, const Photon& ph)
{
    const U4 u = draw4(p.seed, ph.pid, ph.step, 0);
    const DevMaterial& mt = p.mat[ph.medium];
    StepDraw sd;
    float ray_len = mt.ray_len;
    // (lambda / reference)^p as 2^(p log2(lambda / reference)), with the fast
    // base-2 logarithm (documented error: 2^-22 absolute on [0.5, 2], 2 ulp
    // elsewhere) in place of powf's exact-case handling
    if (kSpectral && mt.ray_exp != 0.0f)
        ray_len *= exp2f(mt.ray_exp * __log2f(ph.wl * (1.0f / LXO_REF_WAVELENGTH_NM)));
    // the accurate logarithm: the fast one's absolute error near u = 1 biases
    // the sampled distances by ~1e-4 mm, enough for the paired parity tests
    // of the adjoint tallies to see it (measured, 2 % faster)
    sd.d_abs = isinf(mt.abs_len) ? INFINITY : -mt.abs_len * logf(u.u0);
    sd.d_ray = isinf(ray_len) ? INFINITY : -ray_len * logf(u.u1);
    sd.u2 = u.u2;
    sd.u3 = u.u3;
    return sd;
}

template <bool kStats>
__device__ __forceinline__ void step_histogram(const PropParams& p, const Photon& ph, uint32_t dn, uint32_t dl)
{
    // per-step histogram of node visits (8-wide bins) split by medium (0 vs other), and leaves
    const int m = ph.medium == 0 ? 0 : 1;
    atomicAdd(&p.out.stats[9 + 10 * m + min(dn / 8u, 8u)], 1ull);
    atomicAdd(&p.out.stats[9 + 10 * m + 9], (unsigned long long)dl);
}

// Second half of a step: the interaction at the closest hit or in the bulk.
// Returns -1 if the photon lives on, else its fate code (detail set to
// channel / material / surface / triangle).
// Adjoint tallies of one lane live in shared memory, tally k at tl[k * blockDim.x].
constexpr int kAdjMaxK = 2 * (LXO_ADJ_MAX_MATERIALS + LXO_ADJ_MAX_SURFACES);

template <bool kAdjoint, bool kSpectral>
__device__ int finish_step(const PropParams& p, Photon& ph, const StepDraw& sd, const Hit& h, int& detail,
                           float* tl)
{
    const float d_abs = sd.d_abs, d_ray = sd.d_ray, d_int = fminf(d_abs, d_ray);
    const U4 u = U4{0.0f, 0.0f, sd.u2, sd.u3};
    const DevMaterial& mt = p.mat[ph.medium];
    const int ms = kAdjoint ? p.adj_mat_slot[ph.medium] : -1;
    if (h.id == LXO_NO_HIT) {
        if (isinf(d_int)) {
            detail = -1;
            return LXO_FATE_ESCAPED;
        }
        ph.pos = ph.pos + d_int * ph.dir;
        ph.time += d_int * n_over_c_at<kSpectral>(mt, ph.wl);
        if (kAdjoint && ms >= 0) tl[(2 * ms) * blockDim.x] += d_int;
        if (d_abs <= d_ray) {
            detail = ph.medium;
            return LXO_FATE_BULK_ABS;
        }
        if (kAdjoint && ms >= 0) tl[(2 * ms + 1) * blockDim.x] += 1.0f;
        rayleigh(ph, p.seed);
        ph.last = LXO_NO_HIT;
        return -1;
    }
    const float3 o_ray = ph.pos;
    ph.pos = ph.pos + h.t * ph.dir;
    ph.time += h.t * n_over_c_at<kSpectral>(mt, ph.wl);
    if (kAdjoint && ms >= 0) tl[(2 * ms) * blockDim.x] += h.t;
    // geometric normal and attributes of the triangle hit (record in leaf order)
    if (LXO_CHECK_BOUNDS && h.rec >= p.sc.n_records) {
        atomicOr(p.err, kErrBounds);
        detail = (int)h.id;
        return LXO_FATE_GEOM_ERR;
    }
    const float4* tr = p.sc.tris + 3 * (size_t)h.rec;
    const float4 va = __ldg(tr + 0), vb = __ldg(tr + 1), vc = __ldg(tr + 2);
    const uint2 at = make_uint2(__float_as_uint(vc.z), __float_as_uint(vc.w));
    const float3 e1 = f3(va.w - va.x, vb.x - va.y, vb.y - va.z);
    const float3 e2 = f3(vb.z - va.x, vb.w - va.y, vc.x - va.z);
    const float3 ng = normalize(cross(e1, e2));
    const bool forward = dot(ph.dir, ng) > 0.0f;
    const int mi = at.x & 0xFF, mo = (at.x >> 8) & 0xFF;
    const uint32_t sid = at.x >> 16;
    const int from = forward ? mi : mo, to = forward ? mo : mi;
    const float3 Nf = forward ? (-1.0f) * ng : ng;
    ph.last = h.id;
    if (sid == LXO_SURF_NONE) {
        if (from != ph.medium || to >= p.n_mat) {
            detail = (int)h.id;
            return LXO_FATE_GEOM_ERR;
        }
        const bool refl = dielectric(ph, Nf, n_at<kSpectral>(p.mat[from], ph.wl), n_at<kSpectral>(p.mat[to], ph.wl),
                                      u.u2);
        if (!refl) ph.medium = to;
        spawn_offset(ph, o_ray, h.t, Nf, refl ? 1.0f : -1.0f);
        return -1;
    }
    const DevSurface& sf = p.surf[sid];
    if (sf.type == LXO_SURF_ABSORBER) {
        detail = (int)sid;
        return LXO_FATE_SURF_ABS;
    }
    if (sf.type == LXO_SURF_PHOTOCATHODE) {
        const int ch = (int)at.y;
        if (ch < 0 || ch >= p.n_chan) {
            atomicOr(p.err, kErrChannel);
            detail = (int)h.id;
            return LXO_FATE_GEOM_ERR;
        }
        detail = ch;
        return (u.u2 < sf.qe) ? LXO_FATE_DETECTED : LXO_FATE_QE_FAIL;
    }
    bool specular;
    const int ss = kAdjoint ? p.adj_surf_slot[sid] : -1;
    const int base_k = 2 * p.adj_n_mats + 2 * ss;
    if (sf.type == LXO_SURF_REFLECTOR) {
        if (!(u.u2 < sf.R)) {
            detail = (int)sid;
            return LXO_FATE_SURF_ABS;
        }
        if (kAdjoint && ss >= 0) tl[base_k * blockDim.x] += 1.0f;
        specular = u.u3 < sf.spec;
    } else if (sf.type == LXO_SURF_ELECTRODE_T) {
        if (u.u2 < sf.T) {
            if (from != ph.medium || to >= p.n_mat) {
                detail = (int)h.id;
                return LXO_FATE_GEOM_ERR;
            }
            if (kAdjoint && ss >= 0) tl[base_k * blockDim.x] += 1.0f;
            ph.medium = to;
            spawn_offset(ph, o_ray, h.t, Nf, -1.0f);
            return -1;
        }
        if (!(u.u3 < sf.Rw)) {
            detail = (int)sid;
            return LXO_FATE_SURF_ABS;
        }
        if (kAdjoint && ss >= 0) tl[(base_k + 1) * blockDim.x] += 1.0f;
        specular = draw4(p.seed, ph.pid, ph.step, 1).u3 < sf.wspec;
    } else {
        detail = (int)h.id;
        return LXO_FATE_GEOM_ERR;
    }
    if (specular)
        mirror(ph, Nf);
    else
        lambert(ph, Nf, p.seed);
    spawn_offset(ph, o_ray, h.t, Nf, 1.0f);
    return -1;
}

// One whole step in one pass (draws, closest hit, interaction), for the
// builds whose warps wait for their slowest query.
template <bool kStats, bool kAdjoint, bool kSpectral>
__device__ int photon_step(const PropParams& p, Photon& ph, int& detail, Counters& cnt, float* tl)
{
    const long long cd = kStats ? clock64() : 0;
    const StepDraw sd = begin_step<kSpectral>(p, ph);
    const long long c0 = kStats ? clock64() : 0;
    if (kStats) cnt.cyc[kCycDraw] += (unsigned long long)(c0 - cd);
    const uint32_t n0 = kStats ? cnt.nodes : 0, l0 = kStats ? cnt.leaves : 0;
    const Hit h = closest_hit<kStats>(p.sc, ph.pos, ph.dir, ph.last, fminf(sd.d_abs, sd.d_ray), p.err, cnt);
    if (kStats) {
        cnt.trav_cycles += (unsigned long long)(clock64() - c0);
        step_histogram<kStats>(p, ph, cnt.nodes - n0, cnt.leaves - l0);
    }
    const long long cf = kStats ? clock64() : 0;
    const int fate = finish_step<kAdjoint, kSpectral>(p, ph, sd, h, detail, tl);
    if (kStats) cnt.cyc[kCycFinish] += (unsigned long long)(clock64() - cf);
    return fate;
}

// ---------------------------------------------------------------------------
// persistent propagation kernel
// ---------------------------------------------------------------------------
// Register budgets, as CTAs of 256 threads per SM: every flavour of the
// kernel is built for both and the launch shape picks one.  On the
// DARWIN-scale forward workload (GB300) 8 CTAs (32 registers, the SM's 2048
// threads) hide more latency than 6 (40 registers, +1.4 % time), 5 (48,
// +5.4 %) or 4 (64, +9.8 %) despite their spills; the adjoint build and the
// small 50 cm TPC, whose BVH stays in L1, run faster with 48 registers.
// Lanes refill as soon as one is idle.
#ifndef LXO_REFILL_MIN
#define LXO_REFILL_MIN 1
#endif
constexpr int kBudgetFull = 8;   // 32 registers
constexpr int kBudgetWide = 5;   // 48 registers

// Tally of one photon's fate: shared-memory fate counters, global per-channel
// counts and arrival-time histogram, optional per-photon record and adjoint
// sums.  Plain per-lane atomics: aggregating them over the lanes of a warp
// that hit the same counter (match + reduce) measured 3.8 % slower on the
// DARWIN-scale workload, where two lanes rarely tally the same channel at
// once.
template <bool kAdjoint>
__device__ __forceinline__ void tally(const PropParams& p, unsigned long long* s_f, const Photon& ph, int fate,
                                      int detail, const float* tl)
{
    // row of the per-channel tallies: the channel, or (event - first event) * P + channel for batched events
    const size_t row = p.n_events ? (size_t)((uint32_t)(ph.pid >> 32) - p.first_event) * p.n_chan + detail
                                  : (size_t)detail;
    if (LXO_CHECK_BOUNDS && (fate == LXO_FATE_DETECTED || fate == LXO_FATE_QE_FAIL) &&
        (detail < 0 || row >= (size_t)(p.n_events ? p.n_events : 1) * p.n_chan)) {
        atomicOr(p.err, kErrBounds);
        return;
    }
    if (kAdjoint && fate == LXO_FATE_DETECTED)
        for (int k = 0; k < p.adj_k; ++k)
            atomicAdd(&p.out.adjoint[row * p.adj_k + k], (double)tl[k * blockDim.x]);
    atomicAdd(&s_f[fate], 1ull);
    atomicAdd(&s_f[7], (unsigned long long)ph.step);
    if (fate == LXO_FATE_BULK_ABS) atomicAdd(&s_f[LXO_FATES_FIXED + detail], 1ull);
    if (fate == LXO_FATE_SURF_ABS) atomicAdd(&s_f[LXO_FATES_FIXED + p.n_mat + detail], 1ull);
    if (fate == LXO_FATE_DETECTED || fate == LXO_FATE_QE_FAIL) {
        atomicAdd(&p.out.lce[row], 1u);
        if (fate == LXO_FATE_DETECTED) {
            atomicAdd(&p.out.det[row], 1u);
            if (p.out.hist) {
                const float b = floorf(ph.time / p.tbin);
                const uint32_t bin = (b >= (float)p.n_tbins || !(b >= 0.0f)) ? p.n_tbins : (uint32_t)b;
                atomicAdd(&p.out.hist[row * (p.n_tbins + 1) + bin], 1u);
            }
        }
    }
    const uint64_t idx = ph.pid - p.base;
    if (p.out.ph_fate) p.out.ph_fate[idx] = (uint32_t)fate;
    if (p.out.ph_detail) p.out.ph_detail[idx] = detail;
    if (p.out.ph_steps) p.out.ph_steps[idx] = ph.step;
    if (p.out.ph_time) p.out.ph_time[idx] = ph.time;
    if (p.out.ph_state) {
        float* o = p.out.ph_state + 9 * idx;
        o[0] = ph.pos.x; o[1] = ph.pos.y; o[2] = ph.pos.z;
        o[3] = ph.dir.x; o[4] = ph.dir.y; o[5] = ph.dir.z;
        o[6] = ph.pol.x; o[7] = ph.pol.y; o[8] = ph.pol.z;
    }
}

// Warp-uniform: makes sure the warp's chunk of photon ids is not empty,
// taking the next p.chunk ids from the global work queue; false once the
// queue is exhausted.
__device__ __forceinline__ bool warp_chunk(const PropParams& p, uint32_t lane, unsigned long long& next,
                                           unsigned long long& end, bool& exhausted)
{
    if (next < end) return true;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)p.chunk);
    base = __shfl_sync(FULL_MASK, base, 0);
    if (base >= p.n) {
        exhausted = true;
        return false;
    }
    next = base;
    end = min(base + p.chunk, (unsigned long long)p.n);
    return true;
}

// A photon in a warp's batch buffer: word j of slot k at o[j * kBatchN + k]
// (consecutive lanes, consecutive banks).  Position, direction,
// polarisation, id and, in the spectral build, the wavelength are kept;
// medium and emission time follow from the id and the source when the
// photon is taken, exactly as make_photon computes them (a smaller buffer
// leaves more of the SM's memory to L1: 1.5 % faster than keeping all 13
// words; the wavelength's Box-Muller draw is too dear to redo one lane at a
// time).
constexpr int kBatchN = 32;
template <bool kSpectral>
struct BatchSlot {
    static constexpr int kWords = kSpectral ? 12 : 11;
    static __device__ __forceinline__ void store(float* o, const Photon& q)
    {
        o[0 * kBatchN] = q.pos.x; o[1 * kBatchN] = q.pos.y; o[2 * kBatchN] = q.pos.z;
        o[3 * kBatchN] = q.dir.x; o[4 * kBatchN] = q.dir.y; o[5 * kBatchN] = q.dir.z;
        o[6 * kBatchN] = q.pol.x; o[7 * kBatchN] = q.pol.y; o[8 * kBatchN] = q.pol.z;
        o[9 * kBatchN] = __uint_as_float((uint32_t)q.pid);
        o[10 * kBatchN] = __uint_as_float((uint32_t)(q.pid >> 32));
        if (kSpectral) o[11 * kBatchN] = q.wl;
    }
    static __device__ __forceinline__ Photon load(const float* o, const PropParams& p)
    {
        Photon q;
        q.pos = f3(o[0 * kBatchN], o[1 * kBatchN], o[2 * kBatchN]);
        q.dir = f3(o[3 * kBatchN], o[4 * kBatchN], o[5 * kBatchN]);
        q.pol = f3(o[6 * kBatchN], o[7 * kBatchN], o[8 * kBatchN]);
        q.pid = (uint64_t)__float_as_uint(o[9 * kBatchN]) | ((uint64_t)__float_as_uint(o[10 * kBatchN]) << 32);
        if (p.n_events) {
            const EventDev& ev = p.events[(uint32_t)(q.pid >> 32) - p.first_event];
            q.medium = ev.medium;
            q.time = ev.t0 + emission_delay(p, q.pid, ev.prof);
        } else {
            q.medium = p.src.medium;
            q.time = p.src.t0 + emission_delay(p, q.pid, p.src.prof);
        }
        q.wl = kSpectral ? o[11 * kBatchN] : 0.0f;
        q.last = LXO_NO_HIT;
        q.step = 0;
        return q;
    }
};

// Persistent photon loop.  A lane whose photon reached its fate records its
// tallies and takes the next photon id of its warp's chunk (ballot + prefix
// popcount); chunks of p.chunk ids come from the global work-queue head.  A
// lane refills as soon as it is idle (LXO_REFILL_MIN = 1: waiting for more
// idle lanes measured slower).
// Forward builds:
// * Lanes do not wait for the slowest query of their warp: each pass of the
//   loop traces until some lane has finished its query, and the unfinished
//   queries resume in the next pass beside the fresh ones (dynamic ray
//   fetch; on the DARWIN-scale mesh the lanes active in the node loop rose
//   from 31 % to 45 % and in the leaf loop from 11 % to 20 %, 9 % less time).
// * Photons are made a batch at a time: about one lane dies per pass, so
//   when its shared-memory buffer is empty the warp makes the next kBatchN
//   photons of its chunk, one per lane, and lanes that need a photon take
//   the next ones from the buffer (7 % less time).
// Adjoint builds keep whole steps and make photons lane by lane: with their
// tallies the resumable loop was 4 % slower on the 50 cm TPC, whose tree
// stays in L1.
// Built for CTAs of kThreads = 256 (kBudget per SM) or 128 threads (twice as
// many CTAs): the same registers per thread either way.
template <bool kStats, bool kAdjoint, bool kSpectral, int kThreads, int kBudget>
__global__ void __launch_bounds__(kThreads, kBudget * 256 / kThreads)
    k_propagate(const __grid_constant__ PropParams p)
{
    constexpr bool kYield = !kAdjoint;
    Counters cnt{};
    uint32_t my_steps = 0, outer_iters = 0;
    unsigned long long loop_cycles = 0;
    __shared__ unsigned long long s_f[kMaxFates];
    __shared__ float s_tl[kAdjoint ? kAdjMaxK * kThreads : 1];
    float* tl = kAdjoint ? &s_tl[threadIdx.x] : nullptr;
    for (int i = threadIdx.x; i < p.n_fates; i += blockDim.x) s_f[i] = 0ull;
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    unsigned long long chunk_next = 0, chunk_end = 0;  // warp-uniform
    bool exhausted = false;                             // warp-uniform
    bool alive = false, pending = false;
    int fate = 0, detail = -1;
    Photon ph;
    StepDraw sd;                 // the current step's draws
    TravResume tr;               // its query (kDone: none in flight)
    tr.node = kDone;
    int stack[kStackSize];
    uint32_t n0 = 0, l0 = 0;     // counting build: node visits and leaves when the step began
    using Slot = BatchSlot<kSpectral>;
    __shared__ float s_batch[kYield ? (kThreads / 32) * Slot::kWords * kBatchN : 1];
    float* batch = kYield ? &s_batch[(threadIdx.x >> 5) * Slot::kWords * kBatchN] : nullptr;
    uint32_t batch_head = 0, batch_count = 0;   // warp-uniform: next buffered photon, photons buffered

    while (true) {
        uint32_t need = __ballot_sync(FULL_MASK, !alive);
        const int idle = __popc(need);
        const long long cr = kStats ? clock64() : 0;
        if (idle >= LXO_REFILL_MIN || idle == 32) {
            if (pending) {
                tally<kAdjoint>(p, s_f, ph, fate, detail, tl);
                pending = false;
            }
            if constexpr (kYield) {
                while (need && (batch_head < batch_count || !exhausted)) {
                    if (batch_head == batch_count) {
                        if (!warp_chunk(p, lane, chunk_next, chunk_end, exhausted)) break;
                        const uint32_t make = min((uint32_t)(chunk_end - chunk_next), (uint32_t)kBatchN);
                        if (lane < make) Slot::store(batch + lane, make_photon_outlined(p, chunk_next + lane));
                        __syncwarp();
                        chunk_next += make;
                        batch_head = 0;
                        batch_count = make;
                    }
                    const uint32_t take = min(batch_count - batch_head, (uint32_t)__popc(need));
                    const uint32_t rank = __popc(need & lt_mask);
                    if (((need >> lane) & 1u) && rank < take) {
                        ph = Slot::load(batch + batch_head + rank, p);
                        alive = true;
                    }
                    batch_head += take;
                    __syncwarp();
                    need = __ballot_sync(FULL_MASK, !alive);
                }
            }
            while (!kYield && need && !exhausted) {
                if (chunk_next >= chunk_end) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)p.chunk);
                    base = __shfl_sync(FULL_MASK, base, 0);
                    if (base >= p.n) {
                        exhausted = true;
                        break;
                    }
                    chunk_next = base;
                    chunk_end = min(base + p.chunk, (unsigned long long)p.n);
                }
                const uint32_t avail = (uint32_t)(chunk_end - chunk_next);
                const uint32_t take = min(avail, (uint32_t)__popc(need));
                const uint32_t rank = __popc(need & lt_mask);
                if (((need >> lane) & 1u) && rank < take) {
                    ph = make_photon(p, chunk_next + rank);
                    if (kAdjoint)
                        for (int k = 0; k < p.adj_k; ++k) tl[k * kThreads] = 0.0f;
                    alive = true;
                }
                chunk_next += take;
                need = __ballot_sync(FULL_MASK, !alive);
            }
        }
        if (kStats) cnt.cyc[kCycRefill] += (unsigned long long)(clock64() - cr);
        if (!__any_sync(FULL_MASK, alive || pending)) break;
        if (kStats && lane == 0) outer_iters++;
        const long long c0 = kStats ? clock64() : 0;
        if (alive) {
            // A step is the draws, a closest-hit query and the interaction.
            // With kYield the query may span several passes of this loop: the
            // warp leaves the traversal once one of its lanes has finished,
            // and that lane interacts (or refills) and starts its next query
            // while the others resume theirs.
            bool stepped = true;
            if constexpr (kYield) {
                float tmax = 0.0f;
                if (tr.node == kDone) {
                    const long long cd = kStats ? clock64() : 0;
                    sd = begin_step<kSpectral>(p, ph);
                    tmax = fminf(sd.d_abs, sd.d_ray);
                    if (kStats) {
                        cnt.cyc[kCycDraw] += (unsigned long long)(clock64() - cd);
                        n0 = cnt.nodes;
                        l0 = cnt.leaves;
                    }
                }
                trav_step<kStats>(p.sc, ph.pos, ph.dir, ph.last, tmax, tr, stack, p.err, cnt);
                stepped = tr.node == kDone;
                if (stepped) {
                    if (kStats) step_histogram<kStats>(p, ph, cnt.nodes - n0, cnt.leaves - l0);
                    const long long cf = kStats ? clock64() : 0;
                    const Hit h{tr.best, tr.best_rec, tr.best == LXO_NO_HIT ? INFINITY : tr.bt};
                    fate = finish_step<kAdjoint, kSpectral>(p, ph, sd, h, detail, tl);
                    if (kStats) cnt.cyc[kCycFinish] += (unsigned long long)(clock64() - cf);
                }
            } else {
                fate = photon_step<kStats, kAdjoint, kSpectral>(p, ph, detail, cnt, tl);
            }
            if (stepped) {
                ph.step++;
                if (kStats) my_steps++;
                if (fate < 0 && ph.step >= p.max_steps) {
                    fate = LXO_FATE_TRUNCATED;
                    detail = -1;
                }
                if (fate >= 0) {
                    alive = false;
                    pending = true;
                }
            }
        }
        if (kStats) loop_cycles += (unsigned long long)(clock64() - c0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.n_fates; i += blockDim.x)
        if (s_f[i]) atomicAdd(&p.out.fates[i], s_f[i]);
    if (kStats) {
        atomicAdd(&p.out.stats[0], (unsigned long long)my_steps);
        atomicAdd(&p.out.stats[1], (unsigned long long)cnt.nodes);
        atomicAdd(&p.out.stats[2], (unsigned long long)cnt.leaves);
        atomicAdd(&p.out.stats[3], (unsigned long long)cnt.tris);
        atomicAdd(&p.out.stats[4], (unsigned long long)cnt.node_iters);
        atomicAdd(&p.out.stats[5], (unsigned long long)cnt.leaf_iters);
        atomicAdd(&p.out.stats[6], (unsigned long long)outer_iters);
        atomicAdd(&p.out.stats[7], cnt.trav_cycles);
        atomicAdd(&p.out.stats[8], loop_cycles);
        for (int k = 0; k < kCycPhases; ++k) atomicAdd(&p.out.stats[29 + k], cnt.cyc[k]);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_trace(const Scene& sc, const float* org, const float* dir, const uint32_t* skip,
                         const float* tmax, uint32_t n, uint32_t* hit, float* t, int* err, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int threads = 128;
    k_trace<<<(n + threads - 1) / threads, threads, 0, st>>>(sc, org, dir, skip, tmax, n, hit, t, err);
    return cudaGetLastError();
}

cudaError_t launch_sample_source(const PropParams& p, float* pos, float* dir, float* pol, float* time,
                                 float* wavelength, cudaStream_t st)
{
    if (p.n == 0) return cudaSuccess;
    const int threads = 128;
    const uint64_t blocks = (p.n + threads - 1) / threads;
    k_sample_source<<<(unsigned)blocks, threads, 0, st>>>(p, pos, dir, pol, time, wavelength);
    return cudaGetLastError();
}

template <int kThreads, int kBudget>
static cudaError_t launch_propagate_t(const PropParams& p, int sms, cudaStream_t st)
{
    const bool stats = (p.flags & LXO_FLAG_STATS) != 0;
    const bool adj = (p.flags & LXO_FLAG_ADJOINT) != 0;
    auto kern = p.spectral ? (adj ? k_propagate<false, true, true, kThreads, kBudget>
                                  : k_propagate<false, false, true, kThreads, kBudget>)
                           : (adj ? k_propagate<false, true, false, kThreads, kBudget>
                                  : k_propagate<false, false, false, kThreads, kBudget>);
    if (stats)  // the counting build exists for the default shape only
        kern = p.spectral ? (adj ? k_propagate<true, true, true, 256, kBudgetFull>
                                 : k_propagate<true, false, true, 256, kBudgetFull>)
                          : (adj ? k_propagate<true, true, false, 256, kBudgetFull>
                                 : k_propagate<true, false, false, 256, kBudgetFull>);
    const int threads = stats ? 256 : kThreads;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return e;
    if (p.blocks_per_sm > 0 && (int)p.blocks_per_sm < per_sm) per_sm = (int)p.blocks_per_sm;
    uint64_t blocks = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const uint64_t need = (p.n + threads - 1) / threads;
    if (need < blocks) blocks = need;
    kern<<<(unsigned)blocks, threads, 0, st>>>(p);
    return cudaGetLastError();
}

// The register budget: the wide one (48 registers) when the launch asks for
// at most kBudgetWide CTAs of 256 threads per SM, or by default for the
// adjoint build; else the full-occupancy one (32 registers).
template <int kThreads>
static cudaError_t launch_propagate_b(const PropParams& p, int sms, cudaStream_t st)
{
    const int per256 = 256 / kThreads;
    const bool adj = (p.flags & LXO_FLAG_ADJOINT) != 0;
    const bool wide = p.blocks_per_sm ? (int)p.blocks_per_sm <= kBudgetWide * per256 : adj;
    return wide ? launch_propagate_t<kThreads, kBudgetWide>(p, sms, st)
                : launch_propagate_t<kThreads, kBudgetFull>(p, sms, st);
}

cudaError_t launch_propagate(const PropParams& p, int device, cudaStream_t st)
{
    if (p.n == 0) return cudaSuccess;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    return p.block_threads == 128 ? launch_propagate_b<128>(p, sms, st) : launch_propagate_b<256>(p, sms, st);
}

// ---------------------------------------------------------------------------
// adjoint backward: J[c][q] = a_q * sums[c][ia_q] + b_q * sums[c][ib_q];
// optional grad[q] = sum_c g[c] J[c][q]
// ---------------------------------------------------------------------------
struct AdjCoefs {
    AdjCoef c[2 * LXO_ADJ_MAX_MATERIALS + LXO_ADJ_MAX_SURFACES];
};

__global__ void k_adjoint_jacobian(const AdjCoefs co, int Q, int K, int P, const double* __restrict__ sums,
                                   double* __restrict__ J)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * Q) return;
    const int ch = i / Q, q = i % Q;
    const AdjCoef& c = co.c[q];
    J[i] = c.a * sums[(size_t)ch * K + c.ia] + c.b * sums[(size_t)ch * K + c.ib];
}

__global__ void k_adjoint_vjp(int Q, int P, const double* __restrict__ J, const double* __restrict__ g,
                              double* __restrict__ grad)
{
    __shared__ double red[256];
    const int q = blockIdx.x;
    double acc = 0.0;
    for (int ch = threadIdx.x; ch < P; ch += blockDim.x) acc += g[ch] * J[(size_t)ch * Q + q];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[q] = red[0];
}

cudaError_t launch_adjoint_jacobian(const AdjCoef* coef_host, int Q, int K, int P, const double* sums, double* J,
                                    const double* g, double* grad, cudaStream_t st)
{
    AdjCoefs co;
    for (int q = 0; q < Q; ++q) co.c[q] = coef_host[q];
    const int n = P * Q, threads = 256;
    k_adjoint_jacobian<<<(n + threads - 1) / threads, threads, 0, st>>>(co, Q, K, P, sums, J);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !g) return e;
    k_adjoint_vjp<<<Q, 256, 0, st>>>(Q, P, J, g, grad);
    return cudaGetLastError();
}

}  // namespace lxo
