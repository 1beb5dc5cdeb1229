// Host BVH builder: binned surface-area heuristic over triangle centroids
// (Wald, "On fast Construction of SAH-based Bounding Volume Hierarchies",
// IEEE RT 2007), parallel over subtrees with std::thread, then laid out for
// the GPU as 64-byte two-child nodes in depth-first order and 48-byte
// triangle records in leaf order.
//
// The triangle test on the device is exact (float32 watertight); the boxes
// only cull, so every box is widened by an absolute margin larger than the
// float rounding of the slab test: the traversal never drops a triangle the
// brute-force argmin would return.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "lxo_internal.h"

namespace lxo {
namespace {

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    }
    void grow(const Box& b) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
    }
    void grow(const float* p) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
    }
    double area() const {
        double dx = std::max(0.0f, hi[0] - lo[0]), dy = std::max(0.0f, hi[1] - lo[1]),
               dz = std::max(0.0f, hi[2] - lo[2]);
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Ref {
    Box b;
    float c[3];
    uint32_t id;
};

struct TmpNode {
    Box b;
    int32_t left, right;    // -1 for a leaf
    uint32_t first, count;
    uint32_t depth;
};

// surface-area heuristic: cost of a triangle test relative to a node visit
#ifndef LXO_SAH_CI
#define LXO_SAH_CI 1.0
#endif
constexpr double kSahTriCost = LXO_SAH_CI;

struct Builder {
    std::vector<Ref>& refs;
    TmpNode* nodes;
    std::atomic<uint32_t> n_nodes{0};
    std::atomic<int> threads_free;
    uint32_t leaf_size, bins;
    std::atomic<uint32_t> max_depth{0};

    Builder(std::vector<Ref>& r, TmpNode* n, uint32_t ls, uint32_t nb, int nthreads)
        : refs(r), nodes(n), threads_free(nthreads - 1), leaf_size(ls), bins(nb) {}

    uint32_t alloc() { return n_nodes.fetch_add(1); }

    void make_leaf(uint32_t idx, uint32_t first, uint32_t count) {
        nodes[idx].left = nodes[idx].right = -1;
        nodes[idx].first = first;
        nodes[idx].count = count;
    }

    // builds the subtree of refs[first, first+count) into node idx
    void build(uint32_t idx, uint32_t first, uint32_t count, uint32_t depth) {
        Box b, cb;
        b.reset();
        cb.reset();
        for (uint32_t i = first; i < first + count; ++i) {
            b.grow(refs[i].b);
            cb.grow(refs[i].c);
        }
        nodes[idx].b = b;
        nodes[idx].depth = depth;
        uint32_t md = max_depth.load();
        while (depth > md && !max_depth.compare_exchange_weak(md, depth)) {}
        if (count == 1) {
            make_leaf(idx, first, count);
            return;
        }
        // binned SAH over the three axes
        int best_axis = -1;
        uint32_t best_split = 0;
        double best_cost = INFINITY;
        const double leaf_cost = kSahTriCost * (double)count;
        uint32_t cnt[64], right_cnt[64];
        Box bb[64];
        double right_area[64];
        for (int a = 0; a < 3; ++a) {
            float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.0f)) continue;
            double scale = (double)bins / (double)ext;
            for (uint32_t k = 0; k < bins; ++k) { cnt[k] = 0; bb[k].reset(); }
            for (uint32_t i = first; i < first + count; ++i) {
                int k = (int)(((double)refs[i].c[a] - cb.lo[a]) * scale);
                k = std::min(std::max(k, 0), (int)bins - 1);
                cnt[k]++;
                bb[k].grow(refs[i].b);
            }
            Box acc;
            acc.reset();
            uint32_t c = 0;
            for (int k = (int)bins - 1; k >= 1; --k) {
                acc.grow(bb[k]);
                c += cnt[k];
                right_area[k] = acc.area();
                right_cnt[k] = c;
            }
            acc.reset();
            c = 0;
            for (uint32_t k = 0; k + 1 < bins; ++k) {
                acc.grow(bb[k]);
                c += cnt[k];
                uint32_t rc = right_cnt[k + 1];
                if (c == 0 || rc == 0) continue;
                double cost = 1.0 + kSahTriCost * (acc.area() * c + right_area[k + 1] * rc) / std::max(b.area(), 1e-30);
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_split = k + 1;
                }
            }
        }
        const bool too_deep = depth + 28 >= (uint32_t)kMaxDepth;
        if (best_axis < 0 || too_deep) {
            if (count <= leaf_size) {
                make_leaf(idx, first, count);
                return;
            }
            // no usable split plane (coincident centroids) or deep: median split by index
            uint32_t half = count / 2;
            int a = 0;
            for (int k = 1; k < 3; ++k)
                if (cb.hi[k] - cb.lo[k] > cb.hi[a] - cb.lo[a]) a = k;
            std::nth_element(refs.begin() + first, refs.begin() + first + half, refs.begin() + first + count,
                             [a](const Ref& x, const Ref& y) { return x.c[a] < y.c[a] || (x.c[a] == y.c[a] && x.id < y.id); });
            split_children(idx, first, half, count, depth);
            return;
        }
        if (count <= leaf_size && best_cost >= leaf_cost) {
            make_leaf(idx, first, count);
            return;
        }
        const int a = best_axis;
        const double scale = (double)bins / (double)(cb.hi[a] - cb.lo[a]);
        const float lo = cb.lo[a];
        const uint32_t split = best_split;
        auto mid = std::partition(refs.begin() + first, refs.begin() + first + count, [&](const Ref& r) {
            int k = (int)(((double)r.c[a] - lo) * scale);
            k = std::min(std::max(k, 0), (int)bins - 1);
            return (uint32_t)k < split;
        });
        uint32_t nl = (uint32_t)(mid - (refs.begin() + first));
        if (nl == 0 || nl == count) nl = count / 2;
        split_children(idx, first, nl, count, depth);
    }

    void split_children(uint32_t idx, uint32_t first, uint32_t nl, uint32_t count, uint32_t depth) {
        uint32_t l = alloc(), r = alloc();
        nodes[idx].left = (int32_t)l;
        nodes[idx].right = (int32_t)r;
        nodes[idx].first = 0;
        nodes[idx].count = 0;
        const uint32_t big = 1u << 16;
        if (count > big && threads_free.fetch_sub(1) > 0) {
            std::thread t([=] { build(l, first, nl, depth + 1); });
            build(r, first + nl, count - nl, depth + 1);
            t.join();
            threads_free.fetch_add(1);
        } else {
            if (count > big) threads_free.fetch_add(1);
            build(l, first, nl, depth + 1);
            build(r, first + nl, count - nl, depth + 1);
        }
    }
};

}  // namespace

namespace {

// Bounding box of the part of triangle v (3 x 3 floats) inside box [lo, hi]:
// Sutherland-Hodgman clipping in double against the six planes, the result
// rounded outwards to float.  Returns false if nothing is inside.
bool clipped_box(const float* v, const double lo[3], const double hi[3], Box& out)
{
    double poly[2][12][3];
    int n = 3, cur = 0;
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) poly[0][k][a] = v[3 * k + a];
    for (int a = 0; a < 3 && n; ++a) {
        for (int side = 0; side < 2 && n; ++side) {
            const double bound = side ? hi[a] : lo[a];
            const double sgn = side ? -1.0 : 1.0;  // inside: sgn * (x - bound) >= 0
            int m = 0;
            for (int k = 0; k < n; ++k) {
                const double* P = poly[cur][k];
                const double* Q = poly[cur][(k + 1) % n];
                const double dp = sgn * (P[a] - bound), dq = sgn * (Q[a] - bound);
                if (dp >= 0) {
                    for (int b = 0; b < 3; ++b) poly[cur ^ 1][m][b] = P[b];
                    ++m;
                }
                if ((dp >= 0) != (dq >= 0)) {
                    const double t = dp / (dp - dq);
                    for (int b = 0; b < 3; ++b) poly[cur ^ 1][m][b] = P[b] + t * (Q[b] - P[b]);
                    poly[cur ^ 1][m][a] = bound;
                    ++m;
                }
            }
            n = m;
            cur ^= 1;
        }
    }
    if (n == 0) return false;
    double blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            blo[a] = std::min(blo[a], poly[cur][k][a]);
            bhi[a] = std::max(bhi[a], poly[cur][k][a]);
        }
    for (int a = 0; a < 3; ++a) {
        out.lo[a] = std::nextafter((float)blo[a], -INFINITY);
        out.hi[a] = std::nextafter((float)bhi[a], INFINITY);
    }
    return true;
}

// Early split clipping (Ernst & Greiner, RT 2007): a triangle whose box is
// longer than max_ext is given several references, splitting its box at the
// midpoint of the longest axis, each reference bounded by the clipped part of
// the triangle (the union of the reference boxes still contains the triangle).
void split_refs(const float* v, uint32_t id, const Box& b, float max_ext, int depth, std::vector<Ref>& out)
{
    int a = 0;
    for (int k = 1; k < 3; ++k)
        if (b.hi[k] - b.lo[k] > b.hi[a] - b.lo[a]) a = k;
    if (b.hi[a] - b.lo[a] <= max_ext || depth >= 12) {
        Ref r;
        r.b = b;
        for (int k = 0; k < 3; ++k) r.c[k] = 0.5f * (b.lo[k] + b.hi[k]);
        r.id = id;
        out.push_back(r);
        return;
    }
    const double mid = 0.5 * ((double)b.lo[a] + (double)b.hi[a]);
    for (int half = 0; half < 2; ++half) {
        double lo[3], hi[3];
        for (int k = 0; k < 3; ++k) { lo[k] = b.lo[k]; hi[k] = b.hi[k]; }
        if (half == 0) hi[a] = mid; else lo[a] = mid;
        Box cb;
        if (!clipped_box(v, lo, hi, cb)) continue;
        for (int k = 0; k < 3; ++k) {  // never larger than the parent
            cb.lo[k] = std::max(cb.lo[k], b.lo[k]);
            cb.hi[k] = std::min(cb.hi[k], b.hi[k]);
        }
        split_refs(v, id, cb, max_ext, depth + 1, out);
    }
}

}  // namespace

namespace {

// kd top of a planar cluster: halves the cell rectangle [i0,i1) x [j0,j1)
// along its longer side down to single cells; returns the tmp node of the
// subtree or -1 if it holds no triangle.
int32_t kd_top(Builder& B, const std::vector<int32_t>& cell_root, int nu, int i0, int i1, int j0, int j1)
{
    if (i1 - i0 == 1 && j1 - j0 == 1) return cell_root[(size_t)j0 * nu + i0];
    int32_t l, r;
    if (i1 - i0 >= j1 - j0) {
        const int m = (i0 + i1) / 2;
        l = kd_top(B, cell_root, nu, i0, m, j0, j1);
        r = kd_top(B, cell_root, nu, m, i1, j0, j1);
    } else {
        const int m = (j0 + j1) / 2;
        l = kd_top(B, cell_root, nu, i0, i1, j0, m);
        r = kd_top(B, cell_root, nu, i0, i1, m, j1);
    }
    if (l < 0) return r;
    if (r < 0) return l;
    const uint32_t idx = B.alloc();
    TmpNode& nd = B.nodes[idx];
    nd.b = B.nodes[l].b;
    nd.b.grow(B.nodes[r].b);
    nd.left = l;
    nd.right = r;
    nd.first = nd.count = 0;
    nd.depth = 0;
    return (int32_t)idx;
}

Ref make_ref(const float* tri_v, uint32_t id)
{
    Ref r;
    r.b.reset();
    for (int j = 0; j < 3; ++j) r.b.grow(&tri_v[9ull * id + 3 * j]);
    for (int a = 0; a < 3; ++a) r.c[a] = 0.5f * (r.b.lo[a] + r.b.hi[a]);
    r.id = id;
    return r;
}

}  // namespace

int build_bvh(const float* tri_v, uint32_t nt, const int32_t* cluster_of, int n_clusters, uint32_t leaf_size,
              uint32_t bins, uint32_t n_threads, float expand, BvhHost* out, char* err, size_t err_len)
{
    auto t0 = std::chrono::steady_clock::now();
    if (nt == 0 || nt >= (1u << 28)) {
        snprintf(err, err_len, "build_bvh: triangle count %u out of range [1, 2^28)", nt);
        return -1;
    }
    if (n_clusters < 0 || n_clusters > kMaxClusters || (n_clusters > 0 && !cluster_of)) {
        snprintf(err, err_len, "build_bvh: %d clusters (max %d)", n_clusters, kMaxClusters);
        return -1;
    }
    if (leaf_size == 0) leaf_size = 4;
    if (leaf_size > 8) leaf_size = 8;
    if (bins == 0) bins = 16;
    bins = std::min(std::max(bins, 4u), 64u);
    if (n_threads == 0) n_threads = std::max(1u, std::thread::hardware_concurrency());

    // ---- planar clusters: slab, grid, triangle -> cells ----------------------
    struct Cl {
        Box b;
        uint32_t n = 0;
        int axis = 2, u = 0, v = 1, nu = 1, nv = 1;
        double cell = 1.0;
        std::vector<uint32_t> cell_count, cell_first;
    };
    std::vector<Cl> cl(n_clusters);
    std::vector<uint8_t> in_main(nt, 1);
    for (uint32_t i = 0; i < nt && n_clusters; ++i) {
        const int c = cluster_of[i];
        if (c < 0) continue;
        if (c >= n_clusters) {
            snprintf(err, err_len, "build_bvh: triangle %u in cluster %d >= %d", i, c, n_clusters);
            return -1;
        }
        if (cl[c].n == 0) cl[c].b.reset();
        for (int j = 0; j < 3; ++j) cl[c].b.grow(&tri_v[9ull * i + 3 * j]);
        cl[c].n++;
    }
    for (int c = 0; c < n_clusters; ++c) {
        Cl& k = cl[c];
        if (k.n == 0) continue;
        float ext[3];
        for (int a = 0; a < 3; ++a) ext[a] = k.b.hi[a] - k.b.lo[a];
        k.axis = (ext[0] <= ext[1] && ext[0] <= ext[2]) ? 0 : (ext[1] <= ext[2] ? 1 : 2);
        k.u = (k.axis + 1) % 3;
        k.v = (k.axis + 2) % 3;
        const double area = std::max(1e-6, (double)ext[k.u] * ext[k.v]);
        k.cell = std::max((double)expand * 64.0, std::sqrt(area / std::max(1.0, k.n / 16.0)));
        k.nu = std::max(1, (int)std::ceil((ext[k.u] + 2.0 * expand) / k.cell));
        k.nv = std::max(1, (int)std::ceil((ext[k.v] + 2.0 * expand) / k.cell));
        if ((double)k.nu * k.nv > 16e6) {
            k.cell *= std::sqrt((double)k.nu * k.nv / 16e6);
            k.nu = std::max(1, (int)std::ceil((ext[k.u] + 2.0 * expand) / k.cell));
            k.nv = std::max(1, (int)std::ceil((ext[k.v] + 2.0 * expand) / k.cell));
        }
        k.cell_count.assign((size_t)k.nu * k.nv, 0);
    }
    // cell range of a triangle's box (widened); big triangles stay in the main tree
    auto cell_range = [&](const Cl& k, const Box& b, int& i0, int& i1, int& j0, int& j1) {
        const double ou = (double)k.b.lo[k.u] - expand, ov = (double)k.b.lo[k.v] - expand;
        i0 = std::max(0, (int)std::floor(((double)b.lo[k.u] - expand - ou) / k.cell));
        i1 = std::min(k.nu - 1, (int)std::floor(((double)b.hi[k.u] + expand - ou) / k.cell));
        j0 = std::max(0, (int)std::floor(((double)b.lo[k.v] - expand - ov) / k.cell));
        j1 = std::min(k.nv - 1, (int)std::floor(((double)b.hi[k.v] + expand - ov) / k.cell));
    };
    uint64_t n_dup = 0;
    for (uint32_t i = 0; i < nt && n_clusters; ++i) {
        const int c = cluster_of[i];
        if (c < 0 || cl[c].n == 0) continue;
        Cl& k = cl[c];
        const Ref r = make_ref(tri_v, i);
        int i0, i1, j0, j1;
        cell_range(k, r.b, i0, i1, j0, j1);
        if ((int64_t)(i1 - i0 + 1) * (j1 - j0 + 1) > 64) continue;  // stays in the main tree
        in_main[i] = 0;
        for (int j = j0; j <= j1; ++j)
            for (int ii = i0; ii <= i1; ++ii) k.cell_count[(size_t)j * k.nu + ii]++;
        n_dup += (uint64_t)(i1 - i0 + 1) * (j1 - j0 + 1);
    }
    // main-tree references, big triangles split into clipped references
    float scene_ext = 0.0f;
    {
        Box sb;
        sb.reset();
        for (uint64_t k = 0; k < 3ull * nt; ++k) sb.grow(&tri_v[3 * k]);
        for (int a = 0; a < 3; ++a) scene_ext = std::max(scene_ext, sb.hi[a] - sb.lo[a]);
    }
#ifndef LXO_ESC_DIV
#define LXO_ESC_DIV 32.0f
#endif
    const float max_ext = LXO_ESC_DIV > 0.0f ? scene_ext / LXO_ESC_DIV : INFINITY;
    std::vector<Ref> main_refs;
    for (uint32_t i = 0; i < nt; ++i) {
        if (!in_main[i]) continue;
        const Ref r = make_ref(tri_v, i);
        float e = 0.0f;
        for (int a = 0; a < 3; ++a) e = std::max(e, r.b.hi[a] - r.b.lo[a]);
        if (e <= max_ext) main_refs.push_back(r);
        else split_refs(&tri_v[9ull * i], i, r.b, max_ext, 0, main_refs);
    }
    const uint64_t n_main = main_refs.size();
    const uint64_t n_refs = n_main + n_dup;
    if (n_refs >= (1ull << 28)) {
        snprintf(err, err_len, "build_bvh: %llu triangle records exceed 2^28", (unsigned long long)n_refs);
        return -1;
    }
    std::vector<Ref> refs(n_refs);
    {
        for (uint64_t k = 0; k < n_main; ++k) refs[k] = main_refs[k];
        std::vector<Ref>().swap(main_refs);
        uint64_t off = n_main;
        for (int c = 0; c < n_clusters; ++c) {
            Cl& kc = cl[c];
            kc.cell_first.assign(kc.cell_count.size(), 0);
            for (size_t q = 0; q < kc.cell_count.size(); ++q) {
                kc.cell_first[q] = (uint32_t)off;
                off += kc.cell_count[q];
            }
        }
        std::vector<std::vector<uint32_t>> fill(n_clusters);
        for (int c = 0; c < n_clusters; ++c) fill[c].assign(cl[c].cell_count.size(), 0);
        for (uint32_t i = 0; i < nt && n_clusters; ++i) {
            const int c = cluster_of[i];
            if (c < 0 || in_main[i]) continue;
            Cl& kc = cl[c];
            const Ref r = make_ref(tri_v, i);
            int i0, i1, j0, j1;
            cell_range(kc, r.b, i0, i1, j0, j1);
            const double ou = (double)kc.b.lo[kc.u] - expand, ov = (double)kc.b.lo[kc.v] - expand;
            for (int j = j0; j <= j1; ++j)
                for (int ii = i0; ii <= i1; ++ii) {
                    const size_t q = (size_t)j * kc.nu + ii;
                    // the reference's box is clipped to its cell (widened by the margin): a
                    // ray reaching this part of the triangle passes through this cell
                    Ref rc = r;
                    const float cu0 = (float)(ou + ii * kc.cell - expand), cu1 = (float)(ou + (ii + 1) * kc.cell + expand);
                    const float cv0 = (float)(ov + j * kc.cell - expand), cv1 = (float)(ov + (j + 1) * kc.cell + expand);
                    rc.b.lo[kc.u] = std::max(rc.b.lo[kc.u], cu0);
                    rc.b.hi[kc.u] = std::min(rc.b.hi[kc.u], cu1);
                    rc.b.lo[kc.v] = std::max(rc.b.lo[kc.v], cv0);
                    rc.b.hi[kc.v] = std::min(rc.b.hi[kc.v], cv1);
                    for (int a = 0; a < 3; ++a) rc.c[a] = 0.5f * (rc.b.lo[a] + rc.b.hi[a]);
                    refs[kc.cell_first[q] + fill[c][q]++] = rc;
                }
        }
    }

    // ---- trees ----------------------------------------------------------------
    TmpNode* nodes = (TmpNode*)malloc(sizeof(TmpNode) * (2ull * n_refs + 4ull * 16e6 + 8));
    if (!nodes) {
        snprintf(err, err_len, "build_bvh: out of host memory");
        return -1;
    }
    Builder B(refs, nodes, leaf_size, bins, (int)n_threads);
    int32_t main_tmp = -1;
    if (n_main) {
        main_tmp = (int32_t)B.alloc();
        B.build((uint32_t)main_tmp, 0, (uint32_t)n_main, 0);
    }
    std::vector<std::vector<int32_t>> cell_root(n_clusters);
    std::vector<int32_t> cl_root(n_clusters, -1);
    for (int c = 0; c < n_clusters; ++c) {
        Cl& kc = cl[c];
        if (kc.n == 0) continue;
        const size_t ncell = kc.cell_count.size();
        cell_root[c].assign(ncell, -1);
        std::atomic<size_t> next{0};
        auto work = [&]() {
            for (size_t q = next.fetch_add(1); q < ncell; q = next.fetch_add(1)) {
                if (!kc.cell_count[q]) continue;
                const uint32_t r = B.alloc();
                B.build(r, kc.cell_first[q], kc.cell_count[q], 0);
                cell_root[c][q] = (int32_t)r;
            }
        };
        std::vector<std::thread> th;
        for (uint32_t t = 1; t < n_threads; ++t) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        cl_root[c] = kd_top(B, cell_root[c], kc.nu, 0, kc.nu, 0, kc.nv);
    }
    const uint32_t n_tmp = B.n_nodes.load();

    // ---- layout: depth-first per tree, main tree first ------------------------
    std::vector<uint32_t> gpu_index(n_tmp, 0xFFFFFFFFu);
    uint32_t n_internal = 0, n_leaves = 0, max_depth = 0;
    auto dfs = [&](int32_t root) {
        if (root < 0) return;
        std::vector<std::pair<uint32_t, uint32_t>> st{{(uint32_t)root, 1u}};
        while (!st.empty()) {
            auto [i, d] = st.back();
            st.pop_back();
            max_depth = std::max(max_depth, d);
            if (nodes[i].left < 0) { ++n_leaves; continue; }
            gpu_index[i] = n_internal++;
            st.push_back({(uint32_t)nodes[i].right, d + 1});
            st.push_back({(uint32_t)nodes[i].left, d + 1});
        }
    };
    const bool main_leaf = main_tmp >= 0 && nodes[main_tmp].left < 0;
    uint32_t main_wrap = 0xFFFFFFFFu;
    if (main_leaf) main_wrap = n_internal++;  // a one-leaf root node wraps a leaf main tree
    dfs(main_tmp);
    for (int c = 0; c < n_clusters; ++c) dfs(cl_root[c]);
    out->n_nodes = std::max(1u, n_internal);
    out->n_leaves = n_leaves;
    out->n_records = (uint32_t)n_refs;
    out->max_depth = max_depth + 1;
    out->nodes = (float4*)calloc(4ull * out->n_nodes, sizeof(float4));
    out->tris = (float4*)malloc(sizeof(float4) * 3ull * n_refs);
    uint32_t n_cells = 0;
    for (int c = 0; c < n_clusters; ++c) n_cells += (uint32_t)cl[c].cell_count.size();
    out->cells = (int32_t*)malloc(sizeof(int32_t) * std::max(1u, n_cells));
    if (!out->nodes || !out->tris || !out->cells) {
        free(nodes);
        free_bvh(out);
        snprintf(err, err_len, "build_bvh: out of host memory");
        return -1;
    }
    for (uint64_t k = 0; k < n_refs; ++k) {
        const float* v = &tri_v[9ull * refs[k].id];
        float4* r = &out->tris[3ull * k];
        const uint32_t id = refs[k].id;
        float idf;
        memcpy(&idf, &id, 4);
        r[0] = make_float4(v[0], v[1], v[2], v[3]);
        r[1] = make_float4(v[4], v[5], v[6], v[7]);
        r[2] = make_float4(v[8], idf, 0.0f, 0.0f);
    }
    auto child_ref = [&](int32_t c) -> int32_t {
        if (c < 0) return kEmptyChild;
        if (nodes[c].left >= 0) return (int32_t)gpu_index[c];
        const uint32_t enc = (nodes[c].first << 3) | (nodes[c].count - 1);
        return ~(int32_t)enc;
    };
    auto put_box = [&](float4* f, int slot, const Box& b) {
        for (int a = 0; a < 3; ++a) {
            const float lo = b.lo[a] - expand, hi = b.hi[a] + expand;
            if (slot == 0) { f[a].x = lo; f[a].y = hi; }
            else { f[a].z = lo; f[a].w = hi; }
        }
    };
    double sah = 0.0;
    const double root_area = main_tmp >= 0 ? std::max(nodes[main_tmp].b.area(), 1e-30) : 1.0;
    for (uint32_t i = 0; i < n_tmp; ++i) {
        if (gpu_index[i] == 0xFFFFFFFFu) continue;
        sah += nodes[i].b.area() / root_area;
        float4* f = &out->nodes[4ull * gpu_index[i]];
        put_box(f, 0, nodes[nodes[i].left].b);
        put_box(f, 1, nodes[nodes[i].right].b);
        int32_t r4[4] = {child_ref(nodes[i].left), child_ref(nodes[i].right), 0, 0};
        memcpy(&f[3], r4, 16);
    }
    if (main_leaf) {
        float4* f = &out->nodes[4ull * main_wrap];
        // a one-leaf tree: the leaf in both slots, so the traversal never has
        // to test for a missing child (the leaf is tested twice, the second
        // test finding nothing closer)
        put_box(f, 0, nodes[main_tmp].b);
        put_box(f, 1, nodes[main_tmp].b);
        int32_t r4[4] = {child_ref(main_tmp), child_ref(main_tmp), 0, 0};
        memcpy(&f[3], r4, 16);
    }
    out->main_root = main_tmp < 0 ? kEmptyChild : (main_leaf ? (int32_t)main_wrap : child_ref(main_tmp));
    out->n_clusters = 0;
    uint32_t cell_off = 0;
    for (int c = 0; c < n_clusters; ++c) {
        const Cl& kc = cl[c];
        if (kc.n == 0 || cl_root[c] < 0) continue;
        ClusterHost& h = out->clusters[out->n_clusters++];
        h.axis = kc.axis;
        h.slab_lo = kc.b.lo[kc.axis] - expand;
        h.slab_hi = kc.b.hi[kc.axis] + expand;
        h.u0 = (float)((double)kc.b.lo[kc.u] - expand);
        h.v0 = (float)((double)kc.b.lo[kc.v] - expand);
        h.inv_cell = (float)(1.0 / kc.cell);
        h.nu = kc.nu;
        h.nv = kc.nv;
        h.root = child_ref(cl_root[c]);
        h.cells_offset = cell_off;
        for (size_t q = 0; q < kc.cell_count.size(); ++q) out->cells[cell_off + q] = child_ref(cell_root[c][q]);
        cell_off += (uint32_t)kc.cell_count.size();
    }
    out->n_cells = cell_off;
    free(nodes);
    out->sah_cost = sah;
    out->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return 0;
}

int detect_layers(const float* tri_v, uint32_t nt, int32_t* cluster_of)
{
    for (uint32_t i = 0; i < nt; ++i) cluster_of[i] = -1;
    Box sb;
    sb.reset();
    for (uint64_t k = 0; k < 3ull * nt; ++k) sb.grow(&tri_v[3 * k]);
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, sb.hi[a] - sb.lo[a]);
    const float thin = 0.004f * ext, wide = 0.01f * ext, tol = 3.0f;
    struct Grp { uint32_t n; int axis; std::vector<uint32_t> ids; };
    std::vector<Grp> groups;
    for (int axis : {2, 0, 1}) {
        std::vector<std::pair<float, uint32_t>> small;  // (lo, id)
        for (uint32_t i = 0; i < nt; ++i) {
            if (cluster_of[i] >= 0) continue;
            float lo = INFINITY, hi = -INFINITY;
            for (int j = 0; j < 3; ++j) {
                lo = std::min(lo, tri_v[9ull * i + 3 * j + axis]);
                hi = std::max(hi, tri_v[9ull * i + 3 * j + axis]);
            }
            if (hi - lo <= thin) small.push_back({lo, i});
        }
        std::sort(small.begin(), small.end());
        size_t g0 = 0;
        float glo = 0.0f, ghi = -INFINITY;
        auto close = [&](size_t g1) {
            if (g1 - g0 >= 32768 && ghi - glo <= wide) {
                Grp g{(uint32_t)(g1 - g0), axis, {}};
                for (size_t k = g0; k < g1; ++k) g.ids.push_back(small[k].second);
                groups.push_back(std::move(g));
            }
        };
        for (size_t k = 0; k < small.size(); ++k) {
            const uint32_t i = small[k].second;
            float hi = -INFINITY;
            for (int j = 0; j < 3; ++j) hi = std::max(hi, tri_v[9ull * i + 3 * j + axis]);
            if (k == 0 || small[k].first > ghi + tol) {
                if (k) close(k);
                g0 = k;
                glo = small[k].first;
                ghi = hi;
            } else {
                ghi = std::max(ghi, hi);
            }
        }
        if (!small.empty()) close(small.size());
        // mark this axis' groups so other axes do not take their triangles
        for (auto& g : groups)
            if (g.axis == axis)
                for (uint32_t id : g.ids) cluster_of[id] = 0;
    }
    for (uint32_t i = 0; i < nt; ++i) cluster_of[i] = -1;
    std::sort(groups.begin(), groups.end(), [](const Grp& x, const Grp& y) { return x.n > y.n; });
    const int n = std::min((int)groups.size(), kMaxClusters);
    for (int c = 0; c < n; ++c)
        for (uint32_t id : groups[c].ids) cluster_of[id] = c;
    return n;
}

void free_bvh(BvhHost* b)
{
    free(b->nodes);
    free(b->tris);
    free(b->cells);
    b->nodes = nullptr;
    b->tris = nullptr;
    b->cells = nullptr;
}

}  // namespace lxo
