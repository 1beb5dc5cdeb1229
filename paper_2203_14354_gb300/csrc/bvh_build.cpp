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
        const double leaf_cost = (double)count;
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
                double cost = 1.0 + (acc.area() * c + right_area[k + 1] * rc) / std::max(b.area(), 1e-30);
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

int build_bvh(const float* tri_v, uint32_t nt, uint32_t leaf_size, uint32_t bins, uint32_t n_threads,
              float expand, BvhHost* out, char* err, size_t err_len)
{
    auto t0 = std::chrono::steady_clock::now();
    if (nt == 0 || nt >= (1u << 28)) {
        snprintf(err, err_len, "build_bvh: triangle count %u out of range [1, 2^28)", nt);
        return -1;
    }
    if (leaf_size == 0) leaf_size = 4;
    if (leaf_size > 8) leaf_size = 8;
    if (bins == 0) bins = 16;
    bins = std::min(std::max(bins, 4u), 64u);
    if (n_threads == 0) n_threads = std::max(1u, std::thread::hardware_concurrency());
    std::vector<Ref> refs(nt);
    for (uint32_t i = 0; i < nt; ++i) {
        Ref& r = refs[i];
        r.b.reset();
        for (int j = 0; j < 3; ++j) r.b.grow(&tri_v[9ull * i + 3 * j]);
        for (int a = 0; a < 3; ++a) r.c[a] = 0.5f * (r.b.lo[a] + r.b.hi[a]);
        r.id = i;
    }
    TmpNode* nodes = (TmpNode*)malloc(sizeof(TmpNode) * (2ull * nt + 1));
    if (!nodes) {
        snprintf(err, err_len, "build_bvh: out of host memory");
        return -1;
    }
    Builder B(refs, nodes, leaf_size, bins, (int)n_threads);
    uint32_t root = B.alloc();
    B.build(root, 0, nt, 0);
    const uint32_t n_tmp = B.n_nodes.load();
    // layout: depth-first, internal nodes only; a root leaf gets a one-leaf root node
    std::vector<uint32_t> gpu_index(n_tmp, 0xFFFFFFFFu);
    uint32_t n_internal = 0, n_leaves = 0;
    {
        std::vector<uint32_t> st{root};
        while (!st.empty()) {
            uint32_t i = st.back();
            st.pop_back();
            if (nodes[i].left < 0) { ++n_leaves; continue; }
            gpu_index[i] = n_internal++;
            st.push_back((uint32_t)nodes[i].right);
            st.push_back((uint32_t)nodes[i].left);
        }
    }
    const bool root_leaf = nodes[root].left < 0;
    if (root_leaf) n_internal = 1;
    out->n_nodes = n_internal;
    out->n_leaves = n_leaves;
    out->n_records = nt;
    out->max_depth = B.max_depth.load() + 1;
    out->nodes = (float4*)malloc(sizeof(float4) * 4ull * n_internal);
    out->tris = (float4*)malloc(sizeof(float4) * 3ull * nt);
    if (!out->nodes || !out->tris) {
        free(nodes);
        free_bvh(out);
        snprintf(err, err_len, "build_bvh: out of host memory");
        return -1;
    }
    // triangle records in leaf order (refs are already grouped by leaf)
    for (uint32_t k = 0; k < nt; ++k) {
        const float* v = &tri_v[9ull * refs[k].id];
        float4* r = &out->tris[3ull * k];
        uint32_t id = refs[k].id;
        float idf;
        memcpy(&idf, &id, 4);
        r[0] = make_float4(v[0], v[1], v[2], v[3]);
        r[1] = make_float4(v[4], v[5], v[6], v[7]);
        r[2] = make_float4(v[8], idf, 0.0f, 0.0f);
    }
    auto child_ref = [&](uint32_t c) -> int32_t {
        if (nodes[c].left >= 0) return (int32_t)gpu_index[c];
        uint32_t enc = (nodes[c].first << 3) | (nodes[c].count - 1);
        return ~(int32_t)enc;
    };
    auto put_box = [&](float4* f, int slot, const Box& b) {
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) { lo[a] = b.lo[a] - expand; hi[a] = b.hi[a] + expand; }
        for (int a = 0; a < 3; ++a) {
            if (slot == 0) { f[a].x = lo[a]; f[a].y = hi[a]; }
            else { f[a].z = lo[a]; f[a].w = hi[a]; }
        }
    };
    double sah = 0.0;
    const double root_area = std::max(nodes[root].b.area(), 1e-30);
    if (root_leaf) {
        float4* f = &out->nodes[0];
        memset(f, 0, 4 * sizeof(float4));
        put_box(f, 0, nodes[root].b);
        int32_t refs2[4] = {child_ref(root), kEmptyChild, 0, 0};
        memcpy(&f[3], refs2, 16);
        sah = nodes[root].count;
    } else {
        for (uint32_t i = 0; i < n_tmp; ++i) {
            if (nodes[i].left < 0) {
                sah += nodes[i].b.area() / root_area * nodes[i].count;
                continue;
            }
            sah += nodes[i].b.area() / root_area;
            float4* f = &out->nodes[4ull * gpu_index[i]];
            put_box(f, 0, nodes[nodes[i].left].b);
            put_box(f, 1, nodes[nodes[i].right].b);
            int32_t r4[4] = {child_ref((uint32_t)nodes[i].left), child_ref((uint32_t)nodes[i].right), 0, 0};
            memcpy(&f[3], r4, 16);
        }
    }
    free(nodes);
    out->sah_cost = sah;
    out->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return 0;
}

void free_bvh(BvhHost* b)
{
    free(b->nodes);
    free(b->tris);
    b->nodes = nullptr;
    b->tris = nullptr;
}

}  // namespace lxo
