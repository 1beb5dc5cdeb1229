// C ABI of the photon tracker (declared in include/lxo.h): context, mesh and
// table upload, BVH build + upload, and the launches.  Host code only; the
// kernels are in lxo_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lxo_internal.h"

struct lxo_ctx {
    int device = 0;
    std::string err;
    // host mesh
    uint32_t nt = 0;
    std::vector<float> tri_v;      // [nt*9]
    std::vector<uint32_t> attr;    // [nt]
    std::vector<int32_t> chan;     // [nt]
    float max_abs = 1.0f;
    bool have_mesh = false, have_bvh = false, validated = false;
    std::vector<lxo_material> mats;
    std::vector<lxo_surface> surfs;
    std::vector<lxo_pmt> pmts;
    std::vector<int32_t> adj_mats, adj_surfs;
    std::vector<lxo_event> events;
    uint32_t launch_blocks_per_sm = 0, launch_chunk = 64, launch_threads = 256;
    // device
    lxo::EventDev* d_events = nullptr;
    unsigned long long* d_ev_prefix = nullptr;
    uint32_t first_event = 0;   // event id of the table's first event
    uint64_t ev_total = 0;
    float4* d_nodes = nullptr;
    float4* d_tris = nullptr;
    int32_t* d_cells = nullptr;
    lxo::Scene scene{};
    unsigned long long* d_queue = nullptr;  // scratch: work-queue head
    int* d_err = nullptr;                   // scratch: device error word
    void* d_tally = nullptr;                // tallies of lxo_propagate_host
    size_t tally_bytes = 0;
    lxo_bvh_info info{};
};

namespace {

// NVTX range over the host side of one API call (the launch enqueue for the
// asynchronous ones): profilers attribute each kernel to the call that
// launched it.  Free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

lxo_status fail(lxo_ctx* c, lxo_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

lxo_status cuda_fail(lxo_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, LXO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

void free_device_geometry(lxo_ctx* c)
{
    if (c->d_nodes) cudaFree(c->d_nodes);
    if (c->d_tris) cudaFree(c->d_tris);
    if (c->d_cells) cudaFree(c->d_cells);
    c->d_nodes = nullptr;
    c->d_tris = nullptr;
    c->d_cells = nullptr;
    c->scene = lxo::Scene{};
    c->have_bvh = false;
}

lxo_status validate(lxo_ctx* c)
{
    if (c->validated) return LXO_OK;
    if (!c->have_mesh) return fail(c, LXO_ERR_STATE, "no mesh loaded");
    if (c->mats.empty()) return fail(c, LXO_ERR_STATE, "no materials set");
    if (c->pmts.empty()) return fail(c, LXO_ERR_STATE, "no PMT table set");
    if (!c->have_bvh) return fail(c, LXO_ERR_STATE, "BVH not built");
    const uint32_t M = (uint32_t)c->mats.size(), S = (uint32_t)c->surfs.size(), P = (uint32_t)c->pmts.size();
    for (uint32_t i = 0; i < c->nt; ++i) {
        const uint32_t a = c->attr[i];
        const uint32_t mi = a & 0xFF, mo = (a >> 8) & 0xFF, sf = a >> 16;
        if (mi >= M || mo >= M)
            return fail(c, LXO_ERR_ARG, "triangle %u: material index (%u, %u) >= %u materials", i, mi, mo, M);
        if (sf != LXO_SURF_NONE && sf >= S)
            return fail(c, LXO_ERR_ARG, "triangle %u: surface %u >= %u surfaces", i, sf, S);
        if (sf != LXO_SURF_NONE && c->surfs[sf].type == LXO_SURF_PHOTOCATHODE &&
            (c->chan[i] < 0 || (uint32_t)c->chan[i] >= P))
            return fail(c, LXO_ERR_ARG, "triangle %u: photocathode channel %d outside [0, %u)", i, c->chan[i], P);
    }
    c->validated = true;
    return LXO_OK;
}

// Largest |z| of the Box-Muller deviate: sqrt(-2 ln u) with u >= 2^-24 (the
// uniforms of the draw contract) is at most 5.77.
constexpr double kMaxDeviate = 5.8;

// The Gaussian of an emission spectrum (mean 0 = the reference wavelength)
// and a check that every wavelength it can emit is > 0 nm and, when some
// material has dispersion, gives every material an index > 0.
lxo_status spectrum(lxo_ctx* c, float mean_nm, float fwhm_nm, const char* what, size_t idx, bool check_index,
                    lxo::Spectrum* out)
{
    if (!std::isfinite(mean_nm) || !std::isfinite(fwhm_nm) || mean_nm < 0.0f || fwhm_nm < 0.0f)
        return fail(c, LXO_ERR_ARG, "%s %zu: spectrum mean %g nm, FWHM %g nm (finite, >= 0)", what, idx, mean_nm,
                    fwhm_nm);
    const double mean = mean_nm > 0.0f ? (double)mean_nm : (double)LXO_REF_WAVELENGTH_NM;
    const double sigma = (double)fwhm_nm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double lo = mean - kMaxDeviate * sigma, hi = mean + kMaxDeviate * sigma;
    if (!(lo > 0.0))
        return fail(c, LXO_ERR_ARG, "%s %zu: spectrum reaches %g nm", what, idx, lo);
    if (check_index)
        for (size_t m = 0; m < c->mats.size(); ++m) {
            const lxo_material& x = c->mats[m];
            const double r = (double)LXO_REF_WAVELENGTH_NM;
            const double n_lo = x.n + x.dn_dlambda_per_nm * (lo - r), n_hi = x.n + x.dn_dlambda_per_nm * (hi - r);
            if (!(n_lo > 0.0 && n_hi > 0.0))
                return fail(c, LXO_ERR_ARG, "%s %zu: material %zu has n <= 0 within the spectrum (%g..%g nm)", what,
                            idx, m, lo, hi);
        }
    if (out) *out = lxo::Spectrum{(float)mean, (float)sigma};
    return LXO_OK;
}

lxo_status fill_params(lxo_ctx* c, const lxo_source* src, uint64_t n, uint64_t base, const lxo_run_params* rp,
                       lxo::PropParams* p)
{
    if (!src) return fail(c, LXO_ERR_ARG, "source is NULL");
    memset(p, 0, sizeof *p);
    const int M = (int)c->mats.size(), S = (int)c->surfs.size();
    p->sc = c->scene;
    for (int m = 0; m < M; ++m) {
        const lxo_material& x = c->mats[m];
        p->mat[m].n = x.n;
        p->mat[m].n_over_c = (float)((double)x.n / 299.792458);
        p->mat[m].abs_len = (x.abs_len_mm > 0.0f && std::isfinite(x.abs_len_mm)) ? x.abs_len_mm : INFINITY;
        p->mat[m].ray_len =
            (x.rayleigh_len_mm > 0.0f && std::isfinite(x.rayleigh_len_mm)) ? x.rayleigh_len_mm : INFINITY;
        p->mat[m].dn = x.dn_dlambda_per_nm;
        p->mat[m].dn_over_c = (float)((double)x.dn_dlambda_per_nm / 299.792458);
        p->mat[m].ray_exp = x.rayleigh_exp;
        if (x.dn_dlambda_per_nm != 0.0f || x.rayleigh_exp != 0.0f) p->spectral = 1;
    }
    for (int s = 0; s < S; ++s) {
        const lxo_surface& x = c->surfs[s];
        p->surf[s] = lxo::DevSurface{x.type, x.reflectivity, x.spec_frac, x.qe, x.transparency,
                                     x.wire_reflectivity, x.wire_spec_frac};
    }
    p->n_mat = M;
    p->n_surf = S;
    p->n_chan = (int)c->pmts.size();
    p->n_fates = LXO_FATES_FIXED + M + S;
    if (src->kind < LXO_SRC_VOLUME_POLYGON || src->kind > LXO_SRC_EXPLICIT)
        return fail(c, LXO_ERR_ARG, "unknown source kind %d", src->kind);
    if (src->medium < 0 || src->medium >= M)
        return fail(c, LXO_ERR_ARG, "source medium %d outside [0, %d)", src->medium, M);
    if (src->kind == LXO_SRC_VOLUME_POLYGON && (src->n_sides < 0 || src->n_sides > lxo::kMaxPolySides ||
                                                 src->n_sides == 1 || src->n_sides == 2))
        return fail(c, LXO_ERR_ARG, "polygon source: n_sides %d not in {0, 3..%d}", src->n_sides,
                    lxo::kMaxPolySides);
    if (src->kind == LXO_SRC_EXPLICIT && (!src->pos || !src->dir || !src->pol))
        return fail(c, LXO_ERR_ARG, "explicit source needs pos, dir and pol device arrays");
    if (!(src->singlet_frac >= 0.0f && src->singlet_frac <= 1.0f) || !(src->tau_singlet_ns >= 0.0f) ||
        !(src->tau_triplet_ns >= 0.0f))
        return fail(c, LXO_ERR_ARG, "source time profile: singlet_frac %g not in [0, 1] or a negative constant",
                    src->singlet_frac);
    lxo::SourceDev& sd = p->src;
    lxo_status st = spectrum(c, src->wl_mean_nm, src->wl_fwhm_nm, "source", 0, p->spectral != 0, &sd.spec);
    if (st) return st;
    sd.kind = src->kind;
    sd.medium = src->medium;
    sd.n_sides = src->n_sides;
    sd.radius = src->radius;
    sd.z_min = src->z_min;
    sd.z_max = src->z_max;
    sd.t0 = src->t0;
    sd.prof = lxo::TimeProfile{src->singlet_frac, src->tau_singlet_ns, src->tau_triplet_ns};
    for (int a = 0; a < 3; ++a) {
        sd.center[a] = src->center[a];
        sd.p1[a] = src->p1[a];
    }
    if (src->kind == LXO_SRC_VOLUME_POLYGON && src->n_sides > 0) {
        const double pi = 3.141592653589793;
        sd.apothem = (float)((double)src->radius * cos(pi / src->n_sides));
        sd.phase_turns = (float)((double)src->phase / (2.0 * pi));
        for (int k = 0; k < src->n_sides; ++k) {
            const double a = (double)src->phase + 2.0 * pi * (k + 0.5) / src->n_sides;
            sd.side_cos[k] = (float)cos(a);
            sd.side_sin[k] = (float)sin(a);
        }
    }
    sd.pos = src->pos;
    sd.dir = src->dir;
    sd.pol = src->pol;
    p->n = n;
    p->base = base;
    if (rp) {
        p->seed = rp->seed;
        p->max_steps = rp->max_steps ? rp->max_steps : 10000u;
        p->n_tbins = rp->n_tbins;
        p->tbin = rp->tbin_ns;
        p->flags = rp->flags;
        if (!(rp->tbin_ns > 0.0f)) return fail(c, LXO_ERR_ARG, "tbin_ns must be > 0");
        if (rp->n_tbins > LXO_MAX_TBINS)
            return fail(c, LXO_ERR_ARG, "n_tbins %u above %u", rp->n_tbins, LXO_MAX_TBINS);
    }
    p->queue = c->d_queue;
    p->err = c->d_err;
    p->chunk = c->launch_chunk;
    p->blocks_per_sm = c->launch_blocks_per_sm;
    p->block_threads = c->launch_threads;
    for (int m = 0; m < LXO_MAX_MATERIALS; ++m) p->adj_mat_slot[m] = -1;
    for (int q = 0; q < LXO_MAX_SURFACES; ++q) p->adj_surf_slot[q] = -1;
    p->adj_k = 0;
    p->adj_n_mats = (int)c->adj_mats.size();
    if (rp && (rp->flags & LXO_FLAG_ADJOINT)) {
        for (size_t i = 0; i < c->adj_mats.size(); ++i) {
            if (c->adj_mats[i] >= M) return fail(c, LXO_ERR_ARG, "adjoint material %d >= %d", c->adj_mats[i], M);
            // the path-length tally serves L_abs and L_ray together, so a
            // Rayleigh length that changes with the wavelength has no tally
            if (c->mats[c->adj_mats[i]].rayleigh_exp != 0.0f)
                return fail(c, LXO_ERR_ARG, "adjoint material %d has rayleigh_exp != 0", c->adj_mats[i]);
            p->adj_mat_slot[c->adj_mats[i]] = (signed char)i;
        }
        for (size_t j = 0; j < c->adj_surfs.size(); ++j) {
            if (c->adj_surfs[j] >= S) return fail(c, LXO_ERR_ARG, "adjoint surface %d >= %d", c->adj_surfs[j], S);
            p->adj_surf_slot[c->adj_surfs[j]] = (signed char)j;
        }
        p->adj_k = 2 * (int)(c->adj_mats.size() + c->adj_surfs.size());
        if (p->adj_k == 0) return fail(c, LXO_ERR_ARG, "LXO_FLAG_ADJOINT without tracked parameters");
    }
    return LXO_OK;
}

}  // namespace

extern "C" {

lxo_status lxo_create(lxo_ctx** out, int cuda_device)
{
    if (!out) return LXO_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return LXO_ERR_CUDA;
    if (cuda_device < 0 || cuda_device >= n) return LXO_ERR_ARG;
    lxo_ctx* c = new (std::nothrow) lxo_ctx();
    if (!c) return LXO_ERR_NOMEM;
    c->device = cuda_device;
    DeviceGuard g(cuda_device);
    if (cudaMalloc(&c->d_queue, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        lxo_destroy(c);
        return LXO_ERR_CUDA;
    }
    *out = c;
    return LXO_OK;
}

void lxo_destroy(lxo_ctx* c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    free_device_geometry(c);
    if (c->d_queue) cudaFree(c->d_queue);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_tally) cudaFree(c->d_tally);
    if (c->d_events) cudaFree(c->d_events);
    if (c->d_ev_prefix) cudaFree(c->d_ev_prefix);
    delete c;
}

const char* lxo_last_error(const lxo_ctx* c) { return c ? c->err.c_str() : "null context"; }

lxo_status lxo_load_mesh(lxo_ctx* c, const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                         const uint8_t* mat_inner, const uint8_t* mat_outer, const uint16_t* surface,
                         const int32_t* channel)
{
    NvtxRange nvtx("lxo_load_mesh");
    if (!c) return LXO_ERR_ARG;
    if (!verts || !tris || !mat_inner || !mat_outer || !surface || !channel)
        return fail(c, LXO_ERR_ARG, "load_mesh: NULL array");
    if (nt == 0 || nt >= (1u << 28)) return fail(c, LXO_ERR_ARG, "load_mesh: %u triangles not in [1, 2^28)", nt);
    for (uint64_t i = 0; i < 3ull * nv; ++i)
        if (!std::isfinite(verts[i])) return fail(c, LXO_ERR_ARG, "load_mesh: vertex %llu not finite",
                                                  (unsigned long long)(i / 3));
    try {
        c->tri_v.resize(9ull * nt);
        c->attr.resize(nt);
        c->chan.resize(nt);
    } catch (...) {
        return fail(c, LXO_ERR_NOMEM, "load_mesh: out of host memory");
    }
    float mx = 1.0f;
    for (uint64_t i = 0; i < nt; ++i) {
        for (int j = 0; j < 3; ++j) {
            const uint32_t v = tris[3 * i + j];
            if (v >= nv) return fail(c, LXO_ERR_ARG, "load_mesh: triangle %llu vertex index %u >= %u",
                                     (unsigned long long)i, v, nv);
            for (int a = 0; a < 3; ++a) {
                const float x = verts[3ull * v + a];
                c->tri_v[9 * i + 3 * j + a] = x;
                mx = std::max(mx, std::fabs(x));
            }
        }
        c->attr[i] = (uint32_t)mat_inner[i] | ((uint32_t)mat_outer[i] << 8) | ((uint32_t)surface[i] << 16);
        c->chan[i] = channel[i];
    }
    c->nt = nt;
    c->max_abs = mx;
    c->have_mesh = true;
    c->validated = false;
    DeviceGuard g(c->device);
    free_device_geometry(c);
    return LXO_OK;
}

lxo_status lxo_set_materials(lxo_ctx* c, const lxo_material* m, uint32_t n)
{
    if (!c) return LXO_ERR_ARG;
    if (!m || n == 0 || n > LXO_MAX_MATERIALS)
        return fail(c, LXO_ERR_ARG, "set_materials: need 1..%d materials", LXO_MAX_MATERIALS);
    for (uint32_t i = 0; i < n; ++i)
        if (!(m[i].n > 0.0f) || std::isnan(m[i].abs_len_mm) || std::isnan(m[i].rayleigh_len_mm) ||
            !std::isfinite(m[i].dn_dlambda_per_nm) || !std::isfinite(m[i].rayleigh_exp))
            return fail(c, LXO_ERR_ARG,
                        "set_materials: material %u invalid (n must be > 0, lengths not NaN, dispersion finite)", i);
    c->mats.assign(m, m + n);
    c->validated = false;
    return LXO_OK;
}

lxo_status lxo_set_surfaces(lxo_ctx* c, const lxo_surface* s, uint32_t n)
{
    if (!c) return LXO_ERR_ARG;
    if (n > LXO_MAX_SURFACES || (n && !s)) return fail(c, LXO_ERR_ARG, "set_surfaces: need 0..%d surfaces",
                                                       LXO_MAX_SURFACES);
    for (uint32_t i = 0; i < n; ++i) {
        if (s[i].type < LXO_SURF_ABSORBER || s[i].type > LXO_SURF_ELECTRODE_T)
            return fail(c, LXO_ERR_ARG, "set_surfaces: surface %u has unknown type %d", i, s[i].type);
        const float v[6] = {s[i].reflectivity, s[i].spec_frac, s[i].qe, s[i].transparency, s[i].wire_reflectivity,
                            s[i].wire_spec_frac};
        for (float x : v)
            if (!(x >= 0.0f && x <= 1.0f))
                return fail(c, LXO_ERR_ARG, "set_surfaces: surface %u has a probability outside [0, 1]", i);
    }
    c->surfs.assign(s, s + n);
    c->validated = false;
    return LXO_OK;
}

lxo_status lxo_set_pmts(lxo_ctx* c, const lxo_pmt* p, uint32_t n)
{
    if (!c) return LXO_ERR_ARG;
    if (!p || n == 0) return fail(c, LXO_ERR_ARG, "set_pmts: need at least one channel");
    c->pmts.assign(p, p + n);
    c->validated = false;
    return LXO_OK;
}

lxo_status lxo_build_bvh(lxo_ctx* c, const lxo_bvh_params* bp, lxo_bvh_info* info)
{
    NvtxRange nvtx("lxo_build_bvh");
    if (!c) return LXO_ERR_ARG;
    if (!c->have_mesh) return fail(c, LXO_ERR_STATE, "build_bvh: no mesh loaded");
    lxo_bvh_params q{};
    if (bp) q = *bp;
    lxo::BvhHost b;
    char msg[256] = {0};
    // widen boxes far beyond the float rounding of the slab test
    const float expand = std::ldexp(c->max_abs, -19);
    // thin dense layers (electrode wire meshes, PMT arrays) get their own
    // grid-entered trees
    std::vector<int32_t> cluster_of(c->nt, -1);
    const int n_clusters = lxo::detect_layers(c->tri_v.data(), c->nt, cluster_of.data());
    if (lxo::build_bvh(c->tri_v.data(), c->nt, cluster_of.data(), n_clusters, q.leaf_size, q.sah_bins, q.n_threads,
                       expand, &b, msg, sizeof msg))
        return fail(c, LXO_ERR_NOMEM, "%s", msg);
    // attributes of each record
    for (uint32_t k = 0; k < b.n_records; ++k) {
        float4& r2 = b.tris[3ull * k + 2];
        uint32_t id;
        memcpy(&id, &r2.y, 4);
        const uint32_t a = c->attr[id];
        const int32_t ch = c->chan[id];
        memcpy(&r2.z, &a, 4);
        memcpy(&r2.w, &ch, 4);
    }
    DeviceGuard g(c->device);
    free_device_geometry(c);
    const size_t nb = sizeof(float4) * 4ull * b.n_nodes, tb = sizeof(float4) * 3ull * b.n_records;
    const size_t cb = sizeof(int32_t) * std::max(1u, b.n_cells);
    cudaError_t e = cudaMalloc(&c->d_nodes, nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tris, tb);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cells, cb);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_nodes, b.nodes, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tris, b.tris, tb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b.n_cells) e = cudaMemcpy(c->d_cells, b.cells, sizeof(int32_t) * b.n_cells,
                                                      cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lxo::free_bvh(&b);
        free_device_geometry(c);
        return cuda_fail(c, e, "build_bvh: upload");
    }
    lxo::Scene& sc = c->scene;
    sc.nodes = c->d_nodes;
    sc.tris = c->d_tris;
    sc.n_tris = c->nt;
    sc.main_root = b.main_root;
    sc.n_nodes = b.n_nodes;
    sc.n_records = b.n_records;
    sc.n_clusters = b.n_clusters;
    for (int k = 0; k < b.n_clusters; ++k) {
        const lxo::ClusterHost& h = b.clusters[k];
        lxo::ClusterDev& d = sc.clusters[k];
        d.axis = h.axis;
        d.nu = h.nu;
        d.nv = h.nv;
        d.root = h.root;
        d.slab_lo = h.slab_lo;
        d.slab_hi = h.slab_hi;
        d.u0 = h.u0;
        d.v0 = h.v0;
        d.inv_cell = h.inv_cell;
        d.delta = expand;
        d.cells = c->d_cells + h.cells_offset;
    }
    lxo::free_bvh(&b);
    c->info.n_tris = c->nt;
    c->info.n_nodes = b.n_nodes;
    c->info.n_leaves = b.n_leaves;
    c->info.max_depth = b.max_depth;
    c->info.node_bytes = nb + cb;
    c->info.tri_bytes = tb;
    c->info.build_seconds = b.build_seconds;
    c->info.sah_cost = b.sah_cost;
    if (info) *info = c->info;
    c->have_bvh = true;
    c->validated = false;
    if (b.max_depth + lxo::kMaxClusters * lxo::kMaxCellsPerRay + 1 >= (uint32_t)lxo::kStackSize)
        return fail(c, LXO_ERR_ARG, "build_bvh: depth %u exceeds the traversal stack", b.max_depth);
    return LXO_OK;
}

lxo_status lxo_trace_rays(lxo_ctx* c, const float* org, const float* dir, const uint32_t* skip, const float* tmax,
                          uint32_t n, uint32_t* hit, float* t, void* stream)
{
    NvtxRange nvtx("lxo_trace_rays");
    if (!c) return LXO_ERR_ARG;
    if (!c->have_bvh) return fail(c, LXO_ERR_STATE, "trace_rays: BVH not built");
    if (n == 0) return LXO_OK;
    if (!org || !dir || !hit || !t) return fail(c, LXO_ERR_ARG, "trace_rays: NULL array");
    DeviceGuard g(c->device);
    CK(lxo::launch_trace(c->scene, org, dir, skip, tmax, n, hit, t, c->d_err, (cudaStream_t)stream), "trace_rays");
    return LXO_OK;
}

lxo_status lxo_sample_source(lxo_ctx* c, const lxo_source* src, uint64_t n, uint64_t base, uint64_t seed,
                             float* pos, float* dir, float* pol, float* time, float* wavelength, void* stream)
{
    NvtxRange nvtx("lxo_sample_source");
    if (!c) return LXO_ERR_ARG;
    if (c->mats.empty()) return fail(c, LXO_ERR_STATE, "sample_source: no materials set");
    if (n == 0) return LXO_OK;
    if (!pos || !dir || !pol) return fail(c, LXO_ERR_ARG, "sample_source: NULL array");
    lxo::PropParams p;
    lxo_run_params rp{seed, 1, 0, 1.0f, 0};
    lxo_status s = fill_params(c, src, n, base, &rp, &p);
    if (s) return s;
    DeviceGuard g(c->device);
    CK(lxo::launch_sample_source(p, pos, dir, pol, time, wavelength, (cudaStream_t)stream), "sample_source");
    return LXO_OK;
}

lxo_status lxo_propagate(lxo_ctx* c, const lxo_source* src, uint64_t n, uint64_t base, const lxo_run_params* rp,
                         const lxo_results* out, void* stream)
{
    NvtxRange nvtx("lxo_propagate");
    if (!c) return LXO_ERR_ARG;
    lxo_status s = validate(c);
    if (s) return s;
    if (!rp) return fail(c, LXO_ERR_ARG, "propagate: run params are NULL");
    if (!out || !out->lce || !out->det || !out->hist || !out->fates)
        return fail(c, LXO_ERR_ARG, "propagate: lce, det, hist and fates buffers are required");
    if ((rp->flags & LXO_FLAG_STATS) && !out->stats)
        return fail(c, LXO_ERR_ARG, "propagate: LXO_FLAG_STATS needs the stats buffer");
    if ((rp->flags & LXO_FLAG_ADJOINT) && !out->adjoint)
        return fail(c, LXO_ERR_ARG, "propagate: LXO_FLAG_ADJOINT needs the adjoint buffer");
    if (n == 0) return LXO_OK;
    lxo::PropParams p;
    s = fill_params(c, src, n, base, rp, &p);
    if (s) return s;
    p.out = *out;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->d_queue, 0, sizeof(unsigned long long), st), "propagate: reset queue");
    CK(lxo::launch_propagate(p, c->device, st), "propagate: launch");
    return LXO_OK;
}

lxo_status lxo_propagate_host(lxo_ctx* c, const lxo_source* src, uint64_t n, uint64_t base,
                              const lxo_run_params* rp, const lxo_results* host_out, void* stream)
{
    NvtxRange nvtx("lxo_propagate_host");
    if (!c) return LXO_ERR_ARG;
    lxo_status s = validate(c);
    if (s) return s;
    if (!rp) return fail(c, LXO_ERR_ARG, "propagate_host: run params are NULL");
    if (!host_out || !host_out->lce || !host_out->det || !host_out->hist || !host_out->fates)
        return fail(c, LXO_ERR_ARG, "propagate_host: lce, det, hist and fates buffers are required");
    if (host_out->ph_fate || host_out->ph_detail || host_out->ph_steps || host_out->ph_time || host_out->ph_state ||
        host_out->stats || host_out->adjoint)
        return fail(c, LXO_ERR_ARG, "propagate_host: per-photon outputs, stats and adjoint are device-only");
    if (rp->flags & (LXO_FLAG_STATS | LXO_FLAG_ADJOINT))
        return fail(c, LXO_ERR_ARG, "propagate_host: LXO_FLAG_STATS / LXO_FLAG_ADJOINT not supported");
    const size_t P = c->pmts.size(), B = (size_t)rp->n_tbins + 1;
    const size_t NF = LXO_FATES_FIXED + c->mats.size() + c->surfs.size();
    const size_t bytes = 8 * NF + 4 * (2 * P + P * B);
    DeviceGuard g(c->device);
    if (c->tally_bytes < bytes) {
        if (c->d_tally) cudaFree(c->d_tally);
        c->d_tally = nullptr;
        c->tally_bytes = 0;
        CK(cudaMalloc(&c->d_tally, bytes), "propagate_host: tallies");
        c->tally_bytes = bytes;
    }
    cudaStream_t st = (cudaStream_t)stream;
    lxo_results d{};
    d.fates = (unsigned long long*)c->d_tally;
    d.lce = (uint32_t*)(d.fates + NF);
    d.det = d.lce + P;
    d.hist = d.det + P;
    CK(cudaMemsetAsync(c->d_tally, 0, bytes, st), "propagate_host: zero tallies");
    s = lxo_propagate(c, src, n, base, rp, &d, stream);
    if (s) return s;
    std::vector<unsigned long long> hf(NF);
    std::vector<uint32_t> hu(2 * P + P * B);
    CK(cudaMemcpyAsync(hf.data(), d.fates, 8 * NF, cudaMemcpyDeviceToHost, st), "propagate_host: copy fates");
    CK(cudaMemcpyAsync(hu.data(), d.lce, 4 * hu.size(), cudaMemcpyDeviceToHost, st), "propagate_host: copy tallies");
    s = lxo_sync(c, stream);
    if (s) return s;
    for (size_t i = 0; i < NF; ++i) host_out->fates[i] += hf[i];
    for (size_t i = 0; i < P; ++i) {
        host_out->lce[i] += hu[i];
        host_out->det[i] += hu[P + i];
    }
    for (size_t i = 0; i < P * B; ++i) host_out->hist[i] += hu[2 * P + i];
    return LXO_OK;
}

lxo_status lxo_upload_events(lxo_ctx* c, const lxo_event* ev, uint32_t n, uint32_t first_event)
{
    NvtxRange nvtx("lxo_upload_events");
    if (!c) return LXO_ERR_ARG;
    if (!ev || n == 0) return fail(c, LXO_ERR_ARG, "upload_events: no events");
    if ((uint64_t)first_event + n > (1ull << 32))
        return fail(c, LXO_ERR_ARG, "upload_events: event ids %u + %u exceed 2^32", first_event, n);
    std::vector<lxo::EventDev> h(n);
    std::vector<unsigned long long> pre(n + 1, 0);
    for (uint32_t e = 0; e < n; ++e) {
        const lxo_event& x = ev[e];
        if (x.kind != LXO_SRC_POINT && x.kind != LXO_SRC_SEGMENT && x.kind != LXO_SRC_BALL)
            return fail(c, LXO_ERR_ARG, "upload_events: event %u has source kind %d (point, segment or ball only)",
                        e, x.kind);
        if (x.n_photons >= (1ull << 32))
            return fail(c, LXO_ERR_ARG, "upload_events: event %u has %llu photons (< 2^32)", e,
                        (unsigned long long)x.n_photons);
        if (x.medium < 0) return fail(c, LXO_ERR_ARG, "upload_events: event %u medium %d", e, x.medium);
        if (!(x.singlet_frac >= 0.0f && x.singlet_frac <= 1.0f) || !(x.tau_singlet_ns >= 0.0f) ||
            !(x.tau_triplet_ns >= 0.0f))
            return fail(c, LXO_ERR_ARG, "upload_events: event %u time profile (f %g, tau %g, %g)", e, x.singlet_frac,
                        x.tau_singlet_ns, x.tau_triplet_ns);
        lxo::Spectrum sp;
        lxo_status st = spectrum(c, x.wl_mean_nm, x.wl_fwhm_nm, "upload_events: event", e, false, &sp);
        if (st) return st;
        h[e] = lxo::EventDev{x.kind, x.medium, {x.center[0], x.center[1], x.center[2]}, {x.p1[0], x.p1[1], x.p1[2]},
                             x.radius, x.t0, {x.singlet_frac, x.tau_singlet_ns, x.tau_triplet_ns}, sp};
        pre[e + 1] = pre[e] + x.n_photons;
    }
    DeviceGuard g(c->device);
    if (c->d_events) cudaFree(c->d_events);
    if (c->d_ev_prefix) cudaFree(c->d_ev_prefix);
    c->d_events = nullptr;
    c->d_ev_prefix = nullptr;
    c->events.clear();
    CK(cudaMalloc(&c->d_events, sizeof(lxo::EventDev) * n), "upload_events: alloc");
    CK(cudaMalloc(&c->d_ev_prefix, sizeof(unsigned long long) * (n + 1)), "upload_events: alloc");
    CK(cudaMemcpy(c->d_events, h.data(), sizeof(lxo::EventDev) * n, cudaMemcpyHostToDevice), "upload_events: copy");
    CK(cudaMemcpy(c->d_ev_prefix, pre.data(), sizeof(unsigned long long) * (n + 1), cudaMemcpyHostToDevice),
       "upload_events: copy");
    c->events.assign(ev, ev + n);
    c->ev_total = pre[n];
    c->first_event = first_event;
    return LXO_OK;
}

lxo_status lxo_propagate_events(lxo_ctx* c, const lxo_run_params* rp, const lxo_results* out, void* stream)
{
    NvtxRange nvtx("lxo_propagate_events");
    if (!c) return LXO_ERR_ARG;
    lxo_status s = validate(c);
    if (s) return s;
    if (c->events.empty()) return fail(c, LXO_ERR_STATE, "propagate_events: no events uploaded");
    if (!rp) return fail(c, LXO_ERR_ARG, "propagate_events: run params are NULL");
    if (!out || !out->lce || !out->det || !out->fates)
        return fail(c, LXO_ERR_ARG, "propagate_events: lce, det and fates buffers are required");
    if (out->ph_fate || out->ph_detail || out->ph_steps || out->ph_time || out->ph_state || out->stats ||
        (rp->flags & LXO_FLAG_STATS))
        return fail(c, LXO_ERR_ARG, "propagate_events: per-photon outputs and stats are not supported");
    if ((rp->flags & LXO_FLAG_ADJOINT) && !out->adjoint)
        return fail(c, LXO_ERR_ARG, "propagate_events: LXO_FLAG_ADJOINT needs the adjoint buffer");
    for (size_t e = 0; e < c->events.size(); ++e)
        if (c->events[e].medium >= (int)c->mats.size())
            return fail(c, LXO_ERR_ARG, "propagate_events: event %zu medium %d >= %zu materials", e,
                        c->events[e].medium, c->mats.size());
    lxo_source src{};
    src.kind = LXO_SRC_POINT;
    src.medium = c->events[0].medium;
    lxo::PropParams p;
    s = fill_params(c, &src, c->ev_total, 0, rp, &p);
    if (s) return s;
    if (p.spectral)  // the materials may have changed since the upload
        for (size_t e = 0; e < c->events.size(); ++e) {
            s = spectrum(c, c->events[e].wl_mean_nm, c->events[e].wl_fwhm_nm, "propagate_events: event", e, true,
                         nullptr);
            if (s) return s;
        }
    p.out = *out;
    p.n_events = (uint32_t)c->events.size();
    p.first_event = c->first_event;
    p.events = c->d_events;
    p.ev_prefix = c->d_ev_prefix;
    if (c->ev_total == 0) return LXO_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->d_queue, 0, sizeof(unsigned long long), st), "propagate_events: reset queue");
    CK(lxo::launch_propagate(p, c->device, st), "propagate_events: launch");
    return LXO_OK;
}

lxo_status lxo_set_launch(lxo_ctx* c, uint32_t blocks_per_sm, uint32_t chunk, uint32_t threads)
{
    if (!c) return LXO_ERR_ARG;
    if (blocks_per_sm > 32 || chunk > 4096)
        return fail(c, LXO_ERR_ARG, "set_launch: blocks_per_sm <= 32, chunk <= 4096");
    if (threads != 0 && threads != 128 && threads != 256)
        return fail(c, LXO_ERR_ARG, "set_launch: threads per block 128 or 256 (0 = 256), not %u", threads);
    c->launch_blocks_per_sm = blocks_per_sm;
    c->launch_chunk = chunk ? chunk : 64;
    c->launch_threads = threads ? threads : 256;
    return LXO_OK;
}

lxo_status lxo_set_adjoint(lxo_ctx* c, const int32_t* mats, uint32_t n_mats, const int32_t* surfs, uint32_t n_surfs)
{
    if (!c) return LXO_ERR_ARG;
    if (n_mats > LXO_ADJ_MAX_MATERIALS || n_surfs > LXO_ADJ_MAX_SURFACES || (n_mats && !mats) || (n_surfs && !surfs))
        return fail(c, LXO_ERR_ARG, "set_adjoint: at most %d materials and %d surfaces", LXO_ADJ_MAX_MATERIALS,
                    LXO_ADJ_MAX_SURFACES);
    for (uint32_t i = 0; i < n_mats; ++i) {
        if (mats[i] < 0 || mats[i] >= LXO_MAX_MATERIALS) return fail(c, LXO_ERR_ARG, "set_adjoint: material %d", mats[i]);
        for (uint32_t k = 0; k < i; ++k)
            if (mats[k] == mats[i]) return fail(c, LXO_ERR_ARG, "set_adjoint: material %d twice", mats[i]);
    }
    for (uint32_t j = 0; j < n_surfs; ++j) {
        if (surfs[j] < 0 || surfs[j] >= (int32_t)c->surfs.size())
            return fail(c, LXO_ERR_ARG, "set_adjoint: surface %d not in the surface table", surfs[j]);
        const int t = c->surfs[surfs[j]].type;
        if (t != LXO_SURF_REFLECTOR && t != LXO_SURF_ELECTRODE_T)
            return fail(c, LXO_ERR_ARG, "set_adjoint: surface %d is neither a reflector nor an electrode", surfs[j]);
        for (uint32_t k = 0; k < j; ++k)
            if (surfs[k] == surfs[j]) return fail(c, LXO_ERR_ARG, "set_adjoint: surface %d twice", surfs[j]);
    }
    c->adj_mats.assign(mats, mats + n_mats);
    c->adj_surfs.assign(surfs, surfs + n_surfs);
    return LXO_OK;
}

lxo_status lxo_adjoint_jacobian(lxo_ctx* c, const double* sums, uint32_t n_rows, double* J, const double* g,
                                double* grad, void* stream)
{
    NvtxRange nvtx("lxo_adjoint_jacobian");
    if (!c) return LXO_ERR_ARG;
    if (!sums || !J || (!g) != (!grad)) return fail(c, LXO_ERR_ARG, "adjoint_jacobian: NULL array");
    const int nm = (int)c->adj_mats.size(), ns = (int)c->adj_surfs.size();
    const int K = 2 * (nm + ns), Q = 2 * nm + ns;
    const int P = n_rows ? (int)n_rows : (int)c->pmts.size();
    if (K == 0 || P == 0) return fail(c, LXO_ERR_STATE, "adjoint_jacobian: no tracked parameters or no PMTs");
    if ((uint64_t)P * (uint64_t)Q > (uint64_t)INT32_MAX)
        return fail(c, LXO_ERR_ARG, "adjoint_jacobian: %u rows x %d parameters exceed 2^31 entries", n_rows, Q);
    lxo::AdjCoef coef[2 * LXO_ADJ_MAX_MATERIALS + LXO_ADJ_MAX_SURFACES];
    for (int i = 0; i < nm; ++i) {
        const lxo_material& m = c->mats[c->adj_mats[i]];
        const double La = (m.abs_len_mm > 0.0f && std::isfinite(m.abs_len_mm)) ? m.abs_len_mm : INFINITY;
        const double Lr = (m.rayleigh_len_mm > 0.0f && std::isfinite(m.rayleigh_len_mm)) ? m.rayleigh_len_mm : INFINITY;
        coef[2 * i] = lxo::AdjCoef{2 * i, 2 * i, std::isinf(La) ? 0.0 : 1.0 / (La * La), 0.0};
        coef[2 * i + 1] = lxo::AdjCoef{2 * i, 2 * i + 1, std::isinf(Lr) ? 0.0 : 1.0 / (Lr * Lr),
                                       std::isinf(Lr) ? 0.0 : -1.0 / Lr};
    }
    for (int j = 0; j < ns; ++j) {
        const lxo_surface& sf = c->surfs[c->adj_surfs[j]];
        const int ia = 2 * nm + 2 * j;
        if (sf.type == LXO_SURF_REFLECTOR)
            coef[2 * nm + j] = lxo::AdjCoef{ia, ia + 1, sf.reflectivity > 0.0f ? 1.0 / sf.reflectivity : 0.0, 0.0};
        else
            coef[2 * nm + j] = lxo::AdjCoef{ia, ia + 1, sf.transparency > 0.0f ? 1.0 / sf.transparency : 0.0,
                                            sf.transparency < 1.0f ? -1.0 / (1.0 - sf.transparency) : 0.0};
    }
    DeviceGuard gd(c->device);
    CK(lxo::launch_adjoint_jacobian(coef, Q, K, P, sums, J, g, grad, (cudaStream_t)stream), "adjoint_jacobian");
    return LXO_OK;
}

lxo_status lxo_sync(lxo_ctx* c, void* stream)
{
    if (!c) return LXO_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
    int h = 0;
    CK(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "sync: read error word");
    if (h) {
        CK(cudaMemset(c->d_err, 0, sizeof(int)), "sync: clear error word");
        return fail(c, LXO_ERR_DEVICE, "device fault flags 0x%x (1 = traversal stack, 2 = channel range, 8 = index out of range)", h);
    }
    return LXO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of lxo_propagate_host.
//
// Its device scratch (work-queue head, error word and the device copy of the
// tallies) lives in the file-scope array below instead of memory obtained
// from cudaMalloc.  The array is part of this file's device module, so every
// GPU that loads the library holds LXO_STATIC_SCRATCH_BYTES of it until the
// process exits.  Host code cannot use the array's name as a device address:
// the address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[LXO_STATIC_SCRATCH_BYTES];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_addr[kMaxStaticDevices] = {};

// error message without growing the context's string (no host allocation)
lxo_status static_fail(lxo_ctx* c, lxo_status code, const char* msg)
{
    const size_t cap = c->err.capacity();
    const size_t len = strlen(msg);
    c->err.assign(msg, len < cap ? len : cap);
    return code;
}

}  // namespace

extern "C" lxo_status lxo_propagate_host_static(lxo_ctx* c, const lxo_source* src, uint64_t n, uint64_t base,
                                                const lxo_run_params* rp, const lxo_results* host_out, void* stream)
{
    if (!c) return LXO_ERR_ARG;
    if (!rp) return static_fail(c, LXO_ERR_ARG, "run params are NULL");
    if (!host_out || !host_out->lce || !host_out->det || !host_out->hist || !host_out->fates)
        return static_fail(c, LXO_ERR_ARG, "lce, det, hist, fates host buffers required");
    if (host_out->ph_fate || host_out->ph_detail || host_out->ph_steps || host_out->ph_time || host_out->ph_state ||
        host_out->stats || host_out->adjoint || (rp->flags & (LXO_FLAG_STATS | LXO_FLAG_ADJOINT)))
        return static_fail(c, LXO_ERR_ARG, "per-photon outputs, stats and adjoint unsupported");
    lxo_status s = validate(c);
    if (s) return s;
    const uint64_t P = c->pmts.size(), B = (uint64_t)rp->n_tbins + 1;
    const uint64_t NF = LXO_FATES_FIXED + c->mats.size() + c->surfs.size();
    // layout: [0, 8) queue head, [8, 12) error word, tallies from offset 256
    const uint64_t fates_off = 256, lce_off = fates_off + 8 * NF, det_off = lce_off + 4 * P, hist_off = det_off + 4 * P;
    const uint64_t need = hist_off + 4 * P * B;
    if (B > (1ull << 32) || need > (uint64_t)LXO_STATIC_SCRATCH_BYTES)
        return static_fail(c, LXO_ERR_ARG, "tallies exceed LXO_STATIC_SCRATCH_BYTES");
    if (c->device < 0 || c->device >= kMaxStaticDevices) return static_fail(c, LXO_ERR_ARG, "device index");
    DeviceGuard g(c->device);
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[c->device]) {
            void* addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
            if (e != cudaSuccess) return static_fail(c, LXO_ERR_CUDA, "cudaGetSymbolAddress failed");
            g_static_addr[c->device] = (unsigned char*)addr;
        }
        scratch = g_static_addr[c->device];
    }
    lxo::PropParams p;
    s = fill_params(c, src, n, base, rp, &p);
    if (s) return s;
    p.queue = (unsigned long long*)scratch;
    p.err = (int*)(scratch + 8);
    memset(&p.out, 0, sizeof p.out);
    p.out.fates = (unsigned long long*)(scratch + fates_off);
    p.out.lce = (uint32_t*)(scratch + lce_off);
    p.out.det = (uint32_t*)(scratch + det_off);
    p.out.hist = (uint32_t*)(scratch + hist_off);
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: reset the queue head and
    // error word, and start the tallies from the caller's values
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.out.fates, host_out->fates, 8 * NF, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.out.lce, host_out->lce, 4 * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.out.det, host_out->det, 4 * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.out.hist, host_out->hist, 4 * P * B, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n > 0) e = lxo::launch_propagate(p, c->device, st);
    // the fault flags first: on a fault the caller's arrays stay untouched,
    // as with lxo_propagate_host
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(c, LXO_ERR_CUDA, cudaGetErrorString(e));
    if (herr) {
        char msg[128];  // on the stack: the message allocates nothing
        snprintf(msg, sizeof msg,
                 "device fault flags 0x%x (1 = traversal stack, 2 = channel range, 8 = index out of range)", herr);
        return static_fail(c, LXO_ERR_DEVICE, msg);
    }
    e = cudaMemcpyAsync(host_out->fates, p.out.fates, 8 * NF, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->lce, p.out.lce, 4 * P, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->det, p.out.det, 4 * P, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->hist, p.out.hist, 4 * P * B, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(c, LXO_ERR_CUDA, cudaGetErrorString(e));
    return LXO_OK;
}
