/*
 * CPU oracle of the optical-photon tracker -- TEST INFRASTRUCTURE ONLY.
 * Only the tests, the entry module's smoke() and bench.py's CPU-baseline leg
 * load this file's library.  See oracle.h for the contract.
 *
 * Each function names the passage of the paper (or the published method) it
 * follows.  Physics in double, intersection in float32 (same precision as the
 * kernel: the closest hit is a floating-point argmin).
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 */
#define _POSIX_C_SOURCE 200809L
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define NO_HIT 0xFFFFFFFFu
#define SURF_NONE 0xFFFFu
#define C_MM_PER_NS 299.792458
#define TWO_PI 6.283185307179586
#define PI_D 3.141592653589793
#define SOURCE_STEP 0xFFFFFFFFu
/* Table 2 quotes every optical constant at 175 nm */
#define REF_WAVELENGTH_NM 175.0
#define MAX_TRIES 64
#define N_FIXED 8 /* fate counters before the per-material block */

typedef struct { float lo[3], hi[3]; int32_t left, right; uint32_t first, count; } onode;

struct orc_scene {
    uint32_t nt;
    float* v;        /* [nt*9] vertices in index order */
    uint8_t* mi;
    uint8_t* mo;
    uint16_t* sf;
    int32_t* ch;
    uint32_t* order; /* triangle ids in BVH leaf order */
    onode* nodes;
    uint32_t n_nodes;
    int n_mat;
    double mat[64][5];  /* n, L_abs, L_ray (at the reference wavelength), dn/dlambda per nm, Rayleigh exponent */
    int n_surf;
    int stype[256];
    double sp[256][6];
    int n_chan;
    int n_amat, amat[4], n_asurf, asurf[8];
    int mat_slot[64], surf_slot[256];  /* tracked index or -1 */
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As   */
/* Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies whose    */
/* high halves are xored with the other counter words and the key; the key   */
/* is bumped by the Weyl constants between rounds.                           */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1): the top 23 bits plus one half, times 2^-23 (never 0 or 1) */
double orc_uniform(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

static void draw4(uint64_t seed, uint64_t pid, uint32_t step, uint32_t draw, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), step, draw};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox(ctr, key, o);
    for (int i = 0; i < 4; ++i) u[i] = orc_uniform(o[i]);
}

/* ------------------------------------------------------------------------ */
/* small vector helpers (double)                                             */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3])
{
    double l = norm3(a);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* orthonormal basis (t1, t2) perpendicular to unit n: Duff et al.,
 * "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017. */
static void onb(const double n[3], double t1[3], double t2[3])
{
    double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    t1[0] = 1.0 + sgn * n[0] * n[0] * a; t1[1] = sgn * b; t1[2] = -sgn * n[0];
    t2[0] = b; t2[1] = sgn + n[1] * n[1] * a; t2[2] = -n[1];
}

/* ------------------------------------------------------------------------ */
/* Watertight ray/triangle intersection in float32: Woop, Benthin, Wald,     */
/* "Watertight Ray/Triangle Intersection", JCGT 2(1), 2013.  The ray is      */
/* sheared so it runs along +z from the origin; the 2-D edge functions U, V, */
/* W are taken in float and redone in double when one is exactly zero; the  */
/* hit distance is T/det.  Every operation is a single rounded float op in  */
/* the written order (the file is compiled with -ffp-contract=off).          */
/* ------------------------------------------------------------------------ */
typedef struct { int kx, ky, kz; float Sx, Sy, Sz; float o[3]; } wray;

static wray wray_setup(const float o[3], const float d[3])
{
    wray r;
    float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    int kz = (ax >= ay) ? ((ax >= az) ? 0 : 2) : ((ay >= az) ? 1 : 2);
    int kx = kz + 1; if (kx == 3) kx = 0;
    int ky = kx + 1; if (ky == 3) ky = 0;
    if (d[kz] < 0.0f) { int tmp = kx; kx = ky; ky = tmp; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = d[kx] / d[kz];
    r.Sy = d[ky] / d[kz];
    r.Sz = 1.0f / d[kz];
    r.o[0] = o[0]; r.o[1] = o[1]; r.o[2] = o[2];
    return r;
}

static int wray_hit(const wray* r, const float* v, float tmax, float* t_out)
{
    float A[3], B[3], C[3];
    for (int i = 0; i < 3; ++i) {
        A[i] = v[i] - r->o[i];
        B[i] = v[3 + i] - r->o[i];
        C[i] = v[6 + i] - r->o[i];
    }
    float Ax = A[r->kx] - r->Sx * A[r->kz];
    float Ay = A[r->ky] - r->Sy * A[r->kz];
    float Bx = B[r->kx] - r->Sx * B[r->kz];
    float By = B[r->ky] - r->Sy * B[r->kz];
    float Cx = C[r->kx] - r->Sx * C[r->kz];
    float Cy = C[r->ky] - r->Sy * C[r->kz];
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        double CxBy = (double)Cx * (double)By, CyBx = (double)Cy * (double)Bx;
        U = (float)(CxBy - CyBx);
        double AxCy = (double)Ax * (double)Cy, AyCx = (double)Ay * (double)Cx;
        V = (float)(AxCy - AyCx);
        double BxAy = (double)Bx * (double)Ay, ByAx = (double)By * (double)Ax;
        W = (float)(BxAy - ByAx);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
    float det = U + V + W;
    if (det == 0.0f) return 0;
    float Az = r->Sz * A[r->kz];
    float Bz = r->Sz * B[r->kz];
    float Cz = r->Sz * C[r->kz];
    float T = U * Az + V * Bz + W * Cz;
    float t = T / det;
    if (!(t > 0.0f) || !(t <= tmax)) return 0;
    *t_out = t;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* BVH: plain median split on the widest centroid axis, leaves of <= 4.      */
/* Its result is the brute-force argmin (checked by the tests): boxes are    */
/* tested in double with a 1e-3 mm margin, far wider than float rounding.    */
/* ------------------------------------------------------------------------ */
typedef struct { float c[3]; uint32_t id; } cref;

static void tri_bounds(const float* v, float lo[3], float hi[3])
{
    for (int i = 0; i < 3; ++i) {
        float a = v[i], b = v[3 + i], c = v[6 + i];
        float mn = a < b ? a : b; mn = mn < c ? mn : c;
        float mx = a > b ? a : b; mx = mx > c ? mx : c;
        lo[i] = mn; hi[i] = mx;
    }
}

/* order of two references by (centroid[axis], id); the axis is an argument
 * so that scenes can be built from several threads at once */
static int cref_cmp(const cref* a, const cref* b, int axis)
{
    float x = a->c[axis], y = b->c[axis];
    if (x < y) return -1;
    if (x > y) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

/* quickselect by (centroid[axis], id) so the split is deterministic; the
 * last few elements are put in order by insertion */
static void select_kth(cref* a, uint32_t n, uint32_t k, int axis)
{
    uint32_t lo = 0, hi = n - 1;
    while (hi > lo + 16) {
        cref piv = a[lo + (hi - lo) / 2];
        uint32_t i = lo, j = hi;
        while (i <= j) {
            while (cref_cmp(&a[i], &piv, axis) < 0) ++i;
            while (cref_cmp(&a[j], &piv, axis) > 0) --j;
            if (i <= j) {
                cref t = a[i]; a[i] = a[j]; a[j] = t;
                ++i;
                if (j == 0) break;
                --j;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return;
    }
    for (uint32_t i = lo + 1; i <= hi; ++i) {
        cref t = a[i];
        uint32_t j = i;
        while (j > lo && cref_cmp(&t, &a[j - 1], axis) < 0) {
            a[j] = a[j - 1];
            --j;
        }
        a[j] = t;
    }
}

static uint32_t build_rec(orc_scene* s, cref* refs, uint32_t first, uint32_t count)
{
    uint32_t idx = s->n_nodes++;
    onode* nd = &s->nodes[idx];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = first; i < first + count; ++i) {
        float tl[3], th[3];
        tri_bounds(&s->v[9 * (uint64_t)refs[i].id], tl, th);
        for (int a = 0; a < 3; ++a) {
            if (tl[a] < lo[a]) lo[a] = tl[a];
            if (th[a] > hi[a]) hi[a] = th[a];
            if (refs[i].c[a] < clo[a]) clo[a] = refs[i].c[a];
            if (refs[i].c[a] > chi[a]) chi[a] = refs[i].c[a];
        }
    }
    memcpy(nd->lo, lo, sizeof lo);
    memcpy(nd->hi, hi, sizeof hi);
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->first = first;
        nd->count = count;
        return idx;
    }
    int axis = 0;
    float ext = chi[0] - clo[0];
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; axis = a; }
    uint32_t half = count / 2;
    select_kth(refs + first, count, half, axis);
    int32_t l = (int32_t)build_rec(s, refs, first, half);
    int32_t r = (int32_t)build_rec(s, refs, first + half, count - half);
    nd = &s->nodes[idx];
    nd->left = l;
    nd->right = r;
    nd->first = 0;
    nd->count = 0;
    return idx;
}

orc_scene* orc_scene_new(const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                         const uint8_t* mat_inner, const uint8_t* mat_outer,
                         const uint16_t* surface, const int32_t* channel)
{
    if (!verts || !tris || nt == 0) return NULL;
    for (uint64_t i = 0; i < 3ull * nt; ++i)
        if (tris[i] >= nv) return NULL;
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->nt = nt;
    s->v = (float*)malloc(sizeof(float) * 9ull * nt);
    s->mi = (uint8_t*)malloc(nt);
    s->mo = (uint8_t*)malloc(nt);
    s->sf = (uint16_t*)malloc(2ull * nt);
    s->ch = (int32_t*)malloc(4ull * nt);
    for (uint64_t i = 0; i < nt; ++i) {
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 3; ++a) s->v[9 * i + 3 * j + a] = verts[3ull * tris[3 * i + j] + a];
        s->mi[i] = mat_inner ? mat_inner[i] : 0;
        s->mo[i] = mat_outer ? mat_outer[i] : 0;
        s->sf[i] = surface ? surface[i] : SURF_NONE;
        s->ch[i] = channel ? channel[i] : -1;
    }
    cref* refs = (cref*)malloc(sizeof(cref) * nt);
    for (uint32_t i = 0; i < nt; ++i) {
        const float* v = &s->v[9ull * i];
        for (int a = 0; a < 3; ++a) refs[i].c[a] = (v[a] + v[3 + a] + v[6 + a]) / 3.0f;
        refs[i].id = i;
    }
    s->nodes = (onode*)malloc(sizeof(onode) * (2ull * nt + 1));
    s->n_nodes = 0;
    build_rec(s, refs, 0, nt);
    s->order = (uint32_t*)malloc(4ull * nt);
    for (uint32_t i = 0; i < nt; ++i) s->order[i] = refs[i].id;
    free(refs);
    s->n_chan = 0;
    for (int i = 0; i < 64; ++i) s->mat_slot[i] = -1;
    for (int i = 0; i < 256; ++i) s->surf_slot[i] = -1;
    return s;
}

void orc_scene_free(orc_scene* s)
{
    if (!s) return;
    free(s->v); free(s->mi); free(s->mo); free(s->sf); free(s->ch); free(s->order); free(s->nodes);
    free(s);
}

int orc_set_materials(orc_scene* s, const double* m, int n)
{
    if (n < 1 || n > 64) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 5; ++j) s->mat[i][j] = m[5 * i + j];
    s->n_mat = n;
    return 0;
}

int orc_set_surfaces(orc_scene* s, const int* types, const double* p, int n)
{
    if (n < 0 || n > 256) return -1;
    for (int i = 0; i < n; ++i) {
        s->stype[i] = types[i];
        for (int j = 0; j < 6; ++j) s->sp[i][j] = p[6 * i + j];
    }
    s->n_surf = n;
    return 0;
}

int orc_set_channels(orc_scene* s, int n_channels)
{
    s->n_chan = n_channels;
    return 0;
}

int orc_set_adjoint(orc_scene* s, const int* mats, int n_mats, const int* surfs, int n_surfs)
{
    if (n_mats < 0 || n_mats > 4 || n_surfs < 0 || n_surfs > 8) return -1;
    for (int i = 0; i < 64; ++i) s->mat_slot[i] = -1;
    for (int i = 0; i < 256; ++i) s->surf_slot[i] = -1;
    for (int i = 0; i < n_mats; ++i) {
        if (mats[i] < 0 || mats[i] >= 64) return -1;
        s->amat[i] = mats[i];
        s->mat_slot[mats[i]] = i;
    }
    for (int j = 0; j < n_surfs; ++j) {
        if (surfs[j] < 0 || surfs[j] >= 256) return -1;
        s->asurf[j] = surfs[j];
        s->surf_slot[surfs[j]] = j;
    }
    s->n_amat = n_mats;
    s->n_asurf = n_surfs;
    return 0;
}

/* Score of a detected path (the photon never was absorbed):
 *  bulk absorption over length l in material of absorption length L: exp(-l/L)
 *    -> d/dL log = l / L^2
 *  Rayleigh: N scatters over length l: L^-N exp(-l/L) -> d/dL log = l/L^2 - N/L
 *  each reflection on a reflector of reflectivity R: factor R -> n / R
 *  electrode of transparency T: T per pass, (1-T) R_w per wire reflection
 *    -> n_T / T - n_W / (1 - T) */
void orc_jacobian(const orc_scene* s, const double* sums, double* J)
{
    const int K = 2 * s->n_amat + 2 * s->n_asurf, Q = 2 * s->n_amat + s->n_asurf;
    for (int c = 0; c < s->n_chan; ++c) {
        const double* t = &sums[(size_t)c * K];
        double* j = &J[(size_t)c * Q];
        for (int i = 0; i < s->n_amat; ++i) {
            const double La = s->mat[s->amat[i]][1], Lr = s->mat[s->amat[i]][2];
            j[2 * i] = isinf(La) ? 0.0 : t[2 * i] / (La * La);
            j[2 * i + 1] = isinf(Lr) ? 0.0 : t[2 * i] / (Lr * Lr) - t[2 * i + 1] / Lr;
        }
        for (int q = 0; q < s->n_asurf; ++q) {
            const int sid = s->asurf[q];
            const double* sp = s->sp[sid];
            const double a = t[2 * s->n_amat + 2 * q], b = t[2 * s->n_amat + 2 * q + 1];
            double g = 0.0;
            if (s->stype[sid] == ORC_REFLECTOR) g = a / sp[0];
            else if (s->stype[sid] == ORC_ELECTRODE_T) g = a / sp[3] - b / (1.0 - sp[3]);
            j[2 * s->n_amat + q] = g;
        }
    }
}

/* slab test in double against a box widened by 1e-3 mm */
static int box_overlap(const onode* nd, const double o[3], const double inv[3], double tmax)
{
    double t0 = -1e-3, t1 = tmax + 1e-3;
    for (int a = 0; a < 3; ++a) {
        double lo = (double)nd->lo[a] - 1e-3, hi = (double)nd->hi[a] + 1e-3;
        if (isinf(inv[a])) {
            if (o[a] < lo || o[a] > hi) return 0;
            continue;
        }
        double ta = (lo - o[a]) * inv[a], tb = (hi - o[a]) * inv[a];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* closest hit: smallest t in (0, tmax], ties to the smallest triangle id */
static uint32_t closest_hit(const orc_scene* s, const float o[3], const float d[3], uint32_t skip,
                            float tmax, float* t_out, int brute)
{
    wray r = wray_setup(o, d);
    uint32_t best = NO_HIT;
    float bt = tmax;
    if (brute) {
        for (uint32_t i = 0; i < s->nt; ++i) {
            float t;
            if (i == skip) continue;
            if (wray_hit(&r, &s->v[9ull * i], bt, &t)) {
                if (t < bt || (t == bt && (best == NO_HIT || i < best))) { bt = t; best = i; }
            }
        }
        *t_out = bt;
        return best;
    }
    double od[3] = {o[0], o[1], o[2]}, inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = (d[a] == 0.0f) ? INFINITY : 1.0 / (double)d[a];
    uint32_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const onode* nd = &s->nodes[stack[--sp]];
        double lim = isinf(bt) ? INFINITY : (double)bt * (1.0 + 1e-5);
        if (!box_overlap(nd, od, inv, lim)) continue;
        if (nd->left < 0) {
            for (uint32_t k = nd->first; k < nd->first + nd->count; ++k) {
                uint32_t i = s->order[k];
                float t;
                if (i == skip) continue;
                if (wray_hit(&r, &s->v[9ull * i], bt, &t)) {
                    if (t < bt || (t == bt && (best == NO_HIT || i < best))) { bt = t; best = i; }
                }
            }
        } else {
            stack[sp++] = (uint32_t)nd->left;
            stack[sp++] = (uint32_t)nd->right;
        }
    }
    *t_out = bt;
    return best;
}

void orc_trace(const orc_scene* s, uint64_t n, const float* org, const float* dir,
               const uint32_t* skip, const float* tmax, uint32_t* hit, float* t, int brute)
{
    for (uint64_t i = 0; i < n; ++i) {
        float tt;
        uint32_t h = closest_hit(s, &org[3 * i], &dir[3 * i], skip ? skip[i] : NO_HIT,
                                 tmax ? tmax[i] : INFINITY, &tt, brute);
        hit[i] = h;
        t[i] = (h == NO_HIT) ? INFINITY : tt;
    }
}

/* ------------------------------------------------------------------------ */
/* Fresnel amplitudes (Born & Wolf, Sec. 1.5): s and p reflection and        */
/* transmission coefficients for n1 -> n2; p basis vectors are s x k of each */
/* wave.  Paper Sec. 2.2: the only surfaces whose reflectivity is computed   */
/* from refractive indices are quartz, LXe and GXe.                          */
/* ------------------------------------------------------------------------ */
void orc_fresnel(double n1, double n2, double cos_i, double out[6])
{
    double eta = n1 / n2;
    double sin_t2 = eta * eta * (1.0 - cos_i * cos_i);
    if (sin_t2 >= 1.0) {
        out[0] = 1.0; out[1] = 1.0; out[2] = 0.0; out[3] = 0.0; out[4] = 0.0; out[5] = 1.0;
        return;
    }
    double cos_t = sqrt(1.0 - sin_t2);
    out[0] = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    out[1] = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
    out[2] = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);
    out[3] = 2.0 * n1 * cos_i / (n2 * cos_i + n1 * cos_t);
    out[4] = cos_t;
    out[5] = 0.0;
}

/* One dielectric boundary interaction of a linearly polarised photon:
 * P(reflect) = cs^2 Rs + cp^2 Rp; the outgoing polarisation is the coherent
 * sum of the s and p amplitudes (magnitudes only under total internal
 * reflection).  Normal incidence (k parallel to N, plane of incidence
 * undefined, Appendix item 1) takes s = eps. */
int orc_dielectric(const double k[3], const double eps[3], const double N[3], double n1, double n2,
                   double u, double k_out[3], double eps_out[3], double* p_reflect)
{
    double cos_i = -dot3(k, N);
    double s[3];
    cross3(k, N, s);
    if (norm3(s) < 1e-6) {
        s[0] = eps[0]; s[1] = eps[1]; s[2] = eps[2];
    } else {
        normalize3(s);
    }
    double p_in[3];
    cross3(s, k, p_in);
    double cs = dot3(eps, s), cp = dot3(eps, p_in);
    double f[6];
    orc_fresnel(n1, n2, cos_i, f);
    int tir = f[5] != 0.0;
    double pr = tir ? 1.0 : cs * cs * f[0] * f[0] + cp * cp * f[1] * f[1];
    if (p_reflect) *p_reflect = pr;
    if (u < pr) {
        for (int a = 0; a < 3; ++a) k_out[a] = k[a] + 2.0 * cos_i * N[a];
        normalize3(k_out);
        double pr_v[3];
        cross3(s, k_out, pr_v);
        double as = tir ? cs : cs * f[0], ap = tir ? cp : cp * f[1];
        for (int a = 0; a < 3; ++a) eps_out[a] = as * s[a] + ap * pr_v[a];
        normalize3(eps_out);
        return 1;
    }
    double eta = n1 / n2, cos_t = f[4];
    for (int a = 0; a < 3; ++a) k_out[a] = eta * k[a] + (eta * cos_i - cos_t) * N[a];
    normalize3(k_out);
    double pt_v[3];
    cross3(s, k_out, pt_v);
    for (int a = 0; a < 3; ++a) eps_out[a] = cs * f[2] * s[a] + cp * f[3] * pt_v[a];
    normalize3(eps_out);
    return 0;
}

/* Specular reflection off a reflector (Sec. 2.2: the specular share of a
 * reflector's reflections): the direction mirrors about the surface,
 * k' = k + 2 cos(i) N; the polarisation mirrors like a field reflected by a
 * perfect conductor, whose tangential part changes sign and whose normal
 * part is kept, eps' = -eps + 2 (eps.N) N, then made exactly transverse to
 * k' and unit.  N is the unit normal on the incident side. */
void orc_mirror(const double k[3], const double eps[3], const double N[3], double k_out[3], double eps_out[3])
{
    double cos_i = -dot3(k, N);
    double pe = dot3(eps, N);
    for (int a = 0; a < 3; ++a) {
        k_out[a] = k[a] + 2.0 * cos_i * N[a];
        eps_out[a] = -eps[a] + 2.0 * pe * N[a];
    }
    normalize3(k_out);
    double c = dot3(eps_out, k_out);
    for (int a = 0; a < 3; ++a) eps_out[a] -= c * k_out[a];
    normalize3(eps_out);
}

/* Rayleigh scattering of a linearly polarised photon (dipole law, Appendix
 * item 3): the new direction k' has density proportional to
 * 1 - (k'.eps)^2 = sin^2(psi), psi the angle between k' and eps; the new
 * polarisation is eps projected perpendicular to k'.  Sampled exactly in the
 * frame whose pole is eps: c = cos(psi) has density (3/4)(1 - c^2) on
 * [-1, 1], whose CDF (3 (c + 1) - (c^3 + 1)) / 4 = u0 is the cubic
 * c^3 - 3c = 2 - 4 u0; its root in [-1, 1] is c = 2 cos((acos(1 - 2 u0) + 4 pi) / 3)
 * (with c = 2 cos(x), c^3 - 3c = 2 cos(3x)).  The azimuth about eps is
 * 2 pi u1, measured in the orthonormal basis onb(eps).  One Philox call:
 * draw index 1 of the step. */
void orc_rayleigh(const double k[3], const double eps[3], uint64_t pid, uint32_t step, uint64_t seed,
                  double k_out[3], double eps_out[3])
{
    (void)k;
    double u[4];
    draw4(seed, pid, step, 1, u);
    double c = 2.0 * cos((acos(1.0 - 2.0 * u[0]) + 4.0 * PI_D) / 3.0);
    double sn = sqrt(fmax(0.0, 1.0 - c * c)), ph = TWO_PI * u[1];
    double e1[3], e2[3];
    onb(eps, e1, e2);
    for (int a = 0; a < 3; ++a) k_out[a] = c * eps[a] + sn * (cos(ph) * e1[a] + sin(ph) * e2[a]);
    normalize3(k_out);
    double ce = dot3(k_out, eps);
    for (int a = 0; a < 3; ++a) eps_out[a] = eps[a] - ce * k_out[a];
    normalize3(eps_out);
}

/* random linear polarisation perpendicular to unit k from angle alpha */
static void random_pol(const double k[3], double alpha, double eps[3])
{
    double e1[3], e2[3];
    onb(k, e1, e2);
    double ca = cos(alpha), sa = sin(alpha);
    for (int a = 0; a < 3; ++a) eps[a] = ca * e1[a] + sa * e2[a];
    normalize3(eps);
}

/* Lambertian (diffuse) reflection about N, the normal on the incident side:
 * cos(theta) = sqrt(u0), azimuth 2 pi u1, new random polarisation from u2
 * (draw index 1 of the step). */
void orc_lambert(const double N[3], uint64_t pid, uint32_t step, uint64_t seed, double k_out[3], double eps_out[3])
{
    double u[4];
    draw4(seed, pid, step, 1, u);
    double c = sqrt(u[0]), sn = sqrt(fmax(0.0, 1.0 - c * c)), ph = TWO_PI * u[1];
    double t1[3], t2[3];
    onb(N, t1, t2);
    for (int a = 0; a < 3; ++a) k_out[a] = c * N[a] + sn * (cos(ph) * t1[a] + sin(ph) * t2[a]);
    normalize3(k_out);
    random_pol(k_out, TWO_PI * u[2], eps_out);
}

/* ------------------------------------------------------------------------ */
/* Photon source (Sec. 3: positions uniform in the active region, isotropic; */
/* point sources for the LCE maps; 175 nm, random linear polarisation).     */
/* Draws use step index 0xFFFFFFFF: draw 0 = (cos theta, azimuth, pol angle, */
/* z or segment fraction); draws 1.. = position tries.                      */
/* ------------------------------------------------------------------------ */
static int inside_polygon(double x, double y, int n, double R, double phase)
{
    if (n <= 0) return x * x + y * y <= R * R;
    double ap = R * cos(PI_D / n);
    for (int k = 0; k < n; ++k) {
        double a = phase + TWO_PI * (k + 0.5) / n;
        if (x * cos(a) + y * sin(a) > ap) return 0;
    }
    return 1;
}

static void source_photon(const orc_source* src, uint64_t pid, uint64_t idx, uint64_t seed,
                          double pos[3], double dir[3], double pol[3], int* medium, double* t0, double* wl)
{
    const double* p = src->src;
    int kind = (int)p[0];
    *medium = (int)p[1];
    *t0 = p[13];
    /* scintillation time profile (Sec. 2.2, Table 2): the delay after t0
     * follows the singlet exponential (constant p[15]) with probability
     * p[14], else the triplet one (p[16]); own draw (source step, last draw
     * index): u0 picks the component, u1 the exponential delay */
    if (p[15] != 0.0 || p[16] != 0.0) {
        double w[4];
        draw4(seed, pid, SOURCE_STEP, 0xFFFFFFFFu, w);
        double tau = w[0] < p[14] ? p[15] : p[16];
        *t0 += -tau * log(w[1]);
    }
    /* emission spectrum (Sec. 2.2, Table 2): a Gaussian of mean p[17] (0 =
     * the reference wavelength) and full width at half maximum p[18], so
     * sigma = FWHM / (2 sqrt(2 ln 2)); the standard normal deviate is the
     * Box-Muller transform of u2, u3 of the emission draw */
    *wl = p[17] > 0.0 ? p[17] : REF_WAVELENGTH_NM;
    if (p[18] > 0.0) {
        double w[4];
        draw4(seed, pid, SOURCE_STEP, 0xFFFFFFFFu, w);
        double sigma = p[18] / (2.0 * sqrt(2.0 * log(2.0)));
        *wl += sigma * sqrt(-2.0 * log(w[2])) * cos(TWO_PI * w[3]);
    }
    if (kind == ORC_SRC_EXPLICIT) {
        for (int a = 0; a < 3; ++a) {
            pos[a] = src->explicit_pos[3 * idx + a];
            dir[a] = src->explicit_dir[3 * idx + a];
            pol[a] = src->explicit_pol[3 * idx + a];
        }
        normalize3(dir);
        double c = dot3(pol, dir);
        for (int a = 0; a < 3; ++a) pol[a] -= c * dir[a];
        normalize3(pol);
        return;
    }
    double u[4];
    draw4(seed, pid, SOURCE_STEP, 0, u);
    double c = 2.0 * u[0] - 1.0, sn = sqrt(fmax(0.0, 1.0 - c * c)), ph = TWO_PI * u[1];
    dir[0] = sn * cos(ph); dir[1] = sn * sin(ph); dir[2] = c;
    random_pol(dir, TWO_PI * u[2], pol);
    if (kind == ORC_SRC_POINT) {
        for (int a = 0; a < 3; ++a) pos[a] = p[7 + a];
    } else if (kind == ORC_SRC_SEGMENT) {
        for (int a = 0; a < 3; ++a) pos[a] = p[7 + a] + u[3] * (p[10 + a] - p[7 + a]);
    } else if (kind == ORC_SRC_BALL) {
        double R = p[3];
        pos[0] = p[7]; pos[1] = p[8]; pos[2] = p[9];
        for (uint32_t tr = 0; tr < MAX_TRIES; ++tr) {
            double w[4];
            draw4(seed, pid, SOURCE_STEP, 1 + tr, w);
            double x = R * (2.0 * w[0] - 1.0), y = R * (2.0 * w[1] - 1.0), z = R * (2.0 * w[2] - 1.0);
            if (x * x + y * y + z * z <= R * R) {
                pos[0] = p[7] + x; pos[1] = p[8] + y; pos[2] = p[9] + z;
                break;
            }
        }
    } else { /* VOLUME_POLYGON */
        int n = (int)p[2];
        double R = p[3], phase = p[4];
        pos[0] = 0.0; pos[1] = 0.0;
        pos[2] = p[5] + u[3] * (p[6] - p[5]);
        for (uint32_t tr = 0; tr < MAX_TRIES; ++tr) {
            double w[4];
            draw4(seed, pid, SOURCE_STEP, 1 + tr, w);
            double r = R * sqrt(w[0]), a = TWO_PI * w[1];
            double x = r * cos(a), y = r * sin(a);
            if (inside_polygon(x, y, n, R, phase)) { pos[0] = x; pos[1] = y; break; }
            r = R * sqrt(w[2]); a = TWO_PI * w[3];
            x = r * cos(a); y = r * sin(a);
            if (inside_polygon(x, y, n, R, phase)) { pos[0] = x; pos[1] = y; break; }
        }
    }
}

void orc_sample_source(const orc_scene* s, const orc_source* src, uint64_t n, uint64_t base, uint64_t seed,
                       double* pos, double* dir, double* pol, int* medium, double* time, double* wavelength)
{
    (void)s;
    for (uint64_t i = 0; i < n; ++i) {
        double t0, wl;
        int m;
        source_photon(src, base + i, i, seed, &pos[3 * i], &dir[3 * i], &pol[3 * i], &m, &t0, &wl);
        if (medium) medium[i] = m;
        if (time) time[i] = t0;
        if (wavelength) wavelength[i] = wl;
    }
}

/* ------------------------------------------------------------------------ */
/* Propagation of one photon to its fate (Sec. 2.2 and 3): exponential      */
/* absorption and Rayleigh distances, closest surface along the ray, then   */
/* the surface model of the triangle hit.  Per step s the first Philox call */
/* (draw 0) gives u0 -> absorption distance, u1 -> Rayleigh distance,       */
/* u2 -> first surface decision, u3 -> second surface decision; draw 1      */
/* gives the new direction (and u3 of draw 1 decides specular vs diffuse    */
/* for an electrode's wire reflection).                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t* lce;
    uint64_t* det;
    uint64_t* hist;
    uint64_t* fates;
    double* adj;
} tally;

/* Dispersion about the reference wavelength, for a photon of wavelength wl
 * (nm): index n + dn/dlambda (wl - 175), Rayleigh length L_ray (wl/175)^p.
 * With dn/dlambda = 0 and p = 0 every photon sees the Table 2 constants. */
static double index_at(const double* mat, double wl)
{
    return mat[0] + mat[3] * (wl - REF_WAVELENGTH_NM);
}

static double rayleigh_len_at(const double* mat, double wl)
{
    return mat[4] == 0.0 ? mat[2] : mat[2] * pow(wl / REF_WAVELENGTH_NM, mat[4]);
}

static void spawn_offset(double pos[3], const double o_ray[3], double t_hit, const double N[3], double side)
{
    double m = 1.0;
    for (int a = 0; a < 3; ++a) {
        if (fabs(pos[a]) > m) m = fabs(pos[a]);
        if (fabs(o_ray[a]) > m) m = fabs(o_ray[a]);
    }
    if (t_hit > m) m = t_hit;
    double eps = ldexp(m, -18);
    for (int a = 0; a < 3; ++a) pos[a] += side * eps * N[a];
}

static void run_photon(const orc_scene* s, const orc_source* src, uint64_t pid, uint64_t idx, uint64_t seed,
                       uint32_t max_steps, double tbin, uint32_t n_tbins, tally* ty, orc_results* out)
{
    double pos[3], dir[3], pol[3], time, wl;
    int medium;
    source_photon(src, pid, idx, seed, pos, dir, pol, &medium, &time, &wl);
    uint32_t last = NO_HIT;
    uint32_t fate = ORC_TRUNCATED;
    int32_t detail = -1;
    uint32_t step;
    const int M = s->n_mat;
    double tl[24] = {0};  /* adjoint tallies of this photon */
    const int na = s->n_amat;
    for (step = 0; step < max_steps; ++step) {
        double u[4];
        draw4(seed, pid, step, 0, u);
        const double* mat = s->mat[medium];
        double d_abs = isinf(mat[1]) ? INFINITY : -mat[1] * log(u[0]);
        double d_ray = isinf(mat[2]) ? INFINITY : -rayleigh_len_at(mat, wl) * log(u[1]);
        double d_int = d_abs < d_ray ? d_abs : d_ray;
        float of[3] = {(float)pos[0], (float)pos[1], (float)pos[2]};
        float df[3] = {(float)dir[0], (float)dir[1], (float)dir[2]};
        float tmax = isinf(d_int) ? INFINITY : (float)d_int;
        float th;
        uint32_t tri = closest_hit(s, of, df, last, tmax, &th, 0);
        double vel = C_MM_PER_NS / index_at(mat, wl);
        const int ms = s->mat_slot[medium];
        if (tri == NO_HIT) {
            if (isinf(d_int)) { fate = ORC_ESCAPED; detail = -1; break; }
            for (int a = 0; a < 3; ++a) pos[a] += d_int * dir[a];
            time += d_int / vel;
            if (ms >= 0) tl[2 * ms] += d_int;
            if (d_abs <= d_ray) { fate = ORC_BULK_ABS; detail = medium; break; }
            if (ms >= 0) tl[2 * ms + 1] += 1.0;
            double k2[3], e2[3];
            orc_rayleigh(dir, pol, pid, step, seed, k2, e2);
            memcpy(dir, k2, sizeof k2);
            memcpy(pol, e2, sizeof e2);
            last = NO_HIT;
            continue;
        }
        /* advance to the surface */
        double o_ray[3] = {pos[0], pos[1], pos[2]};
        for (int a = 0; a < 3; ++a) pos[a] += (double)th * dir[a];
        time += (double)th / vel;
        if (ms >= 0) tl[2 * ms] += (double)th;
        const float* v = &s->v[9ull * tri];
        double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
        double e2v[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
        double ng[3];
        cross3(e1, e2v, ng);
        normalize3(ng);
        double kn = dot3(dir, ng);
        int forward = kn > 0.0; /* moving from the inner to the outer side */
        int from = forward ? s->mi[tri] : s->mo[tri];
        int to = forward ? s->mo[tri] : s->mi[tri];
        double Nf[3]; /* normal on the incident side */
        for (int a = 0; a < 3; ++a) Nf[a] = forward ? -ng[a] : ng[a];
        uint16_t sid = s->sf[tri];
        last = tri;
        if (sid == SURF_NONE) {
            if (from != medium || to >= M) { fate = ORC_GEOM_ERR; detail = (int32_t)tri; break; }
            double k2[3], e2[3];
            int refl = orc_dielectric(dir, pol, Nf, index_at(s->mat[from], wl), index_at(s->mat[to], wl), u[2],
                                      k2, e2, NULL);
            memcpy(dir, k2, sizeof k2);
            memcpy(pol, e2, sizeof e2);
            if (!refl) medium = to;
            spawn_offset(pos, o_ray, th, Nf, refl ? 1.0 : -1.0);
            continue;
        }
        int type = s->stype[sid];
        const double* sp = s->sp[sid];
        const int ss = s->surf_slot[sid];
        if (type == ORC_ABSORBER) { fate = ORC_SURF_ABS; detail = sid; break; }
        if (type == ORC_PHOTOCATHODE) {
            int c = s->ch[tri];
            if (c < 0 || c >= s->n_chan) { fate = ORC_GEOM_ERR; detail = (int32_t)tri; break; }
            if (u[2] < sp[2]) { fate = ORC_DETECTED; } else { fate = ORC_QE_FAIL; }
            detail = c;
            break;
        }
        int reflect_specular = -1; /* -1: no reflection */
        if (type == ORC_REFLECTOR) {
            if (!(u[2] < sp[0])) { fate = ORC_SURF_ABS; detail = sid; break; }
            if (ss >= 0) tl[2 * na + 2 * ss] += 1.0;
            reflect_specular = u[3] < sp[1];
        } else if (type == ORC_ELECTRODE_T) {
            if (u[2] < sp[3]) { /* passes between the wires */
                if (from != medium || to >= M) { fate = ORC_GEOM_ERR; detail = (int32_t)tri; break; }
                if (ss >= 0) tl[2 * na + 2 * ss] += 1.0;
                medium = to;
                spawn_offset(pos, o_ray, th, Nf, -1.0);
                continue;
            }
            if (!(u[3] < sp[4])) { fate = ORC_SURF_ABS; detail = sid; break; }
            if (ss >= 0) tl[2 * na + 2 * ss + 1] += 1.0;
            double w[4];
            draw4(seed, pid, step, 1, w);
            reflect_specular = w[3] < sp[5];
        } else {
            fate = ORC_GEOM_ERR; detail = (int32_t)tri; break;
        }
        if (reflect_specular) {
            double k2[3], e2[3];
            orc_mirror(dir, pol, Nf, k2, e2);
            memcpy(dir, k2, sizeof k2);
            memcpy(pol, e2, sizeof e2);
        } else {
            double k2[3], e2[3];
            orc_lambert(Nf, pid, step, seed, k2, e2);
            memcpy(dir, k2, sizeof k2);
            memcpy(pol, e2, sizeof e2);
        }
        spawn_offset(pos, o_ray, th, Nf, 1.0);
    }
    uint32_t steps = (step < max_steps) ? step + 1 : max_steps;
    ty->fates[fate] += 1;
    ty->fates[7] += steps;
    if (fate == ORC_BULK_ABS) ty->fates[N_FIXED + detail] += 1;
    if (fate == ORC_SURF_ABS) ty->fates[N_FIXED + M + detail] += 1;
    if (fate == ORC_DETECTED || fate == ORC_QE_FAIL) ty->lce[detail] += 1;
    if (fate == ORC_DETECTED && ty->adj) {
        const int K = 2 * s->n_amat + 2 * s->n_asurf;
        for (int k = 0; k < K; ++k) ty->adj[(uint64_t)detail * K + k] += tl[k];
    }
    if (fate == ORC_DETECTED) {
        ty->det[detail] += 1;
        double b = floor(time / tbin);
        uint32_t bin = (b >= (double)n_tbins || !(b >= 0.0)) ? n_tbins : (uint32_t)b;
        ty->hist[(uint64_t)detail * (n_tbins + 1) + bin] += 1;
    }
    if (out->ph_fate) out->ph_fate[idx] = fate;
    if (out->ph_detail) out->ph_detail[idx] = detail;
    if (out->ph_steps) out->ph_steps[idx] = steps;
    if (out->ph_time) out->ph_time[idx] = (float)time;
    if (out->ph_state) {
        float* o = out->ph_state + 9 * idx;
        for (int a = 0; a < 3; ++a) {
            o[a] = (float)pos[a];
            o[3 + a] = (float)dir[a];
            o[6 + a] = (float)pol[a];
        }
    }
}

typedef struct {
    const orc_scene* s;
    const orc_source* src;
    uint64_t lo, hi, base, seed;
    uint32_t max_steps, n_tbins;
    double tbin;
    orc_results* out;
    tally ty;
} job;

static void* worker(void* arg)
{
    job* j = (job*)arg;
    for (uint64_t i = j->lo; i < j->hi; ++i)
        run_photon(j->s, j->src, j->base + i, i, j->seed, j->max_steps, j->tbin, j->n_tbins, &j->ty, j->out);
    return NULL;
}

int orc_propagate(const orc_scene* s, const orc_source* src, uint64_t n, uint64_t base, uint64_t seed,
                  uint32_t max_steps, double tbin_ns, uint32_t n_tbins, orc_results* out, int n_threads)
{
    if (!s || !src || !out || s->n_mat < 1 || s->n_chan < 1 || tbin_ns <= 0.0 || n_tbins > (1u << 24)) return -1;
    int medium0 = (int)src->src[1];
    if (medium0 < 0 || medium0 >= s->n_mat) return -1;
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > n) n_threads = n ? (int)n : 1;
    const uint64_t P = (uint64_t)s->n_chan;
    const uint64_t NF = N_FIXED + (uint64_t)s->n_mat + (uint64_t)s->n_surf;
    job* jobs = (job*)calloc((size_t)n_threads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        job* j = &jobs[t];
        j->s = s; j->src = src; j->base = base; j->seed = seed;
        j->max_steps = max_steps; j->n_tbins = n_tbins; j->tbin = tbin_ns; j->out = out;
        j->lo = n * (uint64_t)t / (uint64_t)n_threads;
        j->hi = n * (uint64_t)(t + 1) / (uint64_t)n_threads;
        j->ty.lce = (uint64_t*)calloc(P, 8);
        j->ty.det = (uint64_t*)calloc(P, 8);
        j->ty.hist = (uint64_t*)calloc(P * (n_tbins + 1ull), 8);
        j->ty.fates = (uint64_t*)calloc(NF, 8);
        const uint64_t K = 2ull * s->n_amat + 2ull * s->n_asurf;
        j->ty.adj = (out->adjoint && K) ? (double*)calloc(P * K, 8) : NULL;
        pthread_create(&th[t], NULL, worker, j);
    }
    for (int t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        job* j = &jobs[t];
        for (uint64_t c = 0; c < P; ++c) {
            if (out->lce) out->lce[c] += j->ty.lce[c];
            if (out->det) out->det[c] += j->ty.det[c];
        }
        if (out->hist)
            for (uint64_t c = 0; c < P * (n_tbins + 1ull); ++c) out->hist[c] += j->ty.hist[c];
        if (out->fates)
            for (uint64_t c = 0; c < NF; ++c) out->fates[c] += j->ty.fates[c];
        if (j->ty.adj) {
            const uint64_t K = 2ull * s->n_amat + 2ull * s->n_asurf;
            for (uint64_t c = 0; c < P * K; ++c) out->adjoint[c] += j->ty.adj[c];
            free(j->ty.adj);
        }
        free(j->ty.lce); free(j->ty.det); free(j->ty.hist); free(j->ty.fates);
    }
    free(jobs);
    free(th);
    return 0;
}
