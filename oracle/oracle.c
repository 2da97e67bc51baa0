/*
 * oracle.c -- plain, slow FP64 CPU restatement of the path-traced light-transport estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no code, header, table or constant generator
 * with the CUDA path: the two meet only in the written definitions below and in the seeded
 * scene generators that feed both.
 *
 * What it computes ("Megakernel vs Wavefront GPU Path Tracing"):
 *   - Eq. 1 (light transport equation) estimated by Eq. 2 (Monte Carlo mean of f/p) along
 *     paths whose throughput is the product of BSDF x |cos| over the sampling pdf (Eq. 3).
 *   - The forward path-tracing loop of Sec. 2.2: generate the camera ray, extend the path to the
 *     next scattering point, accumulate radiance, sample a new direction and update the
 *     throughput, repeat until the maximum path length.
 *   - The shadow-evaluation stage named in Sec. 3 (next-event estimation toward area lights) and
 *     the Russian-roulette termination named in Sec. 3.1.
 *   - Multi-sample pixels (Sec. 6.2): image = mean over the pixel's samples, summed in sample order.
 *   - Forward-mode derivatives of the same estimator with dual numbers (per-material albedo and
 *     emission), used to check the GPU adjoint.
 *
 * Readings where the paper is silent (each is listed with its reason in the design notes):
 *   - random numbers: counter-based PCG hash (Jarzynski & Olano, JCGT 2020) keyed by
 *     (seed, pixel, sample, bounce, dim); u = (h >> 8) * 2^-24, exact in FP32 and FP64; the pixel
 *     jitter optionally follows the paper's Halton (2,3) sequence with a per-pixel Cranley-Patterson
 *     rotation, in 24-bit fixed point;
 *   - NEE only, no MIS: a BSDF-sampled hit on a listed light adds its emission only at bounce 0
 *     or after a delta bounce; emitters not in the light list always add; the light pmf is
 *     proportional to area; lights and all emission are one-sided (front face by winding);
 *   - max_depth = number of vertices; the last vertex adds emission and stops;
 *   - Russian roulette from bounce rr_start: q = clamp(max(tp), 0.05, 0.95) or a fixed q;
 *   - BSDFs: Lambert; GGX conductor with alpha = max(roughness^2, 1e-4), height-correlated
 *     Smith G2, visible-normal sampling (Heitz 2018), Schlick F with F0 = albedo; smooth
 *     dielectric with exact unpolarised Fresnel, reflect with probability F, radiance scaled by
 *     (eta_i/eta_t)^2 on refraction, tint = albedo;
 *   - geometric normals only; two-sided intersection; Moller-Trumbore with inclusive
 *     barycentric bounds and t > 0; equal t resolved to the lower triangle id;
 *   - ray offset: origin += eps * n on the outgoing side, eps = 1e-4 * max(1, max|p|);
 *     shadow rays end at the light sample lifted by eps (same rule) along the light's normal.
 *
 * Parity pins (tests/test_oracle_*.py): BVH closest hit == brute force; closed-form
 * intersections; Lambert/GGX/dielectric identities (reciprocity, sampled-weight == f cos/pdf,
 * normalisation, R + T = 1, Schlick and Fresnel limits); white-furnace series; the
 * differential-area-to-rectangle form factor, also with the rectangle light cut into triangles of
 * very unequal area; the pinhole camera's geometry (centre ray at the target, half-angles vfov/2
 * and atan(tan(vfov/2) W/H), square pixels, row 0 at the top, +x to the right); light picks
 * counted against area / total area; a glass-in-furnace identity; dual numbers == central finite
 * differences of the oracle itself and == the furnace derivative series.  The camera and
 * light-pick pins are also run on copies of this file with planted mistakes, which must fail them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAXK 8          /* maximum number of tangent directions carried by the dual numbers */
#define OR_MAT_LAMBERT 0u
#define OR_MAT_GGX 1u
#define OR_MAT_DIELECTRIC 2u

/* ------------------------------------------------------------------ vectors (FP64) */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r; r.x = x; r.y = y; r.z = z; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static v3 nrm(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------ random numbers */
/* PCG hash of one 32-bit word (Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 2020):
 * one LCG step, then the PCG RXS-M-XS output permutation. */
uint32_t or_pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

/* Per-path key: seed (both halves), then pixel, then sample, each folded by one hash. */
uint32_t or_path_key(uint64_t seed, uint32_t pixel, uint32_t sample) {
    uint32_t k = or_pcg_hash((uint32_t)(seed >> 32));
    k = or_pcg_hash((uint32_t)seed ^ k);
    k = or_pcg_hash(pixel ^ k);
    k = or_pcg_hash(sample ^ k);
    return k;
}

/* Uniform for (bounce, dim) of a path: 24 high bits of the hash, scaled by 2^-24. */
double or_u01(uint32_t path_key, uint32_t bounce, uint32_t dim) {
    uint32_t h = or_pcg_hash(path_key ^ or_pcg_hash((bounce << 4) | dim));
    return (double)(h >> 8) * (1.0 / 16777216.0);
}

/* Dimensions used at each bounce. */
enum { D_JX = 0, D_JY = 1, D_LIGHT = 2, D_LU = 3, D_LV = 4, D_LOBE = 5, D_DIR0 = 6, D_DIR1 = 7, D_RR = 8 };

void or_u01_batch(uint64_t seed, const uint32_t* pixel, const uint32_t* sample, const uint32_t* bounce,
                  const uint32_t* dim, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = or_u01(or_path_key(seed, pixel[i], sample[i]), bounce[i], dim[i]);
}

/* ------------------------------------------------------------------ pixel jitter (Sec. 2.3)
 * The ray-generation stage jitters each camera ray inside its pixel.  Two samplers:
 *   OR_SAMPLER_PCG: u0, u1 = the path's uniforms of bounce 0, dims D_JX and D_JY;
 *   OR_SAMPLER_HALTON: the paper's Halton sequence in bases 2 and 3 over the pixel's sample index,
 *     shifted per pixel by a Cranley-Patterson rotation (Cranley & Patterson 1976) modulo 1.
 * Everything is a 24-bit fixed-point fraction, so FP32 and FP64 see the same numbers:
 *   radical inverse (van der Corput / Halton 1960): s = sum_k d_k b^k has phi_b(s) = sum_k d_k b^-(k+1);
 *   with K digits (b^K >= 2^32 > s) that is R / b^K with R = sum_k d_k b^(K-1-k), kept as
 *   floor(2^24 R / b^K);
 *   rotation of dim d: the top 24 bits of the hash of (seed, pixel, sample 2^32 - 1) for (bounce 0, d)
 *   (that sample index is never rendered: sample_offset + spp < 2^32);
 *   u_d = ((phi(s) + rotation_d) mod 2^24) * 2^-24. */
#define OR_SAMPLER_PCG 0u
#define OR_SAMPLER_HALTON 1u

uint32_t or_radical_inverse24(uint32_t base, uint32_t s) {
    uint64_t bk = 1;
    int K = 0;
    while (bk < (1ull << 32)) {
        bk *= base;
        ++K;
    }
    uint64_t R = 0;
    uint32_t t = s;
    for (int k = 0; k < K; ++k) {   /* reverse the K base-b digits of s */
        R = R * base + t % base;
        t /= base;
    }
    return (uint32_t)((R << 24) / bk);
}

static uint32_t hash24(uint32_t key, uint32_t bounce, uint32_t dim) {
    return or_pcg_hash(key ^ or_pcg_hash((bounce << 4) | dim)) >> 8;
}

static void pixel_jitter(uint32_t sampler, uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t key, double* u0,
                         double* u1) {
    if (sampler == OR_SAMPLER_HALTON) {
        uint32_t kp = or_path_key(seed, pixel, 0xFFFFFFFFu);
        uint32_t j0 = (or_radical_inverse24(2, sample) + hash24(kp, 0, D_JX)) & 0xFFFFFFu;
        uint32_t j1 = (or_radical_inverse24(3, sample) + hash24(kp, 0, D_JY)) & 0xFFFFFFu;
        *u0 = (double)j0 / 16777216.0;
        *u1 = (double)j1 / 16777216.0;
    } else {
        *u0 = or_u01(key, 0, D_JX);
        *u1 = or_u01(key, 0, D_JY);
    }
}

void or_pixel_jitter_batch(uint32_t sampler, uint64_t seed, const uint32_t* pixel, const uint32_t* sample, int64_t n,
                           double* out) {
    for (int64_t i = 0; i < n; ++i)
        pixel_jitter(sampler, seed, pixel[i], sample[i], or_path_key(seed, pixel[i], sample[i]), out + 2 * i,
                     out + 2 * i + 1);
}

/* ------------------------------------------------------------------ scene */
typedef struct {
    uint32_t type;
    double albedo[3];
    double emission;
    double roughness;
    double ior;
} omat;

typedef struct {
    double lo[3], hi[3];
    int64_t left, right;     /* children (internal) */
    int64_t first, count;    /* range in `order` (leaf, count > 0) */
} onode;

typedef struct or_scene {
    int64_t n_tris;
    v3 *p0, *p1, *p2;
    uint32_t* mat;
    unsigned char* is_light;
    int64_t n_mats;
    omat* mats;
    double env[3];
    int64_t n_lights;
    int64_t* light_tri;      /* light triangles in ascending triangle id */
    double* light_cdf;       /* inclusive prefix sums of area / total area */
    double light_area;       /* total light area */
    int64_t n_nodes;
    onode* nodes;
    int64_t* order;
} or_scene;

static double tri_area(const or_scene* s, int64_t i) {
    return 0.5 * sqrt(dot(cross(sub(s->p1[i], s->p0[i]), sub(s->p2[i], s->p0[i])),
                          cross(sub(s->p1[i], s->p0[i]), sub(s->p2[i], s->p0[i]))));
}

/* ------------------------------------------------------------------ BVH (object-median split)
 * A plain acceleration structure: it never changes which triangle is found, because boxes are
 * padded outward and a box is skipped only when its entry distance is strictly beyond the best
 * hit so far (ties on t still reach the lower id).  Pinned against the brute-force loop. */
static void nth_element(int64_t* a, int64_t n, int64_t k, const double* cen, int axis) {
#define KEY(i) cen[3 * a[i] + axis]
    int64_t lo = 0, hi = n - 1;
    while (hi > lo) {
        double pivot = KEY((lo + hi) / 2);
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (KEY(i) < pivot) i++;
            while (KEY(j) > pivot) j--;
            if (i <= j) { int64_t t = a[i]; a[i] = a[j]; a[j] = t; i++; j--; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else break;
    }
#undef KEY
}

static int64_t build_node(or_scene* s, const double* cen, int64_t first, int64_t count) {
    int64_t id = s->n_nodes++;
    onode* nd = &s->nodes[id];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = first; i < first + count; ++i) {
        int64_t t = s->order[i];
        v3 p[3] = {s->p0[t], s->p1[t], s->p2[t]};
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                double c = comp(p[v], k);
                if (c < nd->lo[k]) nd->lo[k] = c;
                if (c > nd->hi[k]) nd->hi[k] = c;
            }
        for (int k = 0; k < 3; ++k) {
            double c = cen[3 * t + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    }
    for (int k = 0; k < 3; ++k) {  /* pad outward so FP64 slab rounding can never cull a true hit */
        double pad = 1e-9 * (1.0 + fabs(nd->lo[k]) + fabs(nd->hi[k]));
        nd->lo[k] -= pad;
        nd->hi[k] += pad;
    }
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->first = first;
        nd->count = count;
        return id;
    }
    int axis = 0;
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    int64_t half = count / 2;
    nth_element(s->order + first, count, half, cen, axis);
    nd->count = 0;
    int64_t l = build_node(s, cen, first, half);
    int64_t r = build_node(s, cen, first + half, count - half);
    s->nodes[id].left = l;  /* re-index: s->nodes is not reallocated, but keep it explicit */
    s->nodes[id].right = r;
    s->nodes[id].first = 0;
    s->nodes[id].count = 0;
    return id;
}

static void build_bvh(or_scene* s) {
    s->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n_tris > 0 ? s->n_tris : 1));
    s->nodes = (onode*)malloc(sizeof(onode) * (size_t)(2 * s->n_tris + 1));
    double* cen = (double*)malloc(sizeof(double) * 3 * (size_t)(s->n_tris > 0 ? s->n_tris : 1));
    for (int64_t i = 0; i < s->n_tris; ++i) {
        s->order[i] = i;
        v3 c = scl(add(add(s->p0[i], s->p1[i]), s->p2[i]), 1.0 / 3.0);
        cen[3 * i] = c.x; cen[3 * i + 1] = c.y; cen[3 * i + 2] = c.z;
    }
    s->n_nodes = 0;
    if (s->n_tris > 0) build_node(s, cen, 0, s->n_tris);
    free(cen);
}

/* Replace albedo and emission (the differentiable parameters). */
void or_scene_set_materials(or_scene* s, const float* albedo, const float* emission) {
    for (int64_t m = 0; m < s->n_mats; ++m) {
        for (int c = 0; c < 3; ++c) s->mats[m].albedo[c] = (double)albedo[3 * m + c];
        s->mats[m].emission = (double)emission[m];
    }
}

static or_scene* scene_alloc(int64_t n_tris) {
    or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
    s->n_tris = n_tris;
    size_t nt = (size_t)(n_tris > 0 ? n_tris : 1);
    s->p0 = (v3*)malloc(sizeof(v3) * nt);
    s->p1 = (v3*)malloc(sizeof(v3) * nt);
    s->p2 = (v3*)malloc(sizeof(v3) * nt);
    s->mat = (uint32_t*)malloc(sizeof(uint32_t) * nt);
    s->is_light = (unsigned char*)calloc(nt, 1);
    return s;
}

static or_scene* scene_finish(or_scene* s, int64_t n_mats, const uint32_t* mat_type, const float* mat_albedo,
                              const float* mat_emission, const float* mat_roughness, const float* mat_ior,
                              const float* env);

or_scene* or_scene_create(const float* verts, int64_t n_verts, const uint32_t* tris, int64_t n_tris,
                          const uint32_t* tri_mat, int64_t n_mats, const uint32_t* mat_type,
                          const float* mat_albedo, const float* mat_emission, const float* mat_roughness,
                          const float* mat_ior, const float* env) {
    (void)n_verts;
    or_scene* s = scene_alloc(n_tris);
    for (int64_t i = 0; i < n_tris; ++i) {
        const float* a = verts + 3 * (size_t)tris[3 * i];
        const float* b = verts + 3 * (size_t)tris[3 * i + 1];
        const float* c = verts + 3 * (size_t)tris[3 * i + 2];
        s->p0[i] = mk(a[0], a[1], a[2]);
        s->p1[i] = mk(b[0], b[1], b[2]);
        s->p2[i] = mk(c[0], c[1], c[2]);
        s->mat[i] = tri_mat[i];
    }
    return scene_finish(s, n_mats, mat_type, mat_albedo, mat_emission, mat_roughness, mat_ior, env);
}

/* A scene given as world-space triangle corners in FP64 (n_tris x 3 x 3): used for instanced
 * scenes, whose instances the caller has already placed in the world (triangle order = instances
 * in order, each mesh's triangles in order; that order is the triangle id). */
or_scene* or_scene_create_corners(const double* corners, int64_t n_tris, const uint32_t* tri_mat, int64_t n_mats,
                                  const uint32_t* mat_type, const float* mat_albedo, const float* mat_emission,
                                  const float* mat_roughness, const float* mat_ior, const float* env) {
    or_scene* s = scene_alloc(n_tris);
    for (int64_t i = 0; i < n_tris; ++i) {
        const double* c = corners + 9 * (size_t)i;
        s->p0[i] = mk(c[0], c[1], c[2]);
        s->p1[i] = mk(c[3], c[4], c[5]);
        s->p2[i] = mk(c[6], c[7], c[8]);
        s->mat[i] = tri_mat[i];
    }
    return scene_finish(s, n_mats, mat_type, mat_albedo, mat_emission, mat_roughness, mat_ior, env);
}

static or_scene* scene_finish(or_scene* s, int64_t n_mats, const uint32_t* mat_type, const float* mat_albedo,
                              const float* mat_emission, const float* mat_roughness, const float* mat_ior,
                              const float* env) {
    const int64_t n_tris = s->n_tris;
    s->n_mats = n_mats;
    s->mats = (omat*)calloc((size_t)(n_mats > 0 ? n_mats : 1), sizeof(omat));
    for (int64_t m = 0; m < n_mats; ++m) {
        s->mats[m].type = mat_type[m];
        s->mats[m].roughness = mat_roughness[m];
        s->mats[m].ior = mat_ior[m];
    }
    or_scene_set_materials(s, mat_albedo, mat_emission);
    for (int c = 0; c < 3; ++c) s->env[c] = env[c];
    /* The light list is fixed here: triangles whose material emits at creation time. */
    s->n_lights = 0;
    for (int64_t i = 0; i < n_tris; ++i)
        if (s->mats[s->mat[i]].emission > 0.0) s->n_lights++;
    s->light_tri = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n_lights > 0 ? s->n_lights : 1));
    s->light_cdf = (double*)malloc(sizeof(double) * (size_t)(s->n_lights > 0 ? s->n_lights : 1));
    int64_t j = 0;
    double acc = 0.0;
    for (int64_t i = 0; i < n_tris; ++i)
        if (s->mats[s->mat[i]].emission > 0.0) {
            s->is_light[i] = 1;
            s->light_tri[j] = i;
            acc += tri_area(s, i);
            s->light_cdf[j] = acc;
            j++;
        }
    s->light_area = acc;
    for (j = 0; j < s->n_lights; ++j) s->light_cdf[j] = acc > 0.0 ? s->light_cdf[j] / acc : 0.0;
    build_bvh(s);
    return s;
}

void or_scene_destroy(or_scene* s) {
    if (!s) return;
    free(s->p0); free(s->p1); free(s->p2); free(s->mat); free(s->is_light); free(s->mats);
    free(s->light_tri); free(s->light_cdf); free(s->nodes); free(s->order);
    free(s);
}

int64_t or_scene_n_lights(const or_scene* s) { return s->n_lights; }
double or_scene_light_area(const or_scene* s) { return s->light_area; }

/* ------------------------------------------------------------------ intersection */
/* Moller-Trumbore: hit when det != 0, 0 <= u, 0 <= v, u + v <= 1 and tmin < t < tmax. */
static int hit_tri(const or_scene* s, int64_t i, v3 o, v3 d, double tmin, double tmax,
                   double* t_out, double* u_out, double* v_out) {
    v3 e1 = sub(s->p1[i], s->p0[i]);
    v3 e2 = sub(s->p2[i], s->p0[i]);
    v3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 tv = sub(o, s->p0[i]);
    double u = dot(tv, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    v3 q = cross(tv, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    double t = dot(e2, q) * inv;
    if (!(t > tmin && t < tmax)) return 0;
    *t_out = t; *u_out = u; *v_out = v;
    return 1;
}

/* Whether a ray meets a (padded) box within [0, tmax]; *t_entry = its entry distance. */
static int box_hit(const onode* nd, v3 o, v3 d, double tmax, double* t_entry) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), dk = comp(d, k);
        if (dk == 0.0) {
            if (ok < nd->lo[k] || ok > nd->hi[k]) return 0;
            continue;
        }
        double a = (nd->lo[k] - ok) / dk, b = (nd->hi[k] - ok) / dk;
        if (a > b) { double t = a; a = b; b = t; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    *t_entry = t0;
    return 1;
}

static void consider(const or_scene* s, int64_t i, v3 o, v3 d, double* bt, int64_t* bi, double* bu, double* bv) {
    double t, u, v;
    if (hit_tri(s, i, o, d, 0.0, INFINITY, &t, &u, &v))
        if (t < *bt || (t == *bt && i < *bi)) { *bt = t; *bi = i; *bu = u; *bv = v; }
}

/* Closest hit with t > 0; equal t goes to the lower triangle id.  Returns the id or -1. */
static int64_t closest_hit(const or_scene* s, v3 o, v3 d, int use_bvh, double* t_out, double* u_out, double* v_out) {
    double bt = INFINITY, bu = 0.0, bv = 0.0;
    int64_t bi = -1;
    if (!use_bvh || s->n_nodes == 0) {
        for (int64_t i = 0; i < s->n_tris; ++i) consider(s, i, o, d, &bt, &bi, &bu, &bv);
    } else {
        int64_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const onode* nd = &s->nodes[stack[--sp]];
            double te;
            if (!box_hit(nd, o, d, bt, &te)) continue;   /* entry strictly beyond bt: no tie possible */
            if (nd->count > 0) {
                for (int64_t k = nd->first; k < nd->first + nd->count; ++k) consider(s, s->order[k], o, d, &bt, &bi, &bu, &bv);
            } else {
                stack[sp++] = nd->left;
                stack[sp++] = nd->right;
            }
        }
    }
    *t_out = bt; *u_out = bu; *v_out = bv;
    return bi;
}

/* Any triangle with 0 < t < tmax. */
static int occluded(const or_scene* s, v3 o, v3 d, double tmax, int use_bvh) {
    double t, u, v;
    if (!use_bvh || s->n_nodes == 0) {
        for (int64_t i = 0; i < s->n_tris; ++i)
            if (hit_tri(s, i, o, d, 0.0, tmax, &t, &u, &v)) return 1;
        return 0;
    }
    int64_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* nd = &s->nodes[stack[--sp]];
        double te;
        if (!box_hit(nd, o, d, tmax, &te)) continue;
        if (nd->count > 0) {
            for (int64_t k = nd->first; k < nd->first + nd->count; ++k)
                if (hit_tri(s, s->order[k], o, d, 0.0, tmax, &t, &u, &v)) return 1;
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return 0;
}

void or_intersect_batch(const or_scene* s, const double* o, const double* d, int64_t n, int use_bvh,
                        double* t, int64_t* prim, double* u, double* v) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        prim[i] = closest_hit(s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                              use_bvh, &t[i], &u[i], &v[i]);
}

void or_occluded_batch(const or_scene* s, const double* o, const double* d, const double* tmax, int64_t n,
                       int use_bvh, int32_t* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        out[i] = occluded(s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]), tmax[i], use_bvh);
}

/* ------------------------------------------------------------------ dual-number colours
 * A colour value with `nd` tangent directions: derivative of each channel along each
 * parameter direction.  With nd = 0 this is plain FP64 arithmetic. */
typedef struct { double v[3]; double d[OR_MAXK][3]; } dc;

static dc dc_const(double r, double g, double b) {
    dc x;
    memset(&x, 0, sizeof(x));
    x.v[0] = r; x.v[1] = g; x.v[2] = b;
    return x;
}
static dc dc_mul(dc a, dc b, int nd) {
    dc r;
    for (int c = 0; c < 3; ++c) r.v[c] = a.v[c] * b.v[c];
    for (int k = 0; k < nd; ++k)
        for (int c = 0; c < 3; ++c) r.d[k][c] = a.d[k][c] * b.v[c] + a.v[c] * b.d[k][c];
    return r;
}
static dc dc_scale(dc a, double s, int nd) {
    dc r;
    for (int c = 0; c < 3; ++c) r.v[c] = a.v[c] * s;
    for (int k = 0; k < nd; ++k)
        for (int c = 0; c < 3; ++c) r.d[k][c] = a.d[k][c] * s;
    return r;
}
static dc dc_add(dc a, dc b, int nd) {
    dc r;
    for (int c = 0; c < 3; ++c) r.v[c] = a.v[c] + b.v[c];
    for (int k = 0; k < nd; ++k)
        for (int c = 0; c < 3; ++c) r.d[k][c] = a.d[k][c] + b.d[k][c];
    return r;
}

/* Parameter directions: dir_a[k][m][c] for albedo, dir_e[k][m] for emission. */
typedef struct { int nd; int64_t n_mats; const double* dir_a; const double* dir_e; } dirs_t;

static dc mat_albedo(const or_scene* s, int64_t m, const dirs_t* dr) {
    dc a = dc_const(s->mats[m].albedo[0], s->mats[m].albedo[1], s->mats[m].albedo[2]);
    for (int k = 0; k < dr->nd; ++k)
        for (int c = 0; c < 3; ++c) a.d[k][c] = dr->dir_a[((size_t)k * dr->n_mats + m) * 3 + c];
    return a;
}
/* Emitted radiance Le = e * (1, 1, 1). */
static dc mat_emission(const or_scene* s, int64_t m, const dirs_t* dr) {
    double e = s->mats[m].emission;
    dc r = dc_const(e, e, e);
    for (int k = 0; k < dr->nd; ++k)
        for (int c = 0; c < 3; ++c) r.d[k][c] = dr->dir_e[(size_t)k * dr->n_mats + m];
    return r;
}

/* ------------------------------------------------------------------ BSDFs */
/* Orthonormal basis around a unit normal: the branch-free construction of Duff et al.
 * ("Building an Orthonormal Basis, Revisited", JCGT 2017), applied in a fixed rotated frame.
 * The construction switches between two bases where the normal's z crosses 0; every tangent
 * field on the sphere is discontinuous somewhere, and here the switch is moved off the coordinate
 * planes (where floors and walls put their normals) by building the basis for R n and rotating it
 * back.  R = Rodrigues rotation about (1, 2, 3) / sqrt(14) by 1 radian. */
static double g_onb_R[3][3];

__attribute__((constructor)) static void init_onb_frame(void) {
    double k[3] = {1.0, 2.0, 3.0}, l = sqrt(14.0), c = cos(1.0), sn = sin(1.0);
    for (int i = 0; i < 3; ++i) k[i] /= l;
    double K[3][3] = {{0.0, -k[2], k[1]}, {k[2], 0.0, -k[0]}, {-k[1], k[0], 0.0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) g_onb_R[i][j] = (i == j ? c : 0.0) + sn * K[i][j] + (1.0 - c) * k[i] * k[j];
}

static v3 rot(v3 a) {   /* R a */
    return mk(g_onb_R[0][0] * a.x + g_onb_R[0][1] * a.y + g_onb_R[0][2] * a.z,
              g_onb_R[1][0] * a.x + g_onb_R[1][1] * a.y + g_onb_R[1][2] * a.z,
              g_onb_R[2][0] * a.x + g_onb_R[2][1] * a.y + g_onb_R[2][2] * a.z);
}
static v3 rot_t(v3 a) { /* R^T a */
    return mk(g_onb_R[0][0] * a.x + g_onb_R[1][0] * a.y + g_onb_R[2][0] * a.z,
              g_onb_R[0][1] * a.x + g_onb_R[1][1] * a.y + g_onb_R[2][1] * a.z,
              g_onb_R[0][2] * a.x + g_onb_R[1][2] * a.y + g_onb_R[2][2] * a.z);
}

static void onb(v3 n, v3* t, v3* b) {
    v3 m = rot(n);
    double sign = copysign(1.0, m.z);
    double a = -1.0 / (sign + m.z);
    double bb = m.x * m.y * a;
    *t = rot_t(mk(1.0 + sign * m.x * m.x * a, sign * bb, -sign * m.x));
    *b = rot_t(mk(bb, sign + m.y * m.y * a, -m.y));
}

static double ggx_alpha(double roughness) {
    double a = roughness * roughness;
    return a < 1e-4 ? 1e-4 : a;
}
/* Trowbridge-Reitz (GGX) normal distribution, cos_h = n.h. */
static double ggx_D(double alpha, double cos_h) {
    double a2 = alpha * alpha;
    double den = cos_h * cos_h * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * den * den);
}
/* Smith Lambda for GGX, cos_v = n.v > 0. */
static double ggx_lambda(double alpha, double cos_v) {
    double c2 = cos_v * cos_v;
    double tan2 = (1.0 - c2) / c2;
    return 0.5 * (-1.0 + sqrt(1.0 + alpha * alpha * tan2));
}
/* Schlick Fresnel with F0 = albedo, as a dual colour (linear in albedo). */
static dc schlick(dc f0, double cos_t, int nd) {
    double m = 1.0 - cos_t;
    double m5 = m * m * m * m * m;
    dc r;
    for (int c = 0; c < 3; ++c) r.v[c] = f0.v[c] + (1.0 - f0.v[c]) * m5;
    for (int k = 0; k < nd; ++k)
        for (int c = 0; c < 3; ++c) r.d[k][c] = f0.d[k][c] * (1.0 - m5);
    return r;
}

/* BSDF value f(wo, wi) for the non-delta materials; n faces wo.  Zero unless both directions
 * lie on n's side (both are reflection-only). */
static dc bsdf_eval(const omat* m, dc a, v3 n, v3 wo, v3 wi, int nd) {
    double co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0 || ci <= 0.0 || m->type == OR_MAT_DIELECTRIC) return dc_const(0, 0, 0);
    if (m->type == OR_MAT_LAMBERT) return dc_scale(a, 1.0 / OR_PI, nd);
    double alpha = ggx_alpha(m->roughness);
    v3 h = nrm(add(wo, wi));
    double D = ggx_D(alpha, dot(n, h));
    double G2 = 1.0 / (1.0 + ggx_lambda(alpha, co) + ggx_lambda(alpha, ci));
    dc F = schlick(a, dot(wi, h), nd);
    return dc_scale(F, D * G2 / (4.0 * co * ci), nd);
}

/* Solid-angle density with which bsdf_sample draws wi (non-delta materials; n faces wo), for the
 * multiple-importance weights:
 *   Lambert: cos(n, wi) / pi (cosine-weighted hemisphere);
 *   GGX: the visible-normal density D_wo(h) = G1(wo) max(0, wo.h) D(h) / (n.wo) (Heitz 2018) times
 *   the Jacobian 1 / (4 wo.h) of wi = reflect(wo, h):  G1(wo) D(h) / (4 n.wo). */
static double bsdf_pdf(const omat* m, v3 n, v3 wo, v3 wi) {
    double co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0 || ci <= 0.0 || m->type == OR_MAT_DIELECTRIC) return 0.0;
    if (m->type == OR_MAT_LAMBERT) return ci / OR_PI;
    double alpha = ggx_alpha(m->roughness);
    v3 h = nrm(add(wo, wi));
    double g1 = 1.0 / (1.0 + ggx_lambda(alpha, co));
    return g1 * ggx_D(alpha, dot(n, h)) / (4.0 * co);
}

/* Power heuristic with exponent 2 (Veach, "Robust Monte Carlo Methods for Light Transport
 * Simulation", 1997): weight of the strategy with density pa against pb. */
static double power_heuristic(double pa, double pb) {
    double a2 = pa * pa, b2 = pb * pb;
    return a2 + b2 > 0.0 ? a2 / (a2 + b2) : 0.0;
}

/* Visible-normal sample of GGX in the local frame (n = +z), from the construction of Heitz,
 * "Sampling the GGX Distribution of Visible Normals", JCGT 2018: stretch the view vector to the
 * hemisphere configuration, sample a point on the projected disk (warped toward the visible
 * half), lift it to the hemisphere and unstretch. */
static v3 ggx_vndf(v3 wo, double alpha, double u1, double u2) {
    v3 vh = nrm(mk(alpha * wo.x, alpha * wo.y, wo.z));
    double lensq = vh.x * vh.x + vh.y * vh.y;
    v3 T1 = lensq > 0.0 ? scl(mk(-vh.y, vh.x, 0.0), 1.0 / sqrt(lensq)) : mk(1.0, 0.0, 0.0);
    v3 T2 = cross(vh, T1);
    double r = sqrt(u1), phi = 2.0 * OR_PI * u2;
    double t1 = r * cos(phi), t2 = r * sin(phi);
    double sh = 0.5 * (1.0 + vh.z);
    t2 = (1.0 - sh) * sqrt(1.0 - t1 * t1) + sh * t2;
    double tz = 1.0 - t1 * t1 - t2 * t2;
    v3 nh = add(add(scl(T1, t1), scl(T2, t2)), scl(vh, sqrt(tz > 0.0 ? tz : 0.0)));
    return nrm(mk(alpha * nh.x, alpha * nh.y, nh.z > 0.0 ? nh.z : 0.0));
}

/* Exact unpolarised Fresnel reflectance of a smooth dielectric interface; ci = cos of the
 * incident angle (> 0).  Returns 1 on total internal reflection; *ct = cos of transmission. */
static double fresnel_dielectric(double ci, double eta_i, double eta_t, double* ct_out) {
    double eta = eta_i / eta_t;
    double s2 = eta * eta * (1.0 - ci * ci);
    if (s2 >= 1.0) { *ct_out = 0.0; return 1.0; }
    double ct = sqrt(1.0 - s2);
    double rs = (eta_i * ci - eta_t * ct) / (eta_i * ci + eta_t * ct);
    double rp = (eta_t * ci - eta_i * ct) / (eta_t * ci + eta_i * ct);
    *ct_out = ct;
    return 0.5 * (rs * rs + rp * rp);
}

/* BSDF sampling outcome codes (also folded into the branch signature). */
enum { S_LAMBERT = 0, S_GGX = 1, S_GGX_INVALID = 2, S_REFLECT = 3, S_REFRACT = 4, S_TIR = 5 };

typedef struct {
    v3 wi;
    dc weight;    /* f |cos| / pdf */
    int valid;
    int delta;
    int side;     /* +1: leaves on n's side, -1: transmitted */
    int code;
} bsample;

/* Sample a direction.  n faces wo; ng is the winding normal (for dielectric orientation). */
static bsample bsdf_sample(const omat* m, dc a, v3 n, v3 ng, v3 wo, double u5, double u6, double u7, int nd) {
    bsample r;
    memset(&r, 0, sizeof(r));
    r.valid = 1; r.side = 1;
    if (m->type == OR_MAT_LAMBERT) {
        v3 t, b;
        onb(n, &t, &b);
        double rr = sqrt(u6), phi = 2.0 * OR_PI * u7, z = 1.0 - u6;
        r.wi = add(add(scl(t, rr * cos(phi)), scl(b, rr * sin(phi))), scl(n, sqrt(z > 0.0 ? z : 0.0)));
        r.weight = a;                        /* (a/pi) cos / (cos/pi) */
        r.code = S_LAMBERT;
        return r;
    }
    if (m->type == OR_MAT_GGX) {
        v3 t, b;
        onb(n, &t, &b);
        v3 wol = mk(dot(wo, t), dot(wo, b), dot(wo, n));
        double alpha = ggx_alpha(m->roughness);
        v3 ml = ggx_vndf(wol, alpha, u6, u7);
        double c = dot(wol, ml);
        v3 wil = sub(scl(ml, 2.0 * c), wol);
        if (wil.z <= 0.0) { r.valid = 0; r.code = S_GGX_INVALID; r.weight = dc_const(0, 0, 0); return r; }
        r.wi = add(add(scl(t, wil.x), scl(b, wil.y)), scl(n, wil.z));
        double g1 = 1.0 / (1.0 + ggx_lambda(alpha, wol.z));
        double g2 = 1.0 / (1.0 + ggx_lambda(alpha, wol.z) + ggx_lambda(alpha, wil.z));
        r.weight = dc_scale(schlick(a, c, nd), g2 / g1, nd);   /* F G2 / G1(wo) */
        r.code = S_GGX;
        return r;
    }
    /* smooth dielectric */
    double co = dot(wo, ng);
    int entering = co > 0.0;
    double eta_i = entering ? 1.0 : m->ior, eta_t = entering ? m->ior : 1.0;
    double ci = fabs(co), ct;
    double F = fresnel_dielectric(ci, eta_i, eta_t, &ct);
    r.delta = 1;
    if (u5 < F) {
        r.wi = sub(scl(n, 2.0 * ci), wo);
        r.weight = a;
        r.code = F >= 1.0 ? S_TIR : S_REFLECT;
    } else {
        double eta = eta_i / eta_t;
        r.wi = add(scl(wo, -eta), scl(n, eta * ci - ct));
        r.weight = dc_scale(a, eta * eta, nd);
        r.side = -1;
        r.code = S_REFRACT;
    }
    return r;
}

/* Test exports for the BSDF pins (FP64, nd = 0). */
void or_bsdf_eval(uint32_t type, const double* albedo, double roughness, const double* n, const double* wo,
                  const double* wi, double* f_out) {
    omat m; memset(&m, 0, sizeof(m));
    m.type = type; m.roughness = roughness; m.ior = 1.5;
    dc a = dc_const(albedo[0], albedo[1], albedo[2]);
    dc f = bsdf_eval(&m, a, mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), 0);
    for (int c = 0; c < 3; ++c) f_out[c] = f.v[c];
}

int or_bsdf_sample(uint32_t type, const double* albedo, double roughness, double ior, const double* n,
                   const double* ng, const double* wo, double u5, double u6, double u7, double* wi_out,
                   double* weight_out, int32_t* code_out) {
    omat m; memset(&m, 0, sizeof(m));
    m.type = type; m.roughness = roughness; m.ior = ior;
    dc a = dc_const(albedo[0], albedo[1], albedo[2]);
    bsample s = bsdf_sample(&m, a, mk(n[0], n[1], n[2]), mk(ng[0], ng[1], ng[2]), mk(wo[0], wo[1], wo[2]), u5, u6, u7, 0);
    wi_out[0] = s.wi.x; wi_out[1] = s.wi.y; wi_out[2] = s.wi.z;
    for (int c = 0; c < 3; ++c) weight_out[c] = s.weight.v[c];
    *code_out = s.code;
    return s.valid;
}

double or_bsdf_pdf(uint32_t type, double roughness, const double* n, const double* wo, const double* wi) {
    omat m; memset(&m, 0, sizeof(m));
    m.type = type; m.roughness = roughness; m.ior = 1.5;
    return bsdf_pdf(&m, mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]));
}

void or_onb(const double* n, double* t, double* b) {
    v3 tt, bb;
    onb(mk(n[0], n[1], n[2]), &tt, &bb);
    t[0] = tt.x; t[1] = tt.y; t[2] = tt.z;
    b[0] = bb.x; b[1] = bb.y; b[2] = bb.z;
}

double or_fresnel_dielectric(double ci, double eta_i, double eta_t) {
    double ct;
    return fresnel_dielectric(ci, eta_i, eta_t, &ct);
}

double or_ggx_D(double roughness, double cos_h) { return ggx_D(ggx_alpha(roughness), cos_h); }
double or_ggx_G1(double roughness, double cos_v) { return 1.0 / (1.0 + ggx_lambda(ggx_alpha(roughness), cos_v)); }

/* ------------------------------------------------------------------ the estimator */
typedef struct {
    uint32_t max_depth;
    uint32_t rr_start;
    double rr_fixed;     /* > 0: fixed survival probability; else clamp(max(tp), 0.05, 0.95) */
    int use_bvh;
    int mis;             /* combine NEE and BSDF-sampled light hits with the power heuristic */
} ropts;

/* Option bits of the exported render calls. */
#define OR_OPT_HALTON 1u
#define OR_OPT_MIS 2u

/* Optional per-path event log (testing aid): up to OR_MAX_EVENTS events of (bounce << 4 | kind,
 * value) with two diagnostic numbers each. */
#define OR_MAX_EVENTS 64
typedef struct {
    uint32_t* ev;      /* OR_MAX_EVENTS x 2 */
    double* pay;       /* OR_MAX_EVENTS x 2 */
    uint32_t n;
} evlog;

static void log_event(evlog* lg, uint32_t b, uint32_t kind, uint32_t value, double f0, double f1) {
    if (!lg || lg->n >= OR_MAX_EVENTS) return;
    lg->ev[2 * lg->n] = (b << 4) | kind;
    lg->ev[2 * lg->n + 1] = value;
    lg->pay[2 * lg->n] = f0;
    lg->pay[2 * lg->n + 1] = f1;
    lg->n++;
}

/* Branch signature: XOR over the path's events of hash(hash((bounce << 4) | kind) ^ value), so the
 * order in which a pipeline learns the events does not matter.  kind 0: hit triangle id (miss:
 * 0xFFFFFFFF); 1: NEE (light index << 2 | shadow ray cast << 1 | visible); 2: BSDF outcome code;
 * 3: Russian roulette survival. */
static uint32_t sig_event(uint32_t bounce, uint32_t kind, uint32_t value) {
    return or_pcg_hash(or_pcg_hash((bounce << 4) | kind) ^ value);
}

/* Light index j with cdf[j-1] <= u < cdf[j] (first entry whose inclusive cdf exceeds u). */
static int64_t pick_light(const or_scene* s, double u) {
    int64_t lo = 0, hi = s->n_lights - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (s->light_cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* The light-pick step on its own: out[i] = light index drawn by uniform u[i]. */
void or_pick_light_batch(const or_scene* s, const double* u, int64_t n, int64_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = s->n_lights > 0 ? pick_light(s, u[i]) : -1;
}

/* Triangle id of each light, in light-index order (n_lights entries). */
void or_scene_light_tris(const or_scene* s, int64_t* out) {
    for (int64_t j = 0; j < s->n_lights; ++j) out[j] = s->light_tri[j];
}

/* One path from ray (o, d).  Adds radiance into L (dual), counts rays, writes the branch
 * signature.  Follows the steps of Sec. 2.2 with NEE (Sec. 3) and Russian roulette (Sec. 3.1). */
static void trace(const or_scene* s, v3 o, v3 d, uint32_t key, const ropts* op, const dirs_t* dr,
                  dc* L_out, uint32_t* sig_out, uint64_t rays[2], evlog* lg) {
    int nd = dr->nd;
    dc tp = dc_const(1, 1, 1), L = dc_const(0, 0, 0);
    int prev_delta = 1;
    double prev_pdf = 0.0;   /* solid-angle density of the BSDF sample that produced the ray */
    uint32_t sig = 0u;
    for (uint32_t b = 0; b < op->max_depth; ++b) {
        /* step 2: extend the path to the next scattering point */
        double t, hu, hv;
        rays[0]++;
        int64_t tri = closest_hit(s, o, d, op->use_bvh, &t, &hu, &hv);
        if (tri < 0) {
            L = dc_add(L, dc_mul(tp, dc_const(s->env[0], s->env[1], s->env[2]), nd), nd);
            sig ^= sig_event(b, 0, 0xFFFFFFFFu);
            log_event(lg, b, 0, 0xFFFFFFFFu, INFINITY, tp.v[0]);
            break;
        }
        sig ^= sig_event(b, 0, (uint32_t)tri);
        log_event(lg, b, 0, (uint32_t)tri, t, tp.v[0]);
        v3 ng = nrm(cross(sub(s->p1[tri], s->p0[tri]), sub(s->p2[tri], s->p0[tri])));
        v3 x = add(o, scl(d, t));
        int64_t mi = s->mat[tri];
        const omat* m = &s->mats[mi];
        int front = dot(d, ng) < 0.0;
        /* step 3: accumulate emitted radiance.  A listed light hit by a BSDF sample after a
         * non-delta vertex is left to NEE, or with MIS weighted against the density with which NEE
         * would have drawn this point: (1 / total light area) * t^2 / cos at the light. */
        if (front && (!s->is_light[tri] || b == 0 || prev_delta))
            L = dc_add(L, dc_mul(tp, mat_emission(s, mi, dr), nd), nd);
        else if (front && op->mis) {
            double p_light = t * t / (-dot(d, ng) * s->light_area);
            double w = power_heuristic(prev_pdf, p_light);
            L = dc_add(L, dc_scale(dc_mul(tp, mat_emission(s, mi, dr), nd), w, nd), nd);
        }
        if (b + 1 == op->max_depth) break;
        v3 wo = scl(d, -1.0);
        v3 n = front ? ng : scl(ng, -1.0);
        double mx = fabs(x.x);
        if (fabs(x.y) > mx) mx = fabs(x.y);
        if (fabs(x.z) > mx) mx = fabs(x.z);
        double eps = 1e-4 * (mx > 1.0 ? mx : 1.0);
        dc a = mat_albedo(s, mi, dr);
        /* shadow evaluation: next-event estimation toward an area-sampled light point */
        if (m->type != OR_MAT_DIELECTRIC && s->n_lights > 0) {
            int64_t j = pick_light(s, or_u01(key, b, D_LIGHT));
            int64_t lt = s->light_tri[j];
            double su = sqrt(or_u01(key, b, D_LU)), u4 = or_u01(key, b, D_LV);
            double b0 = 1.0 - su, b1 = u4 * su, b2 = 1.0 - b0 - b1;
            v3 y = add(add(scl(s->p0[lt], b0), scl(s->p1[lt], b1)), scl(s->p2[lt], b2));
            v3 nl = nrm(cross(sub(s->p1[lt], s->p0[lt]), sub(s->p2[lt], s->p0[lt])));
            v3 os = add(x, scl(n, eps));
            v3 dv = sub(y, os);
            double dist2 = dot(dv, dv), dist = sqrt(dist2);
            v3 wi = scl(dv, 1.0 / dist);
            double cx = dot(n, wi), cl = -dot(wi, nl);
            uint32_t cast = 0, vis = 0;
            if (cx > 0.0 && cl > 0.0) {
                cast = 1;
                rays[1]++;
                /* the shadow ray ends eps off the light surface, on its emitting side, so that the
                 * light's own (coplanar) triangles can never occlude it, at any angle */
                double my = fabs(y.x);
                if (fabs(y.y) > my) my = fabs(y.y);
                if (fabs(y.z) > my) my = fabs(y.z);
                v3 ys = add(y, scl(nl, 1e-4 * (my > 1.0 ? my : 1.0)));
                v3 sv = sub(ys, os);
                double sdist = sqrt(dot(sv, sv));
                vis = !occluded(s, os, scl(sv, 1.0 / sdist), sdist, op->use_bvh);
                if (vis) {
                    dc f = bsdf_eval(m, a, n, wo, wi, nd);
                    double g = cx * cl * s->light_area / dist2;
                    if (op->mis) g *= power_heuristic(dist2 / (cl * s->light_area), bsdf_pdf(m, n, wo, wi));
                    L = dc_add(L, dc_scale(dc_mul(dc_mul(tp, f, nd), mat_emission(s, s->mat[lt], dr), nd), g, nd), nd);
                }
            }
            sig ^= sig_event(b, 1, ((uint32_t)j << 2) | (cast << 1) | vis);
            log_event(lg, b, 1, ((uint32_t)j << 2) | (cast << 1) | vis, cx, cl);
        }
        /* step 4: sample a new direction and update the throughput (Eq. 3) */
        bsample bs = bsdf_sample(m, a, n, ng, wo, or_u01(key, b, D_LOBE), or_u01(key, b, D_DIR0),
                                 or_u01(key, b, D_DIR1), nd);
        sig ^= sig_event(b, 2, (uint32_t)bs.code);
        log_event(lg, b, 2, (uint32_t)bs.code, bs.weight.v[0], bs.wi.x);
        if (!bs.valid) break;
        tp = dc_mul(tp, bs.weight, nd);
        prev_delta = bs.delta;
        prev_pdf = bs.delta ? 0.0 : bsdf_pdf(m, n, wo, bs.wi);
        if (b >= op->rr_start) {
            double q;
            if (op->rr_fixed > 0.0) q = op->rr_fixed;
            else {
                q = tp.v[0];
                if (tp.v[1] > q) q = tp.v[1];
                if (tp.v[2] > q) q = tp.v[2];
                q = q < 0.05 ? 0.05 : (q > 0.95 ? 0.95 : q);
            }
            int survive = or_u01(key, b, D_RR) < q;
            sig ^= sig_event(b, 3, (uint32_t)survive);
            log_event(lg, b, 3, (uint32_t)survive, q, or_u01(key, b, D_RR));
            if (!survive) break;
            tp = dc_scale(tp, 1.0 / q, nd);
        }
        o = add(x, scl(n, eps * (double)bs.side));
        d = bs.wi;
    }
    *L_out = L;
    *sig_out = sig;
}

typedef struct {
    v3 eye, u, v, w;
    double th, tw;
    uint32_t W, H;
} ocam;

static ocam make_cam(const float* eye, const float* target, const float* up, float vfov_deg, uint32_t W, uint32_t H) {
    ocam c;
    c.eye = mk(eye[0], eye[1], eye[2]);
    c.w = nrm(sub(c.eye, mk(target[0], target[1], target[2])));
    c.u = nrm(cross(mk(up[0], up[1], up[2]), c.w));
    c.v = cross(c.w, c.u);
    c.th = tan((double)vfov_deg * OR_PI / 360.0);
    c.tw = c.th * (double)W / (double)H;
    c.W = W; c.H = H;
    return c;
}

/* Step 1: camera ray through (x + u0, y + u1) of a pinhole camera; y = 0 is the top row. */
static void camera_ray(const ocam* c, uint32_t pixel, double u0, double u1, v3* o, v3* d) {
    uint32_t x = pixel % c->W, y = pixel / c->W;
    double sx = ((double)x + u0) / (double)c->W;
    double sy = ((double)y + u1) / (double)c->H;
    *o = c->eye;
    *d = nrm(sub(add(scl(c->u, (2.0 * sx - 1.0) * c->tw), scl(c->v, (1.0 - 2.0 * sy) * c->th)), c->w));
}

/* The ray-generation step on its own, for explicit (pixel, u0, u1): o_out, d_out are n x 3. */
void or_camera_rays(const float* eye, const float* target, const float* up, float vfov_deg, uint32_t W, uint32_t H,
                    const uint32_t* pixel, const double* u0, const double* u1, int64_t n, double* o_out,
                    double* d_out) {
    ocam cam = make_cam(eye, target, up, vfov_deg, W, H);
    for (int64_t i = 0; i < n; ++i) {
        v3 o, d;
        camera_ray(&cam, pixel[i], u0[i], u1[i], &o, &d);
        o_out[3 * i] = o.x; o_out[3 * i + 1] = o.y; o_out[3 * i + 2] = o.z;
        d_out[3 * i] = d.x; d_out[3 * i + 1] = d.y; d_out[3 * i + 2] = d.z;
    }
}

static int nthreads(int want) {
#ifdef _OPENMP
    return want > 0 ? want : omp_get_max_threads();
#else
    (void)want;
    return 1;
#endif
}

/* Per-path radiance (and tangents) for the listed path ids (path = pixel * spp + sample). */
void or_render_paths(const or_scene* s, const float* eye, const float* target, const float* up, float vfov_deg,
                     uint32_t W, uint32_t H, uint32_t spp, uint32_t max_depth, uint64_t seed, uint32_t rr_start,
                     double rr_fixed, uint32_t opts, int use_bvh, const uint64_t* path_ids, int64_t n, int nd,
                     const double* dir_a, const double* dir_e, int n_threads, double* L_out, double* dL_out,
                     uint32_t* sig_out, uint64_t* rays_out) {
    ocam cam = make_cam(eye, target, up, vfov_deg, W, H);
    ropts op = {max_depth, rr_start, rr_fixed, use_bvh, (opts & OR_OPT_MIS) != 0};
    dirs_t dr = {nd > OR_MAXK ? OR_MAXK : nd, s->n_mats, dir_a, dir_e};
    uint64_t r0 = 0, r1 = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads(n_threads)) reduction(+ : r0, r1)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t pixel = (uint32_t)(path_ids[i] / spp), sample = (uint32_t)(path_ids[i] % spp);
        uint32_t key = or_path_key(seed, pixel, sample);
        double u0, u1;
        pixel_jitter(opts & OR_OPT_HALTON, seed, pixel, sample, key, &u0, &u1);
        v3 o, d;
        camera_ray(&cam, pixel, u0, u1, &o, &d);
        dc L;
        uint32_t sig;
        uint64_t rays[2] = {0, 0};
        trace(s, o, d, key, &op, &dr, &L, &sig, rays, NULL);
        for (int c = 0; c < 3; ++c) L_out[3 * i + c] = L.v[c];
        if (dL_out)
            for (int k = 0; k < dr.nd; ++k)
                for (int c = 0; c < 3; ++c) dL_out[((size_t)i * dr.nd + k) * 3 + c] = L.d[k][c];
        if (sig_out) sig_out[i] = sig;
        r0 += rays[0];
        r1 += rays[1];
    }
    if (rays_out) { rays_out[0] = r0; rays_out[1] = r1; }
}

/* Image of the listed pixels: mean over spp samples, summed in increasing sample order. */
void or_render_pixels(const or_scene* s, const float* eye, const float* target, const float* up, float vfov_deg,
                      uint32_t W, uint32_t H, uint32_t spp, uint32_t max_depth, uint64_t seed, uint32_t rr_start,
                      double rr_fixed, uint32_t opts, int use_bvh, const uint32_t* pixels, int64_t n, int n_threads,
                      double* img_out, uint64_t* rays_out) {
    ocam cam = make_cam(eye, target, up, vfov_deg, W, H);
    ropts op = {max_depth, rr_start, rr_fixed, use_bvh, (opts & OR_OPT_MIS) != 0};
    dirs_t dr = {0, s->n_mats, NULL, NULL};
    uint64_t r0 = 0, r1 = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads(n_threads)) reduction(+ : r0, r1)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0, 0, 0};
        for (uint32_t smp = 0; smp < spp; ++smp) {
            uint32_t key = or_path_key(seed, pixels[i], smp);
            double u0, u1;
            pixel_jitter(opts & OR_OPT_HALTON, seed, pixels[i], smp, key, &u0, &u1);
            v3 o, d;
            camera_ray(&cam, pixels[i], u0, u1, &o, &d);
            dc L;
            uint32_t sig;
            uint64_t rays[2] = {0, 0};
            trace(s, o, d, key, &op, &dr, &L, &sig, rays, NULL);
            for (int c = 0; c < 3; ++c) acc[c] += L.v[c];
            r0 += rays[0];
            r1 += rays[1];
        }
        for (int c = 0; c < 3; ++c) img_out[3 * i + c] = spp > 0 ? acc[c] / (double)spp : 0.0;
    }
    if (rays_out) { rays_out[0] = r0; rays_out[1] = r1; }
}

/* Paths started from explicit rays (closed-form tests): ray i uses path key keys[i]. */
void or_trace_rays(const or_scene* s, const double* o, const double* d, const uint32_t* keys, int64_t n,
                   uint32_t max_depth, uint32_t rr_start, double rr_fixed, uint32_t opts, int use_bvh, int nd,
                   const double* dir_a, const double* dir_e, int n_threads, double* L_out, double* dL_out) {
    ropts op = {max_depth, rr_start, rr_fixed, use_bvh, (opts & OR_OPT_MIS) != 0};
    dirs_t dr = {nd > OR_MAXK ? OR_MAXK : nd, s->n_mats, dir_a, dir_e};
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads(n_threads))
    for (int64_t i = 0; i < n; ++i) {
        dc L;
        uint32_t sig;
        uint64_t rays[2] = {0, 0};
        trace(s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), nrm(mk(d[3 * i], d[3 * i + 1], d[3 * i + 2])), keys[i],
              &op, &dr, &L, &sig, rays, NULL);
        for (int c = 0; c < 3; ++c) L_out[3 * i + c] = L.v[c];
        if (dL_out)
            for (int k = 0; k < dr.nd; ++k)
                for (int c = 0; c < 3; ++c) dL_out[((size_t)i * dr.nd + k) * 3 + c] = L.d[k][c];
    }
}

/* Event logs of the listed paths (testing aid: locate the first decision where two
 * implementations part ways).  ev: n x 64 x 2 u32, pay: n x 64 x 2 f64, n_ev: n. */
void or_trace_path_events(const or_scene* s, const float* eye, const float* target, const float* up, float vfov_deg,
                          uint32_t W, uint32_t H, uint32_t spp, uint32_t max_depth, uint64_t seed, uint32_t rr_start,
                          double rr_fixed, uint32_t opts, const uint64_t* path_ids, int64_t n, uint32_t* ev, double* pay,
                          uint32_t* n_ev, double* L_out) {
    ocam cam = make_cam(eye, target, up, vfov_deg, W, H);
    ropts op = {max_depth, rr_start, rr_fixed, 1, (opts & OR_OPT_MIS) != 0};
    dirs_t dr = {0, s->n_mats, NULL, NULL};
    for (int64_t i = 0; i < n; ++i) {
        uint32_t pixel = (uint32_t)(path_ids[i] / spp), sample = (uint32_t)(path_ids[i] % spp);
        uint32_t key = or_path_key(seed, pixel, sample);
        double u0, u1;
        pixel_jitter(opts & OR_OPT_HALTON, seed, pixel, sample, key, &u0, &u1);
        v3 o, d;
        camera_ray(&cam, pixel, u0, u1, &o, &d);
        evlog lg = {ev + (size_t)i * 2 * OR_MAX_EVENTS, pay + (size_t)i * 2 * OR_MAX_EVENTS, 0};
        dc L;
        uint32_t sig;
        uint64_t rays[2] = {0, 0};
        trace(s, o, d, key, &op, &dr, &L, &sig, rays, &lg);
        n_ev[i] = lg.n;
        for (int c = 0; c < 3; ++c) L_out[3 * i + c] = L.v[c];
    }
}

int or_max_tangents(void) { return OR_MAXK; }
