// pt_device.cuh -- device-side building blocks shared by every kernel of the path tracer:
// vector math, the counter-based random numbers, the pinhole camera, the three BSDFs and the
// shading step of one path vertex.  The megakernel, the wavefront stages, the adjoint and the
// batched kernels all call these same functions, so the two execution orders compute identical
// FP32 values (the wavefront only stores them between kernels).
//
// Paper: "Megakernel vs Wavefront GPU Path Tracing".  Eq. 1-3 (light transport, Monte Carlo,
// path throughput), Sec. 2.2 (the five steps of forward path tracing), Sec. 2.3 (ray generation,
// intersection, shading, accumulation stages), Sec. 3 (shadow evaluation), Sec. 3.1 (Russian
// roulette, compaction).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pt_types.h"

namespace pt {

// ------------------------------------------------------------------ float3 helpers
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
// Dot and cross products with explicit fused multiply-adds.  The kernels are compiled with
// -fmad=false, so the compiler never fuses on its own (which it would do differently per kernel);
// these explicit FMAs are the same instructions in every kernel.
__device__ __forceinline__ float dot(float3 a, float3 b) { return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(__fmaf_rn(a.y, b.z, -(a.z * b.y)), __fmaf_rn(a.z, b.x, -(a.x * b.z)), __fmaf_rn(a.x, b.y, -(a.y * b.x)));
}
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float maxc(float3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }
// Products and sums that cross a kernel boundary in the wavefront are rounded explicitly, so the
// compiler cannot fuse them differently in the megakernel (bitwise-equal images).
__device__ __forceinline__ float3 mul_rn(float3 a, float3 b) {
    return f3(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y), __fmul_rn(a.z, b.z));
}
__device__ __forceinline__ float3 add_rn(float3 a, float3 b) {
    return f3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}

// ------------------------------------------------------------------ random numbers
// PCG hash of one word (Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 2020): one LCG
// step followed by the RXS-M-XS output permutation.
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
// Per-path key from (seed, pixel, sample); uniforms then need one more hash per (bounce, dim).
__device__ __forceinline__ uint32_t path_key(uint64_t seed, uint32_t pixel, uint32_t sample) {
    uint32_t k = pcg_hash((uint32_t)(seed >> 32));
    k = pcg_hash((uint32_t)seed ^ k);
    k = pcg_hash(pixel ^ k);
    return pcg_hash(sample ^ k);
}
// u in [0, 1) on the 2^-24 grid (exact in FP32).
__device__ __forceinline__ float u01(uint32_t key, uint32_t bounce, uint32_t dim) {
    uint32_t h = pcg_hash(key ^ pcg_hash((bounce << 4) | dim));
    return (float)(h >> 8) * 5.9604644775390625e-8f;
}
enum : uint32_t { D_JX = 0, D_JY = 1, D_LIGHT = 2, D_LU = 3, D_LV = 4, D_LOBE = 5, D_DIR0 = 6, D_DIR1 = 7, D_RR = 8 };
enum : uint32_t { SAMPLER_PCG = 0, SAMPLER_HALTON = SAMPLER_HALTON_ID };

// Branch signature event (order-free XOR of per-event hashes; testing aid).
__device__ __forceinline__ uint32_t sig_event(uint32_t bounce, uint32_t kind, uint32_t value) {
    return pcg_hash(pcg_hash((bounce << 4) | kind) ^ value);
}

// ------------------------------------------------------------------ camera (ray generation stage)
// Sub-pixel jitter (Sec. 2.3).  SAMPLER_PCG: the path's uniforms of bounce 0, dims D_JX / D_JY.
// SAMPLER_HALTON: the Halton sequence in bases 2 and 3 over the pixel's sample index, shifted per
// pixel by a Cranley-Patterson rotation modulo 1.  All terms are 24-bit fixed-point fractions, so
// the value is exact in FP32: phi_2(s) is s bit-reversed (top 24 bits); phi_3(s) reverses the 21
// base-3 digits of s into R and takes floor(2^24 R / 3^21); the rotation of dim d is the top 24
// bits of the hash of (seed, pixel, sample 2^32 - 1) for (bounce 0, d).
__device__ __forceinline__ uint32_t halton3_24(uint32_t s) {
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        r = r * 3u + s % 3u;
        s /= 3u;
    }
    return (uint32_t)((r << 24) / 10460353203ull);    // 3^21
}

__device__ __forceinline__ void pixel_jitter(uint32_t sampler, uint64_t seed, uint32_t pixel, uint32_t sample,
                                             uint32_t key, float& u0, float& u1) {
    if (sampler == SAMPLER_HALTON) {
        const uint32_t kp = path_key(seed, pixel, 0xFFFFFFFFu);
        const uint32_t r0 = pcg_hash(kp ^ pcg_hash(D_JX)) >> 8, r1 = pcg_hash(kp ^ pcg_hash(D_JY)) >> 8;
        u0 = (float)(((__brev(sample) >> 8) + r0) & 0xFFFFFFu) * 5.9604644775390625e-8f;
        u1 = (float)((halton3_24(sample) + r1) & 0xFFFFFFu) * 5.9604644775390625e-8f;
    } else {
        u0 = u01(key, 0, D_JX);
        u1 = u01(key, 0, D_JY);
    }
}

// Pinhole ray through (x + u0, y + u1); row 0 at the top (Sec. 2.3 ray generation, Sec. 2.2 step 1).
__device__ __forceinline__ void camera_ray(const DevCamera& c, uint32_t pixel, float u0, float u1, float3& o,
                                           float3& d) {
    uint32_t y = pixel / c.W, x = pixel - y * c.W;
    float sx = ((float)x + u0) / (float)c.W;
    float sy = ((float)y + u1) / (float)c.H;
    float a = 2.0f * sx - 1.0f, b = 1.0f - 2.0f * sy;
    o = f3(c.ex, c.ey, c.ez);
    d = normalize(f3(c.ux, c.uy, c.uz) * a + f3(c.vx, c.vy, c.vz) * b - f3(c.wx, c.wy, c.wz));
}

// ------------------------------------------------------------------ materials and BSDFs
struct MatV {
    uint32_t type;
    float3 albedo;
    float emission;
    float roughness;
    float ior;
};
__device__ __forceinline__ MatV load_mat(const DevMat* mats, uint32_t m) {
    const float4* p = reinterpret_cast<const float4*>(mats + m);
    float4 a = __ldg(p), b = __ldg(p + 1);
    MatV r;
    r.type = __float_as_uint(a.x);
    r.albedo = f3(a.y, a.z, a.w);
    r.emission = b.x;
    r.roughness = b.y;
    r.ior = b.z;
    return r;
}

// Orthonormal basis around a unit normal: the branch-free construction of Duff et al. ("Building an
// Orthonormal Basis, Revisited", JCGT 2017) applied in a fixed rotated frame.  The construction
// switches basis where z crosses 0; building it for R n and rotating back moves that switch off the
// coordinate planes, where scene normals (floors, walls) concentrate, so FP32 rounding of an
// axis-aligned normal cannot flip the sampled direction.  R = Rodrigues rotation about
// (1, 2, 3) / sqrt(14) by 1 radian (entries rounded to FP32).
__device__ __forceinline__ float3 onb_rot(float3 a) {
    return f3(5.731378794e-01f * a.x - 6.090066433e-01f * a.y + 5.482918024e-01f * a.z,
              7.403488159e-01f * a.x + 6.716445088e-01f * a.y - 2.787928283e-02f * a.z,
              -3.512785137e-01f * a.x + 4.219058752e-01f * a.y + 8.358222246e-01f * a.z);
}
__device__ __forceinline__ float3 onb_rot_t(float3 a) {
    return f3(5.731378794e-01f * a.x + 7.403488159e-01f * a.y - 3.512785137e-01f * a.z,
              -6.090066433e-01f * a.x + 6.716445088e-01f * a.y + 4.219058752e-01f * a.z,
              5.482918024e-01f * a.x - 2.787928283e-02f * a.y + 8.358222246e-01f * a.z);
}
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
    float3 m = onb_rot(n);
    float sign = copysignf(1.0f, m.z);
    float a = -1.0f / (sign + m.z);
    float bb = m.x * m.y * a;
    t = onb_rot_t(f3(1.0f + sign * m.x * m.x * a, sign * bb, -sign * m.x));
    b = onb_rot_t(f3(bb, sign + m.y * m.y * a, -m.y));
}

__device__ __forceinline__ float ggx_alpha(float r) { return fmaxf(r * r, 1e-4f); }
// Trowbridge-Reitz normal distribution from cos^2 and sin^2 of the half-vector angle.  The
// denominator cos^2 (a^2 - 1) + 1 is evaluated as cos^2 a^2 + sin^2 with sin^2 from a cross product:
// for sharp lobes (a^2 ~ 1e-5) the first form loses every significant digit in FP32.
__device__ __forceinline__ float ggx_D(float alpha, float cos2_h, float sin2_h) {
    float a2 = alpha * alpha;
    float den = cos2_h * a2 + sin2_h;
    return a2 / (3.14159265358979f * den * den);
}
// Smith Lambda of GGX for cos_v = n.v > 0.
__device__ __forceinline__ float ggx_lambda(float alpha, float cos_v) {
    float c2 = cos_v * cos_v;
    float tan2 = (1.0f - c2) / c2;
    return 0.5f * (-1.0f + sqrtf(1.0f + alpha * alpha * tan2));
}

struct BsdfEval {
    float3 f;      // BSDF value
    float3 dfa;    // d f / d albedo, per channel (f is linear in albedo per channel)
};
// f(wo, wi) of the non-delta materials; n faces wo.  Zero unless both directions are on n's side.
__device__ __forceinline__ BsdfEval bsdf_eval(const MatV& m, float3 n, float3 wo, float3 wi) {
    BsdfEval r;
    r.f = f3(0.f, 0.f, 0.f);
    r.dfa = r.f;
    float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f || m.type == MAT_DIELECTRIC) return r;
    if (m.type == MAT_LAMBERT) {
        const float inv_pi = 0.318309886183791f;
        r.f = m.albedo * inv_pi;
        r.dfa = f3(inv_pi, inv_pi, inv_pi);
        return r;
    }
    float alpha = ggx_alpha(m.roughness);
    float3 h = normalize(wo + wi);
    float ch = dot(n, h);
    float3 nxh = cross(n, h);
    float D = ggx_D(alpha, ch * ch, dot(nxh, nxh));
    float G2 = 1.0f / (1.0f + ggx_lambda(alpha, co) + ggx_lambda(alpha, ci));
    float mm = 1.0f - dot(wi, h);
    float m5 = mm * mm * mm * mm * mm;
    float k = D * G2 / (4.0f * co * ci);
    float3 F = f3(m.albedo.x + (1.0f - m.albedo.x) * m5, m.albedo.y + (1.0f - m.albedo.y) * m5,
                  m.albedo.z + (1.0f - m.albedo.z) * m5);
    r.f = F * k;
    float d1 = (1.0f - m5) * k;
    r.dfa = f3(d1, d1, d1);
    return r;
}

// Solid-angle density with which bsdf_sample draws wi (non-delta materials; n faces wo), for the
// multiple-importance weights: Lambert cos(n, wi) / pi; GGX the visible-normal density
// G1(wo) max(0, wo.h) D(h) / (n.wo) (Heitz 2018) times the reflection Jacobian 1 / (4 wo.h), i.e.
// G1(wo) D(h) / (4 n.wo).
__device__ __forceinline__ float bsdf_pdf(const MatV& m, float3 n, float3 wo, float3 wi) {
    float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f || m.type == MAT_DIELECTRIC) return 0.0f;
    if (m.type == MAT_LAMBERT) return ci * 0.318309886183791f;
    float alpha = ggx_alpha(m.roughness);
    float3 h = normalize(wo + wi);
    float ch = dot(n, h);
    float3 nxh = cross(n, h);
    float g1 = 1.0f / (1.0f + ggx_lambda(alpha, co));
    return g1 * ggx_D(alpha, ch * ch, dot(nxh, nxh)) / (4.0f * co);
}

// Power heuristic with exponent 2 (Veach 1997): weight of the strategy with density pa against pb.
__device__ __forceinline__ float power_heuristic(float pa, float pb) {
    float a2 = pa * pa, b2 = pb * pb;
    return a2 + b2 > 0.0f ? a2 / (a2 + b2) : 0.0f;
}

// Visible-normal sample of GGX in the local frame (n = +z), after Heitz, "Sampling the GGX
// Distribution of Visible Normals" (JCGT 2018): stretch, sample the projected disk warped toward the
// visible half, lift to the hemisphere, unstretch.
__device__ __forceinline__ float3 ggx_vndf(float3 wo, float alpha, float u1, float u2) {
    float3 vh = normalize(f3(alpha * wo.x, alpha * wo.y, wo.z));
    float lensq = vh.x * vh.x + vh.y * vh.y;
    float3 T1 = lensq > 0.0f ? f3(-vh.y, vh.x, 0.0f) * (1.0f / sqrtf(lensq)) : f3(1.0f, 0.0f, 0.0f);
    float3 T2 = cross(vh, T1);
    float r = sqrtf(u1);
    float sp, cp;
    sincosf(6.28318530717959f * u2, &sp, &cp);
    float t1 = r * cp, t2 = r * sp;
    float sh = 0.5f * (1.0f + vh.z);
    t2 = (1.0f - sh) * sqrtf(1.0f - t1 * t1) + sh * t2;
    float tz = 1.0f - t1 * t1 - t2 * t2;
    float3 nh = T1 * t1 + T2 * t2 + vh * sqrtf(fmaxf(tz, 0.0f));
    return normalize(f3(alpha * nh.x, alpha * nh.y, fmaxf(nh.z, 0.0f)));
}

enum : uint32_t { S_LAMBERT = 0, S_GGX = 1, S_GGX_INVALID = 2, S_REFLECT = 3, S_REFRACT = 4, S_TIR = 5 };

struct BsdfSample {
    float3 wi;
    float3 w;      // f |cos| / pdf
    float3 dwa;    // d w / d albedo, per channel
    bool valid;
    bool delta;
    float side;    // +1 leaves on n's side, -1 transmitted
    uint32_t code;
};

// Sample a continuation direction (Sec. 2.2 step 4).  n faces wo; ng is the winding normal.
__device__ __forceinline__ BsdfSample bsdf_sample(const MatV& m, float3 n, float3 ng, float3 wo, float u5,
                                                  float u6, float u7) {
    BsdfSample r;
    r.valid = true;
    r.delta = false;
    r.side = 1.0f;
    if (m.type == MAT_LAMBERT) {
        float3 t, b;
        onb(n, t, b);
        float rr = sqrtf(u6);
        float sp, cp;
        sincosf(6.28318530717959f * u7, &sp, &cp);
        r.wi = t * (rr * cp) + b * (rr * sp) + n * sqrtf(fmaxf(1.0f - u6, 0.0f));
        r.w = m.albedo;                     // (a / pi) cos / (cos / pi)
        r.dwa = f3(1.f, 1.f, 1.f);
        r.code = S_LAMBERT;
        return r;
    }
    if (m.type == MAT_GGX) {
        float3 t, b;
        onb(n, t, b);
        float3 wol = f3(dot(wo, t), dot(wo, b), dot(wo, n));
        float alpha = ggx_alpha(m.roughness);
        float3 ml = ggx_vndf(wol, alpha, u6, u7);
        float c = dot(wol, ml);
        float3 wil = ml * (2.0f * c) - wol;
        if (wil.z <= 0.0f) {
            r.valid = false;
            r.code = S_GGX_INVALID;
            r.w = f3(0.f, 0.f, 0.f);
            r.dwa = r.w;
            r.wi = n;
            return r;
        }
        r.wi = t * wil.x + b * wil.y + n * wil.z;
        float g1 = 1.0f / (1.0f + ggx_lambda(alpha, wol.z));
        float g2 = 1.0f / (1.0f + ggx_lambda(alpha, wol.z) + ggx_lambda(alpha, wil.z));
        float mm = 1.0f - c;
        float m5 = mm * mm * mm * mm * mm;
        float k = g2 / g1;
        float3 F = f3(m.albedo.x + (1.0f - m.albedo.x) * m5, m.albedo.y + (1.0f - m.albedo.y) * m5,
                      m.albedo.z + (1.0f - m.albedo.z) * m5);
        r.w = F * k;                        // F G2 / G1(wo)
        float d1 = (1.0f - m5) * k;
        r.dwa = f3(d1, d1, d1);
        r.code = S_GGX;
        return r;
    }
    // smooth dielectric: exact unpolarised Fresnel, reflect with probability F
    float co = dot(wo, ng);
    bool entering = co > 0.0f;
    float eta_i = entering ? 1.0f : m.ior, eta_t = entering ? m.ior : 1.0f;
    float ci = fabsf(co);
    float eta = eta_i / eta_t;
    float s2 = eta * eta * (1.0f - ci * ci);
    float F, ct = 0.0f;
    if (s2 >= 1.0f) {
        F = 1.0f;
    } else {
        ct = sqrtf(1.0f - s2);
        float rs = (eta_i * ci - eta_t * ct) / (eta_i * ci + eta_t * ct);
        float rp = (eta_t * ci - eta_i * ct) / (eta_t * ci + eta_i * ct);
        F = 0.5f * (rs * rs + rp * rp);
    }
    r.delta = true;
    if (u5 < F) {
        r.wi = n * (2.0f * ci) - wo;
        r.w = m.albedo;
        r.dwa = f3(1.f, 1.f, 1.f);
        r.code = F >= 1.0f ? S_TIR : S_REFLECT;
    } else {
        r.wi = wo * (-eta) + n * (eta * ci - ct);
        float e2 = eta * eta;                  // radiance scale (eta_i / eta_t)^2
        r.w = m.albedo * e2;
        r.dwa = f3(e2, e2, e2);
        r.side = -1.0f;
        r.code = S_REFRACT;
    }
    return r;
}

// ------------------------------------------------------------------ one path vertex
// Everything the shading stage decides at a hit (Sec. 2.2 steps 3-4, Sec. 3 shadow evaluation,
// Sec. 3.1 Russian roulette).  The shadow ray is returned, not traced: the megakernel traces it at
// once, the wavefront appends it to the shadow queue.
struct Vertex {
    uint32_t mat;           // material id of the hit triangle
    uint32_t prim;          // original triangle id
    bool emit_counted;      // emission term added (front face and light-list rule, or MIS)
    float emit_w;           // its weight: 1, or the MIS weight of a BSDF-sampled light hit
    float3 emit;            // tp * Le * emit_w when counted
    bool last;              // b == max_depth - 1: stop after emission
    bool nee;               // an NEE light sample was drawn (non-delta material, lights exist)
    float nee_cx, nee_cl;   // the two cosines that decide whether the shadow ray is cast
    uint32_t light_j;       // light index drawn
    uint32_t light_mat;     // its material
    bool cast;              // shadow ray needed (both cosines positive)
    float3 s_o, s_d;        // shadow ray origin and unit direction
    float s_tmax;           // (1 - 1e-4) * distance
    float3 contrib;         // tp * f * Le_light * G * A  (added if unoccluded)
    float3 nee_g;           // f * G * A (no tp, no Le): for the adjoint
    float3 nee_dfa;         // df/da * G * A * Le_light: for the adjoint
    bool cont;              // the path continues
    uint32_t bsdf_code;
    bool delta;
    float3 w;               // throughput multiplier of this vertex (BSDF weight / q)
    float3 dwa;             // d w / d albedo
    int rr;                 // -1: no roulette at this bounce, 0: killed, 1: survived
    float rr_q;             // survival probability used
    float3 no, nd, ntp;     // continuation ray and throughput
    float pdf;              // solid-angle density of the continuation sample (MIS only; 0 if delta)
};

// Light index with cdf[j-1] <= u < cdf[j] (first entry whose inclusive cdf exceeds u).
__device__ __forceinline__ uint32_t pick_light(const DevScene& s, float u) {
    uint32_t lo = 0, hi = s.n_lights - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(s.light_cdf + mid) > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Shade the hit of ray (o, d) at distance t on reordered triangle `tri`.  MIS = false compiles the
// multiple-importance terms out (the megakernels are instantiated both ways, since the extra code
// costs them registers); with MIS = true they apply when p.mis is set.
template <bool MIS = true, bool INST = false>
__device__ __forceinline__ Vertex shade_vertex(const DevScene& s, const RenderParams& p, uint32_t key, uint32_t b,
                                               float3 o, float3 d, float3 tp, bool prev_delta, float prev_pdf,
                                               float t, uint32_t tri, uint32_t inst = 0xFFFFFFFFu) {
    Vertex V;
    const float4* tr = s.tris + 3 * (size_t)tri;
    float4 t0 = __ldg(tr), t1 = __ldg(tr + 1), t2 = __ldg(tr + 2);
    V.prim = __float_as_uint(t0.w);
    V.mat = __float_as_uint(t1.w);
    bool is_light = __float_as_uint(t2.w) != 0u;
    float3 ng;
    if (INST) {
        // two-level scene: the mesh's object-space edges taken to the world by the instance's
        // rotation/scale rows; the instance may replace the material
        const float4* ip = s.inst + 8 * (size_t)inst;
        const float4 i3 = __ldg(ip + 3), m0 = __ldg(ip + 4), m1 = __ldg(ip + 5), m2 = __ldg(ip + 6);
        const float3 e1 = xyz(t1), e2 = xyz(t2);
        const float3 E1 = f3(dot(xyz(m0), e1), dot(xyz(m1), e1), dot(xyz(m2), e1));
        const float3 E2 = f3(dot(xyz(m0), e2), dot(xyz(m1), e2), dot(xyz(m2), e2));
        ng = normalize(cross(E1, E2));
        V.prim += __float_as_uint(i3.y);
        const uint32_t mw = __float_as_uint(i3.z);
        if (mw != 0u) {
            V.mat = (mw & 0x7FFFFFFFu) - 1u;
            is_light = (mw >> 31) != 0u;
        }
    } else {
        ng = normalize(cross(xyz(t1), xyz(t2)));
    }
    float3 x = o + d * t;
    MatV m = load_mat(s.mats, V.mat);
    bool front = dot(d, ng) < 0.0f;
    // step 3: accumulate emitted radiance (listed lights only at bounce 0 or after a delta bounce;
    // with MIS, also after a non-delta bounce, weighted against the density with which NEE would
    // have drawn this point: (1 / total light area) * t^2 / cos at the light)
    V.emit_counted = front && (!is_light || b == 0 || prev_delta);
    V.emit_w = 1.0f;
    if (MIS && !V.emit_counted && front && p.mis) {
        V.emit_counted = true;
        V.emit_w = power_heuristic(prev_pdf, t * t / (-dot(d, ng) * s.light_area));
    }
    const float Le_w = m.emission * V.emit_w;
    V.emit = V.emit_counted ? mul_rn(tp, f3(Le_w, Le_w, Le_w)) : f3(0.f, 0.f, 0.f);
    V.pdf = 0.0f;
    V.last = (b + 1 == p.max_depth);
    V.nee = false;
    V.cast = false;
    V.cont = false;
    V.rr = -1;
    V.rr_q = 0.f;
    V.nee_cx = 0.f;
    V.nee_cl = 0.f;
    V.light_j = 0;
    V.light_mat = 0;
    V.nee_g = f3(0.f, 0.f, 0.f);
    V.nee_dfa = V.nee_g;
    V.contrib = V.nee_g;
    V.w = V.nee_g;
    V.dwa = V.nee_g;
    V.delta = false;
    V.bsdf_code = 0;
    if (V.last) return V;
    float3 wo = -d;
    float3 n = front ? ng : -ng;
    float mx = fmaxf(fabsf(x.x), fmaxf(fabsf(x.y), fabsf(x.z)));
    float eps = 1e-4f * fmaxf(mx, 1.0f);
    // shadow evaluation: next-event estimation toward an area-sampled light point
    if (m.type != MAT_DIELECTRIC && s.n_lights > 0) {
        V.nee = true;
        uint32_t j = pick_light(s, u01(key, b, D_LIGHT));
        V.light_j = j;
        const float4* lp = s.lights + 3 * (size_t)j;
        float4 l0 = __ldg(lp), l1 = __ldg(lp + 1), l2 = __ldg(lp + 2);
        V.light_mat = __float_as_uint(l0.w);
        float su = sqrtf(u01(key, b, D_LU)), u4 = u01(key, b, D_LV);
        float b0 = 1.0f - su, b1 = u4 * su, b2 = 1.0f - b0 - b1;
        float3 P0 = xyz(l0), P1 = xyz(l1), P2 = xyz(l2);
        float3 y = P0 * b0 + P1 * b1 + P2 * b2;
        float3 nl = normalize(cross(P1 - P0, P2 - P0));
        float3 os = x + n * eps;
        float3 dv = y - os;
        float dist2 = dot(dv, dv), dist = sqrtf(dist2);
        float3 wi = dv * (1.0f / dist);
        float cx = dot(n, wi), cl = -dot(wi, nl);
        V.nee_cx = cx;
        V.nee_cl = cl;
        if (cx > 0.0f && cl > 0.0f) {
            V.cast = true;
            BsdfEval fe = bsdf_eval(m, n, wo, wi);
            float g = cx * cl * s.light_area / dist2;
            if (MIS && p.mis) g = g * power_heuristic(dist2 / (cl * s.light_area), bsdf_pdf(m, n, wo, wi));
            MatV lm = load_mat(s.mats, V.light_mat);
            float3 Le = f3(lm.emission, lm.emission, lm.emission);
            V.nee_g = fe.f * g;
            V.nee_dfa = fe.dfa * g * lm.emission;
            V.contrib = mul_rn(mul_rn(tp, V.nee_g), Le);
            // the shadow ray ends eps off the light surface on its emitting side: the light's own
            // coplanar triangles cannot occlude it, even at grazing angles
            float my = fmaxf(fabsf(y.x), fmaxf(fabsf(y.y), fabsf(y.z)));
            float3 ys = y + nl * (1e-4f * fmaxf(my, 1.0f));
            float3 sv = ys - os;
            float sdist = sqrtf(dot(sv, sv));
            V.s_o = os;
            V.s_d = sv * (1.0f / sdist);
            V.s_tmax = sdist;
        }
    }
    // step 4: sample a continuation and update the throughput (Eq. 3)
    BsdfSample bs = bsdf_sample(m, n, ng, wo, u01(key, b, D_LOBE), u01(key, b, D_DIR0), u01(key, b, D_DIR1));
    V.bsdf_code = bs.code;
    if (!bs.valid) return V;
    float3 ntp = mul_rn(tp, bs.w);
    V.w = bs.w;
    V.dwa = bs.dwa;
    V.delta = bs.delta;
    if (b >= p.rr_start) {
        float q = p.rr_fixed > 0.0f ? p.rr_fixed : fminf(fmaxf(maxc(ntp), 0.05f), 0.95f);
        V.rr_q = q;
        bool survive = u01(key, b, D_RR) < q;
        V.rr = survive ? 1 : 0;
        if (!survive) return V;
        ntp = f3(__fdiv_rn(ntp.x, q), __fdiv_rn(ntp.y, q), __fdiv_rn(ntp.z, q));
        V.w = f3(__fdiv_rn(V.w.x, q), __fdiv_rn(V.w.y, q), __fdiv_rn(V.w.z, q));
        V.dwa = V.dwa * (1.0f / q);
    }
    V.cont = true;
    V.ntp = ntp;
    V.no = x + n * (eps * bs.side);
    V.nd = bs.wi;
    if (MIS && p.mis && !bs.delta) V.pdf = bsdf_pdf(m, n, wo, bs.wi);
    return V;
}

}  // namespace pt
