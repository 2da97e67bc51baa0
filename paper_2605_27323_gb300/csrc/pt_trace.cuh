// pt_trace.cuh -- BVH traversal (the scene-intersection stage of Sec. 2.3, "extend" of Sec. 2.2
// step 2, and the shadow-evaluation query of Sec. 3), written for CUDA cores: the paper's hardware
// ray queries are not reachable here, so traversal is a software loop over a host-built binary
// BVH.
//
// Node layout (64 bytes, one 128-bit load per row, both children's boxes in the parent):
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (ref0, ref1, -, -)     ref: internal node index, or 0x80000000 | first << 3 | (count - 1)
// Triangle record (48 bytes): (v0.xyz, prim id) (e1 = v1 - v0, material) (e2 = v2 - v0, is_light).
//
// Closest hit: Moller-Trumbore with inclusive barycentric bounds and t > 0; equal t goes to the
// lower original triangle id, so the result does not depend on traversal order.  Box tests are
// conservative (the far distance is widened by a few ulps) so rounding cannot cull a true hit.
#pragma once
#include "pt_device.cuh"

namespace pt {

constexpr int kStack = 64;                   // the builder caps tree depth below this
constexpr uint32_t kMaxSteps = 1u << 22;     // traversal step cap (fault guard, never reached)
constexpr uint32_t kMiss = 0xFFFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;

struct Hit {
    float t;
    uint32_t tri;    // reordered triangle index, kMiss on miss
};

__device__ __forceinline__ float3 ray_rcp(float3 d) {
    // 1/d with zero components replaced by a tiny signed value: slabs stay finite and NaN-free
    float x = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
    float y = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
    float z = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
    return f3(1.0f / x, 1.0f / y, 1.0f / z);
}

// Slab test of one box against [0, tmax]; returns whether it is hit and the entry distance.
__device__ __forceinline__ bool box_test(float lox, float hix, float loy, float hiy, float loz, float hiz, float3 o,
                                         float3 id, float tmax, float& tn) {
    float x0 = (lox - o.x) * id.x, x1 = (hix - o.x) * id.x;
    float y0 = (loy - o.y) * id.y, y1 = (hiy - o.y) * id.y;
    float z0 = (loz - o.z) * id.z, z1 = (hiz - o.z) * id.z;
    float a = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.0f));
    float b = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
    tn = a;
    return a <= b * 1.0000005f;
}

// Moller-Trumbore test of one triangle record; t in (0, tmax) by the caller's rule.
__device__ __forceinline__ bool tri_test(const float4* __restrict__ tris, uint32_t i, float3 o, float3 d, float& t,
                                         uint32_t& prim) {
    const float4* p = tris + 3 * (size_t)i;
    float4 a = __ldg(p), e1 = __ldg(p + 1), e2 = __ldg(p + 2);
    float3 E1 = xyz(e1), E2 = xyz(e2);
    float3 pv = cross(d, E2);
    float det = dot(E1, pv);
    if (det == 0.0f) return false;
    float inv = 1.0f / det;
    float3 tv = o - xyz(a);
    float u = dot(tv, pv) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    float3 qv = cross(tv, E1);
    float v = dot(d, qv) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    t = dot(E2, qv) * inv;
    prim = __float_as_uint(a.w);
    return true;
}

__device__ __forceinline__ void load_node(const float4* __restrict__ nodes, uint32_t i, float4& n0, float4& n1,
                                          float4& n2, uint2& refs) {
    const float4* p = nodes + 4 * (size_t)i;
    n0 = __ldg(p);
    n1 = __ldg(p + 1);
    n2 = __ldg(p + 2);
    float4 n3 = __ldg(p + 3);
    refs = make_uint2(__float_as_uint(n3.x), __float_as_uint(n3.y));
}

// Closest hit, plain order: one loop that takes a node step or a leaf step per iteration.  The
// wavefront's traversal kernels use it (measured faster there than the while-while order).
__device__ __forceinline__ Hit trace_closest_plain(const DevScene& s, float3 o, float3 d) {
    float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss;
    uint32_t stack_ref[kStack];
    float stack_t[kStack];
    int sp = 0;
    uint32_t ref = 0;          // the root is always an internal node
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, ref, n0, n1, n2, r);
            float t0, t1;
            bool h0 = box_test(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, o, id, tbest, t0);
            bool h1 = box_test(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, o, id, tbest, t1);
            if (h0 && h1) {
                bool first0 = t0 <= t1;
                if (sp < kStack) {
                    stack_ref[sp] = first0 ? r.y : r.x;
                    stack_t[sp] = first0 ? t1 : t0;
                    ++sp;
                } else {
                    atomicOr(s.status, ST_TRAVERSAL);
                }
                ref = first0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t k = 0; k < cnt; ++k) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f &&
                    (t < tbest || (t == tbest && prim < bprim))) {
                    tbest = t;
                    best = first + k;
                    bprim = prim;
                }
            }
        }
        if (steps >= kMaxSteps) {
            atomicOr(s.status, ST_TRAVERSAL);
            break;
        }
        bool found = false;        // pop the next subtree whose entry is not beyond the best hit
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= tbest * 1.0000005f) {
                ref = stack_ref[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
        ++steps;
    }
    Hit h;
    h.t = tbest;
    h.tri = best;
    return h;
}

// Any hit with 0 < t < tmax, plain order.
__device__ __forceinline__ bool trace_any_plain(const DevScene& s, float3 o, float3 d, float tmax) {
    float3 id = ray_rcp(d);
    uint32_t stack_ref[kStack];
    int sp = 0;
    uint32_t ref = 0;
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, ref, n0, n1, n2, r);
            float t0, t1;
            bool h0 = box_test(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, o, id, tmax, t0);
            bool h1 = box_test(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, o, id, tmax, t1);
            if (h0 && h1) {
                if (sp < kStack) stack_ref[sp++] = r.y;
                else atomicOr(s.status, ST_TRAVERSAL);
                ref = r.x;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t k = 0; k < cnt; ++k) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f && t < tmax) return true;
            }
        }
        if (steps >= kMaxSteps) {
            atomicOr(s.status, ST_TRAVERSAL);
            return false;
        }
        if (sp == 0) return false;
        ref = stack_ref[--sp];
        ++steps;
    }
}

constexpr uint32_t kDone = 0x7FFFFFFFu;     // "traversal finished" (no internal node has this index)
constexpr uint32_t kNoLeaf = 0u;            // no postponed leaf (0 is the root, never a leaf ref)

// Closest hit along o + t d, t > 0.  "While-while" order (after Aila & Laine,
// "Understanding the Efficiency of Ray Traversal on GPUs", 2009): each lane walks internal nodes,
// setting aside the first leaf it reaches, until every lane of the warp holds a leaf; then the
// lanes test their leaves together.  Keeping node steps and triangle steps in separate loops keeps
// the warp on one code path; the hit found does not depend on the visiting order (ties on t go to
// the lower triangle id).
__device__ __forceinline__ Hit trace_closest_ww(const DevScene& s, float3 o, float3 d) {
    const float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss;
    uint32_t stack_ref[kStack];
    float stack_t[kStack];
    int sp = 0;
    uint32_t node = 0, leaf = kNoLeaf;
    uint32_t steps = 0;
    auto pop = [&]() -> uint32_t {
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= tbest * 1.0000005f) return stack_ref[sp];
        }
        return kDone;
    };
    while (node != kDone || leaf != kNoLeaf) {
        // walk internal nodes; set aside the first leaf reached
        while (node != kDone && !(node & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, node, n0, n1, n2, r);
            float t0, t1;
            const bool h0 = box_test(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, o, id, tbest, t0);
            const bool h1 = box_test(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, o, id, tbest, t1);
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                if (sp < kStack) {
                    stack_ref[sp] = first0 ? r.y : r.x;
                    stack_t[sp] = first0 ? t1 : t0;
                    ++sp;
                } else {
                    atomicOr(s.status, ST_TRAVERSAL);
                }
                node = first0 ? r.x : r.y;
            } else if (h0 || h1) {
                node = h0 ? r.x : r.y;
            } else {
                node = pop();
            }
            if (node != kDone && (node & kLeafBit) && leaf == kNoLeaf) {
                leaf = node;
                node = pop();
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                node = kDone;
                leaf = kNoLeaf;
            }
            if (!__any_sync(__activemask(), leaf == kNoLeaf)) break;
        }
        // test the set-aside leaf, then any leaves that follow directly
        while (leaf != kNoLeaf) {
            const uint32_t first = (leaf & 0x7FFFFFFFu) >> 3, cnt = (leaf & 7u) + 1u;
            for (uint32_t k = 0; k < cnt; ++k) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f &&
                    (t < tbest || (t == tbest && prim < bprim))) {
                    tbest = t;
                    best = first + k;
                    bprim = prim;
                }
            }
            leaf = kNoLeaf;
            if (node != kDone && (node & kLeafBit)) {
                leaf = node;
                node = pop();
            }
        }
    }
    Hit h;
    h.t = tbest;
    h.tri = best;
    return h;
}

// Any hit with 0 < t < tmax, in the same while-while order; returns at the first hit.
__device__ __forceinline__ bool trace_any_ww(const DevScene& s, float3 o, float3 d, float tmax) {
    const float3 id = ray_rcp(d);
    uint32_t stack_ref[kStack];
    int sp = 0;
    uint32_t node = 0, leaf = kNoLeaf;
    uint32_t steps = 0;
    auto pop = [&]() -> uint32_t { return sp > 0 ? stack_ref[--sp] : kDone; };
    while (node != kDone || leaf != kNoLeaf) {
        while (node != kDone && !(node & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, node, n0, n1, n2, r);
            float t0, t1;
            const bool h0 = box_test(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, o, id, tmax, t0);
            const bool h1 = box_test(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, o, id, tmax, t1);
            if (h0 && h1) {
                if (sp < kStack) stack_ref[sp++] = r.y;
                else atomicOr(s.status, ST_TRAVERSAL);
                node = r.x;
            } else if (h0 || h1) {
                node = h0 ? r.x : r.y;
            } else {
                node = pop();
            }
            if (node != kDone && (node & kLeafBit) && leaf == kNoLeaf) {
                leaf = node;
                node = pop();
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                return false;
            }
            if (!__any_sync(__activemask(), leaf == kNoLeaf)) break;
        }
        while (leaf != kNoLeaf) {
            const uint32_t first = (leaf & 0x7FFFFFFFu) >> 3, cnt = (leaf & 7u) + 1u;
            for (uint32_t k = 0; k < cnt; ++k) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f && t < tmax) return true;
            }
            leaf = kNoLeaf;
            if (node != kDone && (node & kLeafBit)) {
                leaf = node;
                node = pop();
            }
        }
    }
    return false;
}

// The extend and shadow queries.  WW selects the while-while order (used by the one-thread-per-path
// kernels, where it also lowers register pressure) or the plain loop (used by the wavefront stages).
template <bool WW>
__device__ __forceinline__ Hit trace_closest(const DevScene& s, float3 o, float3 d) {
    return WW ? trace_closest_ww(s, o, d) : trace_closest_plain(s, o, d);
}
template <bool WW>
__device__ __forceinline__ bool trace_any(const DevScene& s, float3 o, float3 d, float tmax) {
    return WW ? trace_any_ww(s, o, d, tmax) : trace_any_plain(s, o, d, tmax);
}

}  // namespace pt
