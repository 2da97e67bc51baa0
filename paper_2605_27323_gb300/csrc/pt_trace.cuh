// pt_trace.cuh -- BVH traversal (the scene-intersection stage of Sec. 2.3, "extend" of Sec. 2.2
// step 2, and the shadow-evaluation query of Sec. 3), written for CUDA cores: the paper's hardware
// ray queries are not reachable here, so traversal is a software loop over a host-built binary
// BVH -- one over all triangles, or (two-level scenes, the paper's TLAS/BLAS structure of Sec. 2.3)
// one over instances whose leaves lead into per-mesh BVHs.
//
// Node layout (64 bytes, one 128-bit load per row, both children's boxes in the parent; each axis
// row pairs the two children so that one packed FP32 operation serves both):
//   n0 = (c0.lo.x, c1.lo.x, c0.hi.x, c1.hi.x)
//   n1 = (c0.lo.y, c1.lo.y, c0.hi.y, c1.hi.y)
//   n2 = (c0.lo.z, c1.lo.z, c0.hi.z, c1.hi.z)
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
    uint32_t prim;   // original triangle id (two-level scenes: the instance's first id + the mesh's)
    uint32_t inst;   // instance (top-level leaf order) of a two-level scene, kMiss otherwise
};

__device__ __forceinline__ float3 ray_rcp(float3 d) {
    // 1/d with zero components replaced by a tiny signed value: slabs stay finite and NaN-free
    float x = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
    float y = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
    float z = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
    return f3(__frcp_rn(x), __frcp_rn(y), __frcp_rn(z));   // correctly rounded, as 1.0f / x
}



// Slab test of one box against [0, tmax]: whether it is hit and its entry distance (the largest
// near-plane distance, at least 0); hit when the entry is at most the exit (the smallest far-plane
// distance, at most tmax) widened by a few ulps, so that rounding cannot cull a true hit.
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

// Slab test of a node's two child boxes against [0, tmax]: whether each is hit and its entry distance.
// Rows nx, ny, nz hold (c0.lo, c1.lo, c0.hi, c1.hi) of one axis, so the plane distances
// (plane - o) * (1/d) of both children come from packed FP32 pairs (sub/mul.rn.f32x2: each half
// rounded exactly as the scalar operation); the entry is the largest near-plane distance (at least 0),
// the exit the smallest far-plane distance (at most tmax), and a box counts as hit when entry <= exit
// widened by a few ulps, so that rounding cannot cull a true hit.  PK = false computes the same values
// with box_test, one child at a time (for the register-bound one-thread-per-path kernels' two-level
// walks, where the packed pairs cost spills).
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpk2(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long slab2(float lo0, float lo1, float o, float id) {
    unsigned long long d, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(lo0, lo1)), "l"(pk2(o, o)));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(d), "l"(pk2(id, id)));
    return r;
}
template <bool PK = true>
__device__ __forceinline__ void box_test2(float4 nx, float4 ny, float4 nz, float3 o, float3 id, float tmax,
                                          float& t0, float& t1, bool& h0, bool& h1) {
    if constexpr (!PK) {
        h0 = box_test(nx.x, nx.z, ny.x, ny.z, nz.x, nz.z, o, id, tmax, t0);
        h1 = box_test(nx.y, nx.w, ny.y, ny.w, nz.y, nz.w, o, id, tmax, t1);
        return;
    }
    float xa0, xa1, xb0, xb1, ya0, ya1, yb0, yb1, za0, za1, zb0, zb1;
    unpk2(slab2(nx.x, nx.y, o.x, id.x), xa0, xa1);
    unpk2(slab2(nx.z, nx.w, o.x, id.x), xb0, xb1);
    unpk2(slab2(ny.x, ny.y, o.y, id.y), ya0, ya1);
    unpk2(slab2(ny.z, ny.w, o.y, id.y), yb0, yb1);
    unpk2(slab2(nz.x, nz.y, o.z, id.z), za0, za1);
    unpk2(slab2(nz.z, nz.w, o.z, id.z), zb0, zb1);
    const float a0 = fmaxf(fmaxf(fminf(xa0, xb0), fminf(ya0, yb0)), fmaxf(fminf(za0, zb0), 0.0f));
    const float e0 = fminf(fminf(fmaxf(xa0, xb0), fmaxf(ya0, yb0)), fminf(fmaxf(za0, zb0), tmax));
    const float a1 = fmaxf(fmaxf(fminf(xa1, xb1), fminf(ya1, yb1)), fmaxf(fminf(za1, zb1), 0.0f));
    const float e1 = fminf(fminf(fmaxf(xa1, xb1), fmaxf(ya1, yb1)), fminf(fmaxf(za1, zb1), tmax));
    t0 = a0;
    t1 = a1;
    h0 = a0 <= e0 * 1.0000005f;
    h1 = a1 <= e1 * 1.0000005f;
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

// ------------------------------------------------------------------ traversal stacks
// The stack of deferred subtrees (far child and its entry distance) of the single-level walks.
// LocalStack: kStack entries per thread in local memory (cached by L1), a closest-hit entry's reference
// and distance in one 8-byte word (one 64-bit access per push and per pop).  ShortStack<K>: the top K
// entries per thread in shared memory -- per-warp short stacks, 32 lanes side by side in each slot
// row, so a warp's accesses of one slot hit 32 distinct banks -- and the entries below them in
// local memory: a push onto a full shared slice first moves the slice's bottom entry to local
// memory.  A kernel whose walks use ShortStack<K> is launched with K * 8 * blockDim.x bytes of
// dynamic shared memory (stack_smem_bytes).  Both give the same traversal order, hence the same
// hits.  `T` = false keeps subtree references only (any-hit walks need no distances).
extern __shared__ uint32_t g_stack_smem[];

template <bool T>
struct LocalStack {
    // closest-hit walks: (ref, t) in one 8-byte entry; any-hit walks: references only
    uint2 e[T ? kStack : 1];
    uint32_t ref[T ? 1 : kStack];
    int sp = 0;
    __device__ __forceinline__ bool empty() const { return sp == 0; }
    __device__ __forceinline__ bool push(uint32_t r, float tt) {
        if (sp >= kStack) return false;
        if (T) e[sp] = make_uint2(r, __float_as_uint(tt));
        else ref[sp] = r;
        ++sp;
        return true;
    }
    __device__ __forceinline__ void pop(uint32_t& r, float& tt) {
        const uint2 v = e[--sp];
        r = v.x;
        tt = __uint_as_float(v.y);
    }
    __device__ __forceinline__ uint32_t pop_ref() { return ref[--sp]; }
};

template <int K, bool T>
struct ShortStack {
    static_assert(K > 0 && (K & (K - 1)) == 0, "the shared slice holds a power-of-two number of entries");
    uint32_t lref[kStack];
    float lt[T ? kStack : 1];
    int sp = 0;      // entries on the stack
    int base = 0;    // entries [0, base) in local memory, [base, sp) in shared memory
    __device__ __forceinline__ static uint32_t slot(int i) { return (uint32_t)(i & (K - 1)) * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ static uint32_t tslot(int i) { return slot(i) + (uint32_t)K * blockDim.x; }
    __device__ __forceinline__ bool empty() const { return sp == 0; }
    __device__ __forceinline__ bool push(uint32_t r, float tt) {
        if (sp >= kStack) return false;
        if (sp < base) base = sp;              // popped into the local part: the shared slice is empty
        if (sp - base == K) {                  // the shared slice is full: its bottom entry goes to local
            lref[base] = g_stack_smem[slot(base)];
            if (T) lt[base] = __uint_as_float(g_stack_smem[tslot(base)]);
            ++base;
        }
        g_stack_smem[slot(sp)] = r;
        if (T) g_stack_smem[tslot(sp)] = __float_as_uint(tt);
        ++sp;
        return true;
    }
    __device__ __forceinline__ float pop_t() {
        --sp;
        return sp >= base ? __uint_as_float(g_stack_smem[tslot(sp)]) : lt[sp];
    }
    __device__ __forceinline__ uint32_t top_ref() const { return sp >= base ? g_stack_smem[slot(sp)] : lref[sp]; }
    __device__ __forceinline__ void pop(uint32_t& r, float& tt) {
        tt = pop_t();
        r = top_ref();
    }
    __device__ __forceinline__ uint32_t pop_ref() {
        --sp;
        return sp >= base ? g_stack_smem[slot(sp)] : lref[sp];
    }
};

// Shared-memory short-stack entries per thread of the single-level walks in the kernels that offer
// it (extend, shadow, the regenerating megakernel, the hybrid continuation; PT_FLAG_SHORT_STACK).
// 8 measured fastest of 4, 8 and 16 -- and the local stack faster than all three on GB300 (its top
// entries stay in the 256 KB L1, while the short stack costs registers and L1 capacity).
constexpr int kShortStack = 8;
__host__ __device__ constexpr size_t stack_smem_bytes(int k, int block) { return (size_t)k * 8u * (size_t)block; }

template <int SK, bool T>
struct StackOf {
    using type = ShortStack<SK, T>;
};
template <bool T>
struct StackOf<0, T> {
    using type = LocalStack<T>;
};

// Traversal counters of one thread (the counting instantiations): internal nodes visited and
// triangles tested.  NoCount compiles to nothing.
struct NoCount {
    __device__ __forceinline__ void node() {}
    __device__ __forceinline__ void tri() {}
};
struct TravCount {
    uint32_t nodes = 0, tris = 0;
    __device__ __forceinline__ void node() { ++nodes; }
    __device__ __forceinline__ void tri() { ++tris; }
};

// Closest hit: one loop that takes a node step or a leaf step per iteration.
template <class Stk, class C = NoCount>
__device__ __forceinline__ Hit trace_closest_plain(const DevScene& s, float3 o, float3 d, Stk& stk, C& cnt) {
    float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss;
    uint32_t ref = 0;          // the root is always an internal node
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, ref, n0, n1, n2, r);
            cnt.node();
            float t0, t1;
            bool h0, h1;
            box_test2(n0, n1, n2, o, id, tbest, t0, t1, h0, h1);
            if (h0 && h1) {
                bool first0 = t0 <= t1;
                if (!stk.push(first0 ? r.y : r.x, first0 ? t1 : t0)) atomicOr(s.status, ST_TRAVERSAL);
                ref = first0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, n_leaf = (ref & 7u) + 1u;
            for (uint32_t k = 0; k < n_leaf; ++k) {
                float t;
                uint32_t prim;
                cnt.tri();
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
        while (!stk.empty()) {
            uint32_t r;
            float t;
            stk.pop(r, t);
            if (t <= tbest * 1.0000005f) {
                ref = r;
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
    h.prim = bprim;
    h.inst = kMiss;
    return h;
}

// ------------------------------------------------------------------ cooperative walks
// A trace launch with few walks leaves most of the GPU idle, and it then lasts as long as its
// longest walk: a chain of dependent node loads.  Such a launch gives each ray a group of G lanes
// (an aligned power-of-two group of a warp, G <= 32).  Every lane walks depth first as above and
// defers far children to a ring of kStack entries; a lane left without work takes the oldest entry
// (the deferred subtree nearest the root) of a lane in its group that holds one, so the subtrees of
// one ray are walked side by side.  Boxes are culled against the smallest best distance in the
// group, which is never below the final one, so the culling stays conservative and the result --
// the smallest (t, prim) over the group -- is the hit of the single-lane walk.  An any-hit walk ends
// as soon as one lane of the group finds an occluder.  All 32 lanes of the warp run these loops
// together with the same G (shuffles over the full warp); lanes of a group without a ray pass
// valid = false and stay idle.
struct RingStack {
    uint32_t ref[kStack];
    float t[kStack];
    uint32_t bot = 0, top = 0;     // entries [bot, top), indexed modulo kStack
    __device__ __forceinline__ bool empty() const { return bot == top; }
    __device__ __forceinline__ bool push(uint32_t r, float tt) {
        if (top - bot >= (uint32_t)kStack) return false;
        ref[top & (kStack - 1)] = r;
        t[top & (kStack - 1)] = tt;
        ++top;
        return true;
    }
    // the newest entry (the lane's own depth-first order)
    __device__ __forceinline__ void pop(uint32_t& r, float& tt) {
        --top;
        r = ref[top & (kStack - 1)];
        tt = t[top & (kStack - 1)];
    }
    // the oldest entry, handed to an idle lane
    __device__ __forceinline__ void take_bottom(uint32_t& r, float& tt) {
        r = ref[bot & (kStack - 1)];
        tt = t[bot & (kStack - 1)];
        ++bot;
    }
    __device__ __forceinline__ void clear() { bot = top; }
};
static_assert((kStack & (kStack - 1)) == 0, "the ring indexes modulo kStack");

__device__ __forceinline__ uint32_t group_mask(uint32_t G, uint32_t lane) {
    return G == 32u ? 0xFFFFFFFFu : ((1u << G) - 1u) << (lane & ~(G - 1u));
}
__device__ __forceinline__ float group_min(float v, uint32_t G) {
    for (uint32_t o = G >> 1; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
__device__ __forceinline__ uint32_t group_min(uint32_t v, uint32_t G) {
    for (uint32_t o = G >> 1; o; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// One work-sharing step of a group (mask gm): its idle lanes and the lanes that hold deferred
// entries are paired in lane order, and each paired donor moves its oldest entry to its idle lane,
// which takes it up unless its entry distance is beyond `tcull` (closest-hit walks; any-hit walks
// defer entries at distance 0).  Returns whether the whole group is idle with nothing deferred.
__device__ __forceinline__ bool group_share(uint32_t gm, uint32_t lane, bool& busy, uint32_t& ref, RingStack& rs,
                                            float tcull) {
    const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !busy) & gm;
    const uint32_t donors = __ballot_sync(0xFFFFFFFFu, busy && !rs.empty()) & gm;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t pairs = min((uint32_t)__popc(idle), (uint32_t)__popc(donors));
    uint32_t give_r = 0u;
    float give_t = 0.f;
    if (((donors >> lane) & 1u) && (uint32_t)__popc(donors & below) < pairs) rs.take_bottom(give_r, give_t);
    uint32_t from = lane;
    const uint32_t k = (uint32_t)__popc(idle & below);
    if (((idle >> lane) & 1u) && k < pairs) {
        uint32_t m = donors;                  // the k-th donor, counting from the lowest lane
        for (uint32_t i = 0; i < k; ++i) m &= m - 1u;
        from = (uint32_t)__ffs(m) - 1u;
    }
    const uint32_t got_r = __shfl_sync(0xFFFFFFFFu, give_r, from);
    const float got_t = __shfl_sync(0xFFFFFFFFu, give_t, from);
    if (from != lane && got_t <= tcull * 1.0000005f) {
        busy = true;
        ref = got_r;
    }
    return idle == gm;
}

__device__ __forceinline__ Hit trace_closest_group(const DevScene& s, float3 o, float3 d, bool valid, uint32_t G) {
    const uint32_t lane = threadIdx.x & 31u, gm = group_mask(G, lane);
    const float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss;
    bool busy = valid && (lane & (G - 1u)) == 0u;    // the group's first lane starts at the root
    uint32_t ref = 0u;
    RingStack rs;
    uint32_t steps = 0;
    while (true) {
        const float tg = group_min(tbest, G);
        if (busy) {
            if (!(ref & kLeafBit)) {
                float4 n0, n1, n2;
                uint2 r;
                load_node(s.nodes, ref, n0, n1, n2, r);
                float t0, t1;
                bool h0, h1;
                box_test2(n0, n1, n2, o, id, tg, t0, t1, h0, h1);
                if (h0 && h1) {
                    const bool first0 = t0 <= t1;
                    if (!rs.push(first0 ? r.y : r.x, first0 ? t1 : t0)) atomicOr(s.status, ST_TRAVERSAL);
                    ref = first0 ? r.x : r.y;
                } else if (h0 || h1) {
                    ref = h0 ? r.x : r.y;
                } else {
                    busy = false;
                }
            } else {
                const uint32_t first = (ref & 0x7FFFFFFFu) >> 3, n_leaf = (ref & 7u) + 1u;
                for (uint32_t k = 0; k < n_leaf; ++k) {
                    float t;
                    uint32_t prim;
                    if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f &&
                        (t < tbest || (t == tbest && prim < bprim))) {
                        tbest = t;
                        best = first + k;
                        bprim = prim;
                    }
                }
                busy = false;
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                busy = false;
                rs.clear();
            }
        }
        const float tc = fminf(tg, tbest);
        while (!busy && !rs.empty()) {       // the next own subtree whose entry is not beyond the best hit
            float t;
            rs.pop(ref, t);
            busy = t <= tc * 1.0000005f;
        }
        const bool over = group_share(gm, lane, busy, ref, rs, tc);
        if (__all_sync(0xFFFFFFFFu, over)) break;
    }
    // the group's hit: the smallest t, then the smallest original id among equal t
    Hit h;
    h.t = group_min(tbest, G);
    h.prim = group_min(tbest == h.t ? bprim : kMiss, G);
    const uint32_t own = __ballot_sync(0xFFFFFFFFu, tbest == h.t && bprim == h.prim) & gm;
    h.tri = __shfl_sync(0xFFFFFFFFu, best, own ? (uint32_t)__ffs(own) - 1u : lane);
    h.inst = kMiss;
    return h;
}

__device__ __forceinline__ bool trace_any_group(const DevScene& s, float3 o, float3 d, float tmax, bool valid,
                                                uint32_t G) {
    const uint32_t lane = threadIdx.x & 31u, gm = group_mask(G, lane);
    const float3 id = ray_rcp(d);
    bool busy = valid && (lane & (G - 1u)) == 0u, hit = false;
    uint32_t ref = 0u;
    RingStack rs;
    uint32_t steps = 0;
    while (true) {
        if (busy) {
            if (!(ref & kLeafBit)) {
                float4 n0, n1, n2;
                uint2 r;
                load_node(s.nodes, ref, n0, n1, n2, r);
                float t0, t1;
                bool h0, h1;
                box_test2(n0, n1, n2, o, id, tmax, t0, t1, h0, h1);
                if (h0 && h1) {
                    const bool first0 = t0 <= t1;
                    if (!rs.push(first0 ? r.y : r.x, 0.f)) atomicOr(s.status, ST_TRAVERSAL);
                    ref = first0 ? r.x : r.y;
                } else if (h0 || h1) {
                    ref = h0 ? r.x : r.y;
                } else {
                    busy = false;
                }
            } else {
                const uint32_t first = (ref & 0x7FFFFFFFu) >> 3, n_leaf = (ref & 7u) + 1u;
                for (uint32_t k = 0; k < n_leaf && !hit; ++k) {
                    float t;
                    uint32_t prim;
                    hit = tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f && t < tmax;
                }
                busy = false;
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                busy = false;
                rs.clear();
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, hit) & gm) {      // an occluder anywhere ends the group's walk
            busy = false;
            rs.clear();
        }
        if (!busy && !rs.empty()) {
            float t;
            rs.pop(ref, t);
            busy = true;
        }
        const bool over = group_share(gm, lane, busy, ref, rs, 0.f);
        if (__all_sync(0xFFFFFFFFu, over)) break;
    }
    return (__ballot_sync(0xFFFFFFFFu, hit) & gm) != 0u;
}

// Any hit with 0 < t < tmax.
template <class Stk, class C = NoCount>
__device__ __forceinline__ bool trace_any_plain(const DevScene& s, float3 o, float3 d, float tmax, Stk& stk, C& cnt) {
    float3 id = ray_rcp(d);
    uint32_t ref = 0;
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 r;
            load_node(s.nodes, ref, n0, n1, n2, r);
            cnt.node();
            float t0, t1;
            bool h0, h1;
            box_test2(n0, n1, n2, o, id, tmax, t0, t1, h0, h1);
            if (h0 && h1) {       // nearer child first: an occluder near the origin ends the walk sooner
                const bool first0 = t0 <= t1;
                if (!stk.push(first0 ? r.y : r.x, 0.f)) atomicOr(s.status, ST_TRAVERSAL);
                ref = first0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? r.x : r.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, n_leaf = (ref & 7u) + 1u;
            for (uint32_t k = 0; k < n_leaf; ++k) {
                float t;
                uint32_t prim;
                cnt.tri();
                if (tri_test(s.tris, first + k, o, d, t, prim) && t > 0.0f && t < tmax) return true;
            }
        }
        if (steps >= kMaxSteps) {
            atomicOr(s.status, ST_TRAVERSAL);
            return false;
        }
        if (stk.empty()) return false;
        ref = stk.pop_ref();
        ++steps;
    }
}

// ------------------------------------------------------------------ two-level scenes
// The top-level BVH (same node layout) has instances in its leaves.  A ray entering an instance's
// box is taken to the mesh's object space (o' = A o + b, d' = A d, d' not renormalised, so the
// parameter t is the world one) and walks the mesh's BVH from its root; equal t still goes to the
// lower original triangle id (the instance's first id + the mesh-local id).

struct InstRay {
    float3 o, d;
    uint32_t root, prim_base;
};

__device__ __forceinline__ InstRay instance_ray(const DevScene& s, uint32_t k, float3 o, float3 d) {
    const float4* p = s.inst + 8 * (size_t)k;
    const float4 a0 = __ldg(p), a1 = __ldg(p + 1), a2 = __ldg(p + 2), a3 = __ldg(p + 3);
    InstRay r;
    r.o = f3(__fadd_rn(dot(xyz(a0), o), a0.w), __fadd_rn(dot(xyz(a1), o), a1.w), __fadd_rn(dot(xyz(a2), o), a2.w));
    r.d = f3(dot(xyz(a0), d), dot(xyz(a1), d), dot(xyz(a2), d));
    r.root = __float_as_uint(a3.x);
    r.prim_base = __float_as_uint(a3.y);
    return r;
}

// Closest hit inside one mesh (object-space ray), updating the running best over instances.
template <bool PK = true>
__device__ __forceinline__ void blas_closest(const DevScene& s, const InstRay& r, uint32_t k, float& tbest,
                                             uint32_t& best, uint32_t& bprim, uint32_t& binst, uint32_t& steps) {
    const float3 id = ray_rcp(r.d);
    uint32_t stack_ref[kStack];
    float stack_t[kStack];
    int sp = 0;
    uint32_t ref = r.root;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 c;
            load_node(s.nodes, ref, n0, n1, n2, c);
            float t0, t1;
            bool h0, h1;
            box_test2<PK>(n0, n1, n2, r.o, id, tbest, t0, t1, h0, h1);
            if (h0 && h1) {
                bool first0 = t0 <= t1;
                if (sp < kStack) {
                    stack_ref[sp] = first0 ? c.y : c.x;
                    stack_t[sp] = first0 ? t1 : t0;
                    ++sp;
                } else {
                    atomicOr(s.status, ST_TRAVERSAL);
                }
                ref = first0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t q = 0; q < cnt; ++q) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + q, r.o, r.d, t, prim) && t > 0.0f) {
                    const uint32_t gp = r.prim_base + prim;
                    if (t < tbest || (t == tbest && gp < bprim)) {
                        tbest = t;
                        best = first + q;
                        bprim = gp;
                        binst = k;
                    }
                }
            }
        }
        if (steps >= kMaxSteps) {
            atomicOr(s.status, ST_TRAVERSAL);
            return;
        }
        bool found = false;
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= tbest * 1.0000005f) {
                ref = stack_ref[sp];
                found = true;
                break;
            }
        }
        if (!found) return;
        ++steps;
    }
}

template <bool PK = true>
__device__ __forceinline__ bool blas_any(const DevScene& s, const InstRay& r, float tmax, uint32_t& steps) {
    const float3 id = ray_rcp(r.d);
    uint32_t stack_ref[kStack];
    int sp = 0;
    uint32_t ref = r.root;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 c;
            load_node(s.nodes, ref, n0, n1, n2, c);
            float t0, t1;
            bool h0, h1;
            box_test2<PK>(n0, n1, n2, r.o, id, tmax, t0, t1, h0, h1);
            if (h0 && h1) {       // nearer child first, as in the single-level walk
                const bool first0 = t0 <= t1;
                if (sp < kStack) stack_ref[sp++] = first0 ? c.y : c.x;
                else atomicOr(s.status, ST_TRAVERSAL);
                ref = first0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t q = 0; q < cnt; ++q) {
                float t;
                uint32_t prim;
                if (tri_test(s.tris, first + q, r.o, r.d, t, prim) && t > 0.0f && t < tmax) return true;
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

template <bool PK = true>
__device__ __forceinline__ Hit trace_closest_inst(const DevScene& s, float3 o, float3 d) {
    const float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss, binst = kMiss;
    uint32_t stack_ref[kStack];
    float stack_t[kStack];
    int sp = 0;
    uint32_t ref = 0;
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 c;
            load_node(s.tlas, ref, n0, n1, n2, c);
            float t0, t1;
            bool h0, h1;
            box_test2<PK>(n0, n1, n2, o, id, tbest, t0, t1, h0, h1);
            if (h0 && h1) {
                bool first0 = t0 <= t1;
                if (sp < kStack) {
                    stack_ref[sp] = first0 ? c.y : c.x;
                    stack_t[sp] = first0 ? t1 : t0;
                    ++sp;
                } else {
                    atomicOr(s.status, ST_TRAVERSAL);
                }
                ref = first0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t q = 0; q < cnt; ++q) {
                const InstRay r = instance_ray(s, first + q, o, d);
                blas_closest<PK>(s, r, first + q, tbest, best, bprim, binst, steps);
            }
        }
        if (steps >= kMaxSteps) {
            atomicOr(s.status, ST_TRAVERSAL);
            break;
        }
        bool found = false;
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
    h.prim = bprim;
    h.inst = binst;
    return h;
}

template <bool PK = true>
__device__ __forceinline__ bool trace_any_inst(const DevScene& s, float3 o, float3 d, float tmax) {
    const float3 id = ray_rcp(d);
    uint32_t stack_ref[kStack];
    int sp = 0;
    uint32_t ref = 0;
    uint32_t steps = 0;
    while (true) {
        if (!(ref & kLeafBit)) {
            float4 n0, n1, n2;
            uint2 c;
            load_node(s.tlas, ref, n0, n1, n2, c);
            float t0, t1;
            bool h0, h1;
            box_test2<PK>(n0, n1, n2, o, id, tmax, t0, t1, h0, h1);
            if (h0 && h1) {       // nearer child first, as in the single-level walk
                const bool first0 = t0 <= t1;
                if (sp < kStack) stack_ref[sp++] = first0 ? c.y : c.x;
                else atomicOr(s.status, ST_TRAVERSAL);
                ref = first0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            } else if (h0 || h1) {
                ref = h0 ? c.x : c.y;
                if (++steps < kMaxSteps) continue;
            }
        } else {
            uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
            for (uint32_t q = 0; q < cnt; ++q)
                if (blas_any<PK>(s, instance_ray(s, first + q, o, d), tmax, steps)) return true;
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

// Two-level scenes, cooperatively: the same group walk over the top-level tree and, inside each
// instance the ray enters, over the mesh's tree.  A deferred entry also names its instance (kMiss for
// a top-level subtree); a lane that takes up an entry of another instance first takes the ray to
// that instance's object space.  t is the world parameter at both levels, so the group's best
// distance culls both, and the hit -- the smallest (t, original id) with its instance -- is the
// one-lane walk's.
struct RingStackInst {
    uint32_t ref[kStack];
    float t[kStack];
    uint32_t inst[kStack];
    uint32_t bot = 0, top = 0;
    __device__ __forceinline__ bool empty() const { return bot == top; }
    __device__ __forceinline__ bool push(uint32_t r, float tt, uint32_t k) {
        if (top - bot >= (uint32_t)kStack) return false;
        ref[top & (kStack - 1)] = r;
        t[top & (kStack - 1)] = tt;
        inst[top & (kStack - 1)] = k;
        ++top;
        return true;
    }
    __device__ __forceinline__ void pop(uint32_t& r, float& tt, uint32_t& k) {
        --top;
        r = ref[top & (kStack - 1)];
        tt = t[top & (kStack - 1)];
        k = inst[top & (kStack - 1)];
    }
    __device__ __forceinline__ void take_bottom(uint32_t& r, float& tt, uint32_t& k) {
        r = ref[bot & (kStack - 1)];
        tt = t[bot & (kStack - 1)];
        k = inst[bot & (kStack - 1)];
        ++bot;
    }
    __device__ __forceinline__ void clear() { bot = top; }
};

// group_share for two-level walks: a paired idle lane also receives the entry's instance (`k`).
__device__ __forceinline__ bool group_share_inst(uint32_t gm, uint32_t lane, bool& busy, uint32_t& ref, uint32_t& k,
                                                 bool& moved, RingStackInst& rs, float tcull) {
    const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !busy) & gm;
    const uint32_t donors = __ballot_sync(0xFFFFFFFFu, busy && !rs.empty()) & gm;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t pairs = min((uint32_t)__popc(idle), (uint32_t)__popc(donors));
    uint32_t give_r = 0u, give_k = kMiss;
    float give_t = 0.f;
    if (((donors >> lane) & 1u) && (uint32_t)__popc(donors & below) < pairs) rs.take_bottom(give_r, give_t, give_k);
    uint32_t from = lane;
    const uint32_t n = (uint32_t)__popc(idle & below);
    if (((idle >> lane) & 1u) && n < pairs) {
        uint32_t m = donors;
        for (uint32_t i = 0; i < n; ++i) m &= m - 1u;
        from = (uint32_t)__ffs(m) - 1u;
    }
    const uint32_t got_r = __shfl_sync(0xFFFFFFFFu, give_r, from);
    const float got_t = __shfl_sync(0xFFFFFFFFu, give_t, from);
    const uint32_t got_k = __shfl_sync(0xFFFFFFFFu, give_k, from);
    moved = false;
    if (from != lane && got_t <= tcull * 1.0000005f) {
        busy = true;
        ref = got_r;
        k = got_k;
        moved = true;
    }
    return idle == gm;
}

// One step of a two-level group walk at `ref` (level `cur`: kMiss = top level, else an instance,
// whose object-space ray is r with reciprocal direction idr): internal nodes push their far child and
// descend; a top-level leaf sets `cur` to its (first) instance and defers the others; a mesh leaf is
// tested by `leaf`.  Returns whether the lane is still busy.
template <class Leaf>
__device__ __forceinline__ bool inst_group_step(const DevScene& s, float3 o, float3 id, uint32_t& cur, const InstRay& r,
                                                float3 idr, uint32_t& ref, float tcull, bool push_t,
                                                RingStackInst& rs, Leaf leaf) {
    if (!(ref & kLeafBit)) {
        float4 n0, n1, n2;
        uint2 c;
        const bool top = cur == kMiss;
        load_node(top ? s.tlas : s.nodes, ref, n0, n1, n2, c);
        const float3 ro = top ? o : r.o, ri = top ? id : idr;
        float t0, t1;
        bool h0, h1;
        box_test2(n0, n1, n2, ro, ri, tcull, t0, t1, h0, h1);
        if (h0 && h1) {
            const bool first0 = t0 <= t1;
            if (!rs.push(first0 ? c.y : c.x, push_t ? (first0 ? t1 : t0) : 0.f, cur)) atomicOr(s.status, ST_TRAVERSAL);
            ref = first0 ? c.x : c.y;
            return true;
        }
        if (h0 || h1) {
            ref = h0 ? c.x : c.y;
            return true;
        }
        return false;
    }
    if (cur == kMiss) {                       // a top-level leaf: its instances
        const uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = (ref & 7u) + 1u;
        for (uint32_t q = 1; q < cnt; ++q)
            if (!rs.push(kLeafBit | ((first + q) << 3), 0.f, kMiss)) atomicOr(s.status, ST_TRAVERSAL);
        cur = first;                          // the caller takes the ray into it and starts at its root
        return true;
    }
    leaf(ref);
    return false;
}

__device__ __forceinline__ Hit trace_closest_group_inst(const DevScene& s, float3 o, float3 d, bool valid,
                                                        uint32_t G) {
    const uint32_t lane = threadIdx.x & 31u, gm = group_mask(G, lane);
    const float3 id = ray_rcp(d);
    float tbest = __int_as_float(0x7f800000);
    uint32_t best = kMiss, bprim = kMiss, binst = kMiss;
    bool busy = valid && (lane & (G - 1u)) == 0u;
    uint32_t ref = 0u, cur = kMiss;
    InstRay r;
    r.o = o;
    r.d = d;
    r.root = 0u;
    r.prim_base = 0u;
    float3 idr = id;
    auto enter = [&](uint32_t k) {
        cur = k;
        if (k != kMiss) {
            r = instance_ray(s, k, o, d);
            idr = ray_rcp(r.d);
        }
    };
    RingStackInst rs;
    uint32_t steps = 0;
    while (true) {
        const float tg = group_min(tbest, G);
        if (busy) {
            const uint32_t was = cur;
            busy = inst_group_step(s, o, id, cur, r, idr, ref, tg, true, rs, [&](uint32_t lr) {
                const uint32_t first = (lr & 0x7FFFFFFFu) >> 3, cnt = (lr & 7u) + 1u;
                for (uint32_t q = 0; q < cnt; ++q) {
                    float t;
                    uint32_t prim;
                    if (tri_test(s.tris, first + q, r.o, r.d, t, prim) && t > 0.0f) {
                        const uint32_t gp = r.prim_base + prim;
                        if (t < tbest || (t == tbest && gp < bprim)) {
                            tbest = t;
                            best = first + q;
                            bprim = gp;
                            binst = cur;
                        }
                    }
                }
            });
            if (was == kMiss && cur != kMiss) {   // entered an instance: its object-space ray, its root
                enter(cur);
                ref = r.root;
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                busy = false;
                rs.clear();
            }
        }
        const float tc = fminf(tg, tbest);
        while (!busy && !rs.empty()) {
            float t;
            uint32_t k;
            rs.pop(ref, t, k);
            busy = t <= tc * 1.0000005f;
            if (busy && k != cur) enter(k);
        }
        uint32_t k = cur;
        bool moved = false;
        const bool over = group_share_inst(gm, lane, busy, ref, k, moved, rs, tc);
        if (moved && k != cur) enter(k);
        if (__all_sync(0xFFFFFFFFu, over)) break;
    }
    Hit h;
    h.t = group_min(tbest, G);
    h.prim = group_min(tbest == h.t ? bprim : kMiss, G);
    const uint32_t own = __ballot_sync(0xFFFFFFFFu, tbest == h.t && bprim == h.prim) & gm;
    const uint32_t from = own ? (uint32_t)__ffs(own) - 1u : lane;
    h.tri = __shfl_sync(0xFFFFFFFFu, best, from);
    h.inst = __shfl_sync(0xFFFFFFFFu, binst, from);
    return h;
}

__device__ __forceinline__ bool trace_any_group_inst(const DevScene& s, float3 o, float3 d, float tmax, bool valid,
                                                     uint32_t G) {
    const uint32_t lane = threadIdx.x & 31u, gm = group_mask(G, lane);
    const float3 id = ray_rcp(d);
    bool busy = valid && (lane & (G - 1u)) == 0u, hit = false;
    uint32_t ref = 0u, cur = kMiss;
    InstRay r;
    r.o = o;
    r.d = d;
    r.root = 0u;
    r.prim_base = 0u;
    float3 idr = id;
    auto enter = [&](uint32_t k) {
        cur = k;
        if (k != kMiss) {
            r = instance_ray(s, k, o, d);
            idr = ray_rcp(r.d);
        }
    };
    RingStackInst rs;
    uint32_t steps = 0;
    while (true) {
        if (busy) {
            const uint32_t was = cur;
            busy = inst_group_step(s, o, id, cur, r, idr, ref, tmax, false, rs, [&](uint32_t lr) {
                const uint32_t first = (lr & 0x7FFFFFFFu) >> 3, cnt = (lr & 7u) + 1u;
                for (uint32_t q = 0; q < cnt && !hit; ++q) {
                    float t;
                    uint32_t prim;
                    hit = tri_test(s.tris, first + q, r.o, r.d, t, prim) && t > 0.0f && t < tmax;
                }
            });
            if (was == kMiss && cur != kMiss) {
                enter(cur);
                ref = r.root;
            }
            if (++steps >= kMaxSteps) {
                atomicOr(s.status, ST_TRAVERSAL);
                busy = false;
                rs.clear();
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, hit) & gm) {
            busy = false;
            rs.clear();
        }
        if (!busy && !rs.empty()) {
            float t;
            uint32_t k;
            rs.pop(ref, t, k);
            busy = true;
            if (k != cur) enter(k);
        }
        uint32_t k = cur;
        bool moved = false;
        const bool over = group_share_inst(gm, lane, busy, ref, k, moved, rs, 0.f);
        if (moved && k != cur) enter(k);
        if (__all_sync(0xFFFFFFFFu, over)) break;
    }
    return (__ballot_sync(0xFFFFFFFFu, hit) & gm) != 0u;
}

// The extend and shadow queries.  (A "while-while" variant that voted across the warp with
// __any_sync(__activemask(), ...) was tried and removed: its result depended on which paths shared a
// warp -- lanes that are not converged may pass different masks to the vote -- so one path in 33M
// differed between the megakernel and the wavefront.)
// INST selects the two-level traversal at compile time (kernels are instantiated both ways, so the
// single-level kernels carry none of its registers).  SK > 0: the single-level walks keep their top
// SK stack entries in shared memory (the kernel supplies stack_smem_bytes(SK, blockDim.x) of dynamic
// shared memory); the two-level walks keep the local stack.
// `cnt` (TravCount) counts the single-level walks' node visits and triangle tests; the two-level
// walks are not counted.  PK = false: the two-level walks test boxes one at a time (box_test2).
template <bool INST = false, int SK = 0, bool PK = true, class C = NoCount>
__device__ __forceinline__ Hit trace_closest(const DevScene& s, float3 o, float3 d, C& cnt) {
    if constexpr (INST) {
        return trace_closest_inst<PK>(s, o, d);
    } else {
        typename StackOf<SK, true>::type stk;
        return trace_closest_plain(s, o, d, stk, cnt);
    }
}
template <bool INST = false, int SK = 0, bool PK = true>
__device__ __forceinline__ Hit trace_closest(const DevScene& s, float3 o, float3 d) {
    NoCount c;
    return trace_closest<INST, SK, PK>(s, o, d, c);
}
template <bool INST = false, int SK = 0, bool PK = true, class C = NoCount>
__device__ __forceinline__ bool trace_any(const DevScene& s, float3 o, float3 d, float tmax, C& cnt) {
    if constexpr (INST) {
        return trace_any_inst<PK>(s, o, d, tmax);
    } else {
        typename StackOf<SK, false>::type stk;
        return trace_any_plain(s, o, d, tmax, stk, cnt);
    }
}
template <bool INST = false, int SK = 0, bool PK = true>
__device__ __forceinline__ bool trace_any(const DevScene& s, float3 o, float3 d, float tmax) {
    NoCount c;
    return trace_any<INST, SK, PK>(s, o, d, tmax, c);
}

}  // namespace pt
