// pt_common.cuh -- device helpers shared by the kernel translation units: warp-aggregated
// atomics, the per-path event recorders, the megakernel's path and bounce functions (also the
// body of the wavefront's hybrid continuation kernel), the wavefront's scene sources and the
// adjoint's record type and warp-aggregated gradient accumulation.
#pragma once
#include <cstdio>

#include "pt_device.cuh"
#include "pt_launch.h"
#include "pt_trace.cuh"

namespace pt {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Programmatic dependent launch (sm_90+): a stage kernel that the host launches with the
// programmatic-serialization attribute may begin while the previous kernel of its stream drains.
// It first waits until that kernel has finished and its writes are visible (a no-op when launched
// normally), then lets the next kernel of the stream begin its own launch, whose blocks become
// resident as this kernel's blocks exit and wait in the same way.
__device__ __forceinline__ void stage_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch through cudaLaunchKernelEx with the programmatic-serialization attribute when l.pdl is set
// (the kernel must begin with stage_prologue()), else as an ordinary launch.
template <class... KArgs, class... Args>
cudaError_t launch_k(const Launch& l, size_t smem, void (*k)(KArgs...), Args... args) {
    if (!l.pdl) {
        k<<<l.grid, l.block, smem, l.st>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)l.grid);
    cfg.blockDim = dim3((unsigned)l.block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = l.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Warp-aggregated append (stream compaction, Sec. 3.1): every lane of the warp calls it; lanes with
// `want` receive consecutive slots from a single atomicAdd issued by the lowest such lane.
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
    uint32_t mask = __ballot_sync(0xFFFFFFFFu, want);
    if (mask == 0u) return 0u;
    uint32_t leader = __ffs(mask) - 1u;
    uint32_t base = 0u;
    if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + (uint32_t)__popc(mask & ((1u << lane_id()) - 1u));
}

// Warp-granular dynamic work: each warp claims its next queue slots (32, one per lane; 32 / G when
// groups of G lanes share a ray) with one atomic, so warps that drew cheap rays take more batches
// and the grid ends together (a static grid-stride split leaves the SMs waiting on the warps that
// drew the longest rays).
__device__ __forceinline__ uint32_t warp_claim(uint32_t* counter, uint32_t k) {
    uint32_t b = 0u;
    if (lane_id() == 0u) b = atomicAdd(counter, k);
    return __shfl_sync(0xFFFFFFFFu, b, 0);
}
__device__ __forceinline__ uint32_t warp_claim32(uint32_t* counter) { return warp_claim(counter, 32u); }

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane_id() == 0 && v) atomicAdd(dst, v);
}

__device__ __forceinline__ float4 f4(float3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

// ================================================================== megakernel
// Event recorders of one path (compile-time: the production kernel records nothing).
struct NoRec {
    __device__ __forceinline__ void ev(uint32_t, uint32_t, uint32_t, float, float) {}
};
struct SigRec {   // order-free branch signature
    uint32_t sg = 0;
    __device__ __forceinline__ void ev(uint32_t b, uint32_t k, uint32_t v, float, float) { sg ^= sig_event(b, k, v); }
};
struct LogRec {   // event list with two diagnostic numbers per event (testing aid)
    uint32_t* ev_u;
    float* ev_f;
    uint32_t n = 0;
    __device__ __forceinline__ void ev(uint32_t b, uint32_t k, uint32_t v, float f0, float f1) {
        if (n >= kMaxEvents) return;
        ev_u[2 * n] = (b << 4) | k;
        ev_u[2 * n + 1] = v;
        ev_f[2 * n] = f0;
        ev_f[2 * n + 1] = f1;
        ++n;
    }
};

// One whole path (Sec. 2.2 steps 1-5) in registers: the body of the megakernel.
template <class Rec, bool MIS, bool INST>
__device__ __forceinline__ float3 mk_path(const DevScene& s, const DevCamera& c, const RenderParams& p, uint64_t path,
                                          Rec& rec, uint32_t& n_ext, uint32_t& n_shd) {
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    const uint32_t pixel = (uint32_t)(path / p.spp);
    const uint32_t sample = p.sample_offset + (uint32_t)(path - (uint64_t)pixel * p.spp);
    const uint32_t key = path_key(p.seed, pixel, sample);
    float3 o, d;
    float u0, u1;
    pixel_jitter(p.sampler, p.seed, pixel, sample, key, u0, u1);
    camera_ray(c, pixel, u0, u1, o, d);                        // step 1
    float3 tp = f3(1.f, 1.f, 1.f), L = f3(0.f, 0.f, 0.f);
    bool prev_delta = true;
    float prev_pdf = 0.f;
    for (uint32_t b = 0; b < p.max_depth; ++b) {
        ++n_ext;
        Hit h = trace_closest<INST, 0, !INST>(s, o, d);        // step 2
        if (h.tri == kMiss) {
            L = add_rn(L, mul_rn(tp, env));
            rec.ev(b, 0, kMiss, __int_as_float(0x7f800000), tp.x);
            break;
        }
        Vertex V = shade_vertex<MIS, INST>(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri, h.inst);
        rec.ev(b, 0, V.prim, h.t, tp.x);
        if (V.emit_counted) L = add_rn(L, V.emit);             // step 3
        if (V.last) break;
        if (V.nee) {                                           // shadow evaluation
            uint32_t vis = 0;
            if (V.cast) {
                ++n_shd;
                vis = trace_any<INST, 0, !INST>(s, V.s_o, V.s_d, V.s_tmax) ? 0u : 1u;
                if (vis) L = add_rn(L, V.contrib);
            }
            rec.ev(b, 1, (V.light_j << 2) | ((uint32_t)V.cast << 1) | vis, V.nee_cx, V.nee_cl);
        }
        rec.ev(b, 2, V.bsdf_code, V.w.x, V.nd.x);
        if (V.rr >= 0) rec.ev(b, 3, (uint32_t)V.rr, V.rr_q, u01(key, b, D_RR));
        if (!V.cont) break;                                    // step 4 done; step 5: repeat
        o = V.no;
        d = V.nd;
        tp = V.ntp;
        prev_delta = V.delta;
        prev_pdf = V.pdf;
    }
    return L;
}

// One bounce of a path held in registers (extend, shade, shadow evaluation), the loop body of the
// regenerating megakernel and of the wavefront's continuation kernel.  Returns true when the path
// ends; otherwise the state has moved to bounce b + 1.
// SK: shared-memory short-stack entries of the walks (0: local stack; see trace_closest).  cc, ca:
// traversal counters of the closest-hit and any-hit walks (NoCount: none).
template <bool SIG, bool MIS, bool INST, int SK = 0, class C = NoCount>
__device__ __forceinline__ bool mk_bounce(const DevScene& s, const RenderParams& p, float3 env, uint32_t key,
                                          uint32_t& b, float3& o, float3& d, float3& tp, bool& prev_delta,
                                          float& prev_pdf, float3& L, uint32_t& sg, uint32_t& n_ext,
                                          uint32_t& n_shd, C& cc, C& ca) {
    ++n_ext;
    Hit h = trace_closest<INST, SK, !INST>(s, o, d, cc);
    if (h.tri == kMiss) {
        L = add_rn(L, mul_rn(tp, env));
        if (SIG) sg ^= sig_event(b, 0, kMiss);
        return true;
    }
    Vertex V = shade_vertex<MIS, INST>(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri, h.inst);
    if (SIG) sg ^= sig_event(b, 0, V.prim);
    if (V.emit_counted) L = add_rn(L, V.emit);
    if (V.last) return true;
    if (V.nee) {
        uint32_t vis = 0;
        if (V.cast) {
            ++n_shd;
            vis = trace_any<INST, SK, !INST>(s, V.s_o, V.s_d, V.s_tmax, ca) ? 0u : 1u;
            if (vis) L = add_rn(L, V.contrib);
        }
        if (SIG) sg ^= sig_event(b, 1, (V.light_j << 2) | ((uint32_t)V.cast << 1) | vis);
    }
    if (SIG) {
        sg ^= sig_event(b, 2, V.bsdf_code);
        if (V.rr >= 0) sg ^= sig_event(b, 3, (uint32_t)V.rr);
    }
    if (!V.cont) return true;
    o = V.no;
    d = V.nd;
    tp = V.ntp;
    prev_delta = V.delta;
    prev_pdf = V.pdf;
    ++b;
    return false;
}
template <bool SIG, bool MIS, bool INST, int SK = 0>
__device__ __forceinline__ bool mk_bounce(const DevScene& s, const RenderParams& p, float3 env, uint32_t key,
                                          uint32_t& b, float3& o, float3& d, float3& tp, bool& prev_delta,
                                          float& prev_pdf, float3& L, uint32_t& sg, uint32_t& n_ext,
                                          uint32_t& n_shd) {
    NoCount cc, ca;
    return mk_bounce<SIG, MIS, INST, SK>(s, p, env, key, b, o, d, tp, prev_delta, prev_pdf, L, sg, n_ext, n_shd, cc,
                                         ca);
}

// Counting instantiations: the warp's node and triangle counts added to s.trav[k], s.trav[k + 1]
// (all 32 lanes call it, converged).
template <class C>
__device__ __forceinline__ void flush_count(const DevScene& s, const C& c, int k);
template <>
__device__ __forceinline__ void flush_count<NoCount>(const DevScene&, const NoCount&, int) {}
template <>
__device__ __forceinline__ void flush_count<TravCount>(const DevScene& s, const TravCount& c, int k) {
    warp_add_u64(s.trav + k, c.nodes);
    warp_add_u64(s.trav + k + 1, c.tris);
}

// ================================================================== wavefront stages
// Scene sources: where a wavefront kernel finds the scene, camera and path numbering of a queue
// entry.  SingleSrc: one scene passed by value (pt_render).  TableSrc: many scenes in device
// tables, the scene found from the global path id by binary search over the scenes' first path ids
// (pt_render_batch).  The per-path arithmetic is the same shared device code either way.
struct PathLoc {
    uint64_t path;     // global path id (signature index)
    uint32_t pixel, sample, sid;
};

struct SingleSrc {
    DevScene s;
    DevCamera c;
    RenderParams p;
    __device__ __forceinline__ uint64_t base() const { return p.path_begin; }
    __device__ __forceinline__ uint32_t sid_of(uint64_t, uint32_t) const { return 0; }
    __device__ __forceinline__ PathLoc locate(uint64_t base, uint32_t pid) const {
        PathLoc l;
        l.path = base + pid;
        l.pixel = (uint32_t)(l.path / p.spp);
        l.sample = p.sample_offset + (uint32_t)(l.path - (uint64_t)l.pixel * p.spp);
        l.sid = 0;
        return l;
    }
    __device__ __forceinline__ DevScene scene(uint32_t) const { return s; }
    __device__ __forceinline__ DevCamera camera(uint32_t) const { return c; }
    __device__ __forceinline__ RenderParams params(uint32_t) const { return p; }
    // scene id carried in the queue records: none needed for one scene
    __device__ __forceinline__ uint32_t ray_tag(uint32_t, uint32_t flags) const { return flags; }
    __device__ __forceinline__ uint32_t sid_from_ray(float, uint64_t, uint32_t) const { return 0; }
    __device__ __forceinline__ uint32_t shadow_tag(uint32_t light_j, uint32_t) const { return light_j; }
    __device__ __forceinline__ uint32_t sid_from_shadow(float, uint64_t, uint32_t) const { return 0; }
    __device__ __forceinline__ PathLoc locate_in(uint64_t base, uint32_t pid, uint32_t) const { return locate(base, pid); }
};

struct TableSrc {
    BatchTables t;
    RenderParams p;    // depth and roulette (spp per scene and the seed from the tables)
    __device__ __forceinline__ uint64_t base() const { return *t.wave_base; }
    __device__ __forceinline__ uint32_t sid_of(uint64_t base, uint32_t pid) const {
        const uint64_t g = base + pid;
        uint32_t lo = 0, hi = t.n - 1;                  // last scene with off[s] <= g
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (__ldg(t.off + mid) <= g) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ PathLoc locate(uint64_t base, uint32_t pid) const {
        PathLoc l;
        l.sid = sid_of(base, pid);
        l.path = base + pid;
        const uint64_t local = l.path - __ldg(t.off + l.sid);
        const uint32_t spp = __ldg(t.spp + l.sid);
        l.pixel = (uint32_t)(local / spp);
        l.sample = (uint32_t)(local - (uint64_t)l.pixel * spp);
        return l;
    }
    __device__ __forceinline__ DevScene scene(uint32_t sid) const { return t.scenes[sid]; }
    __device__ __forceinline__ DevCamera camera(uint32_t sid) const { return t.cams[sid]; }
    __device__ __forceinline__ RenderParams params(uint32_t sid) const {
        RenderParams q = p;
        q.spp = __ldg(t.spp + sid);
        q.seed = __ldg(t.seed);
        return q;
    }
    // the scene id rides in the records' spare bits: ray d.w = flags | sid << 8; shadow c.w = sid
    __device__ __forceinline__ uint32_t ray_tag(uint32_t sid, uint32_t flags) const { return flags | (sid << 8); }
    __device__ __forceinline__ uint32_t sid_from_ray(float dw, uint64_t, uint32_t) const {
        return __float_as_uint(dw) >> 8;
    }
    __device__ __forceinline__ uint32_t shadow_tag(uint32_t, uint32_t sid) const { return sid; }
    __device__ __forceinline__ uint32_t sid_from_shadow(float cw, uint64_t, uint32_t) const {
        return __float_as_uint(cw);
    }
    __device__ __forceinline__ PathLoc locate_in(uint64_t base, uint32_t pid, uint32_t sid) const {
        PathLoc l;
        l.sid = sid;
        l.path = base + pid;
        const uint64_t local = l.path - __ldg(t.off + sid);
        const uint32_t spp = __ldg(t.spp + sid);
        l.pixel = (uint32_t)(local / spp);
        l.sample = (uint32_t)(local - (uint64_t)l.pixel * spp);
        return l;
    }
};

// ================================================================== adjoint (path replay)
struct AdjRec {
    float3 tp;       // throughput arriving at the vertex
    float3 w;        // throughput multiplier of the continuation (BSDF weight / q)
    float3 dwa;      // d w / d albedo
    float3 nee_g;    // f G A of a visible NEE sample (0 otherwise)
    float3 nee_dfa;  // d(f G A Le_light) / d albedo
    float Le;        // emission of the hit material times its weight when its term is counted
    float we;        // that weight (1, or the MIS weight of a BSDF-sampled light hit)
    float Lj;        // emission of the sampled light's material
    uint32_t mat, lmat;
    uint32_t flags;  // 1: continues, 2: NEE visible, 4: emission counted
};

constexpr uint32_t kNoKey = 0xFFFFFFFFu;

// Warp-aggregated accumulation into per-material gradients: lanes holding the same key add their
// values once (one atomic per distinct key per warp).  All 32 lanes call it; key == kNoKey means
// nothing to add.  v = (d/d albedo rgb, d/d emission).
__device__ __forceinline__ void warp_accumulate(float* acc, float* g_alb, float* g_em, bool smem, uint32_t key,
                                                float4 v) {
    uint32_t pending = __ballot_sync(0xFFFFFFFFu, key != kNoKey);
    while (pending) {
        const uint32_t leader = __ffs(pending) - 1u;
        const uint32_t k = __shfl_sync(0xFFFFFFFFu, key, leader);
        const bool mine = key == k;
        const uint32_t grp = __ballot_sync(0xFFFFFFFFu, mine);
        float4 sum = mine ? v : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int o = 16; o > 0; o >>= 1) {
            sum.x += __shfl_xor_sync(0xFFFFFFFFu, sum.x, o);
            sum.y += __shfl_xor_sync(0xFFFFFFFFu, sum.y, o);
            sum.z += __shfl_xor_sync(0xFFFFFFFFu, sum.z, o);
            sum.w += __shfl_xor_sync(0xFFFFFFFFu, sum.w, o);
        }
        if (lane_id() == leader) {
            if (smem) {
                if (sum.x != 0.f) atomicAdd(&acc[4 * k], sum.x);
                if (sum.y != 0.f) atomicAdd(&acc[4 * k + 1], sum.y);
                if (sum.z != 0.f) atomicAdd(&acc[4 * k + 2], sum.z);
                if (sum.w != 0.f) atomicAdd(&acc[4 * k + 3], sum.w);
            } else {
                if (sum.x != 0.f) atomicAdd(&g_alb[3 * k], sum.x);
                if (sum.y != 0.f) atomicAdd(&g_alb[3 * k + 1], sum.y);
                if (sum.z != 0.f) atomicAdd(&g_alb[3 * k + 2], sum.z);
                if (sum.w != 0.f) atomicAdd(&g_em[k], sum.w);
            }
        }
        pending &= ~grp;
    }
}

}  // namespace pt
