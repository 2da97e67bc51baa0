// pt_kernels.cu -- CUDA kernels of the path tracer for sm_103a.
//
// Megakernel (Sec. 2.2): one thread per path, the whole path in one kernel.
// Wavefront (Sec. 2.3, 3, 3.1): raygen -> per bounce { extend -> (key sort) -> shade -> shadow ->
// prepare } -> accumulate.  Stages are linked by structure-of-arrays queues of 16-byte records
// (128-bit coalesced loads and stores); compaction is a warp-aggregated atomic append into the next
// queue (one atomic per warp instead of one per path), and the prepare step rotates the two-slot
// active count without a host round trip.  Grids are persistent (a multiple of the SM count) and
// stride over the device-side count, so no host read-back or indirect launch is needed.
// Adjoint: path replay (re-trace from the random numbers) with per-vertex records kept per thread,
// reverse accumulation, block-level shared-memory gradient reduction, one global atomic per
// non-zero material entry per block.
#include <cstdio>

#include "pt_device.cuh"
#include "pt_launch.h"
#include "pt_trace.cuh"

namespace pt {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

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
template <class Rec, bool MIS>
__device__ __forceinline__ float3 mk_path(const DevScene& s, const DevCamera& c, const RenderParams& p, uint64_t path,
                                          Rec& rec, unsigned long long& n_ext, unsigned long long& n_shd) {
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
        Hit h = trace_closest(s, o, d);                  // step 2
        if (h.tri == kMiss) {
            L = add_rn(L, mul_rn(tp, env));
            rec.ev(b, 0, kMiss, __int_as_float(0x7f800000), tp.x);
            break;
        }
        Vertex V = shade_vertex<MIS>(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri);
        rec.ev(b, 0, V.prim, h.t, tp.x);
        if (V.emit_counted) L = add_rn(L, V.emit);             // step 3
        if (V.last) break;
        if (V.nee) {                                           // shadow evaluation
            uint32_t vis = 0;
            if (V.cast) {
                ++n_shd;
                vis = trace_any(s, V.s_o, V.s_d, V.s_tmax) ? 0u : 1u;
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

template <bool SIG, bool MIS>
__global__ void __launch_bounds__(256) k_megakernel(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                    float* __restrict__ out_L, float* __restrict__ img,
                                                    uint32_t* __restrict__ sig, unsigned long long* __restrict__ rays) {
    unsigned long long n_ext = 0, n_shd = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_paths; i += stride) {
        const uint64_t path = p.path_begin + i;
        float3 L;
        if (SIG) {
            SigRec r;
            L = mk_path<SigRec, MIS>(s, c, p, path, r, n_ext, n_shd);
            sig[path] = r.sg;
        } else {
            NoRec r;
            L = mk_path<NoRec, MIS>(s, c, p, path, r, n_ext, n_shd);
        }
        if (out_L) {
            out_L[3 * i] = L.x;
            out_L[3 * i + 1] = L.y;
            out_L[3 * i + 2] = L.z;
        } else {
            const uint32_t pixel = (uint32_t)(path / p.spp);
            img[3 * (size_t)pixel] = L.x;
            img[3 * (size_t)pixel + 1] = L.y;
            img[3 * (size_t)pixel + 2] = L.z;
        }
    }
    warp_add_u64(rays, n_ext);
    warp_add_u64(rays + 1, n_shd);
}

// One bounce of a path held in registers (extend, shade, shadow evaluation), the loop body of the
// regenerating megakernel and of the wavefront's continuation kernel.  Returns true when the path
// ends; otherwise the state has moved to bounce b + 1.
template <bool SIG, bool MIS>
__device__ __forceinline__ bool mk_bounce(const DevScene& s, const RenderParams& p, float3 env, uint32_t key,
                                          uint32_t& b, float3& o, float3& d, float3& tp, bool& prev_delta,
                                          float& prev_pdf, float3& L, uint32_t& sg, unsigned long long& n_ext,
                                          unsigned long long& n_shd) {
    ++n_ext;
    Hit h = trace_closest(s, o, d);
    if (h.tri == kMiss) {
        L = add_rn(L, mul_rn(tp, env));
        if (SIG) sg ^= sig_event(b, 0, kMiss);
        return true;
    }
    Vertex V = shade_vertex<MIS>(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri);
    if (SIG) sg ^= sig_event(b, 0, V.prim);
    if (V.emit_counted) L = add_rn(L, V.emit);
    if (V.last) return true;
    if (V.nee) {
        uint32_t vis = 0;
        if (V.cast) {
            ++n_shd;
            vis = trace_any(s, V.s_o, V.s_d, V.s_tmax) ? 0u : 1u;
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

// Persistent megakernel with path regeneration.  Each thread still traces one path at a time from
// its camera ray to termination, one bounce per loop iteration; a lane whose path ended claims the
// next path id (warp-aggregated atomic on a device counter) instead of idling until the longest
// path of its warp finishes.  The per-path arithmetic is that of mk_path, so images are identical.
template <bool SIG, bool MIS>
// Register cap for 8 resident blocks of 128: occupancy outweighs the spills (measured 3.96 -> 3.11 ms
// per 1080p frame against the uncapped 107 registers).
__global__ void __launch_bounds__(128, 8) k_megakernel_regen(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                          float* __restrict__ out_L, float* __restrict__ img,
                                                          uint32_t* __restrict__ sig,
                                                          unsigned long long* __restrict__ rays,
                                                          unsigned long long* __restrict__ next_path) {
    unsigned long long n_ext = 0, n_shd = 0;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    bool active = false, exhausted = false;
    uint64_t i = 0;
    uint32_t pixel = 0, key = 0, b = 0, sg = 0;
    float3 o = f3(0.f, 0.f, 0.f), d = o, tp = o, L = o;
    bool prev_delta = true;
    float prev_pdf = 0.f;
    while (true) {
        const bool want = !active && !exhausted;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, want);
        if (m) {
            const uint32_t leader = __ffs(m) - 1u;
            unsigned long long first = 0;
            if (lane_id() == leader) first = atomicAdd(next_path, (unsigned long long)__popc(m));
            first = __shfl_sync(0xFFFFFFFFu, first, leader);
            if (want) {
                i = first + (uint64_t)__popc(m & ((1u << lane_id()) - 1u));
                if (i < n_paths) {
                    const uint64_t path = p.path_begin + i;
                    pixel = (uint32_t)(path / p.spp);
                    const uint32_t sample = p.sample_offset + (uint32_t)(path - (uint64_t)pixel * p.spp);
                    key = path_key(p.seed, pixel, sample);
                    float u0, u1;
                    pixel_jitter(p.sampler, p.seed, pixel, sample, key, u0, u1);
                    camera_ray(c, pixel, u0, u1, o, d);
                    tp = f3(1.f, 1.f, 1.f);
                    L = f3(0.f, 0.f, 0.f);
                    prev_delta = true;
                    prev_pdf = 0.f;
                    b = 0;
                    sg = 0;
                    active = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        if (active) {
            const bool end = mk_bounce<SIG, MIS>(s, p, env, key, b, o, d, tp, prev_delta, prev_pdf, L, sg, n_ext, n_shd);
            if (end) {
                if (out_L) {
                    out_L[3 * i] = L.x;
                    out_L[3 * i + 1] = L.y;
                    out_L[3 * i + 2] = L.z;
                } else {
                    img[3 * (size_t)pixel] = L.x;
                    img[3 * (size_t)pixel + 1] = L.y;
                    img[3 * (size_t)pixel + 2] = L.z;
                }
                if (SIG) sig[p.path_begin + i] = sg;
                active = false;
            }
        }
    }
    warp_add_u64(rays, n_ext);
    warp_add_u64(rays + 1, n_shd);
}

// Event logs of selected paths (testing aid): the megakernel's path function with a recorder.
__global__ void k_debug_paths(DevScene s, DevCamera c, RenderParams p, const unsigned long long* __restrict__ ids,
                              uint32_t n, uint32_t* __restrict__ ev_u, float* __restrict__ ev_f,
                              uint32_t* __restrict__ n_ev, float* __restrict__ out_L) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long a = 0, b = 0;
    LogRec r;
    r.ev_u = ev_u + (size_t)i * 2 * kMaxEvents;
    r.ev_f = ev_f + (size_t)i * 2 * kMaxEvents;
    float3 L = mk_path<LogRec, true>(s, c, p, ids[i], r, a, b);
    n_ev[i] = r.n;
    out_L[3 * i] = L.x;
    out_L[3 * i + 1] = L.y;
    out_L[3 * i + 2] = L.z;
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

// Ray generation: one queue record per path of the wave, radiance zeroed, active count = n.  The
// wave's first path id is a launch argument here and is published to device memory (wave_base_dev)
// for the kernels of the bounce loop.
template <class Src>
__global__ void __launch_bounds__(256) k_raygen(Src src, uint64_t base, uint32_t n, WfBuffers w,
                                                unsigned long long* wave_base_dev) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const PathLoc l = src.locate(base, i);
        const RenderParams p = src.params(l.sid);
        const uint32_t key = path_key(p.seed, l.pixel, l.sample);
        float3 o, d;
        float u0, u1;
        pixel_jitter(p.sampler, p.seed, l.pixel, l.sample, key, u0, u1);
        camera_ray(src.camera(l.sid), l.pixel, u0, u1, o, d);
        w.q_o[0][i] = f4(o, __uint_as_float(i));
        w.q_d[0][i] = f4(d, __uint_as_float(src.ray_tag(l.sid, 1u)));   // previous vertex "delta": the camera
        w.q_tp[0][i] = make_float4(1.f, 1.f, 1.f, 0.f);
        w.L[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (w.sig) w.sig[l.path] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.counts[0] = n;
        w.counts[1] = 0u;
        w.counts[2] = 0u;
        if (wave_base_dev) *wave_base_dev = base;
    }
}

// Extend: closest hit of every active ray (scene-intersection stage); hit records per queue slot.
template <class Src>
__global__ void __launch_bounds__(256) k_extend(Src src, WfBuffers w, int in) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint64_t base = src.base();
    const float4* __restrict__ qo = w.q_o[in];
    const float4* __restrict__ qd = w.q_d[in];
    float2* __restrict__ hit = w.hit;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        float4 o4 = qo[j], d4 = qd[j];
        Hit h = trace_closest(src.scene(src.sid_from_ray(d4.w, base, __float_as_uint(o4.w))), xyz(o4), xyz(d4));
        hit[j] = make_float2(h.t, __uint_as_float(h.tri));
    }
}

// Key sort before shading (counting sort): keys + block histograms, scan, scatter into `perm`.
template <class Src>
__global__ void __launch_bounds__(256) k_sort_keys(Src src, WfBuffers w, int in, uint32_t mode, uint32_t n_keys) {
    extern __shared__ uint32_t hist_s[];
    for (uint32_t k = threadIdx.x; k < n_keys; k += blockDim.x) hist_s[k] = 0u;
    __syncthreads();
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint64_t base = src.base();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        uint32_t tri = __float_as_uint(w.hit[j].y);
        uint32_t key = n_keys - 1u;                          // misses last
        if (tri != kMiss) {
            const DevScene s = src.scene(src.sid_from_ray(w.q_d[in][j].w, base, __float_as_uint(w.q_o[in][j].w)));
            uint32_t m = __float_as_uint(__ldg(s.tris + 3 * (size_t)tri + 1).w);
            key = mode == 1u ? __float_as_uint(__ldg(reinterpret_cast<const float*>(s.mats + m))) : m;
            key = min(key, n_keys - 2u);
        }
        w.keys[j] = key;
        atomicAdd(&hist_s[key], 1u);
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < n_keys; k += blockDim.x)
        if (hist_s[k]) atomicAdd(&w.bucket[k], hist_s[k]);
}

// Exclusive scan of the bucket counts (one block of 1024 threads, n_keys <= 4096).
__global__ void __launch_bounds__(1024) k_sort_scan(WfBuffers w, uint32_t n_keys) {
    __shared__ uint32_t part[1024];
    const uint32_t t = threadIdx.x;
    uint32_t v[4], sum = 0;
    for (int k = 0; k < 4; ++k) {
        uint32_t idx = 4 * t + k;
        v[k] = idx < n_keys ? w.bucket[idx] : 0u;
        sum += v[k];
    }
    part[t] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {          // Hillis-Steele inclusive scan
        uint32_t x = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    uint32_t run = part[t] - sum;
    for (int k = 0; k < 4; ++k) {
        uint32_t idx = 4 * t + k;
        if (idx < n_keys) w.bucket[idx] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(256) k_sort_scatter(WfBuffers w) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = warp * 32u; base < n; base += n_warps * 32u) {
        uint32_t j = base + lane_id();
        bool valid = j < n;
        uint32_t key = valid ? w.keys[j] : 0xFFFFFFFFu;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
        uint32_t leader = __ffs(peers) - 1u;
        uint32_t rank = __popc(peers & ((1u << lane_id()) - 1u));
        uint32_t off = 0u;
        if (valid && lane_id() == leader) off = atomicAdd(&w.bucket[key], (uint32_t)__popc(peers));
        off = __shfl_sync(0xFFFFFFFFu, off, leader);
        if (valid) w.perm[off + rank] = j;
    }
}

// Shade: emission, NEE sample (-> shadow queue), BSDF sample, roulette, compaction of survivors.
template <class Src, bool SIG>
__global__ void __launch_bounds__(256, 3) k_shade(Src src, WfBuffers w, int in, uint32_t b, bool sorted) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint64_t base = src.base();
    const int out = in ^ 1;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wb = warp * 32u; wb < n; wb += n_warps * 32u) {
        const uint32_t j = wb + lane_id();
        bool want_ray = false, want_shadow = false;
        float4 ro, rd, rtp, so, sd, sc;
        if (j < n) {
            const uint32_t slot = sorted ? w.perm[j] : j;
            const float4 o4 = w.q_o[in][slot], d4 = w.q_d[in][slot], tp4 = w.q_tp[in][slot];
            const float2 hh = w.hit[slot];
            const uint32_t pid = __float_as_uint(o4.w);
            const PathLoc l = src.locate_in(base, pid, src.sid_from_ray(d4.w, base, pid));
            const DevScene s = src.scene(l.sid);
            const float3 tp = xyz(tp4);
            const uint32_t tri = __float_as_uint(hh.y);
            if (tri == kMiss) {
                float3 L = add_rn(xyz(w.L[pid]), mul_rn(tp, f3(s.env_r, s.env_g, s.env_b)));
                w.L[pid] = f4(L, 0.f);
                if (SIG) w.sig[l.path] ^= sig_event(b, 0, kMiss);
            } else {
                const RenderParams p = src.params(l.sid);
                const uint32_t key = path_key(p.seed, l.pixel, l.sample);
                Vertex V = shade_vertex(s, p, key, b, xyz(o4), xyz(d4), tp, (__float_as_uint(d4.w) & 1u) != 0u,
                                        tp4.w, hh.x, tri);
                if (V.emit_counted) {
                    float3 L = add_rn(xyz(w.L[pid]), V.emit);
                    w.L[pid] = f4(L, 0.f);
                }
                uint32_t sg = 0;
                if (SIG) sg = sig_event(b, 0, V.prim);
                if (!V.last) {
                    if (V.nee) {
                        if (V.cast) {
                            want_shadow = true;
                            so = f4(V.s_o, V.s_tmax);
                            sd = f4(V.s_d, __uint_as_float(pid));
                            sc = f4(V.contrib, __uint_as_float(src.shadow_tag(V.light_j, l.sid)));
                        } else if (SIG) {
                            sg ^= sig_event(b, 1, V.light_j << 2);
                        }
                    }
                    if (SIG) {
                        sg ^= sig_event(b, 2, V.bsdf_code);
                        if (V.rr >= 0) sg ^= sig_event(b, 3, (uint32_t)V.rr);
                    }
                    if (V.cont) {
                        want_ray = true;
                        ro = f4(V.no, __uint_as_float(pid));
                        rd = f4(V.nd, __uint_as_float(src.ray_tag(l.sid, V.delta ? 1u : 0u)));
                        rtp = f4(V.ntp, V.pdf);
                    }
                }
                if (SIG) w.sig[l.path] ^= sg;
            }
        }
        const uint32_t k = warp_append(&w.counts[2], want_shadow);
        if (want_shadow) {
            if (k < w.capacity) {
                w.s_o[k] = so;
                w.s_d[k] = sd;
                w.s_c[k] = sc;
            } else {
                atomicOr(src.scene(0).status, ST_QUEUE);
            }
        }
        const uint32_t q = warp_append(&w.counts[1], want_ray);
        if (want_ray) {
            if (q < w.capacity) {
                w.q_o[out][q] = ro;
                w.q_d[out][q] = rd;
                w.q_tp[out][q] = rtp;
            } else {
                atomicOr(src.scene(0).status, ST_QUEUE);
            }
        }
    }
}

// Shadow: any-hit test of each queued shadow ray; unoccluded contributions are added to the path.
// At most one shadow ray per path per bounce, so the read-modify-write of L needs no atomics.
template <class Src, bool SIG>
__global__ void __launch_bounds__(256) k_shadow(Src src, WfBuffers w, uint32_t b) {
    const uint32_t n = min(w.counts[2], w.capacity);
    const uint64_t base = src.base();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const float4 so = w.s_o[j], sd = w.s_d[j], sc = w.s_c[j];
        const uint32_t pid = __float_as_uint(sd.w);
        const bool occ = trace_any(src.scene(src.sid_from_shadow(sc.w, base, pid)), xyz(so), xyz(sd), so.w);
        if (!occ) {
            float3 L = add_rn(xyz(w.L[pid]), xyz(sc));
            w.L[pid] = f4(L, 0.f);
        }
        if (SIG) {
            const uint32_t lj = __float_as_uint(sc.w);
            w.sig[base + pid] ^= sig_event(b, 1, (lj << 2) | 2u | (occ ? 0u : 1u));
        }
    }
}

// ---- hybrid wavefront / megakernel (the hybrid of the paper's future work, Sec. 5): once the
// active count entering a bounce is at most `threshold`, one persistent kernel finishes every
// remaining path in registers (the megakernel's loop body, lanes claiming queue entries as they
// free up) instead of running the remaining bounces as sparse wavefront stages.  The decision is
// taken on the device; k_finish_commit then empties the queue so the remaining stage launches find
// no work.  The arithmetic per path is the same as in the wavefront stages, so images are identical.
template <bool SIG, bool MIS>
__global__ void __launch_bounds__(128, 8) k_finish(SingleSrc src, WfBuffers w, int in, uint32_t b0, uint32_t threshold,
                                                  unsigned long long* __restrict__ claim) {
    __shared__ unsigned int h_s[128];     // [b]: extension rays, [64 + b]: shadow rays of bounce b
    const uint32_t n = min(w.counts[0], w.capacity);
    if (n == 0u || n > threshold) return;  // the same value for every thread of the grid
    for (uint32_t k = threadIdx.x; k < 128u; k += blockDim.x) h_s[k] = 0u;
    __syncthreads();
    const DevScene& s = src.s;
    const RenderParams& p = src.p;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    unsigned long long n_ext = 0, n_shd = 0;
    bool active = false, exhausted = false;
    uint32_t pid = 0, key = 0, b = 0, sg = 0;
    uint64_t path = 0;
    float3 o = f3(0.f, 0.f, 0.f), d = o, tp = o, L = o;
    bool prev_delta = true;
    float prev_pdf = 0.f;
    while (true) {
        const bool want = !active && !exhausted;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, want);
        if (m) {
            const uint32_t leader = __ffs(m) - 1u;
            unsigned long long first = 0;
            if (lane_id() == leader) first = atomicAdd(claim, (unsigned long long)__popc(m));
            first = __shfl_sync(0xFFFFFFFFu, first, leader);
            if (want) {
                const uint64_t j = first + (uint64_t)__popc(m & ((1u << lane_id()) - 1u));
                if (j < n) {
                    const float4 o4 = w.q_o[in][j], d4 = w.q_d[in][j], tp4 = w.q_tp[in][j];
                    pid = __float_as_uint(o4.w);
                    const PathLoc l = src.locate(p.path_begin, pid);
                    path = l.path;
                    key = path_key(p.seed, l.pixel, l.sample);
                    o = xyz(o4);
                    d = xyz(d4);
                    tp = xyz(tp4);
                    prev_delta = (__float_as_uint(d4.w) & 1u) != 0u;
                    prev_pdf = tp4.w;
                    L = xyz(w.L[pid]);
                    b = b0;
                    sg = 0;
                    active = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        if (active) {
            const uint32_t bb = b;
            const unsigned long long shd0 = n_shd;
            atomicAdd(&h_s[bb & 63u], 1u);
            const bool end = mk_bounce<SIG, MIS>(s, p, env, key, b, o, d, tp, prev_delta, prev_pdf, L, sg, n_ext, n_shd);
            if (n_shd != shd0) atomicAdd(&h_s[64u + (bb & 63u)], 1u);
            if (end) {
                w.L[pid] = f4(L, 0.f);
                if (SIG) w.sig[path] ^= sg;
                active = false;
            }
        }
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < 128u; k += blockDim.x)
        if (h_s[k]) atomicAdd(&w.hist[k], (unsigned long long)h_s[k]);
}

__global__ void k_finish_commit(WfBuffers w, uint32_t threshold, unsigned long long* claim) {
    const uint32_t n = min(w.counts[0], w.capacity);
    if (n > 0u && n <= threshold) w.counts[0] = 0u;
    *claim = 0ull;
}

// ---- wavefront adjoint: shading that records what the reverse pass needs instead of adding
// radiance (the same shade_vertex decisions, so the replay follows the forward paths exactly).
__global__ void __launch_bounds__(256, 3) k_shade_adj(SingleSrc src, WfBuffers w, AdjBuffers a, int in, uint32_t b) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint64_t base = src.base();
    const int out = in ^ 1;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const size_t cap = w.capacity;
    for (uint32_t wb = warp * 32u; wb < n; wb += n_warps * 32u) {
        const uint32_t j = wb + lane_id();
        bool want_ray = false, want_shadow = false;
        float4 ro, rd, rtp, so, sd;
        if (j < n) {
            const float4 o4 = w.q_o[in][j], d4 = w.q_d[in][j], tp4 = w.q_tp[in][j];
            const float2 hh = w.hit[j];
            const uint32_t pid = __float_as_uint(o4.w);
            const uint32_t tri = __float_as_uint(hh.y);
            if (tri == kMiss) {
                a.pend[pid] = b | (1u << 8);
            } else {
                const PathLoc l = src.locate(base, pid);
                const RenderParams& p = src.p;
                const uint32_t key = path_key(p.seed, l.pixel, l.sample);
                Vertex V = shade_vertex(src.s, p, key, b, xyz(o4), xyz(d4), xyz(tp4), (__float_as_uint(d4.w) & 1u) != 0u,
                                        tp4.w, hh.x, tri);
                uint32_t flags = V.emit_counted ? 4u : 0u;
                const float Le = V.emit_counted ? __ldg(&src.s.mats[V.mat].emission) * V.emit_w : 0.f;
                float Lj = 0.f;
                float4 r1 = make_float4(0.f, 0.f, 0.f, 0.f), r2 = r1;
                if (!V.last) {
                    if (V.nee && V.cast) {
                        want_shadow = true;
                        flags |= 8u;
                        so = f4(V.s_o, V.s_tmax);
                        sd = f4(V.s_d, __uint_as_float(pid));
                        r2 = f4(V.nee_g, V.nee_dfa.x);
                        Lj = __ldg(&src.s.mats[V.light_mat].emission);
                    }
                    if (V.cont) {
                        want_ray = true;
                        flags |= 1u;
                        r1 = f4(V.w, V.dwa.x);
                        ro = f4(V.no, __uint_as_float(pid));
                        rd = f4(V.nd, __uint_as_float(V.delta ? 1u : 0u));
                        rtp = f4(V.ntp, V.pdf);
                    }
                }
                float4* r = a.rec + 4 * ((size_t)b * cap + pid);
                r[0] = make_float4(tp4.x, tp4.y, tp4.z, __uint_as_float(V.mat));
                r[1] = r1;
                r[2] = r2;
                r[3] = make_float4(Le, Lj, V.emit_w, __uint_as_float(flags | (V.light_mat << 4)));
                if (!V.cont || V.last) a.pend[pid] = b + 1u;
            }
        }
        const uint32_t k = warp_append(&w.counts[2], want_shadow);
        if (want_shadow) {
            if (k < w.capacity) {
                w.s_o[k] = so;
                w.s_d[k] = sd;
            } else {
                atomicOr(src.s.status, ST_QUEUE);
            }
        }
        const uint32_t q = warp_append(&w.counts[1], want_ray);
        if (want_ray) {
            if (q < w.capacity) {
                w.q_o[out][q] = ro;
                w.q_d[out][q] = rd;
                w.q_tp[out][q] = rtp;
            } else {
                atomicOr(src.s.status, ST_QUEUE);
            }
        }
    }
}

// Wavefront adjoint shadow stage: mark the vertex's NEE sample visible when unoccluded.
__global__ void __launch_bounds__(256) k_shadow_adj(SingleSrc src, WfBuffers w, AdjBuffers a, uint32_t b) {
    const uint32_t n = min(w.counts[2], w.capacity);
    const size_t cap = w.capacity;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const float4 so = w.s_o[j], sd = w.s_d[j];
        if (!trace_any(src.s, xyz(so), xyz(sd), so.w)) {
            const uint32_t pid = __float_as_uint(sd.w);
            float* fl = reinterpret_cast<float*>(a.rec + 4 * ((size_t)b * cap + pid) + 3) + 3;
            *fl = __uint_as_float(__float_as_uint(*fl) | 2u);
        }
    }
}

// Prepare (Sec. 3.1): record this bounce's counts, promote the next count, reset the slots.
__global__ void k_prepare(WfBuffers w, uint32_t b) {
    w.hist[b] += w.counts[0];
    w.hist[64 + b] += w.counts[2];
    w.counts[0] = w.counts[1];
    w.counts[1] = 0u;
    w.counts[2] = 0u;
}

// ================================================================== accumulation
__global__ void __launch_bounds__(256) k_reduce(const float* __restrict__ L, uint32_t stride_f, uint64_t pixel_begin,
                                                uint64_t n_pixels, uint32_t spp, float* __restrict__ img) {
    const float inv = 1.0f / (float)spp;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t px = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; px < n_pixels; px += stride) {
        float r = 0.f, g = 0.f, bl = 0.f;
        const float* q = L + px * spp * stride_f;
        for (uint32_t smp = 0; smp < spp; ++smp) {
            r = __fadd_rn(r, q[smp * stride_f]);
            g = __fadd_rn(g, q[smp * stride_f + 1]);
            bl = __fadd_rn(bl, q[smp * stride_f + 2]);
        }
        float* o = img + 3 * (pixel_begin + px);
        o[0] = __fmul_rn(r, inv);
        o[1] = __fmul_rn(g, inv);
        o[2] = __fmul_rn(bl, inv);
    }
}

// Progressive accumulation (the running average of Sec. 2.3): add this call's samples of each
// pixel, in sample order, to the pixel's FP32 running sum and write sum / count (img may be null).
// Continuing the sum is exactly what the one-call reduce does, so frames of k1, k2, ... samples end
// at the image of one call with k1 + k2 + ... samples, bit for bit.
__global__ void __launch_bounds__(256) k_accumulate(const float* __restrict__ L, uint32_t stride_f,
                                                    uint64_t pixel_begin, uint64_t n_pixels, uint32_t spp,
                                                    float* __restrict__ sum, uint32_t count, float* __restrict__ img) {
    const float inv = 1.0f / (float)count;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t px = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; px < n_pixels; px += stride) {
        float* a = sum + 3 * (pixel_begin + px);
        float r = a[0], g = a[1], bl = a[2];
        const float* q = L + px * spp * stride_f;
        for (uint32_t smp = 0; smp < spp; ++smp) {
            r = __fadd_rn(r, q[smp * stride_f]);
            g = __fadd_rn(g, q[smp * stride_f + 1]);
            bl = __fadd_rn(bl, q[smp * stride_f + 2]);
        }
        a[0] = r;
        a[1] = g;
        a[2] = bl;
        if (img) {
            float* o = img + 3 * (pixel_begin + px);
            o[0] = __fmul_rn(r, inv);
            o[1] = __fmul_rn(g, inv);
            o[2] = __fmul_rn(bl, inv);
        }
    }
}

__global__ void k_copy_L(const float4* __restrict__ L4, uint64_t n, float* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float4 v = L4[i];
        out[3 * i] = v.x;
        out[3 * i + 1] = v.y;
        out[3 * i + 2] = v.z;
    }
}

// Batched accumulation: add this wave's samples of each pixel, in sample order, to the pixel's
// running FP32 sum in its scene's output image (zeroed before the first wave).  A pixel split
// between two waves continues from the stored partial sum, so the additions are exactly those of
// the single-scene reduce.
__global__ void __launch_bounds__(256) k_reduce_batch(BatchTables t, const float4* __restrict__ L,
                                                      const BatchSegment* __restrict__ seg, uint32_t n_seg,
                                                      unsigned long long w0, unsigned long long w1,
                                                      unsigned long long n_flat) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_flat; f += stride) {
        uint32_t lo = 0, hi = n_seg - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (seg[mid].flat_begin <= f) lo = mid;
            else hi = mid - 1;
        }
        const BatchSegment sg = seg[lo];
        const uint64_t px = sg.px_begin + (f - sg.flat_begin);
        const uint32_t spp = t.spp[sg.scene];
        const uint64_t first = t.off[sg.scene] + px * spp;
        const uint64_t a = first > w0 ? first : w0;
        const uint64_t e = first + spp < w1 ? first + spp : w1;
        float* o = t.out[sg.scene] + 3 * px;
        float r = o[0], g = o[1], bl = o[2];
        for (uint64_t q = a; q < e; ++q) {
            const float4 v = L[q - w0];
            r = __fadd_rn(r, v.x);
            g = __fadd_rn(g, v.y);
            bl = __fadd_rn(bl, v.z);
        }
        o[0] = r;
        o[1] = g;
        o[2] = bl;
    }
}

// Batched accumulation, last step: sums -> means (the single-scene reduce's final multiply).
__global__ void k_scale_batch(BatchTables t, const unsigned long long* __restrict__ px_off, unsigned long long total) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
        uint32_t lo = 0, hi = t.n - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (px_off[mid] <= f) lo = mid;
            else hi = mid - 1;
        }
        const float inv = 1.0f / (float)t.spp[lo];
        float* o = t.out[lo] + 3 * (f - px_off[lo]);
        o[0] = __fmul_rn(o[0], inv);
        o[1] = __fmul_rn(o[1], inv);
        o[2] = __fmul_rn(o[2], inv);
    }
}

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

// Gradient of sum_p <grad[p], img[p]> with respect to albedo and emission.  Each path is re-traced
// with the forward pass's random numbers and decisions; per vertex b the radiance still to come per
// unit throughput R_b = Le_b + f_b G A Le_light + w_b R_{b+1} is built backward, and
//   d/d albedo(m_b)   += delta * tp_b * (dw_b/da * R_{b+1} + d(NEE_b)/da)
//   d/d emission(m_b) += delta . tp_b                (emission counted at b)
//   d/d emission(light material) += delta . tp_b * f_b G A   (visible NEE)
// Loops are warp-uniform so that the per-vertex adds can be aggregated across the warp.
template <int MAXD>
__global__ void __launch_bounds__(256) k_adjoint(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                 const float* __restrict__ grad, float* __restrict__ g_alb,
                                                 float* __restrict__ g_em, int smem) {
    extern __shared__ float acc[];
    if (smem)
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    const float inv_spp = 1.0f / (float)p.spp;
    AdjRec rec[MAXD];
    for (uint64_t base = warp * 32; base < n_paths; base += n_warps * 32) {
        const uint64_t i = base + lane_id();
        int nv = 0;
        bool end_miss = false;
        float3 delta = f3(0.f, 0.f, 0.f);
        if (i < n_paths) {
            const uint64_t path = p.path_begin + i;
            const uint32_t pixel = (uint32_t)(path / p.spp);
            const uint32_t sample = p.sample_offset + (uint32_t)(path - (uint64_t)pixel * p.spp);
            const uint32_t key = path_key(p.seed, pixel, sample);
            float3 o, d;
            float u0, u1;
            pixel_jitter(p.sampler, p.seed, pixel, sample, key, u0, u1);
            camera_ray(c, pixel, u0, u1, o, d);
            float3 tp = f3(1.f, 1.f, 1.f);
            bool prev_delta = true;
            float prev_pdf = 0.f;
            for (uint32_t b = 0; b < p.max_depth && b < (uint32_t)MAXD; ++b) {
                Hit h = trace_closest(s, o, d);
                if (h.tri == kMiss) {
                    end_miss = true;
                    break;
                }
                Vertex V = shade_vertex(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri);
                AdjRec& r = rec[nv++];
                r.tp = tp;
                r.mat = V.mat;
                r.flags = V.emit_counted ? 4u : 0u;
                r.Le = V.emit_counted ? __ldg(&s.mats[V.mat].emission) * V.emit_w : 0.f;
                r.we = V.emit_w;
                r.lmat = V.light_mat;
                r.nee_g = f3(0.f, 0.f, 0.f);
                r.nee_dfa = r.nee_g;
                r.w = r.nee_g;
                r.dwa = r.nee_g;
                r.Lj = 0.f;
                if (V.last) break;
                if (V.nee && V.cast && !trace_any(s, V.s_o, V.s_d, V.s_tmax)) {
                    r.flags |= 2u;
                    r.nee_g = V.nee_g;
                    r.nee_dfa = V.nee_dfa;
                    r.Lj = __ldg(&s.mats[V.light_mat].emission);
                }
                if (!V.cont) break;
                r.flags |= 1u;
                r.w = V.w;
                r.dwa = V.dwa;
                o = V.no;
                d = V.nd;
                tp = V.ntp;
                prev_delta = V.delta;
                prev_pdf = V.pdf;
            }
            delta = f3(grad[3 * (size_t)pixel], grad[3 * (size_t)pixel + 1], grad[3 * (size_t)pixel + 2]) * inv_spp;
        }
        float3 R = end_miss ? env : f3(0.f, 0.f, 0.f);
        const int nmax = __reduce_max_sync(0xFFFFFFFFu, nv);
        for (int b = nmax - 1; b >= 0; --b) {
            uint32_t key_m = kNoKey, key_l = kNoKey;
            float4 vm = make_float4(0.f, 0.f, 0.f, 0.f), vl = vm;
            if (b < nv) {
                const AdjRec& r = rec[b];
                const float3 dtp = delta * r.tp;
                float3 ga = f3(0.f, 0.f, 0.f);
                float ge = 0.f;
                if (r.flags & 1u) {
                    ga = dtp * r.dwa * R;
                    R = r.w * R;
                }
                if (r.flags & 2u) {
                    ga = ga + dtp * r.nee_dfa;
                    key_l = r.lmat;
                    vl.w = dot(dtp, r.nee_g);
                    R = R + r.nee_g * r.Lj;
                }
                if (r.flags & 4u) {
                    ge = (dtp.x + dtp.y + dtp.z) * r.we;
                    R = R + f3(r.Le, r.Le, r.Le);
                }
                key_m = r.mat;
                vm = make_float4(ga.x, ga.y, ga.z, ge);
            }
            warp_accumulate(acc, g_alb, g_em, smem != 0, key_m, vm);
            warp_accumulate(acc, g_alb, g_em, smem != 0, key_l, vl);
        }
    }
    if (smem) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) {
            float v = acc[k];
            if (v != 0.f) {
                uint32_t m = k >> 2, ch = k & 3u;
                if (ch < 3u) atomicAdd(&g_alb[3 * m + ch], v);
                else atomicAdd(&g_em[m], v);
            }
        }
    }
}

// Wavefront adjoint, reverse pass: one thread per path of the wave (consecutive paths per warp, so
// record loads coalesce and neighbouring pixels share materials), walking the vertex records
// backward with the recursion of k_adjoint.
__global__ void __launch_bounds__(256) k_adjoint_reverse(DevScene s, RenderParams p, WfBuffers w, AdjBuffers a,
                                                         uint32_t n, const float* __restrict__ grad,
                                                         float* __restrict__ g_alb, float* __restrict__ g_em,
                                                         int smem) {
    extern __shared__ float acc[];
    if (smem)
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    const float inv_spp = 1.0f / (float)p.spp;
    const size_t cap = w.capacity;
    for (uint32_t wb = warp * 32u; wb < n; wb += n_warps * 32u) {
        const uint32_t pid = wb + lane_id();
        int nv = 0;
        float3 delta = f3(0.f, 0.f, 0.f), R = f3(0.f, 0.f, 0.f);
        if (pid < n) {
            const uint32_t pe = a.pend[pid];
            nv = (int)(pe & 0xFFu);
            if (pe & 0x100u) R = env;
            const uint64_t path = p.path_begin + pid;
            const uint32_t pixel = (uint32_t)(path / p.spp);
            delta = f3(grad[3 * (size_t)pixel], grad[3 * (size_t)pixel + 1], grad[3 * (size_t)pixel + 2]) * inv_spp;
        }
        const int nmax = __reduce_max_sync(0xFFFFFFFFu, nv);
        for (int b = nmax - 1; b >= 0; --b) {
            uint32_t key_m = kNoKey, key_l = kNoKey;
            float4 vm = make_float4(0.f, 0.f, 0.f, 0.f), vl = vm;
            if (b < nv) {
                const float4* r = a.rec + 4 * ((size_t)b * cap + pid);
                const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
                const uint32_t flags = __float_as_uint(r3.w) & 15u;
                const float3 dtp = delta * xyz(r0);
                float3 ga = f3(0.f, 0.f, 0.f);
                float ge = 0.f;
                if (flags & 1u) {
                    ga = dtp * R * r1.w;
                    R = xyz(r1) * R;
                }
                if ((flags & 10u) == 10u) {            // cast and visible
                    const float3 ng = xyz(r2);
                    ga = ga + dtp * r2.w;
                    key_l = __float_as_uint(r3.w) >> 4;
                    vl.w = dot(dtp, ng);
                    R = R + ng * r3.y;
                }
                if (flags & 4u) {
                    ge = (dtp.x + dtp.y + dtp.z) * r3.z;
                    R = R + f3(r3.x, r3.x, r3.x);
                }
                key_m = __float_as_uint(r0.w);
                vm = make_float4(ga.x, ga.y, ga.z, ge);
            }
            warp_accumulate(acc, g_alb, g_em, smem != 0, key_m, vm);
            warp_accumulate(acc, g_alb, g_em, smem != 0, key_l, vl);
        }
    }
    if (smem) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) {
            float v = acc[k];
            if (v != 0.f) {
                uint32_t m = k >> 2, ch = k & 3u;
                if (ch < 3u) atomicAdd(&g_alb[3 * m + ch], v);
                else atomicAdd(&g_em[m], v);
            }
        }
    }
}

// ================================================================== utilities
__global__ void k_set_materials(DevMat* mats, uint32_t n, const float* albedo, const float* emission) {
    uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    if (albedo) {
        mats[m].ar = albedo[3 * m];
        mats[m].ag = albedo[3 * m + 1];
        mats[m].ab = albedo[3 * m + 2];
    }
    if (emission) mats[m].emission = emission[m];
}

__global__ void __launch_bounds__(256) k_trace_closest(DevScene s, const float* __restrict__ rays, uint32_t n,
                                                       float* __restrict__ t, int32_t* __restrict__ prim) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float* r = rays + 8 * (size_t)i;
        Hit h = trace_closest(s, f3(r[0], r[1], r[2]), f3(r[4], r[5], r[6]));
        t[i] = h.t;
        prim[i] = h.tri == kMiss ? -1 : (int32_t)__float_as_uint(__ldg(s.tris + 3 * (size_t)h.tri).w);
    }
}

__global__ void k_debug_rng(uint64_t seed, const uint32_t* px, const uint32_t* sm, const uint32_t* bo,
                            const uint32_t* dm, uint32_t n, float* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = u01(path_key(seed, px[i], sm[i]), bo[i], dm[i]);
}

// ================================================================== launchers
cudaError_t launch_megakernel_regen(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                                    uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays,
                                    unsigned long long* next_path) {
    if (p.mis) {
        if (sig) k_megakernel_regen<true, true><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path);
        else k_megakernel_regen<false, true><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path);
    } else {
        if (sig) k_megakernel_regen<true, false><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path);
        else k_megakernel_regen<false, false><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path);
    }
    return cudaGetLastError();
}

cudaError_t launch_megakernel(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                              uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays) {
    if (p.mis) {
        if (sig) k_megakernel<true, true><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
        else k_megakernel<false, true><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
    } else {
        if (sig) k_megakernel<true, false><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
        else k_megakernel<false, false><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
    }
    return cudaGetLastError();
}

cudaError_t launch_debug_paths(cudaStream_t st, const DevScene& s, const DevCamera& c, const RenderParams& p,
                               const unsigned long long* ids, uint32_t n, uint32_t* ev_u, float* ev_f, uint32_t* n_ev,
                               float* out_L) {
    if (n == 0) return cudaSuccess;
    k_debug_paths<<<(n + 63) / 64, 64, 0, st>>>(s, c, p, ids, n, ev_u, ev_f, n_ev, out_L);
    return cudaGetLastError();
}

cudaError_t launch_raygen(const Launch& l, const DevCamera& c, const RenderParams& p, uint32_t n, const WfBuffers& w) {
    SingleSrc src{DevScene{}, c, p};
    k_raygen<SingleSrc><<<l.grid, l.block, 0, l.st>>>(src, p.path_begin, n, w, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_extend(const Launch& l, const DevScene& s, const WfBuffers& w, int in, const RenderParams& p) {
    SingleSrc src{s, DevCamera{}, p};
    k_extend<SingleSrc><<<l.grid, l.block, 0, l.st>>>(src, w, in);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Launch& l, const DevScene& s, const WfBuffers& w, int in, uint32_t mode, uint32_t n_keys,
                        const RenderParams& p) {
    cudaError_t e = cudaMemsetAsync(w.bucket, 0, sizeof(uint32_t) * n_keys, l.st);
    if (e != cudaSuccess) return e;
    SingleSrc src{s, DevCamera{}, p};
    k_sort_keys<SingleSrc><<<l.grid, l.block, sizeof(uint32_t) * n_keys, l.st>>>(src, w, in, mode, n_keys);
    k_sort_scan<<<1, 1024, 0, l.st>>>(w, n_keys);
    k_sort_scatter<<<l.grid, l.block, 0, l.st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_shade(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce, bool sorted) {
    SingleSrc src{s, DevCamera{}, p};
    if (w.sig) k_shade<SingleSrc, true><<<l.grid, l.block, 0, l.st>>>(src, w, in, bounce, sorted);
    else k_shade<SingleSrc, false><<<l.grid, l.block, 0, l.st>>>(src, w, in, bounce, sorted);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                          uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    if (w.sig) k_shadow<SingleSrc, true><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
    else k_shadow<SingleSrc, false><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                          uint32_t b0, uint32_t threshold, unsigned long long* claim) {
    SingleSrc src{s, DevCamera{}, p};
    if (p.mis) {
        if (w.sig) k_finish<true, true><<<l.grid, l.block, 0, l.st>>>(src, w, in, b0, threshold, claim);
        else k_finish<false, true><<<l.grid, l.block, 0, l.st>>>(src, w, in, b0, threshold, claim);
    } else {
        if (w.sig) k_finish<true, false><<<l.grid, l.block, 0, l.st>>>(src, w, in, b0, threshold, claim);
        else k_finish<false, false><<<l.grid, l.block, 0, l.st>>>(src, w, in, b0, threshold, claim);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish_commit<<<1, 1, 0, l.st>>>(w, threshold, claim);
    return cudaGetLastError();
}

// ---- batched (TableSrc) launchers
cudaError_t launch_raygen_batch(const Launch& l, const BatchTables& t, const RenderParams& p, uint64_t base, uint32_t n,
                                const WfBuffers& w) {
    TableSrc src{t, p};
    k_raygen<TableSrc><<<l.grid, l.block, 0, l.st>>>(src, base, n, w, t.wave_base);
    return cudaGetLastError();
}

cudaError_t launch_bounce_batch(const Launch& le, const Launch& ls, const Launch& lw, const Launch& lk,
                                const BatchTables& t, const RenderParams& p, const WfBuffers& w, uint32_t b,
                                uint32_t sort_mode, uint32_t n_keys) {
    TableSrc src{t, p};
    const int in = (int)(b & 1u);
    k_extend<TableSrc><<<le.grid, le.block, 0, le.st>>>(src, w, in);
    if (n_keys) {
        cudaError_t e = cudaMemsetAsync(w.bucket, 0, sizeof(uint32_t) * n_keys, lk.st);
        if (e != cudaSuccess) return e;
        k_sort_keys<TableSrc><<<lk.grid, lk.block, sizeof(uint32_t) * n_keys, lk.st>>>(src, w, in, sort_mode, n_keys);
        k_sort_scan<<<1, 1024, 0, lk.st>>>(w, n_keys);
        k_sort_scatter<<<lk.grid, lk.block, 0, lk.st>>>(w);
    }
    k_shade<TableSrc, false><<<ls.grid, ls.block, 0, ls.st>>>(src, w, in, b, n_keys > 0);
    k_shadow<TableSrc, false><<<lw.grid, lw.block, 0, lw.st>>>(src, w, b);
    k_prepare<<<1, 1, 0, le.st>>>(w, b);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const Launch& l, const BatchTables& t, const float4* L, const BatchSegment* seg,
                                uint32_t n_seg, uint64_t w0, uint64_t w1, uint64_t n_flat) {
    if (n_flat == 0) return cudaSuccess;
    k_reduce_batch<<<l.grid, l.block, 0, l.st>>>(t, L, seg, n_seg, w0, w1, n_flat);
    return cudaGetLastError();
}

cudaError_t launch_scale_batch(const Launch& l, const BatchTables& t, const unsigned long long* px_off, uint64_t total) {
    if (total == 0) return cudaSuccess;
    k_scale_batch<<<l.grid, l.block, 0, l.st>>>(t, px_off, total);
    return cudaGetLastError();
}

cudaError_t launch_prepare(cudaStream_t st, const WfBuffers& w, uint32_t bounce) {
    k_prepare<<<1, 1, 0, st>>>(w, bounce);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const Launch& l, const float* L, uint32_t stride, uint64_t pixel_begin, uint64_t n_pixels,
                          uint32_t spp, float* img) {
    k_reduce<<<l.grid, l.block, 0, l.st>>>(L, stride, pixel_begin, n_pixels, spp, img);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const Launch& l, const float* L, uint32_t stride, uint64_t pixel_begin, uint64_t n_pixels,
                              uint32_t spp, float* sum, uint32_t count, float* img) {
    k_accumulate<<<l.grid, l.block, 0, l.st>>>(L, stride, pixel_begin, n_pixels, spp, sum, count, img);
    return cudaGetLastError();
}

cudaError_t launch_copy_L(const Launch& l, const float4* L4, uint64_t n, float* out_L3) {
    k_copy_L<<<l.grid, l.block, 0, l.st>>>(L4, n, out_L3);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                           uint64_t n_paths, const float* grad_img, float* g_albedo, float* g_emission,
                           uint32_t max_depth_cap) {
    size_t smem_bytes = sizeof(float) * 4 * (size_t)s.n_mats;
    int smem = smem_bytes <= 32 * 1024 ? 1 : 0;
    size_t sb = smem ? smem_bytes : 0;
    if (max_depth_cap <= 8)
        k_adjoint<8><<<l.grid, l.block, sb, l.st>>>(s, c, p, n_paths, grad_img, g_albedo, g_emission, smem);
    else if (max_depth_cap <= 16)
        k_adjoint<16><<<l.grid, l.block, sb, l.st>>>(s, c, p, n_paths, grad_img, g_albedo, g_emission, smem);
    else
        k_adjoint<32><<<l.grid, l.block, sb, l.st>>>(s, c, p, n_paths, grad_img, g_albedo, g_emission, smem);
    return cudaGetLastError();
}

cudaError_t launch_shade_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                             const AdjBuffers& a, int in, uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    k_shade_adj<<<l.grid, l.block, 0, l.st>>>(src, w, a, in, bounce);
    return cudaGetLastError();
}

cudaError_t launch_shadow_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                              const AdjBuffers& a, uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    k_shadow_adj<<<l.grid, l.block, 0, l.st>>>(src, w, a, bounce);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reverse(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                                   const AdjBuffers& a, uint32_t n, const float* grad, float* g_albedo,
                                   float* g_emission) {
    size_t smem_bytes = sizeof(float) * 4 * (size_t)s.n_mats;
    int smem = smem_bytes <= 32 * 1024 ? 1 : 0;
    k_adjoint_reverse<<<l.grid, l.block, smem ? smem_bytes : 0, l.st>>>(s, p, w, a, n, grad, g_albedo, g_emission, smem);
    return cudaGetLastError();
}

cudaError_t launch_set_materials(cudaStream_t st, DevMat* mats, uint32_t n, const float* albedo, const float* emission) {
    if (n == 0) return cudaSuccess;
    k_set_materials<<<(n + 255) / 256, 256, 0, st>>>(mats, n, albedo, emission);
    return cudaGetLastError();
}

cudaError_t launch_trace_closest(const Launch& l, const DevScene& s, const float* rays, uint32_t n, float* t,
                                 int32_t* prim) {
    k_trace_closest<<<l.grid, l.block, 0, l.st>>>(s, rays, n, t, prim);
    return cudaGetLastError();
}

cudaError_t launch_debug_rng(const Launch& l, uint64_t seed, const uint32_t* px, const uint32_t* sm,
                             const uint32_t* bo, const uint32_t* dm, uint32_t n, float* out) {
    k_debug_rng<<<(n + 255) / 256, 256, 0, l.st>>>(seed, px, sm, bo, dm, n, out);
    return cudaGetLastError();
}

int max_blocks_per_sm(int which, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (which) {
        case K_MEGA: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel<false, false>, block, 0); break;
        case K_MEGA_REGEN: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel_regen<false, false>, block, 0); break;
        case K_EXTEND: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<SingleSrc>, block, 0); break;
        case K_SHADE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<SingleSrc, false>, block, 0); break;
        case K_SHADOW: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow<SingleSrc, false>, block, 0); break;
        case K_EXTEND_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<TableSrc>, block, 0); break;
        case K_SHADE_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<TableSrc, false>, block, 0); break;
        case K_SHADOW_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow<TableSrc, false>, block, 0); break;
        case K_ADJOINT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<16>, block, 16 * 1024); break;
        case K_SHADE_ADJ: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade_adj, block, 0); break;
        case K_SHADOW_ADJ: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow_adj, block, 0); break;
        case K_FINISH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_finish<false, false>, block, 0); break;
        default: break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace pt
