// pt_k_wave.cu -- the wavefront pipeline (Sec. 2.3, 3, 3.1): raygen -> per bounce { extend ->
// (key sort) -> shade -> shadow -> prepare } -> accumulate.  Stages are linked by structure-of-arrays
// queues of 16-byte records (128-bit coalesced loads and stores); compaction is a warp-aggregated
// atomic append into the next queue (one atomic per warp instead of one per path), and the prepare
// step rotates the two-slot active count without a host round trip.  Grids are persistent (a
// multiple of the SM count) and stride over the device-side count, so no host read-back or
// indirect launch is needed.  Also the batched variants (many scenes, one wavefront).
#include <type_traits>

#include "pt_common.cuh"

namespace pt {

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
        w.counts[4] = 0u;
        w.counts[5] = 0u;
        w.counts[6] = 0u;      // no shadow rays pending for the first trace launch
        if (wave_base_dev) *wave_base_dev = base;
    }
}

// Extend: closest hit of every active ray (scene-intersection stage); hit records per queue slot.
// Registers capped for 6 resident blocks of 256 single-level (extend 2.73 -> 2.68 ms per 1080p step
// against 5 blocks) and 4 two-level (64 registers; 6 blocks measured slower, and without a bound
// ptxas takes 78 registers, leaving 3 blocks: 2.89 -> 3.00 ms per two-level frame).
// SK > 0: the walks keep their top SK stack entries in dynamic shared memory (single-level only).
// CNT: count the walks' node visits and triangle tests into the scene's traversal counters.
template <class Src, bool INST, int SK = 0, bool CNT = false>
__global__ void __launch_bounds__(256, INST ? 4 : 6) k_extend(Src src, WfBuffers w, int in) {
    stage_prologue();
    const uint32_t n = min(w.counts[0], w.capacity);
    if (n == 0u) return;       // an emptied queue: no claims (the same for every thread)
    const uint64_t base = src.base();
    const float4* __restrict__ qo = w.q_o[in];
    const float4* __restrict__ qd = w.q_d[in];
    float2* __restrict__ hit = w.hit;
    typename std::conditional<CNT, TravCount, NoCount>::type cnt;
    for (uint32_t b0 = warp_claim32(&w.counts[4]); b0 < n; b0 = warp_claim32(&w.counts[4])) {
        const uint32_t j = b0 + lane_id();
        if (j >= n) continue;
        float4 o4 = __ldcs(&qo[j]), d4 = __ldcs(&qd[j]);
        Hit h = trace_closest<INST, SK>(src.scene(src.sid_from_ray(d4.w, base, __float_as_uint(o4.w))), xyz(o4), xyz(d4),
                                        cnt);
        hit[j] = make_float2(h.t, __uint_as_float(h.tri));
        if (INST) w.hit_inst[j] = h.inst;
    }
    flush_count(src.scene(0), cnt, 0);
}

// Key sort before shading (counting sort): keys + block histograms, scan, scatter into `perm`.
template <class Src, bool INST>
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
            if (INST) {        // an instance may replace the mesh's material
                const uint32_t mw = __float_as_uint(__ldg(s.inst + 8 * (size_t)w.hit_inst[j] + 3).z);
                if (mw != 0u) m = (mw & 0x7FFFFFFFu) - 1u;
            }
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

// Queue records (rays, hits, shadow rays) are loaded and stored with the streaming cache hint
// (__ldcs / __stcs: evict first from L2).  A bounce's queues (about 100 MB at 1080p) would otherwise
// push the scene (39 MB of nodes, 55 MB of triangles) out of the 126 MB L2, and deep-bounce walks then
// wait on DRAM for every node: with the hint the wavefront frame runs 1-1.5% faster at every depth.

// Shading of one queue entry (emission, NEE sample, BSDF sample, roulette): the records of its
// continuation ray and shadow ray, if any.
struct ShadeOut {
    bool want_ray = false, want_shadow = false;
    float4 ro, rd, rtp, so, sd, sc;
};

template <class Src, bool SIG, bool INST>
__device__ __forceinline__ ShadeOut shade_entry(const Src& src, const WfBuffers& w, int in, uint32_t b, bool sorted,
                                                uint64_t base, uint32_t j) {
    ShadeOut r;
    const uint32_t slot = sorted ? w.perm[j] : j;
    const float4 o4 = __ldcs(&w.q_o[in][slot]), d4 = __ldcs(&w.q_d[in][slot]), tp4 = __ldcs(&w.q_tp[in][slot]);
    const float2 hh = __ldcs(&w.hit[slot]);
    const uint32_t pid = __float_as_uint(o4.w);
    const PathLoc l = src.locate_in(base, pid, src.sid_from_ray(d4.w, base, pid));
    const DevScene s = src.scene(l.sid);
    const float3 tp = xyz(tp4);
    const uint32_t tri = __float_as_uint(hh.y);
    if (tri == kMiss) {
        float3 L = add_rn(xyz(w.L[pid]), mul_rn(tp, f3(s.env_r, s.env_g, s.env_b)));
        w.L[pid] = f4(L, 0.f);
        if (SIG) w.sig[l.path] ^= sig_event(b, 0, kMiss);
        return r;
    }
    const RenderParams p = src.params(l.sid);
    const uint32_t key = path_key(p.seed, l.pixel, l.sample);
    Vertex V = shade_vertex<true, INST>(s, p, key, b, xyz(o4), xyz(d4), tp, (__float_as_uint(d4.w) & 1u) != 0u, tp4.w,
                                        hh.x, tri, INST ? w.hit_inst[slot] : kMiss);
    if (V.emit_counted) {
        float3 L = add_rn(xyz(w.L[pid]), V.emit);
        w.L[pid] = f4(L, 0.f);
    }
    uint32_t sg = 0;
    if (SIG) sg = sig_event(b, 0, V.prim);
    if (!V.last) {
        if (V.nee) {
            if (V.cast) {
                r.want_shadow = true;
                r.so = f4(V.s_o, V.s_tmax);
                r.sd = f4(V.s_d, __uint_as_float(pid));
                r.sc = f4(V.contrib, __uint_as_float(src.shadow_tag(V.light_j, l.sid)));
            } else if (SIG) {
                sg ^= sig_event(b, 1, V.light_j << 2);
            }
        }
        if (SIG) {
            sg ^= sig_event(b, 2, V.bsdf_code);
            if (V.rr >= 0) sg ^= sig_event(b, 3, (uint32_t)V.rr);
        }
        if (V.cont) {
            r.want_ray = true;
            r.ro = f4(V.no, __uint_as_float(pid));
            r.rd = f4(V.nd, __uint_as_float(src.ray_tag(l.sid, V.delta ? 1u : 0u)));
            r.rtp = f4(V.ntp, V.pdf);
        }
    }
    if (SIG) w.sig[l.path] ^= sg;
    return r;
}

template <class Src>
__device__ __forceinline__ void put_shadow(const Src& src, const WfBuffers& w, uint32_t k, const ShadeOut& r) {
    if (k < w.capacity) {
        __stcs(&w.s_o[k], r.so);
        __stcs(&w.s_d[k], r.sd);
        __stcs(&w.s_c[k], r.sc);
    } else {
        atomicOr(src.scene(0).status, ST_QUEUE);
    }
}

template <class Src>
__device__ __forceinline__ void put_ray(const Src& src, const WfBuffers& w, int out, uint32_t q, const ShadeOut& r) {
    if (q < w.capacity) {
        __stcs(&w.q_o[out][q], r.ro);
        __stcs(&w.q_d[out][q], r.rd);
        __stcs(&w.q_tp[out][q], r.rtp);
    } else {
        atomicOr(src.scene(0).status, ST_QUEUE);
    }
}

// Shade: emission, NEE sample (-> shadow queue), BSDF sample, roulette, compaction of survivors: each
// warp appends its survivors with one atomic per queue (warp-aggregated).
template <class Src, bool SIG, bool INST>
__global__ void __launch_bounds__(256, 3) k_shade(Src src, WfBuffers w, int in, uint32_t b, bool sorted) {
    stage_prologue();
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint64_t base = src.base();
    const int out = in ^ 1;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wb = warp * 32u; wb < n; wb += n_warps * 32u) {
        const uint32_t j = wb + lane_id();
        ShadeOut r;
        if (j < n) r = shade_entry<Src, SIG, INST>(src, w, in, b, sorted, base, j);
        const uint32_t k = warp_append(&w.counts[2], r.want_shadow);
        if (r.want_shadow) put_shadow(src, w, k, r);
        const uint32_t q = warp_append(&w.counts[1], r.want_ray);
        if (r.want_ray) put_ray(src, w, out, q, r);
    }
}

// Shadow: any-hit test of each queued shadow ray; unoccluded contributions are added to the path.
// At most one shadow ray per path per bounce, so the read-modify-write of L needs no atomics.
template <class Src, bool SIG, bool INST, int SK = 0, bool CNT = false>
__global__ void __launch_bounds__(256) k_shadow(Src src, WfBuffers w, uint32_t b) {
    const uint32_t n = min(w.counts[2], w.capacity);
    if (n == 0u) return;
    const uint64_t base = src.base();
    typename std::conditional<CNT, TravCount, NoCount>::type cnt;
    for (uint32_t b0 = warp_claim32(&w.counts[5]); b0 < n; b0 = warp_claim32(&w.counts[5])) {
        const uint32_t j = b0 + lane_id();
        if (j >= n) continue;
        const float4 so = __ldcs(&w.s_o[j]), sd = __ldcs(&w.s_d[j]), sc = __ldcs(&w.s_c[j]);
        const uint32_t pid = __float_as_uint(sd.w);
        const bool occ =
            trace_any<INST, SK>(src.scene(src.sid_from_shadow(sc.w, base, pid)), xyz(so), xyz(sd), so.w, cnt);
        if (!occ) {
            float3 L = add_rn(xyz(w.L[pid]), xyz(sc));
            w.L[pid] = f4(L, 0.f);
        }
        if (SIG) {
            const uint32_t lj = __float_as_uint(sc.w);
            w.sig[base + pid] ^= sig_event(b, 1, (lj << 2) | 2u | (occ ? 0u : 1u));
        }
    }
    flush_count(src.scene(0), cnt, 2);
}

// The cooperative form of the fused trace stage: each group of G lanes takes one extension ray, then
// one shadow ray, per claim (trace_closest_group / trace_any_group, or their two-level forms); the
// group's first lane writes the result exactly as the one-lane form does.
constexpr uint32_t kCoopMinLanes = 2u;

template <class Src, bool SIG, bool INST, bool ADJ>
__device__ __noinline__ void trace_groups(const Src& src, const WfBuffers& w, const AdjBuffers& a, int in,
                                             uint32_t b, uint32_t n_ext, uint32_t n_shd, uint32_t G) {
    const uint64_t base = src.base();
    const uint32_t per = 32u / G, sub = lane_id() / G;
    const bool lead = (lane_id() & (G - 1u)) == 0u;
    unsigned long long led = 0;      // walks this lane's group traced, counted once per group
    const float4* __restrict__ qo = w.q_o[in];
    const float4* __restrict__ qd = w.q_d[in];
    for (uint32_t b0 = warp_claim(&w.counts[4], per); b0 < n_ext; b0 = warp_claim(&w.counts[4], per)) {
        const uint32_t j = b0 + sub;
        const bool valid = j < n_ext;
        float4 o4 = make_float4(0.f, 0.f, 0.f, 0.f), d4 = make_float4(0.f, 0.f, 1.f, 0.f);
        if (valid) {
            o4 = __ldcs(&qo[j]);
            d4 = __ldcs(&qd[j]);
        }
        const uint32_t sid = valid ? src.sid_from_ray(d4.w, base, __float_as_uint(o4.w)) : 0u;
        const Hit h = INST ? trace_closest_group_inst(src.scene(sid), xyz(o4), xyz(d4), valid, G)
                           : trace_closest_group(src.scene(sid), xyz(o4), xyz(d4), valid, G);
        if (valid && lead) {
            w.hit[j] = make_float2(h.t, __uint_as_float(h.tri));
            if (INST) w.hit_inst[j] = h.inst;
            ++led;
        }
    }
    for (uint32_t b0 = warp_claim(&w.counts[5], per); b0 < n_shd; b0 = warp_claim(&w.counts[5], per)) {
        const uint32_t k = b0 + sub;
        const bool valid = k < n_shd;
        float4 so = make_float4(0.f, 0.f, 0.f, 0.f), sd = make_float4(0.f, 0.f, 1.f, 0.f);
        float4 sc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            so = __ldcs(&w.s_o[k]);
            sd = __ldcs(&w.s_d[k]);
            if (!ADJ) sc = __ldcs(&w.s_c[k]);
        }
        const uint32_t pid = __float_as_uint(sd.w);
        const uint32_t sid = (valid && !ADJ) ? src.sid_from_shadow(sc.w, base, pid) : 0u;
        const bool occ = INST ? trace_any_group_inst(src.scene(sid), xyz(so), xyz(sd), so.w, valid, G)
                              : trace_any_group(src.scene(sid), xyz(so), xyz(sd), so.w, valid, G);
        if (!valid || !lead) continue;
        ++led;
        if constexpr (ADJ) {
            if (!occ) {
                float* fl = reinterpret_cast<float*>(a.rec + 4 * ((size_t)(b - 1u) * w.capacity + pid) + 3) + 3;
                *fl = __uint_as_float(__float_as_uint(*fl) | 2u);
            }
        } else {
            if (!occ) {
                float3 L = add_rn(xyz(w.L[pid]), xyz(sc));
                w.L[pid] = f4(L, 0.f);
            }
            if (SIG) {
                const uint32_t lj = __float_as_uint(sc.w);
                w.sig[base + pid] ^= sig_event(b - 1u, 1, (lj << 2) | 2u | (occ ? 0u : 1u));
            }
        }
    }
    warp_add_u64(&w.hist[kHistGroupWalks + __ffs((int)G) - 2], led);
}

// Trace (the extend stage of bounce b fused with the shadow stage of bounce b - 1): one launch walks
// the BVH for the continuation rays of bounce b (closest hit, queue `in`, counts[0] entries) and for
// the shadow rays that shading cast at bounce b - 1 (any hit, the shadow queue, counts[6] entries).
// The two sets are independent -- a shadow ray only adds its contribution to its path's radiance, and
// only the next shading reads that radiance -- so each path still adds its terms in the order
// emission(b - 1), NEE(b - 1), emission(b), as in the megakernel.  Warps claim 32 continuation rays
// at a time until none is left and then 32 shadow rays at a time (two loops, so each walk keeps the
// registers it has in its own stage); a launch therefore ends when both sets are done, and the shadow
// walks fill the extension walks' tail instead of running after a stage boundary.
// ADJ: the adjoint replay's variant, whose shadow walks mark the vertex record's NEE sample visible
// (flag 2 of record 3 of bounce b - 1) instead of adding a contribution.
template <class Src, bool SIG, bool INST, bool CNT = false, bool ADJ = false>
__global__ void __launch_bounds__(256, INST ? 4 : 6) k_trace(Src src, WfBuffers w, AdjBuffers a, int in, uint32_t b) {
    stage_prologue();
    const uint32_t n_ext = min(w.counts[0], w.capacity), n_shd = min(w.counts[6], w.capacity);
    if (n_ext + n_shd == 0u) return;       // the same for every thread
    const uint64_t base = src.base();
    // Lanes per walk: 1 while the walks fill the grid; once they are few (the sparse late bounces),
    // the largest power of two G <= 32 with walks x G <= the grid's threads (cooperative walks; the
    // counting instantiations keep the one-lane walk their counts describe).
    // The same for every thread: the counts are fixed during the launch.
    uint32_t G = 1u;
    if constexpr (!CNT) {
        const uint64_t threads = (uint64_t)gridDim.x * blockDim.x;
        while (G < 32u && (uint64_t)(n_ext + n_shd) * (2u * G) <= threads) G *= 2u;
        if (G < kCoopMinLanes) G = 1u;
    }
    if (G > 1u) {
        trace_groups<Src, SIG, INST, ADJ>(src, w, a, in, b, n_ext, n_shd, G);
        return;
    }
    typename std::conditional<CNT, TravCount, NoCount>::type cc, ca;
    {
        const float4* __restrict__ qo = w.q_o[in];
        const float4* __restrict__ qd = w.q_d[in];
        for (uint32_t b0 = warp_claim32(&w.counts[4]); b0 < n_ext; b0 = warp_claim32(&w.counts[4])) {
            const uint32_t j = b0 + lane_id();
            if (j >= n_ext) continue;
            const float4 o4 = __ldcs(&qo[j]), d4 = __ldcs(&qd[j]);
            Hit h = trace_closest<INST, 0>(src.scene(src.sid_from_ray(d4.w, base, __float_as_uint(o4.w))), xyz(o4),
                                           xyz(d4), cc);
            w.hit[j] = make_float2(h.t, __uint_as_float(h.tri));
            if (INST) w.hit_inst[j] = h.inst;
        }
    }
    for (uint32_t b0 = warp_claim32(&w.counts[5]); b0 < n_shd; b0 = warp_claim32(&w.counts[5])) {
        const uint32_t k = b0 + lane_id();
        if (k >= n_shd) continue;
        const float4 so = __ldcs(&w.s_o[k]), sd = __ldcs(&w.s_d[k]);
        const uint32_t pid = __float_as_uint(sd.w);
        if constexpr (ADJ) {
            if (!trace_any<INST, 0>(src.scene(0), xyz(so), xyz(sd), so.w, ca)) {
                float* fl = reinterpret_cast<float*>(a.rec + 4 * ((size_t)(b - 1u) * w.capacity + pid) + 3) + 3;
                *fl = __uint_as_float(__float_as_uint(*fl) | 2u);
            }
        } else {
            const float4 sc = __ldcs(&w.s_c[k]);
            const bool occ =
                trace_any<INST, 0>(src.scene(src.sid_from_shadow(sc.w, base, pid)), xyz(so), xyz(sd), so.w, ca);
            if (!occ) {
                float3 L = add_rn(xyz(w.L[pid]), xyz(sc));
                w.L[pid] = f4(L, 0.f);
            }
            if (SIG) {
                const uint32_t lj = __float_as_uint(sc.w);
                w.sig[base + pid] ^= sig_event(b - 1u, 1, (lj << 2) | 2u | (occ ? 0u : 1u));
            }
        }
    }
    flush_count(src.scene(0), cc, 0);
    flush_count(src.scene(0), ca, 2);
}

// Prepare after shading in the fused pipeline: record this bounce's counts, promote the next count,
// and hand the shadow rays shading just cast to the next trace launch (counts[2] -> counts[6]).
__global__ void k_prepare_fused(WfBuffers w, uint32_t b) {
    stage_prologue();
    w.hist[b] += w.counts[0];
    w.hist[64 + b] += w.counts[2];
    w.counts[0] = w.counts[1];
    w.counts[1] = 0u;
    w.counts[6] = w.counts[2];
    w.counts[2] = 0u;
    w.counts[4] = 0u;
    w.counts[5] = 0u;
}

// Prepare (Sec. 3.1): record this bounce's counts, promote the next count, reset the slots.
__global__ void k_prepare(WfBuffers w, uint32_t b) {
    w.hist[b] += w.counts[0];
    w.hist[64 + b] += w.counts[2];
    w.counts[0] = w.counts[1];
    w.counts[1] = 0u;
    w.counts[2] = 0u;
    w.counts[4] = 0u;      // the extend and shadow stages' work counters
    w.counts[5] = 0u;
}

// ================================================================== accumulation
__global__ void __launch_bounds__(256) k_reduce(const float* __restrict__ L, uint32_t stride_f, uint64_t pixel_begin,
                                                uint64_t n_pixels, uint32_t spp, float* __restrict__ img) {
    stage_prologue();
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


// ------------------------------------------------------------------ launchers

cudaError_t launch_raygen(const Launch& l, const DevCamera& c, const RenderParams& p, uint32_t n, const WfBuffers& w) {
    SingleSrc src{DevScene{}, c, p};
    k_raygen<SingleSrc><<<l.grid, l.block, 0, l.st>>>(src, p.path_begin, n, w, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_extend(const Launch& l, const DevScene& s, const WfBuffers& w, int in, const RenderParams& p) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) return launch_k(l, 0, k_extend<SingleSrc, true>, src, w, in);
    if (p.count_trav) return launch_k(l, 0, k_extend<SingleSrc, false, 0, true>, src, w, in);
    if (p.short_stack)
        return launch_k(l, stack_smem_bytes(kShortStack, l.block), k_extend<SingleSrc, false, kShortStack>, src, w, in);
    return launch_k(l, 0, k_extend<SingleSrc, false>, src, w, in);
}

cudaError_t launch_sort(const Launch& l, const DevScene& s, const WfBuffers& w, int in, uint32_t mode, uint32_t n_keys,
                        const RenderParams& p) {
    cudaError_t e = cudaMemsetAsync(w.bucket, 0, sizeof(uint32_t) * n_keys, l.st);
    if (e != cudaSuccess) return e;
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) k_sort_keys<SingleSrc, true><<<l.grid, l.block, sizeof(uint32_t) * n_keys, l.st>>>(src, w, in, mode, n_keys);
    else k_sort_keys<SingleSrc, false><<<l.grid, l.block, sizeof(uint32_t) * n_keys, l.st>>>(src, w, in, mode, n_keys);
    k_sort_scan<<<1, 1024, 0, l.st>>>(w, n_keys);
    k_sort_scatter<<<l.grid, l.block, 0, l.st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_shade(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce, bool sorted) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) {
        if (w.sig) return launch_k(l, 0, k_shade<SingleSrc, true, true>, src, w, in, bounce, sorted);
        return launch_k(l, 0, k_shade<SingleSrc, false, true>, src, w, in, bounce, sorted);
    }
    if (w.sig) return launch_k(l, 0, k_shade<SingleSrc, true, false>, src, w, in, bounce, sorted);
    return launch_k(l, 0, k_shade<SingleSrc, false, false>, src, w, in, bounce, sorted);
}

cudaError_t launch_shadow(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                          uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) {
        if (w.sig) k_shadow<SingleSrc, true, true><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
        else k_shadow<SingleSrc, false, true><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
    } else {
        const size_t sm = stack_smem_bytes(kShortStack, l.block);
        if (p.count_trav && !w.sig) {
            k_shadow<SingleSrc, false, false, 0, true><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
        } else if (p.short_stack) {
            if (w.sig) k_shadow<SingleSrc, true, false, kShortStack><<<l.grid, l.block, sm, l.st>>>(src, w, bounce);
            else k_shadow<SingleSrc, false, false, kShortStack><<<l.grid, l.block, sm, l.st>>>(src, w, bounce);
        } else {
            if (w.sig) k_shadow<SingleSrc, true, false><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
            else k_shadow<SingleSrc, false, false><<<l.grid, l.block, 0, l.st>>>(src, w, bounce);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_raygen_batch(const Launch& l, const BatchTables& t, const RenderParams& p, uint64_t base, uint32_t n,
                                const WfBuffers& w) {
    TableSrc src{t, p};
    k_raygen<TableSrc><<<l.grid, l.block, 0, l.st>>>(src, base, n, w, t.wave_base);
    return cudaGetLastError();
}

cudaError_t launch_bounce_batch(const Launch& le, const Launch& ls, const Launch& lw, const Launch& lk,
                                const BatchTables& t, const RenderParams& p, const WfBuffers& w, uint32_t b,
                                uint32_t sort_mode, uint32_t n_keys, bool fused) {
    TableSrc src{t, p};
    const int in = (int)(b & 1u);
    // fused and unsorted: the stage kernels are programmatic dependents of the kernel before them
    // (programmatic edges of the captured bounce graph; bounce 0's first launch opens the graph)
    const bool pdl = fused && n_keys == 0;
    Launch lt = lw, lsh = ls;
    lt.pdl = pdl;
    lsh.pdl = pdl;
    cudaError_t e;
    if (fused && b > 0)   // lw: the fused launch (this bounce's extension and the last bounce's shadow walks)
        e = launch_k(lt, 0, k_trace<TableSrc, false, false>, src, w, AdjBuffers{}, in, b);
    else
        e = launch_k(le, 0, k_extend<TableSrc, false>, src, w, in);
    if (e != cudaSuccess) return e;
    if (n_keys) {
        if ((e = cudaMemsetAsync(w.bucket, 0, sizeof(uint32_t) * n_keys, lk.st)) != cudaSuccess) return e;
        k_sort_keys<TableSrc, false><<<lk.grid, lk.block, sizeof(uint32_t) * n_keys, lk.st>>>(src, w, in, sort_mode, n_keys);
        k_sort_scan<<<1, 1024, 0, lk.st>>>(w, n_keys);
        k_sort_scatter<<<lk.grid, lk.block, 0, lk.st>>>(w);
    }
    if ((e = launch_k(lsh, 0, k_shade<TableSrc, false, false>, src, w, in, b, n_keys > 0)) != cudaSuccess) return e;
    if (fused) {
        return launch_prepare_fused(le.st, w, b, pdl);
    } else {
        k_shadow<TableSrc, false, false><<<lw.grid, lw.block, 0, lw.st>>>(src, w, b);
        k_prepare<<<1, 1, 0, le.st>>>(w, b);
    }
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

cudaError_t launch_trace(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    const AdjBuffers a{};
    if (s.tlas) {
        if (w.sig) return launch_k(l, 0, k_trace<SingleSrc, true, true>, src, w, a, in, bounce);
        return launch_k(l, 0, k_trace<SingleSrc, false, true>, src, w, a, in, bounce);
    }
    if (p.count_trav && !w.sig) return launch_k(l, 0, k_trace<SingleSrc, false, false, true>, src, w, a, in, bounce);
    if (w.sig) return launch_k(l, 0, k_trace<SingleSrc, true, false>, src, w, a, in, bounce);
    return launch_k(l, 0, k_trace<SingleSrc, false, false>, src, w, a, in, bounce);
}

cudaError_t launch_trace_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                             const AdjBuffers& a, int in, uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) return launch_k(l, 0, k_trace<SingleSrc, false, true, false, true>, src, w, a, in, bounce);
    return launch_k(l, 0, k_trace<SingleSrc, false, false, false, true>, src, w, a, in, bounce);
}

cudaError_t launch_prepare_fused(cudaStream_t st, const WfBuffers& w, uint32_t bounce, bool pdl) {
    Launch l;
    l.grid = 1;
    l.block = 1;
    l.st = st;
    l.pdl = pdl;
    return launch_k(l, 0, k_prepare_fused, w, bounce);
}

cudaError_t launch_prepare(cudaStream_t st, const WfBuffers& w, uint32_t bounce) {
    k_prepare<<<1, 1, 0, st>>>(w, bounce);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const Launch& l, const float* L, uint32_t stride, uint64_t pixel_begin, uint64_t n_pixels,
                          uint32_t spp, float* img) {
    return launch_k(l, 0, k_reduce, L, stride, pixel_begin, n_pixels, spp, img);
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

// Resident blocks per SM of this unit's kernels (0: not one of them).
int occupancy_wave(int which, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    const size_t sm = stack_smem_bytes(kShortStack, block);   // the short-stack instantiations' shared stacks
    switch (which) {
        case K_EXTEND: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<SingleSrc, false>, block, 0); break;
        case K_SHADE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shade<SingleSrc, false, false>), block, 0); break;
        case K_SHADOW: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shadow<SingleSrc, false, false>), block, 0); break;
        case K_EXTEND_SS:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<SingleSrc, false, kShortStack>, block, sm);
            break;
        case K_SHADOW_SS:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shadow<SingleSrc, false, false, kShortStack>), block, sm);
            break;
        case K_TRACE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_trace<SingleSrc, false, false>), block, 0); break;
        case K_TRACE_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_trace<SingleSrc, false, true>), block, 0); break;
        case K_TRACE_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_trace<TableSrc, false, false>), block, 0); break;
        case K_EXTEND_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<TableSrc, false>, block, 0); break;
        case K_SHADE_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shade<TableSrc, false, false>), block, 0); break;
        case K_SHADOW_BATCH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shadow<TableSrc, false, false>), block, 0); break;
        case K_EXTEND_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend<SingleSrc, true>, block, 0); break;
        case K_SHADE_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shade<SingleSrc, false, true>), block, 0); break;
        case K_SHADOW_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (k_shadow<SingleSrc, false, true>), block, 0); break;
        default: return 0;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace pt
