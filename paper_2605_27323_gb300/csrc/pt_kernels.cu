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
template <bool SIG>
__global__ void __launch_bounds__(256) k_megakernel(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                    float* __restrict__ out_L, float* __restrict__ img,
                                                    uint32_t* __restrict__ sig, unsigned long long* __restrict__ rays) {
    unsigned long long n_ext = 0, n_shd = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_paths; i += stride) {
        const uint64_t path = p.path_begin + i;
        const uint32_t pixel = (uint32_t)(path / p.spp);
        const uint32_t sample = (uint32_t)(path - (uint64_t)pixel * p.spp);
        const uint32_t key = path_key(p.seed, pixel, sample);
        float3 o, d;
        camera_ray(c, pixel, key, o, d);                       // step 1
        float3 tp = f3(1.f, 1.f, 1.f), L = f3(0.f, 0.f, 0.f);
        bool prev_delta = true;
        uint32_t sg = 0;
        for (uint32_t b = 0; b < p.max_depth; ++b) {
            ++n_ext;
            Hit h = trace_closest(s, o, d);                    // step 2
            if (h.tri == kMiss) {
                L = add_rn(L, mul_rn(tp, env));
                if (SIG) sg ^= sig_event(b, 0, kMiss);
                break;
            }
            Vertex V = shade_vertex(s, p, key, b, o, d, tp, prev_delta, h.t, h.tri);
            if (SIG) sg ^= sig_event(b, 0, V.prim);
            if (V.emit_counted) L = add_rn(L, V.emit);         // step 3
            if (V.last) break;
            if (V.nee) {                                       // shadow evaluation
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
            if (!V.cont) break;                                // step 4 done; step 5: repeat
            o = V.no;
            d = V.nd;
            tp = V.ntp;
            prev_delta = V.delta;
        }
        if (out_L) {
            out_L[3 * i] = L.x;
            out_L[3 * i + 1] = L.y;
            out_L[3 * i + 2] = L.z;
        } else {
            img[3 * (size_t)pixel] = L.x;
            img[3 * (size_t)pixel + 1] = L.y;
            img[3 * (size_t)pixel + 2] = L.z;
        }
        if (SIG) sig[path] = sg;
    }
    warp_add_u64(rays, n_ext);
    warp_add_u64(rays + 1, n_shd);
}

// ================================================================== wavefront stages
// Ray generation: one queue record per path of the wave, radiance zeroed, active count = n.
__global__ void __launch_bounds__(256) k_raygen(DevCamera c, RenderParams p, uint32_t n, WfBuffers w) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t path = p.path_begin + i;
        const uint32_t pixel = (uint32_t)(path / p.spp);
        const uint32_t sample = (uint32_t)(path - (uint64_t)pixel * p.spp);
        const uint32_t key = path_key(p.seed, pixel, sample);
        float3 o, d;
        camera_ray(c, pixel, key, o, d);
        w.q_o[0][i] = f4(o, __uint_as_float(i));
        w.q_d[0][i] = f4(d, __uint_as_float(1u));            // previous vertex "delta": the camera
        w.q_tp[0][i] = make_float4(1.f, 1.f, 1.f, 0.f);
        w.L[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (w.sig) w.sig[path] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.counts[0] = n;
        w.counts[1] = 0u;
        w.counts[2] = 0u;
    }
}

// Extend: closest hit of every active ray (scene-intersection stage); hit records per queue slot.
__global__ void __launch_bounds__(256) k_extend(DevScene s, WfBuffers w, int in) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const float4* __restrict__ qo = w.q_o[in];
    const float4* __restrict__ qd = w.q_d[in];
    float2* __restrict__ hit = w.hit;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        float4 o4 = qo[j], d4 = qd[j];
        Hit h = trace_closest(s, xyz(o4), xyz(d4));
        hit[j] = make_float2(h.t, __uint_as_float(h.tri));
    }
}

// Key sort before shading (counting sort): keys + block histograms, scan, scatter into `perm`.
__global__ void __launch_bounds__(256) k_sort_keys(DevScene s, WfBuffers w, uint32_t mode, uint32_t n_keys) {
    extern __shared__ uint32_t hist_s[];
    for (uint32_t k = threadIdx.x; k < n_keys; k += blockDim.x) hist_s[k] = 0u;
    __syncthreads();
    const uint32_t n = min(w.counts[0], w.capacity);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        uint32_t tri = __float_as_uint(w.hit[j].y);
        uint32_t key = n_keys - 1u;                          // misses last
        if (tri != kMiss) {
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
template <bool SIG>
__global__ void __launch_bounds__(256) k_shade(DevScene s, RenderParams p, WfBuffers w, int in, uint32_t b,
                                               bool sorted) {
    const uint32_t n = min(w.counts[0], w.capacity);
    const int out = in ^ 1;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    for (uint32_t base = warp * 32u; base < n; base += n_warps * 32u) {
        const uint32_t j = base + lane_id();
        bool want_ray = false, want_shadow = false;
        float4 ro, rd, rtp, so, sd, sc;
        if (j < n) {
            const uint32_t slot = sorted ? w.perm[j] : j;
            const float4 o4 = w.q_o[in][slot], d4 = w.q_d[in][slot], tp4 = w.q_tp[in][slot];
            const float2 hh = w.hit[slot];
            const uint32_t pid = __float_as_uint(o4.w);
            const uint64_t path = p.path_begin + pid;
            const float3 tp = xyz(tp4);
            const uint32_t tri = __float_as_uint(hh.y);
            if (tri == kMiss) {
                float3 L = add_rn(xyz(w.L[pid]), mul_rn(tp, env));
                w.L[pid] = f4(L, 0.f);
                if (SIG) w.sig[path] ^= sig_event(b, 0, kMiss);
            } else {
                const uint32_t pixel = (uint32_t)(path / p.spp);
                const uint32_t sample = (uint32_t)(path - (uint64_t)pixel * p.spp);
                const uint32_t key = path_key(p.seed, pixel, sample);
                Vertex V = shade_vertex(s, p, key, b, xyz(o4), xyz(d4), tp, (__float_as_uint(d4.w) & 1u) != 0u,
                                        hh.x, tri);
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
                            sc = f4(V.contrib, __uint_as_float(V.light_j));
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
                        rd = f4(V.nd, __uint_as_float(V.delta ? 1u : 0u));
                        rtp = f4(V.ntp, 0.f);
                    }
                }
                if (SIG) w.sig[path] ^= sg;
            }
        }
        const uint32_t k = warp_append(&w.counts[2], want_shadow);
        if (want_shadow) {
            if (k < w.capacity) {
                w.s_o[k] = so;
                w.s_d[k] = sd;
                w.s_c[k] = sc;
            } else {
                atomicOr(s.status, ST_QUEUE);
            }
        }
        const uint32_t q = warp_append(&w.counts[1], want_ray);
        if (want_ray) {
            if (q < w.capacity) {
                w.q_o[out][q] = ro;
                w.q_d[out][q] = rd;
                w.q_tp[out][q] = rtp;
            } else {
                atomicOr(s.status, ST_QUEUE);
            }
        }
    }
}

// Shadow: any-hit test of each queued shadow ray; unoccluded contributions are added to the path.
// At most one shadow ray per path per bounce, so the read-modify-write of L needs no atomics.
template <bool SIG>
__global__ void __launch_bounds__(256) k_shadow(DevScene s, RenderParams p, WfBuffers w, uint32_t b) {
    const uint32_t n = min(w.counts[2], w.capacity);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const float4 so = w.s_o[j], sd = w.s_d[j];
        const bool occ = trace_any(s, xyz(so), xyz(sd), so.w);
        const uint32_t pid = __float_as_uint(sd.w);
        if (!occ) {
            const float4 sc = w.s_c[j];
            float3 L = add_rn(xyz(w.L[pid]), xyz(sc));
            w.L[pid] = f4(L, 0.f);
        }
        if (SIG) {
            const uint32_t lj = __float_as_uint(w.s_c[j].w);
            w.sig[p.path_begin + pid] ^= sig_event(b, 1, (lj << 2) | 2u | (occ ? 0u : 1u));
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

__global__ void k_copy_L(const float4* __restrict__ L4, uint64_t n, float* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float4 v = L4[i];
        out[3 * i] = v.x;
        out[3 * i + 1] = v.y;
        out[3 * i + 2] = v.z;
    }
}

// ================================================================== adjoint (path replay)
struct AdjRec {
    float3 tp;       // throughput arriving at the vertex
    float3 w;        // throughput multiplier of the continuation (BSDF weight / q)
    float3 dwa;      // d w / d albedo
    float3 nee_g;    // f G A of a visible NEE sample (0 otherwise)
    float3 nee_dfa;  // d(f G A Le_light) / d albedo
    float Le;        // emission of the hit material when its term is counted
    float Lj;        // emission of the sampled light's material
    uint32_t mat, lmat;
    uint32_t flags;  // 1: continues, 2: NEE visible, 4: emission counted
};

__device__ __forceinline__ void adj_add(float* acc, float* g_alb, float* g_em, bool smem, uint32_t m, float3 ga,
                                        float ge) {
    if (smem) {
        if (ga.x != 0.f) atomicAdd(&acc[4 * m], ga.x);
        if (ga.y != 0.f) atomicAdd(&acc[4 * m + 1], ga.y);
        if (ga.z != 0.f) atomicAdd(&acc[4 * m + 2], ga.z);
        if (ge != 0.f) atomicAdd(&acc[4 * m + 3], ge);
    } else {
        if (ga.x != 0.f) atomicAdd(&g_alb[3 * m], ga.x);
        if (ga.y != 0.f) atomicAdd(&g_alb[3 * m + 1], ga.y);
        if (ga.z != 0.f) atomicAdd(&g_alb[3 * m + 2], ga.z);
        if (ge != 0.f) atomicAdd(&g_em[m], ge);
    }
}

// Gradient of sum_p <grad[p], img[p]> with respect to albedo and emission.  Each path is re-traced
// with the forward pass's random numbers and decisions; per vertex b the radiance still to come per
// unit throughput R_b = Le_b + f_b G A Le_light + w_b R_{b+1} is built backward, and
//   d/d albedo(m_b)   += delta * tp_b * (dw_b/da * R_{b+1} + d(NEE_b)/da)
//   d/d emission(m_b) += delta . tp_b                (emission counted at b)
//   d/d emission(light material) += delta . tp_b * f_b G A   (visible NEE)
template <int MAXD>
__global__ void __launch_bounds__(256) k_adjoint(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                 const float* __restrict__ grad, float* __restrict__ g_alb,
                                                 float* __restrict__ g_em, int smem) {
    extern __shared__ float acc[];
    if (smem)
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    const float inv_spp = 1.0f / (float)p.spp;
    AdjRec rec[MAXD];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_paths; i += stride) {
        const uint64_t path = p.path_begin + i;
        const uint32_t pixel = (uint32_t)(path / p.spp);
        const uint32_t sample = (uint32_t)(path - (uint64_t)pixel * p.spp);
        const uint32_t key = path_key(p.seed, pixel, sample);
        float3 o, d;
        camera_ray(c, pixel, key, o, d);
        float3 tp = f3(1.f, 1.f, 1.f);
        bool prev_delta = true, end_miss = false;
        int nv = 0;
        for (uint32_t b = 0; b < p.max_depth && b < (uint32_t)MAXD; ++b) {
            Hit h = trace_closest(s, o, d);
            if (h.tri == kMiss) {
                end_miss = true;
                break;
            }
            Vertex V = shade_vertex(s, p, key, b, o, d, tp, prev_delta, h.t, h.tri);
            AdjRec& r = rec[nv++];
            r.tp = tp;
            r.mat = V.mat;
            r.flags = V.emit_counted ? 4u : 0u;
            r.Le = V.emit_counted ? __ldg(&s.mats[V.mat].emission) : 0.f;
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
        }
        const float3 delta = f3(grad[3 * (size_t)pixel], grad[3 * (size_t)pixel + 1], grad[3 * (size_t)pixel + 2]) *
                             inv_spp;
        float3 R = end_miss ? env : f3(0.f, 0.f, 0.f);
        for (int b = nv - 1; b >= 0; --b) {
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
                adj_add(acc, g_alb, g_em, smem != 0, r.lmat, f3(0.f, 0.f, 0.f), dot(dtp, r.nee_g));
                R = R + r.nee_g * r.Lj;
            }
            if (r.flags & 4u) {
                ge = dtp.x + dtp.y + dtp.z;
                R = R + f3(r.Le, r.Le, r.Le);
            }
            adj_add(acc, g_alb, g_em, smem != 0, r.mat, ga, ge);
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
cudaError_t launch_megakernel(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                              uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays) {
    if (sig) k_megakernel<true><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
    else k_megakernel<false><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays);
    return cudaGetLastError();
}

cudaError_t launch_raygen(const Launch& l, const DevCamera& c, const RenderParams& p, uint32_t n, const WfBuffers& w) {
    k_raygen<<<l.grid, l.block, 0, l.st>>>(c, p, n, w);
    return cudaGetLastError();
}

cudaError_t launch_extend(const Launch& l, const DevScene& s, const WfBuffers& w, int in) {
    k_extend<<<l.grid, l.block, 0, l.st>>>(s, w, in);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Launch& l, const DevScene& s, const WfBuffers& w, uint32_t mode, uint32_t n_keys) {
    cudaError_t e = cudaMemsetAsync(w.bucket, 0, sizeof(uint32_t) * n_keys, l.st);
    if (e != cudaSuccess) return e;
    k_sort_keys<<<l.grid, l.block, sizeof(uint32_t) * n_keys, l.st>>>(s, w, mode, n_keys);
    k_sort_scan<<<1, 1024, 0, l.st>>>(w, n_keys);
    k_sort_scatter<<<l.grid, l.block, 0, l.st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_shade(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce, bool sorted) {
    if (w.sig) k_shade<true><<<l.grid, l.block, 0, l.st>>>(s, p, w, in, bounce, sorted);
    else k_shade<false><<<l.grid, l.block, 0, l.st>>>(s, p, w, in, bounce, sorted);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                          uint32_t bounce) {
    if (w.sig) k_shadow<true><<<l.grid, l.block, 0, l.st>>>(s, p, w, bounce);
    else k_shadow<false><<<l.grid, l.block, 0, l.st>>>(s, p, w, bounce);
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
        case K_MEGA: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel<false>, block, 0); break;
        case K_EXTEND: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extend, block, 0); break;
        case K_SHADE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<false>, block, 0); break;
        case K_SHADOW: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow<false>, block, 0); break;
        case K_ADJOINT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<16>, block, 16 * 1024); break;
        default: break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace pt
