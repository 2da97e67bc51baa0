// pt_k_adj.cu -- the path-replay adjoint: the wavefront replay (shading that writes per-vertex
// records, shadow visibility flags) with its reverse pass, and the one-thread-per-path replay;
// gradients are reduced in shared memory with warp-aggregated additions, then one global atomic
// per non-zero material entry per block.
#include "pt_common.cuh"

namespace pt {

// ---- wavefront adjoint: shading that records what the reverse pass needs instead of adding
// radiance (the same shade_vertex decisions, so the replay follows the forward paths exactly).
template <bool INST>
__global__ void __launch_bounds__(256, 3) k_shade_adj(SingleSrc src, WfBuffers w, AdjBuffers a, int in, uint32_t b) {
    stage_prologue();
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
            const float4 o4 = __ldcs(&w.q_o[in][j]), d4 = __ldcs(&w.q_d[in][j]), tp4 = __ldcs(&w.q_tp[in][j]);
            const float2 hh = __ldcs(&w.hit[j]);
            const uint32_t pid = __float_as_uint(o4.w);
            const uint32_t tri = __float_as_uint(hh.y);
            if (tri == kMiss) {
                a.pend[pid] = b | (1u << 8);
            } else {
                const PathLoc l = src.locate(base, pid);
                const RenderParams& p = src.p;
                const uint32_t key = path_key(p.seed, l.pixel, l.sample);
                Vertex V = shade_vertex<true, INST>(src.s, p, key, b, xyz(o4), xyz(d4), xyz(tp4),
                                                    (__float_as_uint(d4.w) & 1u) != 0u, tp4.w, hh.x, tri,
                                                    INST ? w.hit_inst[j] : kMiss);
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
                float4* r = a.rec + 4 * ((size_t)b * cap + pid);   // streamed: read back by the reverse pass
                __stcs(r, make_float4(tp4.x, tp4.y, tp4.z, __uint_as_float(V.mat)));
                __stcs(r + 1, r1);
                __stcs(r + 2, r2);
                __stcs(r + 3, make_float4(Le, Lj, V.emit_w, __uint_as_float(flags | (V.light_mat << 4))));
                if (!V.cont || V.last) a.pend[pid] = b + 1u;
            }
        }
        const uint32_t k = warp_append(&w.counts[2], want_shadow);
        if (want_shadow) {
            if (k < w.capacity) {
                __stcs(&w.s_o[k], so);
                __stcs(&w.s_d[k], sd);
            } else {
                atomicOr(src.s.status, ST_QUEUE);
            }
        }
        const uint32_t q = warp_append(&w.counts[1], want_ray);
        if (want_ray) {
            if (q < w.capacity) {
                __stcs(&w.q_o[out][q], ro);
                __stcs(&w.q_d[out][q], rd);
                __stcs(&w.q_tp[out][q], rtp);
            } else {
                atomicOr(src.s.status, ST_QUEUE);
            }
        }
    }
}

// Wavefront adjoint shadow stage: mark the vertex's NEE sample visible when unoccluded.
template <bool INST>
__global__ void __launch_bounds__(256) k_shadow_adj(SingleSrc src, WfBuffers w, AdjBuffers a, uint32_t b) {
    const uint32_t n = min(w.counts[2], w.capacity);
    if (n == 0u) return;
    const size_t cap = w.capacity;
    for (uint32_t b0 = warp_claim32(&w.counts[5]); b0 < n; b0 = warp_claim32(&w.counts[5])) {
        const uint32_t j = b0 + lane_id();
        if (j >= n) continue;
        const float4 so = __ldcs(&w.s_o[j]), sd = __ldcs(&w.s_d[j]);
        if (!trace_any<INST>(src.s, xyz(so), xyz(sd), so.w)) {
            const uint32_t pid = __float_as_uint(sd.w);
            float* fl = reinterpret_cast<float*>(a.rec + 4 * ((size_t)b * cap + pid) + 3) + 3;
            *fl = __uint_as_float(__float_as_uint(*fl) | 2u);
        }
    }
}

// One vertex's gradient terms v = (d/d albedo rgb, d/d emission) of material k, added by one lane
// into the block's shared accumulators (or the global gradients when they do not fit there).
__device__ __forceinline__ void lane_accumulate(float* acc, float* g_alb, float* g_em, bool smem, uint32_t k,
                                                float4 v) {
    if (smem) {
        if (v.x != 0.f) atomicAdd(&acc[4 * k], v.x);
        if (v.y != 0.f) atomicAdd(&acc[4 * k + 1], v.y);
        if (v.z != 0.f) atomicAdd(&acc[4 * k + 2], v.z);
        if (v.w != 0.f) atomicAdd(&acc[4 * k + 3], v.w);
    } else {
        if (v.x != 0.f) atomicAdd(&g_alb[3 * k], v.x);
        if (v.y != 0.f) atomicAdd(&g_alb[3 * k + 1], v.y);
        if (v.z != 0.f) atomicAdd(&g_alb[3 * k + 2], v.z);
        if (v.w != 0.f) atomicAdd(&g_em[k], v.w);
    }
}

// Gradient of sum_p <grad[p], img[p]> with respect to albedo and emission, one thread per path.
// Each path is re-traced with the forward pass's random numbers and decisions, one bounce per loop
// iteration, recording every vertex; when it ends, the radiance still to come per unit throughput
// R_b = Le_b + f_b G A Le_light + w_b R_{b+1} is built backward over the records, and
//   d/d albedo(m_b)   += delta * tp_b * (dw_b/da * R_{b+1} + d(NEE_b)/da)
//   d/d emission(m_b) += delta . tp_b                (emission counted at b)
//   d/d emission(light material) += delta . tp_b * f_b G A   (visible NEE)
// are added with per-lane shared-memory atomics.  The kernel is persistent and regenerates paths
// like the forward megakernel: a lane whose path is done takes the next path id (warp-aggregated
// claim on `claim`, zero at launch) instead of waiting for the longest path of its warp.
// Registers capped for 8 resident blocks of 128, as the forward megakernel (4.56 -> 4.17 ms per
// 1080p pass against the uncapped 96 registers).
template <int MAXD, bool INST>
__global__ void __launch_bounds__(128, 8) k_adjoint(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                 const float* __restrict__ grad, float* __restrict__ g_alb,
                                                 float* __restrict__ g_em, int smem,
                                                 unsigned long long* __restrict__ claim) {
    extern __shared__ float acc[];
    if (smem)
        for (uint32_t k = threadIdx.x; k < 4 * s.n_mats; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const float3 env = f3(s.env_r, s.env_g, s.env_b);
    const float inv_spp = 1.0f / (float)p.spp;
    AdjRec rec[MAXD];
    bool active = false, exhausted = false;
    uint32_t pixel = 0, key = 0, b = 0;
    int nv = 0;
    float3 o = f3(0.f, 0.f, 0.f), d = o, tp = o;
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
                const uint64_t i = first + (uint64_t)__popc(m & ((1u << lane_id()) - 1u));
                if (i < n_paths) {
                    const uint64_t path = p.path_begin + i;
                    pixel = (uint32_t)(path / p.spp);
                    const uint32_t sample = p.sample_offset + (uint32_t)(path - (uint64_t)pixel * p.spp);
                    key = path_key(p.seed, pixel, sample);
                    float u0, u1;
                    pixel_jitter(p.sampler, p.seed, pixel, sample, key, u0, u1);
                    camera_ray(c, pixel, u0, u1, o, d);
                    tp = f3(1.f, 1.f, 1.f);
                    prev_delta = true;
                    prev_pdf = 0.f;
                    b = 0;
                    nv = 0;
                    active = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        if (!active) continue;
        bool end = true, end_miss = false;
        if (b < p.max_depth && b < (uint32_t)MAXD) {
            const Hit h = trace_closest<INST, 0, !INST>(s, o, d);
            if (h.tri == kMiss) {
                end_miss = true;
            } else {
                Vertex V = shade_vertex<true, INST>(s, p, key, b, o, d, tp, prev_delta, prev_pdf, h.t, h.tri, h.inst);
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
                if (!V.last) {
                    if (V.nee && V.cast && !trace_any<INST, 0, !INST>(s, V.s_o, V.s_d, V.s_tmax)) {
                        r.flags |= 2u;
                        r.nee_g = V.nee_g;
                        r.nee_dfa = V.nee_dfa;
                        r.Lj = __ldg(&s.mats[V.light_mat].emission);
                    }
                    if (V.cont) {
                        r.flags |= 1u;
                        r.w = V.w;
                        r.dwa = V.dwa;
                        o = V.no;
                        d = V.nd;
                        tp = V.ntp;
                        prev_delta = V.delta;
                        prev_pdf = V.pdf;
                        ++b;
                        end = false;
                    }
                }
            }
        }
        if (!end) continue;
        // the path is complete: walk its vertices backward
        const float3 delta =
            f3(grad[3 * (size_t)pixel], grad[3 * (size_t)pixel + 1], grad[3 * (size_t)pixel + 2]) * inv_spp;
        float3 R = end_miss ? env : f3(0.f, 0.f, 0.f);
        for (int k = nv - 1; k >= 0; --k) {
            const AdjRec& r = rec[k];
            const float3 dtp = delta * r.tp;
            float3 ga = f3(0.f, 0.f, 0.f);
            float ge = 0.f;
            if (r.flags & 1u) {
                ga = dtp * r.dwa * R;
                R = r.w * R;
            }
            if (r.flags & 2u) {
                ga = ga + dtp * r.nee_dfa;
                lane_accumulate(acc, g_alb, g_em, smem != 0, r.lmat, make_float4(0.f, 0.f, 0.f, dot(dtp, r.nee_g)));
                R = R + r.nee_g * r.Lj;
            }
            if (r.flags & 4u) {
                ge = (dtp.x + dtp.y + dtp.z) * r.we;
                R = R + f3(r.Le, r.Le, r.Le);
            }
            lane_accumulate(acc, g_alb, g_em, smem != 0, r.mat, make_float4(ga.x, ga.y, ga.z, ge));
        }
        active = false;
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
    stage_prologue();
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


// ------------------------------------------------------------------ launchers
cudaError_t launch_adjoint(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                           uint64_t n_paths, const float* grad_img, float* g_albedo, float* g_emission,
                           uint32_t max_depth_cap, unsigned long long* claim) {
    size_t smem_bytes = sizeof(float) * 4 * (size_t)s.n_mats;
    int smem = smem_bytes <= 32 * 1024 ? 1 : 0;
    size_t sb = smem ? smem_bytes : 0;
#define PT_ADJ(D, I) k_adjoint<D, I><<<l.grid, l.block, sb, l.st>>>(s, c, p, n_paths, grad_img, g_albedo, g_emission, smem, claim)
    // two-level scenes: one instantiation (the record array sized for the deepest paths)
    if (s.tlas) PT_ADJ(32, true);
    else if (max_depth_cap <= 8) PT_ADJ(8, false);
    else if (max_depth_cap <= 16) PT_ADJ(16, false);
    else PT_ADJ(32, false);
#undef PT_ADJ
    return cudaGetLastError();
}

cudaError_t launch_shade_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                             const AdjBuffers& a, int in, uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) return launch_k(l, 0, k_shade_adj<true>, src, w, a, in, bounce);
    return launch_k(l, 0, k_shade_adj<false>, src, w, a, in, bounce);
}

cudaError_t launch_shadow_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                              const AdjBuffers& a, uint32_t bounce) {
    SingleSrc src{s, DevCamera{}, p};
    if (s.tlas) k_shadow_adj<true><<<l.grid, l.block, 0, l.st>>>(src, w, a, bounce);
    else k_shadow_adj<false><<<l.grid, l.block, 0, l.st>>>(src, w, a, bounce);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reverse(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                                   const AdjBuffers& a, uint32_t n, const float* grad, float* g_albedo,
                                   float* g_emission) {
    size_t smem_bytes = sizeof(float) * 4 * (size_t)s.n_mats;
    int smem = smem_bytes <= 32 * 1024 ? 1 : 0;
    return launch_k(l, smem ? smem_bytes : 0, k_adjoint_reverse, s, p, w, a, n, grad, g_albedo, g_emission, smem);
}

// Resident blocks per SM of this unit's kernels (0: not one of them).
int occupancy_adj(int which, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (which) {
        case K_ADJOINT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<16, false>, block, 16 * 1024); break;
        case K_SHADE_ADJ: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade_adj<false>, block, 0); break;
        case K_SHADOW_ADJ: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow_adj<false>, block, 0); break;
        case K_SHADE_ADJ_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade_adj<true>, block, 0); break;
        case K_SHADOW_ADJ_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shadow_adj<true>, block, 0); break;
        default: return 0;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace pt
