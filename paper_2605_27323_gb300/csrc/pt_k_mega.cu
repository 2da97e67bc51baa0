// pt_k_mega.cu -- the persistent megakernel with path regeneration (Sec. 2.2: one thread traces one
// path to termination; a lane whose path ended claims the next one), and the hybrid continuation
// kernel that finishes a wavefront's last sparse bounces with the same bounce function (Sec. 6.1).
#include <type_traits>

#include "pt_common.cuh"

namespace pt {


// Persistent megakernel with path regeneration.  Each thread still traces one path at a time from
// its camera ray to termination, one bounce per loop iteration; a lane whose path ended claims the
// next path id (warp-aggregated atomic on a device counter) instead of idling until the longest
// path of its warp finishes.  The per-path arithmetic is that of mk_path, so images are identical.
template <bool SIG, bool MIS, bool INST, int SK = 0, bool CNT = false>
// Register cap for 8 resident blocks of 128: occupancy outweighs the spills (measured 3.96 -> 3.11 ms
// per 1080p frame against the uncapped 107 registers; for two-level scenes a cap of 6 blocks with
// fewer spills measured slower too, 5.49 -> 6.07 ms).
__global__ void __launch_bounds__(128, 8) k_megakernel_regen(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                          float* __restrict__ out_L, float* __restrict__ img,
                                                          uint32_t* __restrict__ sig,
                                                          unsigned long long* __restrict__ rays,
                                                          unsigned long long* __restrict__ next_path) {
    uint32_t n_ext = 0, n_shd = 0;
    typename std::conditional<CNT, TravCount, NoCount>::type cc, ca;   // closest-hit / any-hit walks
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
            const bool end = mk_bounce<SIG, MIS, INST, SK>(s, p, env, key, b, o, d, tp, prev_delta, prev_pdf, L, sg, n_ext,
                                                         n_shd, cc, ca);
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
    flush_count(s, cc, 0);
    flush_count(s, ca, 2);
}


// ---- hybrid wavefront / megakernel (the hybrid of the paper's future work, Sec. 6.1): once the
// active count entering a bounce is at most `threshold`, one persistent kernel finishes every
// remaining path in registers (the megakernel's loop body, lanes claiming queue entries as they
// free up) instead of running the remaining bounces as sparse wavefront stages.  The decision is
// taken on the device; k_finish_commit then empties the queue so the remaining stage launches find
// no work.  The arithmetic per path is the same as in the wavefront stages, so images are identical.
template <bool SIG, bool MIS, bool INST, int SK = 0>
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
    uint32_t n_ext = 0, n_shd = 0;
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
                    const float4 o4 = __ldcs(&w.q_o[in][j]), d4 = __ldcs(&w.q_d[in][j]), tp4 = __ldcs(&w.q_tp[in][j]);
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
            const uint32_t shd0 = n_shd;
            atomicAdd(&h_s[bb & 63u], 1u);
            const bool end = mk_bounce<SIG, MIS, INST, SK>(s, p, env, key, b, o, d, tp, prev_delta, prev_pdf, L, sg, n_ext,
                                                         n_shd);
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


// ------------------------------------------------------------------ launchers
cudaError_t launch_megakernel_regen(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                                    uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays,
                                    unsigned long long* next_path) {
    // PT_FLAG_SHORT_STACK: the single-level variants keep their top stack entries in shared memory
    const size_t sm = stack_smem_bytes(kShortStack, l.block);
#define PT_REGEN(S, M, I, K) k_megakernel_regen<S, M, I, K><<<l.grid, l.block, K ? sm : 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path)
    if (s.tlas) {            // two-level scenes: one variant, MIS decided at run time
        if (sig) PT_REGEN(true, true, true, 0);
        else PT_REGEN(false, true, true, 0);
    } else if (p.count_trav && !sig) {
        k_megakernel_regen<false, true, false, 0, true>
            <<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays, next_path);
    } else if (p.short_stack) {
        if (sig) PT_REGEN(true, true, false, kShortStack);
        else PT_REGEN(false, true, false, kShortStack);
    } else if (p.mis) {
        if (sig) PT_REGEN(true, true, false, 0);
        else PT_REGEN(false, true, false, 0);
    } else {
        if (sig) PT_REGEN(true, false, false, 0);
        else PT_REGEN(false, false, false, 0);
    }
#undef PT_REGEN
    return cudaGetLastError();
}



cudaError_t launch_finish(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                          uint32_t b0, uint32_t threshold, unsigned long long* claim) {
    SingleSrc src{s, DevCamera{}, p};
    const size_t sm = stack_smem_bytes(kShortStack, l.block);
#define PT_FIN(S, M, I, K) k_finish<S, M, I, K><<<l.grid, l.block, K ? sm : 0, l.st>>>(src, w, in, b0, threshold, claim)
    if (s.tlas) {
        if (w.sig) PT_FIN(true, true, true, 0);
        else PT_FIN(false, true, true, 0);
    } else if (p.short_stack) {
        if (w.sig) PT_FIN(true, true, false, kShortStack);
        else PT_FIN(false, true, false, kShortStack);
    } else if (p.mis) {
        if (w.sig) PT_FIN(true, true, false, 0);
        else PT_FIN(false, true, false, 0);
    } else {
        if (w.sig) PT_FIN(true, false, false, 0);
        else PT_FIN(false, false, false, 0);
    }
#undef PT_FIN
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish_commit<<<1, 1, 0, l.st>>>(w, threshold, claim);
    return cudaGetLastError();
}

// Resident blocks per SM of this unit's kernels (0: not one of them).
int occupancy_mega(int which, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (which) {
        case K_MEGA_REGEN: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel_regen<false, false, false>, block, 0); break;
        case K_MEGA_REGEN_SS:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel_regen<false, true, false, kShortStack>, block,
                                                              stack_smem_bytes(kShortStack, block));
            break;
        case K_MEGA_REGEN_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel_regen<false, true, true>, block, 0); break;
        case K_FINISH_INST: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_finish<false, true, true>, block, 0); break;
        case K_FINISH: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_finish<false, false, false>, block, 0); break;
        case K_FINISH_SS:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_finish<false, true, false, kShortStack>, block,
                                                              stack_smem_bytes(kShortStack, block));
            break;
        default: return 0;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace pt
