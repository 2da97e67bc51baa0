// pt_k_mega_static.cu -- the megakernel in the paper's layout (Sec. 2.2: one thread per path,
// launched over all paths), and the event-log kernel that records every decision of selected paths
// (a testing aid for locating where two implementations part ways).
#include "pt_common.cuh"

namespace pt {

template <bool SIG, bool MIS, bool INST>
__global__ void __launch_bounds__(256) k_megakernel(DevScene s, DevCamera c, RenderParams p, uint64_t n_paths,
                                                    float* __restrict__ out_L, float* __restrict__ img,
                                                    uint32_t* __restrict__ sig, unsigned long long* __restrict__ rays) {
    uint32_t n_ext = 0, n_shd = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_paths; i += stride) {
        const uint64_t path = p.path_begin + i;
        float3 L;
        if (SIG) {
            SigRec r;
            L = mk_path<SigRec, MIS, INST>(s, c, p, path, r, n_ext, n_shd);
            sig[path] = r.sg;
        } else {
            NoRec r;
            L = mk_path<NoRec, MIS, INST>(s, c, p, path, r, n_ext, n_shd);
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

// Event logs of selected paths (testing aid): the megakernel's path function with a recorder.
template <bool INST>
__global__ void k_debug_paths(DevScene s, DevCamera c, RenderParams p, const unsigned long long* __restrict__ ids,
                              uint32_t n, uint32_t* __restrict__ ev_u, float* __restrict__ ev_f,
                              uint32_t* __restrict__ n_ev, float* __restrict__ out_L) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t a = 0, b = 0;
    LogRec r;
    r.ev_u = ev_u + (size_t)i * 2 * kMaxEvents;
    r.ev_f = ev_f + (size_t)i * 2 * kMaxEvents;
    float3 L = mk_path<LogRec, true, INST>(s, c, p, ids[i], r, a, b);
    n_ev[i] = r.n;
    out_L[3 * i] = L.x;
    out_L[3 * i + 1] = L.y;
    out_L[3 * i + 2] = L.z;
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_megakernel(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                              uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays) {
#define PT_MK(S, M, I) k_megakernel<S, M, I><<<l.grid, l.block, 0, l.st>>>(s, c, p, n_paths, out_L, img, sig, rays)
    if (s.tlas) {
        if (sig) PT_MK(true, true, true);
        else PT_MK(false, true, true);
    } else if (p.mis) {
        if (sig) PT_MK(true, true, false);
        else PT_MK(false, true, false);
    } else {
        if (sig) PT_MK(true, false, false);
        else PT_MK(false, false, false);
    }
#undef PT_MK
    return cudaGetLastError();
}

cudaError_t launch_debug_paths(cudaStream_t st, const DevScene& s, const DevCamera& c, const RenderParams& p,
                               const unsigned long long* ids, uint32_t n, uint32_t* ev_u, float* ev_f, uint32_t* n_ev,
                               float* out_L) {
    if (n == 0) return cudaSuccess;
    if (s.tlas) k_debug_paths<true><<<(n + 63) / 64, 64, 0, st>>>(s, c, p, ids, n, ev_u, ev_f, n_ev, out_L);
    else k_debug_paths<false><<<(n + 63) / 64, 64, 0, st>>>(s, c, p, ids, n, ev_u, ev_f, n_ev, out_L);
    return cudaGetLastError();
}

// Resident blocks per SM of this unit's kernels (0: not one of them).
int occupancy_mega_static(int which, int block) {
    if (which != K_MEGA) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_megakernel<false, false, false>, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace pt
