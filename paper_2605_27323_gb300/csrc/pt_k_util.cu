// pt_k_util.cu -- material updates, closest-hit queries, the random-number probe, and the
// occupancy table used to size persistent grids.
#include "pt_common.cuh"

namespace pt {

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

template <bool INST>
__global__ void __launch_bounds__(256) k_trace_closest(DevScene s, const float* __restrict__ rays, uint32_t n,
                                                       float* __restrict__ t, int32_t* __restrict__ prim) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float* r = rays + 8 * (size_t)i;
        Hit h = trace_closest<INST>(s, f3(r[0], r[1], r[2]), f3(r[4], r[5], r[6]));
        t[i] = h.t;
        prim[i] = h.tri == kMiss ? -1 : (int32_t)h.prim;
    }
}

__global__ void k_debug_rng(uint64_t seed, const uint32_t* px, const uint32_t* sm, const uint32_t* bo,
                            const uint32_t* dm, uint32_t n, float* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = u01(path_key(seed, px[i], sm[i]), bo[i], dm[i]);
}


// ------------------------------------------------------------------ launchers
cudaError_t launch_set_materials(cudaStream_t st, DevMat* mats, uint32_t n, const float* albedo, const float* emission) {
    if (n == 0) return cudaSuccess;
    k_set_materials<<<(n + 255) / 256, 256, 0, st>>>(mats, n, albedo, emission);
    return cudaGetLastError();
}

cudaError_t launch_trace_closest(const Launch& l, const DevScene& s, const float* rays, uint32_t n, float* t,
                                 int32_t* prim) {
    if (s.tlas) k_trace_closest<true><<<l.grid, l.block, 0, l.st>>>(s, rays, n, t, prim);
    else k_trace_closest<false><<<l.grid, l.block, 0, l.st>>>(s, rays, n, t, prim);
    return cudaGetLastError();
}

cudaError_t launch_debug_rng(const Launch& l, uint64_t seed, const uint32_t* px, const uint32_t* sm,
                             const uint32_t* bo, const uint32_t* dm, uint32_t n, float* out) {
    k_debug_rng<<<(n + 255) / 256, 256, 0, l.st>>>(seed, px, sm, bo, dm, n, out);
    return cudaGetLastError();
}

int max_blocks_per_sm(int which, int block) {
    int nb = occupancy_mega(which, block);
    if (!nb) nb = occupancy_mega_static(which, block);
    if (!nb) nb = occupancy_wave(which, block);
    if (!nb) nb = occupancy_adj(which, block);
    return nb > 0 ? nb : 1;
}

}  // namespace pt
