// pt_launch.h -- host-callable launchers of the CUDA kernels (defined in the pt_k_*.cu units), used by
// the C-ABI layer (pt_api.cpp).  Every launcher is asynchronous on `st` and returns the launch error.
#pragma once
#include <cstdint>
#include <cuda_runtime_api.h>

#include "pt_types.h"

namespace pt {

struct Launch {
    int grid;
    int block;
    cudaStream_t st;
    bool pdl = false;   // programmatic dependent launch (the wavefront stage kernels; see stage_prologue)
};

// Megakernel (Sec. 2.2): one thread per path, whole path in one kernel.  Writes per-path radiance
// into out_L (stride 3 floats, wave-local index) when non-null, else img (spp == 1: pixel = path).
cudaError_t launch_megakernel(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                              uint64_t n_paths, float* out_L, float* img, uint32_t* sig,
                              unsigned long long* rays);

// Persistent megakernel with path regeneration (next_path: device counter zeroed by the caller).
cudaError_t launch_megakernel_regen(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                                    uint64_t n_paths, float* out_L, float* img, uint32_t* sig, unsigned long long* rays,
                                    unsigned long long* next_path);

// Event logs of selected paths (testing aid).
cudaError_t launch_debug_paths(cudaStream_t st, const DevScene& s, const DevCamera& c, const RenderParams& p,
                               const unsigned long long* ids, uint32_t n, uint32_t* ev_u, float* ev_f, uint32_t* n_ev,
                               float* out_L);

// Wavefront stages (Sec. 2.3, 3.1).  `in` selects the ping-pong queue read this bounce.
cudaError_t launch_raygen(const Launch& l, const DevCamera& c, const RenderParams& p, uint32_t n, const WfBuffers& w);
cudaError_t launch_extend(const Launch& l, const DevScene& s, const WfBuffers& w, int in, const RenderParams& p);
cudaError_t launch_sort(const Launch& l, const DevScene& s, const WfBuffers& w, int in, uint32_t mode, uint32_t n_keys,
                        const RenderParams& p);
cudaError_t launch_shade(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce, bool sorted);
cudaError_t launch_shadow(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                          uint32_t bounce);
cudaError_t launch_prepare(cudaStream_t st, const WfBuffers& w, uint32_t bounce);
// The fused pipeline: the extend stage of bounce b and the shadow stage of bounce b - 1 in one launch
// (the shadow rays pending in counts[6]), and the prepare step that hands shading's new shadow rays on.
cudaError_t launch_trace(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                         uint32_t bounce);
cudaError_t launch_prepare_fused(cudaStream_t st, const WfBuffers& w, uint32_t bounce, bool pdl = false);
// The adjoint replay's fused launch: its shadow walks mark the records of bounce - 1.
cudaError_t launch_trace_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                             const AdjBuffers& a, int in, uint32_t bounce);

// Batched wavefront over device scene tables (TableSrc): raygen of one wave (publishes the wave
// base), one bounce of extend/(sort)/shade/shadow/prepare (capturable: no host-varying arguments),
// accumulation of a wave into the scenes' running sums, and the final sums -> means.
cudaError_t launch_raygen_batch(const Launch& l, const BatchTables& t, const RenderParams& p, uint64_t base, uint32_t n,
                                const WfBuffers& w);
// fused: the shadow walks of bounce b - 1 run in bounce b's extend launch (lw configures that launch);
// otherwise lw configures a shadow stage after shading.
cudaError_t launch_bounce_batch(const Launch& le, const Launch& ls, const Launch& lw, const Launch& lk,
                                const BatchTables& t, const RenderParams& p, const WfBuffers& w, uint32_t b,
                                uint32_t sort_mode, uint32_t n_keys, bool fused);
cudaError_t launch_reduce_batch(const Launch& l, const BatchTables& t, const float4* L, const BatchSegment* seg,
                                uint32_t n_seg, uint64_t w0, uint64_t w1, uint64_t n_flat);
cudaError_t launch_scale_batch(const Launch& l, const BatchTables& t, const unsigned long long* px_off, uint64_t total);

// Accumulation (Sec. 2.3): img[pixel] = (1/spp) * sum_s L[pixel * spp + s], samples in order.
// L has `stride` floats per path (3 or 4), wave-local; pixels [pixel_begin, pixel_begin + n_pixels).
cudaError_t launch_reduce(const Launch& l, const float* L, uint32_t stride, uint64_t pixel_begin, uint64_t n_pixels,
                          uint32_t spp, float* img);
// Copy wave-local float4 radiance into the caller's N_p x 3 buffer at path offset `path_begin`.
cudaError_t launch_copy_L(const Launch& l, const float4* L4, uint64_t n, float* out_L3);
// sum[px] += the pixel's spp samples (in order); img[px] = sum[px] / count unless img is null
cudaError_t launch_accumulate(const Launch& l, const float* L, uint32_t stride, uint64_t pixel_begin, uint64_t n_pixels,
                              uint32_t spp, float* sum, uint32_t count, float* img);
// Hybrid: finish every active path of the wave in one kernel when at most `threshold` are active
// entering bounce b0 (queue `in`), then empty the queue; `claim` is a zeroed device u64.
cudaError_t launch_finish(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w, int in,
                          uint32_t b0, uint32_t threshold, unsigned long long* claim);

// Path-replay adjoint (one thread per path).  grad_img is H x W x 3; `claim` is a device counter
// that must be zero at launch (warps take paths from it).
cudaError_t launch_adjoint(const Launch& l, const DevScene& s, const DevCamera& c, const RenderParams& p,
                           uint64_t n_paths, const float* grad_img, float* g_albedo, float* g_emission,
                           uint32_t max_depth_cap, unsigned long long* claim);

// Wavefront adjoint: shading that writes per-vertex records, the shadow stage that marks visible
// NEE samples, and the reverse pass over one wave's paths.
cudaError_t launch_shade_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                             const AdjBuffers& a, int in, uint32_t bounce);
cudaError_t launch_shadow_adj(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                              const AdjBuffers& a, uint32_t bounce);
cudaError_t launch_adjoint_reverse(const Launch& l, const DevScene& s, const RenderParams& p, const WfBuffers& w,
                                   const AdjBuffers& a, uint32_t n, const float* grad, float* g_albedo,
                                   float* g_emission);

// Utilities.
cudaError_t launch_set_materials(cudaStream_t st, DevMat* mats, uint32_t n, const float* albedo, const float* emission);
cudaError_t launch_trace_closest(const Launch& l, const DevScene& s, const float* rays, uint32_t n, float* t,
                                 int32_t* prim);
cudaError_t launch_debug_rng(const Launch& l, uint64_t seed, const uint32_t* px, const uint32_t* sm,
                             const uint32_t* bo, const uint32_t* dm, uint32_t n, float* out);

// Occupancy helpers.
// occupancy of each kernel unit's kernels (0 when `which` is not one of them)
int occupancy_mega(int which, int block);
int occupancy_mega_static(int which, int block);
int occupancy_wave(int which, int block);
int occupancy_adj(int which, int block);
int max_blocks_per_sm(int which, int block);   // which: 0 megakernel, 1 extend, 2 shade, 3 shadow, 4 adjoint
enum { K_MEGA = 0, K_EXTEND = 1, K_SHADE = 2, K_SHADOW = 3, K_ADJOINT = 4, K_EXTEND_BATCH = 5, K_SHADE_BATCH = 6,
       K_SHADOW_BATCH = 7, K_SHADE_ADJ = 8, K_SHADOW_ADJ = 9,
       K_MEGA_REGEN = 10, K_FINISH = 11, K_MEGA_REGEN_INST = 12, K_FINISH_INST = 13,
       K_EXTEND_INST = 14, K_SHADE_INST = 15, K_SHADOW_INST = 16, K_SHADE_ADJ_INST = 17, K_SHADOW_ADJ_INST = 18,
       // the single-level instantiations whose walks keep a shared-memory short stack
       K_EXTEND_SS = 19, K_SHADOW_SS = 20, K_MEGA_REGEN_SS = 21, K_FINISH_SS = 22,
       K_TRACE = 23, K_TRACE_INST = 24, K_TRACE_BATCH = 25 };

}  // namespace pt
