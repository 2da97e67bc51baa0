// pt_static.cu -- pt_render_wavefront_static: the wavefront render with its queues in one fixed
// file-scope device array, for callers that cannot allocate device memory themselves or let a
// library do it (an application whose memory manager owns every byte of the device, or a
// real-time loop that cannot absorb the implicit synchronisation of cudaMalloc/cudaFree).
//
// The array is kStaticScratchBytes (384 MiB, 0.13% of a GB300's memory: room for 2.2 million paths,
// so a 1-spp 1920x1080 frame renders in one wave); a GPU holds it from the first call on it (CUDA
// loads this file's module, and the array with it, when the call looks up its address) until the
// process exits.  Frames larger than one array's worth of paths are rendered in waves of whole
// pixels.  Every call shares the array: it keeps the previous call's contents, this file clears the
// counters and the call's status word that must start at zero on every call, and calls that overlap
// on the GPU (other streams, other threads) race on it.  The first call on a device looks up the
// array's device address with cudaGetSymbolAddress (the host-side name is only a stand-in); make
// that first call before any stream capture.  Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "pt.h"
#include "pt_launch.h"
#include "pt_types.h"

namespace pt {
pt_status static_set_error(pt_status s, const char* msg);
pt_status static_prepare(pt_scene* sc, const pt_camera* cam, const pt_render_opts* opts, DevScene* view,
                         DevCamera* dc, pt_render_opts* o_out, int* device);
bool static_is_device_ptr(const void* p);
}  // namespace pt

namespace {

constexpr size_t kStaticScratchBytes = 384ull << 20;
constexpr size_t kHeaderBytes = 256 + 8 * pt::kHistWords;  // counters (incl. this call's status word), totals
constexpr uint32_t kStatusWord = 16;            // counts[16]: device status word of this call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the array on `device` (which is current), looked up once per device.
pt_status scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return pt::static_set_error(PT_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            char msg[160];
            std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
            return pt::static_set_error(PT_ERR_CUDA, msg);
        }
        g_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[device];
    return PT_OK;
}

// Paths one wave can hold: the largest capacity whose records (the allocating entry points' layout)
// fit the array after the header.
uint64_t wave_capacity() {
    const size_t avail = kStaticScratchBytes - kHeaderBytes;
    uint64_t cap = avail / pt::kWfBytesPerPath;
    while (cap > 0 && pt::wavefront_bytes(cap) > avail) --cap;
    return cap;
}

pt_status cuda_fail(cudaError_t e, const char* what) {
    char msg[200];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return pt::static_set_error(PT_ERR_CUDA, msg);
}

}  // namespace

extern "C" pt_status pt_render_wavefront_static(pt_scene* scene, const pt_camera* cam, uint32_t spp,
                                                uint32_t max_depth, uint64_t seed, const pt_render_opts* opts,
                                                float* d_out_rgb, void* stream) {
    if (!d_out_rgb) return pt::static_set_error(PT_ERR_INVALID_ARG, "output image is NULL");
    if (spp == 0) return pt::static_set_error(PT_ERR_INVALID_ARG, "spp must be >= 1");
    if (max_depth > 64) return pt::static_set_error(PT_ERR_INVALID_ARG, "max_depth must be <= 64");
    pt::DevScene ds;
    pt::DevCamera dc;
    pt_render_opts o;
    int device = 0;
    pt_status s = pt::static_prepare(scene, cam, opts, &ds, &dc, &o, &device);
    if (s != PT_OK) return s;
    if (o.mode != PT_MODE_WAVEFRONT)
        return pt::static_set_error(PT_ERR_INVALID_ARG, "this entry point renders with the wavefront only (opts->mode)");
    if (o.hybrid_threshold)
        return pt::static_set_error(PT_ERR_INVALID_ARG, "this entry point has no hybrid continuation (opts->hybrid_threshold)");
    if (!pt::static_is_device_ptr(d_out_rgb))
        return pt::static_set_error(PT_ERR_INVALID_ARG, "d_out_rgb must be device memory (this call stages nothing)");
    if (o.d_path_sig && !pt::static_is_device_ptr(o.d_path_sig))
        return pt::static_set_error(PT_ERR_INVALID_ARG, "d_path_sig must be device memory");
    const uint64_t cap_max = wave_capacity();
    if (spp > cap_max) {
        char msg[200];
        std::snprintf(msg, sizeof msg, "spp %u needs %llu bytes per pixel; the static scratch holds %llu paths (%zu MiB)",
                      spp, (unsigned long long)spp * pt::kWfBytesPerPath, (unsigned long long)cap_max,
                      kStaticScratchBytes >> 20);
        return pt::static_set_error(PT_ERR_INVALID_ARG, msg);
    }
    unsigned char* base = nullptr;
    if ((s = scratch_address(device, &base)) != PT_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t n_pixels = (uint64_t)cam->width * cam->height;
    const uint64_t n_paths = n_pixels * spp;
    const uint64_t cap = cap_max - cap_max % spp;

    // the array: counters and histories, then the wavefront records in the allocating layout
    pt::WfBuffers w{};
    w.counts = reinterpret_cast<uint32_t*>(base);
    w.hist = reinterpret_cast<unsigned long long*>(base + 256);
    const size_t used = kHeaderBytes + pt::carve_wavefront_at(reinterpret_cast<char*>(base) + kHeaderBytes, cap, w);
    if (used > kStaticScratchBytes) return pt::static_set_error(PT_ERR_UNSUPPORTED, "static scratch layout overflow");
    w.sig = o.d_path_sig;
    w.capacity = (uint32_t)cap;
    // faults of this call (traversal cap, queue overflow) go to a word of the array, not to the
    // scene's status word, so pt_get_stats keeps describing the scene's last pt_render call
    ds.status = w.counts + kStatusWord;

    cudaError_t e = cudaMemsetAsync(base, 0, kHeaderBytes, st);   // counters, status word, histories
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (max_depth == 0) {
        e = cudaMemsetAsync(d_out_rgb, 0, n_pixels * 12, st);
        if (e == cudaSuccess && o.d_path_sig) e = cudaMemsetAsync(o.d_path_sig, 0, n_paths * 4, st);
        return e == cudaSuccess ? PT_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    const int block = o.block_size ? (int)o.block_size : 256;
    // resident blocks per SM of the three persistent stages, looked up once per call (the two-level
    // instantiations have their own register counts)
    const bool inst = ds.tlas != nullptr;
    // the fused order of pt_render (each bounce's trace launch also walks the shadow rays of the
    // previous shading) unless PT_FLAG_SEPARATE_SHADOW asks for the separate shadow stage
    const bool fused = !(o.flags & PT_FLAG_SEPARATE_SHADOW);
    const int per_extend = pt::max_blocks_per_sm(inst ? pt::K_EXTEND_INST : pt::K_EXTEND, block);
    const int per_shade = pt::max_blocks_per_sm(inst ? pt::K_SHADE_INST : pt::K_SHADE, block);
    const int per_shadow = fused ? 0 : pt::max_blocks_per_sm(inst ? pt::K_SHADOW_INST : pt::K_SHADOW, block);
    const int per_trace = fused ? pt::max_blocks_per_sm(inst ? pt::K_TRACE_INST : pt::K_TRACE, block) : 0;
    auto persistent = [&](int per, uint64_t work) {
        pt::Launch l;
        l.block = block;
        const uint64_t need = (work + block - 1) / block;
        l.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * std::max(per, 1), need));
        l.st = st;
        return l;
    };
    auto plain = [&](uint64_t work) {
        pt::Launch l;
        l.block = 256;
        l.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 8));
        l.st = st;
        return l;
    };
    uint32_t n_keys = 0;
    if (o.sort_mode == PT_SORT_TYPE) n_keys = 4;
    if (o.sort_mode == PT_SORT_MATERIAL) n_keys = std::min<uint32_t>(ds.n_mats + 1, pt::kMaxSortKeys);
    const uint32_t sort_mode = o.sort_mode == PT_SORT_TYPE ? 1u : 2u;
    pt::RenderParams p;
    p.seed = seed;
    p.spp = spp;
    p.max_depth = max_depth;
    p.rr_start = o.rr_start;
    p.rr_fixed = o.rr_fixed;
    p.sampler = (o.flags & PT_FLAG_HALTON) ? pt::SAMPLER_HALTON_ID : 0u;
    p.mis = (o.flags & PT_FLAG_MIS) ? 1u : 0u;
    for (uint64_t w0 = 0; w0 < n_paths; w0 += cap) {
        const uint32_t n = (uint32_t)std::min<uint64_t>(cap, n_paths - w0);
        p.path_begin = w0;
        pt::Launch le = persistent(per_extend, n), ls = persistent(per_shade, n);
        const pt::Launch lw = persistent(per_shadow, n);
        pt::Launch lt = persistent(per_trace, 2ull * n), lr = plain(n / spp);
        // fused: the stage kernels are programmatic dependents of the kernel before them, as in pt_render
        le.pdl = ls.pdl = lt.pdl = lr.pdl = fused && n_keys == 0;
        if ((e = pt::launch_raygen(plain(n), dc, p, n, w)) != cudaSuccess) return cuda_fail(e, "raygen");
        for (uint32_t b = 0; b < max_depth; ++b) {
            const int in = (int)(b & 1u);
            if (!fused || b == 0) {          // no shadow rays are pending before the first shading
                if ((e = pt::launch_extend(le, ds, w, in, p)) != cudaSuccess) return cuda_fail(e, "extend");
            } else if ((e = pt::launch_trace(lt, ds, p, w, in, b)) != cudaSuccess) {
                return cuda_fail(e, "trace");
            }
            if (n_keys && (e = pt::launch_sort(plain(n), ds, w, in, sort_mode, n_keys, p)) != cudaSuccess)
                return cuda_fail(e, "sort");
            if ((e = pt::launch_shade(ls, ds, p, w, in, b, n_keys > 0)) != cudaSuccess) return cuda_fail(e, "shade");
            if (fused) {
                if ((e = pt::launch_prepare_fused(st, w, b, le.pdl)) != cudaSuccess) return cuda_fail(e, "prepare");
                continue;
            }
            if ((e = pt::launch_shadow(lw, ds, p, w, b)) != cudaSuccess) return cuda_fail(e, "shadow");
            if ((e = pt::launch_prepare(st, w, b)) != cudaSuccess) return cuda_fail(e, "prepare");
        }
        if ((e = pt::launch_reduce(lr, reinterpret_cast<const float*>(w.L), 4, w0 / spp, n / spp, spp,
                                   d_out_rgb)) != cudaSuccess)
            return cuda_fail(e, "reduce");
    }
    return PT_OK;
}
