// pt_api.cpp -- the C ABI of include/pt.h: argument validation, scene packing and upload, workspace
// management, and the host side of the megakernel / wavefront / adjoint / batched pipelines.
// Every call is asynchronous on the caller's stream except where the header says otherwise.
#include "pt.h"

#include <cuda_runtime_api.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bvh_build.h"
#include "pt_launch.h"
#include "pt_types.h"

namespace {

thread_local std::string g_err;

pt_status fail(pt_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define PT_CUDA(expr)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(PT_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

#define PT_TRY(expr)                   \
    do {                               \
        pt_status s_ = (expr);         \
        if (s_ != PT_OK) return s_;    \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    pt_status ensure(size_t want) {
        if (bytes >= want && p) return PT_OK;
        release();
        if (want == 0) want = 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(PT_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", want, cudaGetErrorString(e));
        }
        bytes = want;
        return PT_OK;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int sm_count(int device) {
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(device);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    cache[device] = n;
    return n;
}

int blocks_per_sm(int which, int block) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(which, block);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = pt::max_blocks_per_sm(which, block);
    cache[key] = n;
    return n;
}

enum Stage { ST_RAYGEN, ST_EXTEND, ST_SORT, ST_SHADE, ST_SHADOW, ST_REDUCE, ST_MEGA, ST_ADJOINT, ST_COUNT };

// One device allocation carved into the wavefront arrays for `cap` paths (kWfBytesPerPath each).
pt_status carve_wavefront(DevBuf& buf, uint64_t cap, pt::WfBuffers& w) {
    PT_TRY(buf.ensure(pt::wavefront_bytes(cap)));
    pt::carve_wavefront_at(buf.as<char>(), cap, w);
    return PT_OK;
}

}  // namespace

struct pt_scene {
    int device = 0;
    uint64_t n_tris = 0, n_nodes = 0, n_lights = 0;
    uint32_t n_mats = 0;
    float light_area = 0.f;
    float env[3] = {0.f, 0.f, 0.f};
    DevBuf nodes, tris, mats, lights, cdf, status;
    DevBuf tlas, inst;          // two-level scenes: top-level nodes and instance records
    bool instanced = false;
    // workspaces (grown on demand, kept until destroy)
    DevBuf wf;
    uint64_t wf_capacity = 0;
    pt::WfBuffers wfb{};
    DevBuf pathL, img_stage, grad_stage, counters, adj;
    cudaStream_t last_stream = nullptr;
    uint32_t last_mode = 0;
    uint64_t last_paths = 0;
    uint32_t launches = 0;     // kernel launches issued by the last call
    // profiling: stage intervals between events recorded on the launch stream.  Consecutive stages
    // share the event between them (one record per stage boundary: each record costs the stream a
    // couple of microseconds).  A stage's end is recorded when the next stage begins, another
    // stage ends, or the call finishes, so a bookkeeping launch between two stages counts toward
    // the earlier one.
    struct Ev {
        int stage;
        int a, b;      // indices into ev_pool; -1: not recorded
    };
    std::vector<Ev> events;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0, pool_used = 0;
    long ev_pending = -1;     // the stage whose end is still to be recorded
    bool profiling = false;
    std::mutex mu;

    ~pt_scene() {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    }

    pt::DevScene view() const {
        pt::DevScene s;
        s.nodes = nodes.as<const float4>();
        s.tris = tris.as<const float4>();
        s.mats = mats.as<const pt::DevMat>();
        s.lights = lights.as<const float4>();
        s.light_cdf = cdf.as<const float>();
        s.n_lights = (uint32_t)n_lights;
        s.light_area = light_area;
        s.env_r = env[0];
        s.env_g = env[1];
        s.env_b = env[2];
        s.n_mats = n_mats;
        s.status = status.as<uint32_t>();
        s.tlas = instanced ? tlas.as<const float4>() : nullptr;
        s.inst = instanced ? inst.as<const float4>() : nullptr;
        s.trav = trav();
        return s;
    }
    uint32_t* counts() const { return counters.as<uint32_t>(); }
    unsigned long long* hist() const { return reinterpret_cast<unsigned long long*>(counters.as<char>() + 256); }
    unsigned long long* rays() const { return hist() + 128; }

    pt_status ensure_counters() { return counters.ensure(256 + 8 * pt::kHistWords); }
    unsigned long long* trav() const { return hist() + 132; }   // 4 traversal counters
    unsigned long long* next_path() const { return hist() + 130; }
    unsigned long long* finish_claim() const { return hist() + 131; }

    // One allocation carved into the wavefront arrays for `cap` paths per wave.
    pt_status ensure_wf(uint64_t cap) {
        if (wf_capacity >= cap && wf.p) return PT_OK;
        PT_TRY(carve_wavefront(wf, cap, wfb));
        wf_capacity = cap;
        return PT_OK;
    }

    void ev_reset(bool on) {
        profiling = on;
        ev_used = 0;
        pool_used = 0;
        ev_pending = -1;
    }
    pt_status ev_record(cudaStream_t st, int& slot) {
        if (pool_used == ev_pool.size()) {
            cudaEvent_t e = nullptr;
            PT_CUDA(cudaEventCreate(&e));
            ev_pool.push_back(e);
        }
        slot = (int)pool_used++;
        PT_CUDA(cudaEventRecord(ev_pool[slot], st));
        return PT_OK;
    }
    pt_status ev_begin(int stage, cudaStream_t st, size_t& idx) {
        if (!profiling) return PT_OK;
        int e = -1;
        PT_TRY(ev_record(st, e));
        if (ev_pending >= 0) {
            events[ev_pending].b = e;
            ev_pending = -1;
        }
        if (ev_used == events.size()) events.push_back(Ev{stage, -1, -1});
        idx = ev_used++;
        events[idx] = Ev{stage, e, -1};
        return PT_OK;
    }
    pt_status ev_end(size_t idx, cudaStream_t st) {
        if (!profiling) return PT_OK;
        PT_TRY(ev_flush(st));
        ev_pending = (long)idx;
        return PT_OK;
    }
    pt_status ev_flush(cudaStream_t st) {
        if (!profiling || ev_pending < 0) return PT_OK;
        int e = -1;
        PT_TRY(ev_record(st, e));
        events[ev_pending].b = e;
        ev_pending = -1;
        return PT_OK;
    }
};

namespace {

pt_status make_camera(const pt_camera* cam, pt::DevCamera& c) {
    if (!cam) return fail(PT_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width == 0 || cam->height == 0) return fail(PT_ERR_INVALID_ARG, "camera width/height must be > 0");
    if ((uint64_t)cam->width * cam->height >= (1ull << 32))
        return fail(PT_ERR_INVALID_ARG, "camera has more than 2^32 pixels");
    if (!(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f))
        return fail(PT_ERR_INVALID_ARG, "vfov_deg must be in (0, 180)");
    if (!finite3(cam->eye) || !finite3(cam->target) || !finite3(cam->up))
        return fail(PT_ERR_INVALID_ARG, "camera vectors must be finite");
    double e[3], w[3], u[3], v[3];
    for (int k = 0; k < 3; ++k) {
        e[k] = cam->eye[k];
        w[k] = (double)cam->eye[k] - (double)cam->target[k];
    }
    double wl = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(wl > 0)) return fail(PT_ERR_INVALID_ARG, "camera eye equals target");
    for (double& x : w) x /= wl;
    double up[3] = {cam->up[0], cam->up[1], cam->up[2]};
    u[0] = up[1] * w[2] - up[2] * w[1];
    u[1] = up[2] * w[0] - up[0] * w[2];
    u[2] = up[0] * w[1] - up[1] * w[0];
    double ul = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(ul > 0)) return fail(PT_ERR_INVALID_ARG, "camera up is parallel to the view direction");
    for (double& x : u) x /= ul;
    v[0] = w[1] * u[2] - w[2] * u[1];
    v[1] = w[2] * u[0] - w[0] * u[2];
    v[2] = w[0] * u[1] - w[1] * u[0];
    double th = std::tan((double)cam->vfov_deg * M_PI / 360.0);
    double tw = th * (double)cam->width / (double)cam->height;
    c.ex = (float)e[0];
    c.ey = (float)e[1];
    c.ez = (float)e[2];
    c.ux = (float)(u[0] * tw);
    c.uy = (float)(u[1] * tw);
    c.uz = (float)(u[2] * tw);
    c.vx = (float)(v[0] * th);
    c.vy = (float)(v[1] * th);
    c.vz = (float)(v[2] * th);
    c.wx = (float)w[0];
    c.wy = (float)w[1];
    c.wz = (float)w[2];
    c.W = cam->width;
    c.H = cam->height;
    return PT_OK;
}

pt_render_opts default_opts() {
    pt_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = PT_MODE_WAVEFRONT;
    o.rr_start = 3;
    return o;
}

pt_status check_opts(const pt_render_opts& o) {
    if (o.mode > PT_MODE_WAVEFRONT) return fail(PT_ERR_INVALID_ARG, "opts.mode must be 0 or 1");
    if (!(o.rr_fixed >= 0.f && o.rr_fixed <= 1.f)) return fail(PT_ERR_INVALID_ARG, "opts.rr_fixed must be in [0, 1]");
    if (o.sort_mode > PT_SORT_MATERIAL) return fail(PT_ERR_INVALID_ARG, "opts.sort_mode must be 0, 1 or 2");
    if (o.block_size && (o.block_size % 32 || o.block_size < 64 || o.block_size > 256))
        return fail(PT_ERR_INVALID_ARG, "opts.block_size must be 0 or a multiple of 32 in [64, 256]");
    return PT_OK;
}

// The short-stack instantiation of a single-level stage (PT_FLAG_SHORT_STACK), whose occupancy
// includes its shared-memory stacks.
int short_stack_kernel(const pt_scene* sc, int kernel, bool on) {
    if (!on || sc->instanced) return kernel;
    switch (kernel) {
        case pt::K_EXTEND: return pt::K_EXTEND_SS;
        case pt::K_SHADOW: return pt::K_SHADOW_SS;
        case pt::K_MEGA_REGEN: return pt::K_MEGA_REGEN_SS;
        case pt::K_FINISH: return pt::K_FINISH_SS;
        default: return kernel;
    }
}

// The two-level instantiation of a wavefront stage (its register count, hence its occupancy, differs).
int stage_kernel(const pt_scene* sc, int kernel) {
    if (!sc->instanced) return kernel;
    switch (kernel) {
        case pt::K_EXTEND: return pt::K_EXTEND_INST;
        case pt::K_SHADE: return pt::K_SHADE_INST;
        case pt::K_SHADOW: return pt::K_SHADOW_INST;
        case pt::K_SHADE_ADJ: return pt::K_SHADE_ADJ_INST;
        case pt::K_SHADOW_ADJ: return pt::K_SHADOW_ADJ_INST;
        default: return kernel;
    }
}

pt::Launch launch_for(const pt_scene* sc, int kernel, uint32_t block_opt, uint32_t def_block, cudaStream_t st,
                      uint64_t work_upper) {
    kernel = stage_kernel(sc, kernel);
    pt::Launch l;
    l.block = block_opt ? (int)block_opt : (int)def_block;
    int per = blocks_per_sm(kernel, l.block);
    uint64_t grid = (uint64_t)sm_count(sc->device) * (uint64_t)per;
    uint64_t need = (work_upper + l.block - 1) / l.block;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    l.grid = (int)grid;
    l.st = st;
    return l;
}

pt::Launch simple_launch(const pt_scene* sc, cudaStream_t st, uint64_t work) {
    pt::Launch l;
    l.block = 256;
    uint64_t grid = std::min<uint64_t>((work + 255) / 256, (uint64_t)sm_count(sc->device) * 8);
    l.grid = (int)std::max<uint64_t>(grid, 1);
    l.st = st;
    return l;
}

pt_status set_device(const pt_scene* sc) {
    int cur = -1;
    PT_CUDA(cudaGetDevice(&cur));
    if (cur != sc->device) PT_CUDA(cudaSetDevice(sc->device));
    return PT_OK;
}

// The fused wavefront's stage kernels (forward and the adjoint's replay) are launched as programmatic
// dependents of the kernel before them (sm_90+): each may become resident while its predecessor
// drains and waits for it on the device (stage_prologue), which hides the launch gap between
// dependent stages.
constexpr bool kStagePdl = true;

// The wavefront pipeline over one scene and camera, waves of `cap` paths (a multiple of spp).  With
// `accum`, each wave's samples continue the per-pixel running sums and img = sum / count.
pt_status run_wavefront(pt_scene* sc, const pt::DevCamera& cam, const pt::RenderParams& p0, const pt_render_opts& o,
                        uint64_t n_paths, float* img, float* path_L, uint32_t* sig, cudaStream_t st,
                        float* accum = nullptr, uint32_t count = 0) {
    uint64_t cap = o.queue_capacity ? std::min<uint64_t>(o.queue_capacity, n_paths) : n_paths;
    cap = std::max<uint64_t>(cap - cap % p0.spp, p0.spp);
    if (cap >= (1ull << 32)) cap = ((1ull << 32) - (1ull << 20)) / p0.spp * p0.spp;
    PT_TRY(sc->ensure_wf(cap));
    pt::WfBuffers w = sc->wfb;
    w.counts = sc->counts();
    w.hist = sc->hist();
    w.sig = sig;
    w.capacity = (uint32_t)cap;
    const pt::DevScene ds = sc->view();
    uint32_t n_keys = 0;
    if (o.sort_mode == PT_SORT_TYPE) n_keys = 4;                       // 3 types + miss
    if (o.sort_mode == PT_SORT_MATERIAL) n_keys = std::min<uint32_t>(sc->n_mats + 1, pt::kMaxSortKeys);
    const uint32_t sort_mode = o.sort_mode == PT_SORT_TYPE ? 1u : 2u;
    for (uint64_t w0 = 0; w0 < n_paths; w0 += cap) {
        const uint32_t n = (uint32_t)std::min<uint64_t>(cap, n_paths - w0);
        pt::RenderParams p = p0;
        p.path_begin = w0;
        size_t ev = 0;
        PT_TRY(sc->ev_begin(ST_RAYGEN, st, ev));
        PT_CUDA(pt::launch_raygen(simple_launch(sc, st, n), cam, p, n, w));
        PT_TRY(sc->ev_end(ev, st));
        sc->launches += 1;
        // fused: each bounce's extend launch also walks the shadow rays the previous shading cast
        // (no stage boundary between them); the hybrid and the short-stack variant keep the stages apart
        const bool fused = !(o.flags & PT_FLAG_SEPARATE_SHADOW) && !o.hybrid_threshold && !p.short_stack;
        for (uint32_t b = 0; b < p.max_depth; ++b) {
            const int in = (int)(b & 1u);
            if (fused) {
                PT_TRY(sc->ev_begin(ST_EXTEND, st, ev));
                if (b == 0) {     // no shadow rays are pending before the first shading
                    pt::Launch le = launch_for(sc, pt::K_EXTEND, o.block_size, 256, st, n);
                    le.pdl = kStagePdl;
                    PT_CUDA(pt::launch_extend(le, ds, w, in, p));
                } else {
                    pt::Launch lt = launch_for(sc, sc->instanced ? pt::K_TRACE_INST : pt::K_TRACE, o.block_size, 256, st,
                                               2ull * n);
                    lt.pdl = kStagePdl;
                    PT_CUDA(pt::launch_trace(lt, ds, p, w, in, b));
                }
                PT_TRY(sc->ev_end(ev, st));
                bool sorted_f = n_keys > 0;
                if (sorted_f) {
                    PT_TRY(sc->ev_begin(ST_SORT, st, ev));
                    PT_CUDA(pt::launch_sort(simple_launch(sc, st, n), ds, w, in, sort_mode, n_keys, p));
                    PT_TRY(sc->ev_end(ev, st));
                }
                pt::Launch ls = launch_for(sc, pt::K_SHADE, o.block_size, 256, st, n);
                ls.pdl = kStagePdl && !sorted_f;
                PT_TRY(sc->ev_begin(ST_SHADE, st, ev));
                PT_CUDA(pt::launch_shade(ls, ds, p, w, in, b, sorted_f));
                PT_TRY(sc->ev_end(ev, st));
                PT_CUDA(pt::launch_prepare_fused(st, w, b, kStagePdl));
                sc->launches += 3 + (sorted_f ? 3 : 0);
                continue;
            }
            pt::Launch le = launch_for(sc, short_stack_kernel(sc, pt::K_EXTEND, p.short_stack), o.block_size, 256, st, n);
            PT_TRY(sc->ev_begin(ST_EXTEND, st, ev));
            PT_CUDA(pt::launch_extend(le, ds, w, in, p));
            PT_TRY(sc->ev_end(ev, st));
            bool sorted = n_keys > 0;
            if (sorted) {
                PT_TRY(sc->ev_begin(ST_SORT, st, ev));
                PT_CUDA(pt::launch_sort(simple_launch(sc, st, n), ds, w, in, sort_mode, n_keys, p));
                PT_TRY(sc->ev_end(ev, st));
            }
            pt::Launch ls = launch_for(sc, pt::K_SHADE, o.block_size, 256, st, n);
            PT_TRY(sc->ev_begin(ST_SHADE, st, ev));
            PT_CUDA(pt::launch_shade(ls, ds, p, w, in, b, sorted));
            PT_TRY(sc->ev_end(ev, st));
            pt::Launch lw = launch_for(sc, short_stack_kernel(sc, pt::K_SHADOW, p.short_stack), o.block_size, 256, st, n);
            PT_TRY(sc->ev_begin(ST_SHADOW, st, ev));
            PT_CUDA(pt::launch_shadow(lw, ds, p, w, b));
            PT_TRY(sc->ev_end(ev, st));
            PT_CUDA(pt::launch_prepare(st, w, b));
            sc->launches += 4 + (sorted ? 3 : 0);
            if (o.hybrid_threshold && b + 1 < p.max_depth) {
                // hybrid: finish the remaining bounces in one kernel if few paths are left
                const uint32_t thr = (uint32_t)std::min<uint64_t>(o.hybrid_threshold, 0xFFFFFFFFull);
                pt::Launch lf = launch_for(sc, sc->instanced ? pt::K_FINISH_INST : short_stack_kernel(sc, pt::K_FINISH, p.short_stack),
                                           128, 128, st,
                                           std::min<uint64_t>(n, thr));
                PT_TRY(sc->ev_begin(ST_MEGA, st, ev));
                PT_CUDA(pt::launch_finish(lf, ds, p, w, (int)((b + 1) & 1u), b + 1, thr, sc->finish_claim()));
                PT_TRY(sc->ev_end(ev, st));
                sc->launches += 2;
            }
        }
        PT_TRY(sc->ev_begin(ST_REDUCE, st, ev));
        if (accum)
            PT_CUDA(pt::launch_accumulate(simple_launch(sc, st, n / p.spp), reinterpret_cast<const float*>(w.L), 4,
                                          w0 / p.spp, n / p.spp, p.spp, accum, count, img));
        else {
            pt::Launch lr = simple_launch(sc, st, n / p.spp);
            lr.pdl = kStagePdl;
            PT_CUDA(pt::launch_reduce(lr, reinterpret_cast<const float*>(w.L), 4, w0 / p.spp, n / p.spp, p.spp, img));
        }
        if (path_L) PT_CUDA(pt::launch_copy_L(simple_launch(sc, st, n), w.L, n, path_L + 3 * w0));
        PT_TRY(sc->ev_end(ev, st));
        sc->launches += path_L ? 2 : 1;
    }
    return PT_OK;
}

}  // namespace

// Internal helpers for the allocation-free entry point in pt_static.cu (C++ linkage, not exported
// from the ABI).  They only read the scene and convert arguments; none of them allocates.
namespace pt {

pt_status static_set_error(pt_status s, const char* msg) { return fail(s, "%s", msg); }

pt_status static_prepare(pt_scene* sc, const pt_camera* cam, const pt_render_opts* opts, DevScene* view,
                         DevCamera* dc, pt_render_opts* o_out, int* device) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    pt_render_opts o = opts ? *opts : default_opts();
    PT_TRY(check_opts(o));
    PT_TRY(make_camera(cam, *dc));
    PT_TRY(set_device(sc));
    *view = sc->view();
    *o_out = o;
    *device = sc->device;
    return PT_OK;
}

bool static_is_device_ptr(const void* p) { return is_device_ptr(p); }

}  // namespace pt

// ------------------------------------------------------------------ batched rendering
// Process-wide state of pt_render_batch on one device: the wavefront workspace, the device tables
// (scene views, cameras, path and pixel offsets, spp, output pointers, wave segments), counters, a
// private non-blocking stream for graph capture, and the captured bounce-loop graph.
namespace {

struct BatchCtx {
    DevBuf wf, tables, counters;
    pt::WfBuffers wfb{};
    uint64_t capacity = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<uint64_t> graph_key;
    std::mutex mu;
};

BatchCtx* batch_ctx(int device) {
    static std::mutex mu;
    static std::map<int, BatchCtx*> ctxs;   // kept for the life of the process
    std::lock_guard<std::mutex> g(mu);
    BatchCtx*& c = ctxs[device];
    if (!c) c = new BatchCtx();
    return c;
}

template <class T>
size_t put(std::vector<char>& blob, const T* v, size_t count) {
    size_t off = align256(blob.size());
    blob.resize(off + sizeof(T) * count);
    if (count) std::memcpy(blob.data() + off, v, sizeof(T) * count);
    return off;
}

}  // namespace

pt_status batch_render(pt_scene* const* scenes, const pt_camera* cams, const uint32_t* spp, uint32_t n,
                       uint32_t max_depth, uint64_t seed, const pt_render_opts* opts, float* const* d_out,
                       void* stream) {
    if (!scenes || !cams || !spp || !d_out || n == 0) return fail(PT_ERR_INVALID_ARG, "empty batch or NULL arrays");
    if (max_depth > 64) return fail(PT_ERR_INVALID_ARG, "max_depth must be <= 64");
    pt_render_opts o = opts ? *opts : default_opts();
    PT_TRY(check_opts(o));
    const int device = scenes[0] ? scenes[0]->device : -1;
    std::vector<pt::DevScene> views(n);
    std::vector<pt::DevCamera> dcs(n);
    std::vector<unsigned long long> off(n + 1, 0), px_off(n + 1, 0);
    std::vector<uint32_t> spps(n);
    std::vector<float*> outs(n);
    uint32_t max_mats = 1;
    for (uint32_t i = 0; i < n; ++i) {
        if (!scenes[i]) return fail(PT_ERR_INVALID_ARG, "scene %u is NULL", i);
        if (scenes[i]->device != device) return fail(PT_ERR_INVALID_ARG, "scene %u is on another device", i);
        if (scenes[i]->instanced) return fail(PT_ERR_UNSUPPORTED, "scene %u is a two-level scene: batched rendering takes single-level scenes", i);
        if (spp[i] == 0) return fail(PT_ERR_INVALID_ARG, "spp[%u] must be >= 1", i);
        PT_TRY(make_camera(&cams[i], dcs[i]));
        if (!d_out[i] || !is_device_ptr(d_out[i])) return fail(PT_ERR_INVALID_ARG, "d_out[%u] must be device memory", i);
        views[i] = scenes[i]->view();
        spps[i] = spp[i];
        outs[i] = d_out[i];
        max_mats = std::max(max_mats, scenes[i]->n_mats);
        const uint64_t px = (uint64_t)cams[i].width * cams[i].height;
        px_off[i + 1] = px_off[i] + px;
        off[i + 1] = off[i] + px * spp[i];
    }
    const uint64_t total = off[n];
    if (total >= (1ull << 40)) return fail(PT_ERR_INVALID_ARG, "too many paths");
    PT_TRY(set_device(scenes[0]));
    BatchCtx* ctx = batch_ctx(device);
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t cap = o.queue_capacity ? std::min<uint64_t>(o.queue_capacity, total) : std::min<uint64_t>(total, 1ull << 24);
    cap = std::max<uint64_t>(cap, 1);
    if (cap >= (1ull << 32)) cap = (1ull << 32) - (1ull << 20);
    if (ctx->capacity < cap || !ctx->wf.p) {
        if (ctx->graph) {
            cudaGraphExecDestroy(ctx->graph);
            ctx->graph = nullptr;
        }
        PT_CUDA(cudaStreamSynchronize(st));
        PT_TRY(carve_wavefront(ctx->wf, cap, ctx->wfb));
        ctx->capacity = cap;
    }
    PT_TRY(ctx->counters.ensure(256 + 8 * pt::kHistWords));
    // wave segments: runs of pixels of one scene inside each wave
    std::vector<pt::BatchSegment> segs;
    struct Wave {
        uint64_t w0, w1, flat;
        uint32_t seg0, nseg;
    };
    std::vector<Wave> waves;
    // waves: a scene larger than half a wave gets waves of its own (one large BVH in L2 at a time);
    // smaller scenes are packed together up to the capacity
    std::vector<std::pair<uint64_t, uint64_t>> ranges;
    {
        uint64_t cur0 = 0, cur1 = 0;
        for (uint32_t s = 0; s < n; ++s) {
            const uint64_t a0 = off[s], a1 = off[s + 1];
            if (a1 - a0 > cap / 2) {
                if (cur1 > cur0) ranges.push_back({cur0, cur1});
                const uint64_t k = (a1 - a0 + cap - 1) / cap, per = (a1 - a0 + k - 1) / k;
                for (uint64_t x = a0; x < a1; x += per) ranges.push_back({x, std::min(a1, x + per)});
                cur0 = cur1 = a1;
            } else {
                if (a1 - cur0 > cap) {
                    ranges.push_back({cur0, cur1});
                    cur0 = cur1;
                }
                cur1 = a1;
            }
        }
        if (cur1 > cur0) ranges.push_back({cur0, cur1});
    }
    for (const auto& rg : ranges) {
        const uint64_t w0 = rg.first, w1 = rg.second;
        Wave wv{w0, w1, 0, (uint32_t)segs.size(), 0};
        for (uint32_t s = 0; s < n; ++s) {
            if (off[s + 1] <= w0 || off[s] >= w1 || off[s + 1] == off[s]) continue;
            const uint64_t a = std::max(w0, (uint64_t)off[s]) - off[s], b = std::min(w1, (uint64_t)off[s + 1]) - off[s];
            const uint64_t p0 = a / spps[s], p1 = (b + spps[s] - 1) / spps[s];
            pt::BatchSegment sg{s, 0, p0, p1 - p0, wv.flat};
            segs.push_back(sg);
            wv.flat += p1 - p0;
            wv.nseg++;
        }
        waves.push_back(wv);
    }
    std::vector<char> blob;
    const size_t o_sc = put(blob, views.data(), n), o_cam = put(blob, dcs.data(), n), o_off = put(blob, off.data(), n + 1),
                 o_spp = put(blob, spps.data(), n), o_out = put(blob, outs.data(), n),
                 o_px = put(blob, px_off.data(), n + 1), o_seg = put(blob, segs.data(), segs.size());
    const unsigned long long seed64 = seed;
    const size_t o_seed = put(blob, &seed64, 1);
    if (ctx->tables.bytes < blob.size() && ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (ctx->tables.bytes < blob.size()) PT_CUDA(cudaStreamSynchronize(st));
    PT_TRY(ctx->tables.ensure(std::max<size_t>(blob.size(), 1 << 16)));
    PT_CUDA(cudaMemcpyAsync(ctx->tables.p, blob.data(), blob.size(), cudaMemcpyHostToDevice, st));
    char* tb = ctx->tables.as<char>();
    pt::BatchTables t;
    t.scenes = reinterpret_cast<const pt::DevScene*>(tb + o_sc);
    t.cams = reinterpret_cast<const pt::DevCamera*>(tb + o_cam);
    t.off = reinterpret_cast<const unsigned long long*>(tb + o_off);
    t.spp = reinterpret_cast<const uint32_t*>(tb + o_spp);
    t.out = reinterpret_cast<float* const*>(tb + o_out);
    t.n = n;
    t.wave_base = reinterpret_cast<unsigned long long*>(ctx->counters.as<char>() + 128);
    t.seed = reinterpret_cast<const unsigned long long*>(tb + o_seed);
    const unsigned long long* px_dev = reinterpret_cast<const unsigned long long*>(tb + o_px);
    const pt::BatchSegment* seg_dev = reinterpret_cast<const pt::BatchSegment*>(tb + o_seg);
    pt::WfBuffers w = ctx->wfb;
    w.counts = ctx->counters.as<uint32_t>();
    w.hist = reinterpret_cast<unsigned long long*>(ctx->counters.as<char>() + 256);
    w.sig = nullptr;
    w.capacity = (uint32_t)cap;
    PT_CUDA(cudaMemsetAsync(ctx->counters.p, 0, ctx->counters.bytes, st));
    for (uint32_t i = 0; i < n; ++i) PT_CUDA(cudaMemsetAsync(outs[i], 0, (px_off[i + 1] - px_off[i]) * 12, st));
    if (max_depth == 0) return PT_OK;
    pt::RenderParams p;
    p.seed = seed;
    p.path_begin = 0;
    p.spp = 1;
    p.max_depth = max_depth;
    p.rr_start = o.rr_start;
    p.rr_fixed = o.rr_fixed;
    p.sampler = (o.flags & PT_FLAG_HALTON) ? pt::SAMPLER_HALTON_ID : 0u;
    p.mis = (o.flags & PT_FLAG_MIS) ? 1u : 0u;
    uint32_t n_keys = 0;
    if (o.sort_mode == PT_SORT_TYPE) n_keys = 4;
    if (o.sort_mode == PT_SORT_MATERIAL) n_keys = std::min<uint32_t>(max_mats + 1, pt::kMaxSortKeys);
    const uint32_t sort_mode = o.sort_mode == PT_SORT_TYPE ? 1u : 2u;
    const uint32_t block = o.block_size ? o.block_size : 256;
    const int sms = sm_count(device);
    auto persistent = [&](int which, cudaStream_t s_) {
        pt::Launch l;
        l.block = (int)block;
        l.grid = std::max(1, sms * blocks_per_sm(which, (int)block));
        l.st = s_;
        return l;
    };
    auto plain = [&](uint64_t work, cudaStream_t s_) {
        pt::Launch l;
        l.block = 256;
        l.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 8));
        l.st = s_;
        return l;
    };
    const bool fused = !(o.flags & PT_FLAG_SEPARATE_SHADOW);
    auto bounce_loop = [&](cudaStream_t s_) -> pt_status {
        for (uint32_t b = 0; b < max_depth; ++b)
            PT_CUDA(pt::launch_bounce_batch(persistent(pt::K_EXTEND_BATCH, s_), persistent(pt::K_SHADE_BATCH, s_),
                                            persistent(fused ? pt::K_TRACE_BATCH : pt::K_SHADOW_BATCH, s_),
                                            plain(cap, s_), t, p, w, b, sort_mode, n_keys, fused));
        return PT_OK;
    };
    const bool use_graph = !(o.flags & PT_FLAG_NO_GRAPH);
    if (use_graph) {
        // the captured loop depends only on these; tables and counters are read from device memory
        std::vector<uint64_t> key = {cap, max_depth, n_keys, sort_mode, block, o.rr_start, (uint64_t)fused,
                                     (uint64_t)__builtin_bit_cast(uint32_t, o.rr_fixed),
                                     (uint64_t)(uintptr_t)ctx->tables.p, (uint64_t)(uintptr_t)ctx->wf.p, n};
        if (!ctx->graph || ctx->graph_key != key) {
            if (ctx->graph) {
                cudaGraphExecDestroy(ctx->graph);
                ctx->graph = nullptr;
            }
            if (!ctx->cap_stream) PT_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            PT_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            pt_status cs = bounce_loop(ctx->cap_stream);
            cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (cs != PT_OK) {
                if (graph) cudaGraphDestroy(graph);
                return cs;
            }
            if (ce != cudaSuccess) return fail(PT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&ctx->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                ctx->graph = nullptr;
                return fail(PT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            }
            ctx->graph_key = key;
        }
    }
    for (const Wave& wv : waves) {
        const uint32_t nw = (uint32_t)(wv.w1 - wv.w0);
        PT_CUDA(pt::launch_raygen_batch(plain(nw, st), t, p, wv.w0, nw, w));
        if (use_graph) PT_CUDA(cudaGraphLaunch(ctx->graph, st));
        else PT_TRY(bounce_loop(st));
        PT_CUDA(pt::launch_reduce_batch(plain(wv.flat, st), t, w.L, seg_dev + wv.seg0, wv.nseg, wv.w0, wv.w1, wv.flat));
    }
    PT_CUDA(pt::launch_scale_batch(plain(px_off[n], st), t, px_dev, px_off[n]));
    return PT_OK;
}

namespace {

// pt_render and pt_render_progressive.  With `accum` the samples are pixel samples
// sample_offset .. sample_offset + spp - 1, added to the running sums, and the image (if any) is
// sum / (sample_offset + spp).
pt_status render_impl(pt_scene* sc, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                      const pt_render_opts* opts, float* d_out_rgb, float* d_path_L_or_null, void* stream,
                      uint32_t sample_offset, float* accum) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if (!d_out_rgb && !accum) return fail(PT_ERR_INVALID_ARG, "output image is NULL");
    if (spp == 0) return fail(PT_ERR_INVALID_ARG, "spp must be >= 1");
    if (max_depth > 64) return fail(PT_ERR_INVALID_ARG, "max_depth must be <= 64");
    if ((uint64_t)sample_offset + spp > 0xFFFFFFFFull) return fail(PT_ERR_INVALID_ARG, "sample_offset + spp overflows 32 bits");
    pt_render_opts o = opts ? *opts : default_opts();
    PT_TRY(check_opts(o));
    pt::DevCamera dc;
    PT_TRY(make_camera(cam, dc));
    const uint64_t n_pixels = (uint64_t)cam->width * cam->height;
    const uint64_t n_paths = n_pixels * spp;
    if (n_paths >= (1ull << 40)) return fail(PT_ERR_INVALID_ARG, "too many paths");
    if (d_path_L_or_null && !is_device_ptr(d_path_L_or_null)) return fail(PT_ERR_INVALID_ARG, "path_L must be a device pointer");
    if (o.d_path_sig && !is_device_ptr(o.d_path_sig)) return fail(PT_ERR_INVALID_ARG, "d_path_sig must be a device pointer");
    if (accum && !is_device_ptr(accum)) return fail(PT_ERR_INVALID_ARG, "d_accum_rgb must be a device pointer");
    if (accum && d_out_rgb && !is_device_ptr(d_out_rgb))
        return fail(PT_ERR_INVALID_ARG, "d_out_rgb must be a device pointer for progressive rendering");
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool host_out = d_out_rgb && !is_device_ptr(d_out_rgb);
    float* img = d_out_rgb;
    if (host_out) {
        PT_TRY(sc->img_stage.ensure(n_pixels * 12));
        img = sc->img_stage.as<float>();
    }
    const uint32_t count = sample_offset + spp;
    sc->ev_reset((o.flags & PT_FLAG_PROFILE) != 0);
    sc->last_stream = st;
    sc->last_mode = o.mode;
    sc->last_paths = n_paths;
    sc->launches = 0;
    PT_CUDA(cudaMemsetAsync(sc->counters.p, 0, sc->counters.bytes, st));
    PT_CUDA(cudaMemsetAsync(sc->status.p, 0, 4, st));
    if (accum && sample_offset == 0) PT_CUDA(cudaMemsetAsync(accum, 0, n_pixels * 12, st));
    pt::RenderParams p;
    p.seed = seed;
    p.path_begin = 0;
    p.spp = spp;
    p.max_depth = max_depth;
    p.rr_start = o.rr_start;
    p.rr_fixed = o.rr_fixed;
    p.sampler = (o.flags & PT_FLAG_HALTON) ? pt::SAMPLER_HALTON_ID : 0u;
    p.mis = (o.flags & PT_FLAG_MIS) ? 1u : 0u;
    p.short_stack = (o.flags & PT_FLAG_SHORT_STACK) ? 1u : 0u;
    p.count_trav = (o.flags & PT_FLAG_COUNT_TRAVERSAL) ? 1u : 0u;
    p.sample_offset = sample_offset;
    if (max_depth == 0) {
        // every sample is black: the sums are unchanged and the image is sum / count
        if (accum) {
            size_t ev = 0;
            PT_TRY(sc->ev_begin(ST_REDUCE, st, ev));
            PT_CUDA(pt::launch_accumulate(simple_launch(sc, st, n_pixels), nullptr, 3, 0, n_pixels, 0, accum, count, img));
            PT_TRY(sc->ev_end(ev, st));
            sc->launches += 1;
        } else {
            PT_CUDA(cudaMemsetAsync(img, 0, n_pixels * 12, st));
        }
        if (d_path_L_or_null) PT_CUDA(cudaMemsetAsync(d_path_L_or_null, 0, n_paths * 12, st));
        if (o.d_path_sig) PT_CUDA(cudaMemsetAsync(o.d_path_sig, 0, n_paths * 4, st));
    } else if (o.mode == PT_MODE_MEGAKERNEL) {
        float* outL = d_path_L_or_null;
        if (!outL && (spp > 1 || accum)) {
            PT_TRY(sc->pathL.ensure(n_paths * 12));
            outL = sc->pathL.as<float>();
        }
        size_t ev = 0;
        PT_TRY(sc->ev_begin(ST_MEGA, st, ev));
        if (o.flags & PT_FLAG_MK_STATIC) {
            pt::Launch l = launch_for(sc, pt::K_MEGA, o.block_size, 128, st, n_paths);
            PT_CUDA(pt::launch_megakernel(l, sc->view(), dc, p, n_paths, outL, img, o.d_path_sig, sc->rays()));
        } else {
            pt::Launch l = launch_for(sc, sc->instanced ? pt::K_MEGA_REGEN_INST
                                                        : short_stack_kernel(sc, pt::K_MEGA_REGEN, p.short_stack),
                                      o.block_size ? std::min<uint32_t>(o.block_size, 128) : 128, 128,
                                      st, n_paths);
            PT_CUDA(pt::launch_megakernel_regen(l, sc->view(), dc, p, n_paths, outL, img, o.d_path_sig, sc->rays(),
                                                sc->next_path()));
        }
        PT_TRY(sc->ev_end(ev, st));
        sc->launches += 1;
        if (outL) {
            sc->launches += 1;
            PT_TRY(sc->ev_begin(ST_REDUCE, st, ev));
            if (accum)
                PT_CUDA(pt::launch_accumulate(simple_launch(sc, st, n_pixels), outL, 3, 0, n_pixels, spp, accum, count, img));
            else
                PT_CUDA(pt::launch_reduce(simple_launch(sc, st, n_pixels), outL, 3, 0, n_pixels, spp, img));
            PT_TRY(sc->ev_end(ev, st));
        }
    } else {
        PT_TRY(run_wavefront(sc, dc, p, o, n_paths, img, d_path_L_or_null, o.d_path_sig, st, accum, count));
    }
    PT_TRY(sc->ev_flush(st));
    if (host_out) {
        PT_CUDA(cudaMemcpyAsync(d_out_rgb, img, n_pixels * 12, cudaMemcpyDeviceToHost, st));
        PT_CUDA(cudaStreamSynchronize(st));
    }
    return PT_OK;
}

}  // namespace

namespace {

// Material table and environment checks shared by both scene constructors.
pt_status check_materials(const pt_material* mats, uint32_t n_mats, const float* env_radiance) {
    for (uint32_t m = 0; m < n_mats; ++m) {
        const pt_material& M = mats[m];
        if (M.type > PT_MAT_DIELECTRIC) return fail(PT_ERR_INVALID_ARG, "material %u: unknown type %u", m, M.type);
        if (!finite3(M.albedo) || M.albedo[0] < 0 || M.albedo[1] < 0 || M.albedo[2] < 0)
            return fail(PT_ERR_INVALID_ARG, "material %u: albedo must be finite and >= 0", m);
        if (!std::isfinite(M.emission) || M.emission < 0) return fail(PT_ERR_INVALID_ARG, "material %u: emission must be finite and >= 0", m);
        if (!std::isfinite(M.roughness) || M.roughness < 0) return fail(PT_ERR_INVALID_ARG, "material %u: roughness must be finite and >= 0", m);
        if (!std::isfinite(M.ior) || !(M.ior > 0)) return fail(PT_ERR_INVALID_ARG, "material %u: ior must be finite and > 0", m);
    }
    if (env_radiance && (!finite3(env_radiance) || env_radiance[0] < 0 || env_radiance[1] < 0 || env_radiance[2] < 0))
        return fail(PT_ERR_INVALID_ARG, "env_radiance must be finite and >= 0");
    return PT_OK;
}

}  // namespace

extern "C" {

const char* pt_status_string(pt_status s) {
    switch (s) {
        case PT_OK: return "ok";
        case PT_ERR_INVALID_ARG: return "invalid argument";
        case PT_ERR_OOM: return "out of memory";
        case PT_ERR_CUDA: return "CUDA error";
        case PT_ERR_QUEUE_OVERFLOW: return "queue overflow";
        case PT_ERR_TRAVERSAL_LIMIT: return "traversal limit exceeded";
        case PT_ERR_TIMEOUT: return "timeout";
        case PT_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* pt_last_error(void) { return g_err.c_str(); }

pt_status pt_scene_create(const float* verts, uint32_t n_verts, const uint32_t* tris, uint32_t n_tris,
                          const uint32_t* tri_material, const pt_material* mats, uint32_t n_mats,
                          const float env_radiance[3], void* cuda_stream, pt_scene** out) {
    if (!out) return fail(PT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_tris > 0 && (!verts || !tris || !tri_material))
        return fail(PT_ERR_INVALID_ARG, "verts, tris and tri_material are required when n_tris > 0");
    if (n_mats > 0 && !mats) return fail(PT_ERR_INVALID_ARG, "mats is NULL");
    if (n_tris > 0 && n_mats == 0) return fail(PT_ERR_INVALID_ARG, "n_mats must be > 0 when n_tris > 0");
    if (n_mats >= (1u << 28)) return fail(PT_ERR_INVALID_ARG, "n_mats must be < 2^28");
    if (n_tris >= (1u << 28)) return fail(PT_ERR_INVALID_ARG, "n_tris must be < 2^28");
    for (uint64_t i = 0; i < 3ull * n_verts; ++i)
        if (!std::isfinite(verts[i])) return fail(PT_ERR_INVALID_ARG, "vertex %llu is not finite", (unsigned long long)(i / 3));
    for (uint64_t i = 0; i < 3ull * n_tris; ++i)
        if (tris[i] >= n_verts) return fail(PT_ERR_INVALID_ARG, "triangle %llu references vertex %u >= n_verts", (unsigned long long)(i / 3), tris[i]);
    for (uint32_t i = 0; i < n_tris; ++i)
        if (tri_material[i] >= n_mats) return fail(PT_ERR_INVALID_ARG, "triangle %u has material %u >= n_mats", i, tri_material[i]);
    PT_TRY(check_materials(mats, n_mats, env_radiance));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    pt_scene* sc = new (std::nothrow) pt_scene();
    if (!sc) return fail(PT_ERR_OOM, "host allocation failed");
    auto bail = [&](pt_status s) {
        delete sc;
        return s;
    };
    if (cudaGetDevice(&sc->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PT_ERR_CUDA, "no CUDA device"));
    }
    sc->n_tris = n_tris;
    sc->n_mats = n_mats;
    if (env_radiance)
        for (int k = 0; k < 3; ++k) sc->env[k] = env_radiance[k];

    pt::BvhOut bvh;
    std::string err;
    if (!pt::build_bvh(verts, tris, n_tris, bvh, err)) return bail(fail(PT_ERR_INVALID_ARG, "BVH build: %s", err.c_str()));
    sc->n_nodes = bvh.n_internal;

    // triangle records in leaf order: (v0 | prim) (e1 | material) (e2 | is_light)
    std::vector<float> trec(12 * (size_t)n_tris);
    auto bits = [](uint32_t u) {
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    for (uint32_t k = 0; k < n_tris; ++k) {
        uint32_t i = bvh.order[k];
        const float* a = verts + 3 * (size_t)tris[3 * (size_t)i];
        const float* b = verts + 3 * (size_t)tris[3 * (size_t)i + 1];
        const float* c = verts + 3 * (size_t)tris[3 * (size_t)i + 2];
        float* r = &trec[12 * (size_t)k];
        uint32_t m = tri_material[i];
        r[0] = a[0]; r[1] = a[1]; r[2] = a[2]; r[3] = bits(i);
        r[4] = b[0] - a[0]; r[5] = b[1] - a[1]; r[6] = b[2] - a[2]; r[7] = bits(m);
        r[8] = c[0] - a[0]; r[9] = c[1] - a[1]; r[10] = c[2] - a[2];
        r[11] = bits(mats[m].emission > 0.f ? 1u : 0u);
    }
    // light list: triangles whose material emits at creation, ascending id; pmf proportional to area
    std::vector<float> lrec;
    std::vector<double> areas;
    for (uint32_t i = 0; i < n_tris; ++i) {
        uint32_t m = tri_material[i];
        if (!(mats[m].emission > 0.f)) continue;
        const float* a = verts + 3 * (size_t)tris[3 * (size_t)i];
        const float* b = verts + 3 * (size_t)tris[3 * (size_t)i + 1];
        const float* c = verts + 3 * (size_t)tris[3 * (size_t)i + 2];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = (double)b[k] - a[k];
            e2[k] = (double)c[k] - a[k];
        }
        double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
        areas.push_back(0.5 * std::sqrt(cx * cx + cy * cy + cz * cz));
        float rec[12] = {a[0], a[1], a[2], bits(m), b[0], b[1], b[2], 0.f, c[0], c[1], c[2], 0.f};
        lrec.insert(lrec.end(), rec, rec + 12);
    }
    sc->n_lights = areas.size();
    std::vector<float> cdf(std::max<size_t>(areas.size(), 1), 0.f);
    double total = 0;
    for (double a : areas) total += a;
    double acc = 0;
    for (size_t j = 0; j < areas.size(); ++j) {
        acc += areas[j];
        cdf[j] = total > 0 ? (float)(acc / total) : 0.f;
    }
    if (!areas.empty() && total > 0) cdf.back() = 1.0f;
    sc->light_area = (float)total;

    std::vector<pt::DevMat> dm(std::max<uint32_t>(n_mats, 1));
    for (uint32_t m = 0; m < n_mats; ++m) {
        const pt_material& M = mats[m];
        dm[m] = pt::DevMat{M.type, M.albedo[0], M.albedo[1], M.albedo[2], M.emission, M.roughness, M.ior, 0u};
    }

    pt_status s;
    if ((s = sc->nodes.ensure(bvh.nodes.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->tris.ensure(std::max<size_t>(trec.size() * 4, 48))) != PT_OK) return bail(s);
    if ((s = sc->mats.ensure(dm.size() * sizeof(pt::DevMat))) != PT_OK) return bail(s);
    if ((s = sc->lights.ensure(std::max<size_t>(lrec.size() * 4, 48))) != PT_OK) return bail(s);
    if ((s = sc->cdf.ensure(cdf.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->status.ensure(256)) != PT_OK) return bail(s);
    if ((s = sc->ensure_counters()) != PT_OK) return bail(s);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->nodes.p, bvh.nodes.data(), bvh.nodes.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !trec.empty()) e = cudaMemcpyAsync(sc->tris.p, trec.data(), trec.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && trec.empty()) e = cudaMemsetAsync(sc->tris.p, 0, 48, st);   // the never-hit record
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->mats.p, dm.data(), dm.size() * sizeof(pt::DevMat), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !lrec.empty()) e = cudaMemcpyAsync(sc->lights.p, lrec.data(), lrec.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->cdf.p, cdf.data(), cdf.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->status.p, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->counters.p, 0, sc->counters.bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PT_ERR_CUDA, "scene upload: %s", cudaGetErrorString(e)));
    }
    sc->last_stream = st;
    *out = sc;
    return PT_OK;
}

// Two-level scene (the paper's TLAS/BLAS structure, Sec. 2.3): one binned-SAH BVH per mesh over its
// object-space triangles, a top-level BVH over the instances' world boxes, and a light list of
// the instances' emissive triangles placed in the world.  Triangle ids run over the instances in
// order, each mesh's triangles in order.
pt_status pt_scene_create_instanced(uint32_t n_meshes, const float* const* verts, const uint32_t* n_verts,
                                    const uint32_t* const* tris, const uint32_t* n_tris,
                                    const uint32_t* const* tri_material, const pt_instance* instances,
                                    uint32_t n_instances, const pt_material* mats, uint32_t n_mats,
                                    const float env_radiance[3], void* cuda_stream, pt_scene** out) {
    if (!out) return fail(PT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_meshes == 0 || !verts || !n_verts || !tris || !n_tris || !tri_material)
        return fail(PT_ERR_INVALID_ARG, "at least one mesh with its arrays is required");
    if (n_instances == 0 || !instances) return fail(PT_ERR_INVALID_ARG, "at least one instance is required");
    if (n_mats == 0 || !mats) return fail(PT_ERR_INVALID_ARG, "materials are required");
    if (n_mats >= (1u << 28)) return fail(PT_ERR_INVALID_ARG, "n_mats must be < 2^28");
    uint64_t total_records = 0;
    for (uint32_t m = 0; m < n_meshes; ++m) {
        if (n_tris[m] == 0) return fail(PT_ERR_INVALID_ARG, "mesh %u has no triangles", m);
        if (!verts[m] || !tris[m] || !tri_material[m]) return fail(PT_ERR_INVALID_ARG, "mesh %u: NULL array", m);
        for (uint64_t i = 0; i < 3ull * n_verts[m]; ++i)
            if (!std::isfinite(verts[m][i])) return fail(PT_ERR_INVALID_ARG, "mesh %u: vertex %llu is not finite", m, (unsigned long long)(i / 3));
        for (uint64_t i = 0; i < 3ull * n_tris[m]; ++i)
            if (tris[m][i] >= n_verts[m]) return fail(PT_ERR_INVALID_ARG, "mesh %u: triangle %llu references vertex %u >= n_verts", m, (unsigned long long)(i / 3), tris[m][i]);
        for (uint32_t i = 0; i < n_tris[m]; ++i)
            if (tri_material[m][i] >= n_mats) return fail(PT_ERR_INVALID_ARG, "mesh %u: triangle %u has material %u >= n_mats", m, i, tri_material[m][i]);
        total_records += n_tris[m];
    }
    if (total_records >= (1u << 28)) return fail(PT_ERR_INVALID_ARG, "the meshes hold >= 2^28 triangles");
    PT_TRY(check_materials(mats, n_mats, env_radiance));
    // instance transforms and their inverses (FP64)
    std::vector<double> inv(12 * (size_t)n_instances);
    uint64_t total_prims = 0;
    for (uint32_t i = 0; i < n_instances; ++i) {
        const pt_instance& I = instances[i];
        if (I.mesh >= n_meshes) return fail(PT_ERR_INVALID_ARG, "instance %u: mesh %u >= n_meshes", i, I.mesh);
        if (I.material != PT_NO_MATERIAL && I.material >= n_mats)
            return fail(PT_ERR_INVALID_ARG, "instance %u: material %u >= n_mats", i, I.material);
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(I.xform[k])) return fail(PT_ERR_INVALID_ARG, "instance %u: transform is not finite", i);
        const double r[9] = {I.xform[0], I.xform[1], I.xform[2], I.xform[4], I.xform[5], I.xform[6],
                             I.xform[8], I.xform[9], I.xform[10]};
        const double c00 = r[4] * r[8] - r[5] * r[7], c01 = r[5] * r[6] - r[3] * r[8], c02 = r[3] * r[7] - r[4] * r[6];
        const double det = r[0] * c00 + r[1] * c01 + r[2] * c02;
        double scale = 0;
        for (double v : r) scale = std::max(scale, std::fabs(v));
        if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) return fail(PT_ERR_INVALID_ARG, "instance %u: transform is singular", i);
        // inverse of the 3x3 part by cofactors; b = -A t
        double A[9] = {c00 / det, (r[2] * r[7] - r[1] * r[8]) / det, (r[1] * r[5] - r[2] * r[4]) / det,
                       c01 / det, (r[0] * r[8] - r[2] * r[6]) / det, (r[2] * r[3] - r[0] * r[5]) / det,
                       c02 / det, (r[1] * r[6] - r[0] * r[7]) / det, (r[0] * r[4] - r[1] * r[3]) / det};
        const double t[3] = {I.xform[3], I.xform[7], I.xform[11]};
        for (int row = 0; row < 3; ++row) {
            double* o = &inv[12 * (size_t)i + 4 * row];
            o[0] = A[3 * row];
            o[1] = A[3 * row + 1];
            o[2] = A[3 * row + 2];
            o[3] = -(A[3 * row] * t[0] + A[3 * row + 1] * t[1] + A[3 * row + 2] * t[2]);
        }
        total_prims += n_tris[I.mesh];
    }
    if (total_prims >= 0xFFFFFFFFull) return fail(PT_ERR_INVALID_ARG, "the instances hold >= 2^32 - 1 triangles");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    pt_scene* sc = new (std::nothrow) pt_scene();
    if (!sc) return fail(PT_ERR_OOM, "host allocation failed");
    auto bail = [&](pt_status s) {
        delete sc;
        return s;
    };
    if (cudaGetDevice(&sc->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PT_ERR_CUDA, "no CUDA device"));
    }
    sc->instanced = true;
    sc->n_tris = total_prims;
    sc->n_mats = n_mats;
    if (env_radiance)
        for (int k = 0; k < 3; ++k) sc->env[k] = env_radiance[k];
    auto bits = [](uint32_t u) {
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    auto ubits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return u;
    };
    // bottom level: one BVH per mesh, nodes and triangle records concatenated (refs relocated)
    std::vector<float> nodes, trec;
    std::vector<uint32_t> node_base(n_meshes), rec_base(n_meshes);
    for (uint32_t m = 0; m < n_meshes; ++m) {
        pt::BvhOut bvh;
        std::string err;
        if (!pt::build_bvh(verts[m], tris[m], n_tris[m], bvh, err))
            return bail(fail(PT_ERR_INVALID_ARG, "mesh %u: BVH build: %s", m, err.c_str()));
        node_base[m] = (uint32_t)(nodes.size() / 16);
        rec_base[m] = (uint32_t)(trec.size() / 12);
        const uint32_t nb = node_base[m], rb = rec_base[m];
        for (size_t n = 0; n < bvh.nodes.size() / 16; ++n) {
            float f[16];
            std::memcpy(f, &bvh.nodes[16 * n], sizeof f);
            for (int c = 12; c < 14; ++c) {
                uint32_t ref = ubits(f[c]);
                if (ref & 0x80000000u) {
                    const uint32_t first = (ref & 0x7FFFFFFFu) >> 3, cnt = ref & 7u;
                    ref = 0x80000000u | ((first + rb) << 3) | cnt;
                } else {
                    ref += nb;
                }
                f[c] = bits(ref);
            }
            nodes.insert(nodes.end(), f, f + 16);
        }
        for (uint32_t k = 0; k < n_tris[m]; ++k) {
            const uint32_t i = bvh.order[k];
            const float* pa = verts[m] + 3 * (size_t)tris[m][3 * (size_t)i];
            const float* pb = verts[m] + 3 * (size_t)tris[m][3 * (size_t)i + 1];
            const float* pc = verts[m] + 3 * (size_t)tris[m][3 * (size_t)i + 2];
            const uint32_t mat = tri_material[m][i];
            const float r[12] = {pa[0], pa[1], pa[2], bits(i), pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2], bits(mat),
                                 pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2], bits(mats[mat].emission > 0.f ? 1u : 0u)};
            trec.insert(trec.end(), r, r + 12);
        }
    }
    // top level: the instances' world boxes -- the bounds of the mesh's vertices placed in the world
    // (tighter than the placed corners of the object box when the instance rotates), padded a few
    // ulps outward -- built as degenerate triangles (lo, hi, hi) so the same builder applies
    std::vector<std::vector<uint32_t>> used(n_meshes);       // vertices referenced by each mesh
    for (uint32_t m = 0; m < n_meshes; ++m) {
        std::vector<char> mark(n_verts[m], 0);
        for (uint64_t k = 0; k < 3ull * n_tris[m]; ++k) mark[tris[m][k]] = 1;
        for (uint32_t v = 0; v < n_verts[m]; ++v)
            if (mark[v]) used[m].push_back(v);
    }
    std::vector<float> ibox(6 * (size_t)n_instances);
    std::vector<uint32_t> itri(3 * (size_t)n_instances);
    for (uint32_t i = 0; i < n_instances; ++i) {
        const pt_instance& I = instances[i];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (uint32_t v : used[I.mesh]) {
            const float* p = verts[I.mesh] + 3 * (size_t)v;
            for (int r = 0; r < 3; ++r) {
                const double w = I.xform[4 * r] * (double)p[0] + I.xform[4 * r + 1] * (double)p[1] +
                                 I.xform[4 * r + 2] * (double)p[2] + I.xform[4 * r + 3];
                lo[r] = std::min(lo[r], w);
                hi[r] = std::max(hi[r], w);
            }
        }
        double ext = 0;
        for (int r = 0; r < 3; ++r) ext = std::max(ext, std::max(std::fabs(lo[r]), std::fabs(hi[r])));
        const double pad = 1e-6 * ext + 1e-30;
        for (int r = 0; r < 3; ++r) {
            ibox[6 * (size_t)i + r] = std::nextafter((float)(lo[r] - pad), -INFINITY);
            ibox[6 * (size_t)i + 3 + r] = std::nextafter((float)(hi[r] + pad), INFINITY);
        }
        itri[3 * (size_t)i] = 2 * i;
        itri[3 * (size_t)i + 1] = 2 * i + 1;
        itri[3 * (size_t)i + 2] = 2 * i + 1;
    }
    pt::BvhOut top;
    std::string err;
    if (!pt::build_bvh(ibox.data(), itri.data(), n_instances, top, err, 1))
        return bail(fail(PT_ERR_INVALID_ARG, "top-level BVH build: %s", err.c_str()));
    std::vector<uint32_t> prim_base(n_instances);
    {
        uint64_t acc = 0;
        for (uint32_t i = 0; i < n_instances; ++i) {
            prim_base[i] = (uint32_t)acc;
            acc += n_tris[instances[i].mesh];
        }
    }
    // instance records in top-level leaf order, 128 bytes: i0..i2 world-to-object rows (A | b),
    // i3 = (mesh root node, first triangle id, material word, -), i4..i6 object-to-world rows of R;
    // the first 64 bytes are all that taking a ray into the instance reads
    std::vector<float> irec(32 * (size_t)n_instances, 0.f);
    for (uint32_t k = 0; k < n_instances; ++k) {
        const uint32_t i = top.order[k];
        const pt_instance& I = instances[i];
        float* r = &irec[32 * (size_t)k];
        for (int q = 0; q < 12; ++q) r[q] = (float)inv[12 * (size_t)i + q];
        uint32_t mw = 0;
        if (I.material != PT_NO_MATERIAL) mw = (I.material + 1u) | (mats[I.material].emission > 0.f ? 0x80000000u : 0u);
        r[12] = bits(node_base[I.mesh]);
        r[13] = bits(prim_base[i]);
        r[14] = bits(mw);
        for (int row = 0; row < 3; ++row)
            for (int c = 0; c < 3; ++c) r[16 + 4 * row + c] = I.xform[4 * row + c];
    }
    // lights: every instance's emissive triangles in the world, ascending triangle id
    std::vector<float> lrec;
    std::vector<double> areas;
    for (uint32_t i = 0; i < n_instances; ++i) {
        const pt_instance& I = instances[i];
        const uint32_t m = I.mesh;
        for (uint32_t j = 0; j < n_tris[m]; ++j) {
            const uint32_t mat = I.material != PT_NO_MATERIAL ? I.material : tri_material[m][j];
            if (!(mats[mat].emission > 0.f)) continue;
            double w[3][3];
            for (int v = 0; v < 3; ++v) {
                const float* p = verts[m] + 3 * (size_t)tris[m][3 * (size_t)j + v];
                for (int r = 0; r < 3; ++r)
                    w[v][r] = I.xform[4 * r] * (double)p[0] + I.xform[4 * r + 1] * (double)p[1] +
                              I.xform[4 * r + 2] * (double)p[2] + I.xform[4 * r + 3];
            }
            double e1[3], e2[3];
            for (int r = 0; r < 3; ++r) {
                e1[r] = w[1][r] - w[0][r];
                e2[r] = w[2][r] - w[0][r];
            }
            const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                         cz = e1[0] * e2[1] - e1[1] * e2[0];
            areas.push_back(0.5 * std::sqrt(cx * cx + cy * cy + cz * cz));
            const float rec[12] = {(float)w[0][0], (float)w[0][1], (float)w[0][2], bits(mat),
                                   (float)w[1][0], (float)w[1][1], (float)w[1][2], 0.f,
                                   (float)w[2][0], (float)w[2][1], (float)w[2][2], 0.f};
            lrec.insert(lrec.end(), rec, rec + 12);
        }
    }
    sc->n_lights = areas.size();
    std::vector<float> cdf(std::max<size_t>(areas.size(), 1), 0.f);
    double total = 0;
    for (double x : areas) total += x;
    double acc = 0;
    for (size_t j = 0; j < areas.size(); ++j) {
        acc += areas[j];
        cdf[j] = total > 0 ? (float)(acc / total) : 0.f;
    }
    if (!areas.empty() && total > 0) cdf.back() = 1.0f;
    sc->light_area = (float)total;
    sc->n_nodes = nodes.size() / 16 + top.nodes.size() / 16;
    std::vector<pt::DevMat> dm(n_mats);
    for (uint32_t m = 0; m < n_mats; ++m) {
        const pt_material& M = mats[m];
        dm[m] = pt::DevMat{M.type, M.albedo[0], M.albedo[1], M.albedo[2], M.emission, M.roughness, M.ior, 0u};
    }
    pt_status s;
    if ((s = sc->nodes.ensure(nodes.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->tris.ensure(trec.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->tlas.ensure(top.nodes.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->inst.ensure(irec.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->mats.ensure(dm.size() * sizeof(pt::DevMat))) != PT_OK) return bail(s);
    if ((s = sc->lights.ensure(std::max<size_t>(lrec.size() * 4, 48))) != PT_OK) return bail(s);
    if ((s = sc->cdf.ensure(cdf.size() * 4)) != PT_OK) return bail(s);
    if ((s = sc->status.ensure(256)) != PT_OK) return bail(s);
    if ((s = sc->ensure_counters()) != PT_OK) return bail(s);
    cudaError_t e = cudaMemcpyAsync(sc->nodes.p, nodes.data(), nodes.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->tris.p, trec.data(), trec.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->tlas.p, top.nodes.data(), top.nodes.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->inst.p, irec.data(), irec.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->mats.p, dm.data(), dm.size() * sizeof(pt::DevMat), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !lrec.empty()) e = cudaMemcpyAsync(sc->lights.p, lrec.data(), lrec.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->cdf.p, cdf.data(), cdf.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->status.p, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->counters.p, 0, sc->counters.bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PT_ERR_CUDA, "scene upload: %s", cudaGetErrorString(e)));
    }
    sc->last_stream = st;
    *out = sc;
    return PT_OK;
}

void pt_scene_destroy(pt_scene* scene) {
    if (!scene) return;
    if (scene->last_stream) cudaStreamSynchronize(scene->last_stream);
    else cudaDeviceSynchronize();
    cudaGetLastError();
    delete scene;
}

pt_status pt_scene_set_materials(pt_scene* sc, const float* d_albedo, const float* d_emission, void* stream) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if ((d_albedo && !is_device_ptr(d_albedo)) || (d_emission && !is_device_ptr(d_emission)))
        return fail(PT_ERR_INVALID_ARG, "material arrays must be device pointers");
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    PT_CUDA(pt::launch_set_materials(static_cast<cudaStream_t>(stream), sc->mats.as<pt::DevMat>(), sc->n_mats, d_albedo,
                                     d_emission));
    return PT_OK;
}

pt_status pt_scene_info(const pt_scene* sc, uint64_t* n_tris, uint64_t* n_nodes, uint64_t* n_lights, float* light_area,
                        uint64_t* device_bytes) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if (n_tris) *n_tris = sc->n_tris;
    if (n_nodes) *n_nodes = sc->n_nodes;
    if (n_lights) *n_lights = sc->n_lights;
    if (light_area) *light_area = sc->light_area;
    if (device_bytes)
        *device_bytes = sc->nodes.bytes + sc->tris.bytes + sc->tlas.bytes + sc->inst.bytes + sc->mats.bytes +
                        sc->lights.bytes + sc->cdf.bytes + sc->wf.bytes + sc->pathL.bytes + sc->img_stage.bytes +
                        sc->grad_stage.bytes + sc->counters.bytes + sc->adj.bytes;
    return PT_OK;
}

pt_status pt_render(pt_scene* sc, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                    const pt_render_opts* opts, float* d_out_rgb, float* d_path_L_or_null, void* stream) {
    if (!d_out_rgb) return fail(PT_ERR_INVALID_ARG, "output image is NULL");
    return render_impl(sc, cam, spp, max_depth, seed, opts, d_out_rgb, d_path_L_or_null, stream, 0, nullptr);
}

pt_status pt_render_progressive(pt_scene* sc, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                                uint32_t sample_offset, const pt_render_opts* opts, float* d_accum_rgb,
                                float* d_out_rgb_or_null, void* stream) {
    if (!d_accum_rgb) return fail(PT_ERR_INVALID_ARG, "d_accum_rgb is NULL");
    return render_impl(sc, cam, spp, max_depth, seed, opts, d_out_rgb_or_null, nullptr, stream, sample_offset,
                       d_accum_rgb);
}

pt_status pt_render_backward(pt_scene* sc, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                             const pt_render_opts* opts, const float* d_grad_rgb, float* d_grad_albedo,
                             float* d_grad_emission, void* stream) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if (!d_grad_rgb || !d_grad_albedo || !d_grad_emission)
        return fail(PT_ERR_INVALID_ARG, "gradient pointers must be non-NULL");
    if (spp == 0) return fail(PT_ERR_INVALID_ARG, "spp must be >= 1");
    if (max_depth > 32) return fail(PT_ERR_UNSUPPORTED, "backward supports max_depth <= 32");
    if (!is_device_ptr(d_grad_albedo) || !is_device_ptr(d_grad_emission))
        return fail(PT_ERR_INVALID_ARG, "d_grad_albedo and d_grad_emission must be device pointers");
    pt_render_opts o = opts ? *opts : default_opts();
    PT_TRY(check_opts(o));
    pt::DevCamera dc;
    PT_TRY(make_camera(cam, dc));
    const uint64_t n_pixels = (uint64_t)cam->width * cam->height;
    const uint64_t n_paths = n_pixels * spp;
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float* grad = d_grad_rgb;
    if (!is_device_ptr(d_grad_rgb)) {
        PT_TRY(sc->grad_stage.ensure(n_pixels * 12));
        PT_CUDA(cudaMemcpyAsync(sc->grad_stage.p, d_grad_rgb, n_pixels * 12, cudaMemcpyHostToDevice, st));
        grad = sc->grad_stage.as<float>();
    }
    sc->ev_reset((o.flags & PT_FLAG_PROFILE) != 0);
    sc->last_stream = st;
    sc->last_mode = 2;
    sc->last_paths = n_paths;
    sc->launches = 0;
    PT_CUDA(cudaMemsetAsync(sc->counters.p, 0, sc->counters.bytes, st));
    PT_CUDA(cudaMemsetAsync(sc->status.p, 0, 4, st));
    if (max_depth == 0 || sc->n_mats == 0) return PT_OK;
    pt::RenderParams p;
    p.seed = seed;
    p.path_begin = 0;
    p.spp = spp;
    p.max_depth = max_depth;
    p.rr_start = o.rr_start;
    p.rr_fixed = o.rr_fixed;
    p.sampler = (o.flags & PT_FLAG_HALTON) ? pt::SAMPLER_HALTON_ID : 0u;
    p.mis = (o.flags & PT_FLAG_MIS) ? 1u : 0u;
    size_t ev = 0;
    PT_TRY(sc->ev_begin(ST_ADJOINT, st, ev));
    if (o.mode == PT_MODE_MEGAKERNEL) {
        pt::Launch l = launch_for(sc, pt::K_ADJOINT, o.block_size, 128, st, n_paths);
        // the counters were zeroed above; the regenerating megakernel's path counter is free here
        PT_CUDA(pt::launch_adjoint(l, sc->view(), dc, p, n_paths, grad, d_grad_albedo, d_grad_emission, max_depth,
                                   sc->next_path()));
        sc->launches += 1;
    } else {
        // wavefront replay: the forward stages with record-writing shading, then one reverse pass per wave
        const uint64_t per_path = 180 + 64ull * max_depth;
        uint64_t cap = std::min<uint64_t>(n_paths, (8ull << 30) / per_path);
        cap = std::max<uint64_t>(cap - cap % spp, spp);
        if (cap >= (1ull << 32)) cap = ((1ull << 32) - (1ull << 20)) / spp * spp;
        PT_TRY(sc->ensure_wf(cap));
        const size_t rec_bytes = align256(cap * max_depth * 64);
        PT_TRY(sc->adj.ensure(rec_bytes + align256(cap * 4)));
        pt::WfBuffers w = sc->wfb;
        w.counts = sc->counts();
        w.hist = sc->hist();
        w.sig = nullptr;
        w.capacity = (uint32_t)cap;
        pt::AdjBuffers ab;
        ab.rec = sc->adj.as<float4>();
        ab.pend = reinterpret_cast<uint32_t*>(sc->adj.as<char>() + rec_bytes);
        const pt::DevScene ds = sc->view();
        for (uint64_t w0 = 0; w0 < n_paths; w0 += cap) {
            const uint32_t n = (uint32_t)std::min<uint64_t>(cap, n_paths - w0);
            pt::RenderParams pw = p;
            pw.path_begin = w0;
            size_t e2 = 0;
            PT_TRY(sc->ev_begin(ST_RAYGEN, st, e2));
            PT_CUDA(pt::launch_raygen(simple_launch(sc, st, n), dc, pw, n, w));
            PT_TRY(sc->ev_end(e2, st));
            // fused as the forward wavefront: each bounce's extend launch also walks the shadow rays of
            // the previous bounce (marking their records), unless the separate order is asked for
            const bool fused = !(o.flags & PT_FLAG_SEPARATE_SHADOW);
            for (uint32_t b = 0; b < max_depth; ++b) {
                const int in = (int)(b & 1u);
                PT_TRY(sc->ev_begin(ST_EXTEND, st, e2));
                if (fused && b > 0) {
                    pt::Launch lt = launch_for(sc, sc->instanced ? pt::K_TRACE_INST : pt::K_TRACE, o.block_size, 256,
                                               st, 2ull * n);
                    lt.pdl = kStagePdl;
                    PT_CUDA(pt::launch_trace_adj(lt, ds, pw, w, ab, in, b));
                } else {
                    pt::Launch le = launch_for(sc, pt::K_EXTEND, o.block_size, 256, st, n);
                    le.pdl = fused && kStagePdl;
                    PT_CUDA(pt::launch_extend(le, ds, w, in, pw));
                }
                PT_TRY(sc->ev_end(e2, st));
                PT_TRY(sc->ev_begin(ST_SHADE, st, e2));
                pt::Launch ls = launch_for(sc, pt::K_SHADE_ADJ, o.block_size, 256, st, n);
                ls.pdl = fused && kStagePdl;
                PT_CUDA(pt::launch_shade_adj(ls, ds, pw, w, ab, in, b));
                PT_TRY(sc->ev_end(e2, st));
                if (fused) {
                    PT_CUDA(pt::launch_prepare_fused(st, w, b, kStagePdl));
                    continue;
                }
                PT_TRY(sc->ev_begin(ST_SHADOW, st, e2));
                PT_CUDA(pt::launch_shadow_adj(launch_for(sc, pt::K_SHADOW_ADJ, o.block_size, 256, st, n), ds, pw, w, ab, b));
                PT_TRY(sc->ev_end(e2, st));
                PT_CUDA(pt::launch_prepare(st, w, b));
            }
            PT_TRY(sc->ev_begin(ST_REDUCE, st, e2));
            pt::Launch lr = simple_launch(sc, st, n);
            lr.pdl = fused && kStagePdl;
            PT_CUDA(pt::launch_adjoint_reverse(lr, ds, pw, w, ab, n, grad, d_grad_albedo, d_grad_emission));
            PT_TRY(sc->ev_end(e2, st));
            sc->launches += 2 + (fused ? 3 : 4) * max_depth;
        }
    }
    PT_TRY(sc->ev_end(ev, st));
    PT_TRY(sc->ev_flush(st));
    return PT_OK;
}

pt_status pt_trace_closest(pt_scene* sc, const float* d_rays, uint32_t n, float* d_t, int32_t* d_prim, void* stream) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if (n == 0) return PT_OK;
    if (!d_rays || !d_t || !d_prim) return fail(PT_ERR_INVALID_ARG, "NULL buffer");
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sc->last_stream = st;
    PT_CUDA(pt::launch_trace_closest(launch_for(sc, pt::K_EXTEND, 0, 256, st, n), sc->view(), d_rays, n, d_t, d_prim));
    return PT_OK;
}

pt_status pt_debug_rng(uint64_t seed, const uint32_t* px, const uint32_t* sm, const uint32_t* bo, const uint32_t* dm,
                       uint32_t n, float* out, void* stream) {
    if (n == 0) return PT_OK;
    if (!px || !sm || !bo || !dm || !out) return fail(PT_ERR_INVALID_ARG, "NULL buffer");
    pt::Launch l{1, 256, static_cast<cudaStream_t>(stream)};
    PT_CUDA(pt::launch_debug_rng(l, seed, px, sm, bo, dm, n, out));
    return PT_OK;
}

pt_status pt_debug_trace_paths(pt_scene* sc, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                               const pt_render_opts* opts, const uint64_t* d_path_ids, uint32_t n, uint32_t* d_events,
                               float* d_payload, uint32_t* d_n_events, float* d_path_L, void* stream) {
    if (!sc) return fail(PT_ERR_INVALID_ARG, "scene is NULL");
    if (spp == 0) return fail(PT_ERR_INVALID_ARG, "spp must be >= 1");
    if (max_depth > 64) return fail(PT_ERR_INVALID_ARG, "max_depth must be <= 64");
    if (n == 0) return PT_OK;
    if (!d_path_ids || !d_events || !d_payload || !d_n_events || !d_path_L) return fail(PT_ERR_INVALID_ARG, "NULL buffer");
    pt_render_opts o = opts ? *opts : default_opts();
    PT_TRY(check_opts(o));
    pt::DevCamera dc;
    PT_TRY(make_camera(cam, dc));
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sc->last_stream = st;
    pt::RenderParams p;
    p.seed = seed;
    p.path_begin = 0;
    p.spp = spp;
    p.max_depth = max_depth;
    p.rr_start = o.rr_start;
    p.rr_fixed = o.rr_fixed;
    p.sampler = (o.flags & PT_FLAG_HALTON) ? pt::SAMPLER_HALTON_ID : 0u;
    p.mis = (o.flags & PT_FLAG_MIS) ? 1u : 0u;
    PT_CUDA(pt::launch_debug_paths(st, sc->view(), dc, p, reinterpret_cast<const unsigned long long*>(d_path_ids), n,
                                   d_events, d_payload, d_n_events, d_path_L));
    return PT_OK;
}

pt_status pt_get_stats(pt_scene* sc, pt_stats* out) {
    if (!sc || !out) return fail(PT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(sc->mu);
    PT_TRY(set_device(sc));
    PT_CUDA(cudaStreamSynchronize(sc->last_stream));
    std::memset(out, 0, sizeof(*out));
    std::vector<unsigned long long> h(pt::kHistWords);
    uint32_t status = 0;
    PT_CUDA(cudaMemcpy(h.data(), sc->hist(), pt::kHistWords * 8, cudaMemcpyDeviceToHost));
    PT_CUDA(cudaMemcpy(&status, sc->status.p, 4, cudaMemcpyDeviceToHost));
    out->paths = sc->last_paths;
    out->launches_total = sc->launches;
    if (sc->last_mode != PT_MODE_WAVEFRONT) {
        out->extension_rays = h[128];
        out->shadow_rays = h[129];
    } else {
        for (int b = 0; b < 64; ++b) {
            out->extension_rays += h[b];
            out->shadow_rays += h[64 + b];
            out->active[b] = h[b];
            out->shadow_queued[b] = h[64 + b];
            if (h[b]) out->bounces = b + 1;
        }
    }
    out->nodes_closest = h[132];
    out->tris_closest = h[133];
    out->nodes_any = h[134];
    out->tris_any = h[135];
    for (int i = 0; i < 5; ++i) out->group_walks[i] = h[pt::kHistGroupWalks + i];
    out->status = status & pt::ST_TRAVERSAL ? PT_ERR_TRAVERSAL_LIMIT
                : status & pt::ST_QUEUE     ? PT_ERR_QUEUE_OVERFLOW
                : status & pt::ST_TIMEOUT   ? PT_ERR_TIMEOUT
                                            : PT_OK;
    if (sc->profiling) {
        float ms[ST_COUNT] = {};
        uint32_t n_ext = 0, n_shd = 0;
        for (size_t i = 0; i < sc->ev_used; ++i) {
            float t = 0.f;
            const auto& e = sc->events[i];
            if (e.a < 0 || e.b < 0) continue;      // a call that failed before the stage ended
            PT_CUDA(cudaEventElapsedTime(&t, sc->ev_pool[e.a], sc->ev_pool[e.b]));
            ms[sc->events[i].stage] += t;
            if (sc->events[i].stage == ST_EXTEND) ++n_ext;
            if (sc->events[i].stage == ST_SHADOW) ++n_shd;
        }
        out->ms_raygen = ms[ST_RAYGEN];
        out->ms_extend = ms[ST_EXTEND];
        out->ms_sort = ms[ST_SORT];
        out->ms_shade = ms[ST_SHADE];
        out->ms_shadow = ms[ST_SHADOW];
        out->ms_reduce = ms[ST_REDUCE];
        out->ms_megakernel = ms[ST_MEGA];
        out->ms_adjoint = ms[ST_ADJOINT];
        out->launches_extend = n_ext;
        out->launches_shadow = n_shd;
        for (float t : ms) out->ms_total += t;
    }
    return PT_OK;
}

pt_status pt_render_batch(pt_scene* const* scenes, const pt_camera* cams, const uint32_t* spp, uint32_t n,
                          uint32_t max_depth, uint64_t seed, const pt_render_opts* opts, float* const* d_out,
                          void* stream) {
    return batch_render(scenes, cams, spp, n, max_depth, seed, opts, d_out, stream);
}

pt_status pt_autotune_batch(pt_scene* const* scenes, const pt_camera* cams, const uint32_t* spp, uint32_t n,
                            uint32_t max_depth, uint64_t seed, const pt_render_opts* base, float* const* d_out,
                            void* stream, pt_render_opts* best, float* best_ms) {
    if (!best) return fail(PT_ERR_INVALID_ARG, "best is NULL");
    pt_render_opts o = base ? *base : default_opts();
    PT_TRY(check_opts(o));
    o.mode = PT_MODE_WAVEFRONT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t total = 0;
    if (!scenes || !cams || !spp || n == 0) return fail(PT_ERR_INVALID_ARG, "empty batch");
    for (uint32_t i = 0; i < n; ++i) total += (uint64_t)cams[i].width * cams[i].height * spp[i];
    cudaEvent_t e0, e1;
    PT_CUDA(cudaEventCreate(&e0));
    PT_CUDA(cudaEventCreate(&e1));
    auto time_it = [&](const pt_render_opts& c, float& ms) -> pt_status {
        PT_TRY(batch_render(scenes, cams, spp, n, max_depth, seed, &c, d_out, stream));   // warm-up, capture
        float best_t = 1e30f;
        for (int r = 0; r < 2; ++r) {
            PT_CUDA(cudaEventRecord(e0, st));
            PT_TRY(batch_render(scenes, cams, spp, n, max_depth, seed, &c, d_out, stream));
            PT_CUDA(cudaEventRecord(e1, st));
            PT_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            PT_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best_t = std::min(best_t, t);
        }
        ms = best_t;
        return PT_OK;
    };
    // coordinate descent: queue capacity, then block size, then sort granularity
    std::vector<uint64_t> caps;
    for (uint64_t c : {1ull << 21, 1ull << 22, 1ull << 23, 1ull << 24, 1ull << 25})
        if (c < total) caps.push_back(c);
    caps.push_back(std::min<uint64_t>(total, 1ull << 26));
    pt_render_opts cur = o;
    cur.sort_mode = PT_SORT_NONE;
    cur.block_size = 256;
    float cur_ms = 1e30f;
    pt_status s = PT_OK;
    for (uint64_t c : caps) {
        pt_render_opts t = cur;
        t.queue_capacity = c;
        float ms;
        if ((s = time_it(t, ms)) != PT_OK) break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur.queue_capacity = c;
        }
    }
    for (uint32_t bs : {128u}) {
        if (s != PT_OK) break;
        pt_render_opts t = cur;
        t.block_size = bs;
        float ms;
        if ((s = time_it(t, ms)) != PT_OK) break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur.block_size = bs;
        }
    }
    for (uint32_t sm : {(uint32_t)PT_SORT_TYPE, (uint32_t)PT_SORT_MATERIAL}) {
        if (s != PT_OK) break;
        pt_render_opts t = cur;
        t.sort_mode = sm;
        float ms;
        if ((s = time_it(t, ms)) != PT_OK) break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur.sort_mode = sm;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PT_OK) return s;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return PT_OK;
}

}  // extern "C"
