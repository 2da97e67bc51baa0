/*
 * pt.h -- C ABI of the GB300 path tracer (libpt.so).
 *
 * The library renders triangle scenes with the Monte Carlo light-transport estimator of
 * "Megakernel vs Wavefront GPU Path Tracing": Eq. 1 (light transport equation) estimated by
 * Eq. 2 (mean of f/p over samples) along paths whose throughput follows Eq. 3, with the forward
 * path-tracing loop of Sec. 2.2, the shadow-evaluation stage of Sec. 3 (next-event estimation)
 * and Russian roulette (Sec. 3.1).  It runs the estimator two ways (Sec. 2.2 / 2.3): a megakernel
 * (one thread traces one path to termination) and a wavefront pipeline (ray generation, extend
 * traversal, material-sorted shading, shadow traversal, accumulation) linked by device queues
 * with the two-slot active count of Sec. 3.1.  It also provides a path-replay adjoint (gradients
 * of an image loss with respect to per-material albedo and emission) and batched rendering of
 * many scenes in one persistent wavefront.
 *
 * Conventions for every entry point:
 *  - Pointers prefixed d_ are device pointers on the current CUDA device unless stated "host or
 *    device" (then the library detects host memory and stages it through its own device buffer).
 *    The caller owns them; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless stated otherwise; errors in arguments are reported
 *    synchronously by the return value, device-side faults (traversal step cap, queue overflow)
 *    are recorded in a device status word and reported by pt_get_stats.
 *  - Nothing throws; every failure returns a pt_status and sets a thread-local message
 *    (pt_last_error).
 *  - Images are row-major H x W x 3 float32 (linear RGB), row 0 at the top.  Path p = pixel * spp
 *    + sample, pixel = y * W + x.  Per-path buffers are N_p x 3 float32, N_p = W * H * spp.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PT_OK = 0,
    PT_ERR_INVALID_ARG = 1,     /* a pointer, size or option is out of range */
    PT_ERR_OOM = 2,             /* device or host allocation failed */
    PT_ERR_CUDA = 3,            /* a CUDA runtime call failed (message in pt_last_error) */
    PT_ERR_QUEUE_OVERFLOW = 4,  /* a wavefront queue append exceeded its capacity */
    PT_ERR_TRAVERSAL_LIMIT = 5, /* a BVH traversal exceeded its step cap or stack */
    PT_ERR_TIMEOUT = 6,         /* a bounded device wait gave up */
    PT_ERR_UNSUPPORTED = 7      /* valid but not supported (e.g. backward depth > 32) */
} pt_status;

/* Material models (Sec. 3: shading stage; the paper's layered OpenPBR model is reduced to these
 * three lobes).  Le = emission * (1, 1, 1), one-sided (front face by winding). */
enum { PT_MAT_LAMBERT = 0, PT_MAT_GGX = 1, PT_MAT_DIELECTRIC = 2 };

typedef struct {
    uint32_t type;      /* PT_MAT_* */
    float albedo[3];    /* Lambert albedo / GGX F0 (Schlick) / dielectric tint, each in [0, 1] */
    float emission;     /* scalar emitted radiance, >= 0; > 0 at creation puts the material's
                           triangles in the light list */
    float roughness;    /* GGX: alpha = max(roughness^2, 1e-4) */
    float ior;          /* dielectric index of refraction (> 0) */
    uint32_t flags;     /* reserved, 0 */
} pt_material;          /* 32 bytes */

/* Pinhole camera of the ray-generation stage (Sec. 2.3): ray through (x + u0, y + u1). */
typedef struct {
    float eye[3], target[3], up[3];
    float vfov_deg;     /* vertical field of view, (0, 180) */
    uint32_t width, height;
} pt_camera;

enum { PT_MODE_MEGAKERNEL = 0, PT_MODE_WAVEFRONT = 1 };
enum { PT_SORT_NONE = 0, PT_SORT_TYPE = 1, PT_SORT_MATERIAL = 2 };
enum {
    PT_FLAG_PROFILE = 1u,       /* time each stage with CUDA events on the launch stream; read the
                                   times with pt_get_stats after the stream completes */
    PT_FLAG_NO_GRAPH = 2u,      /* batched wavefront: launch the bounce loop directly, not as a CUDA graph */
    PT_FLAG_MK_STATIC = 4u,     /* megakernel: one thread per path, launched over all paths (the paper's
                                   layout) instead of the persistent kernel with path regeneration */
    PT_FLAG_HALTON = 8u,        /* pixel jitter from the Halton sequence in bases 2 and 3 over the pixel's
                                   sample index with a per-pixel Cranley-Patterson rotation (Sec. 2.3),
                                   in 24-bit fixed point; default: the path's PCG uniforms */
    PT_FLAG_MIS = 16u,          /* combine next-event estimation and BSDF-sampled hits on listed lights
                                   with the power heuristic (Veach 1997) instead of leaving those hits
                                   to NEE; the expectation is unchanged, the variance on glossy surfaces
                                   and large lights is lower.  Gradients follow (the weights do not
                                   depend on albedo or emission). */
    PT_FLAG_SHORT_STACK = 32u,  /* pt_render / pt_render_progressive on single-level scenes: the BVH walks
                                   of the extend and shadow stages, the megakernel and the hybrid
                                   continuation keep the top 8 entries of their traversal stacks in shared
                                   memory (per-warp short stacks, 64 bytes per thread), the rest in local
                                   memory.  Same hits and images; slower than the default local-memory
                                   stack on GB300, whose L1 already holds it.  Ignored elsewhere. */
    PT_FLAG_SEPARATE_SHADOW = 128u, /* wavefront (pt_render, pt_render_progressive, pt_render_backward's
                                   wavefront replay, pt_render_batch, pt_render_wavefront_static): run the
                                   shadow stage as its own launch after shading, as the paper's stage list
                                   orders it, instead of walking each bounce's shadow rays in the next
                                   bounce's extend launch.  Same image and gradients; the default fused
                                   order has one stage boundary fewer per bounce, and its trace launches
                                   give each ray a group of lanes when they hold few walks.  The hybrid
                                   continuation and PT_FLAG_SHORT_STACK always use the separate order. */
    PT_FLAG_COUNT_TRAVERSAL = 64u  /* pt_render / pt_render_progressive on single-level scenes without
                                   d_path_sig: the extend and shadow stages and the regenerating
                                   megakernel run instantiations that count the BVH nodes visited and the
                                   triangles tested by every walk (pt_stats nodes_* / tris_*); the
                                   production instantiations count nothing.  Same hits and images. */
};

typedef struct {
    uint32_t mode;              /* PT_MODE_* */
    uint32_t rr_start;          /* first bounce with Russian roulette (Sec. 3.1); >= max_depth: off */
    float rr_fixed;             /* > 0: fixed survival probability; 0: q = clamp(max(tp), .05, .95) */
    uint32_t sort_mode;         /* wavefront: PT_SORT_* key sort before shading */
    uint32_t block_size;        /* threads per block: 0 = default, else a multiple of 32 in [64, 256] */
    uint32_t flags;             /* PT_FLAG_* */
    uint64_t queue_capacity;    /* wavefront: paths per wave; 0 = all paths in one wave */
    uint32_t* d_path_sig;       /* optional device N_p u32: per-path branch signature (testing) */
    uint64_t hybrid_threshold;  /* wavefront (pt_render, pt_render_progressive): when at most this many
                                   paths of a wave are active entering a bounce, one persistent kernel
                                   finishes them all in registers (the megakernel's loop body) instead
                                   of running the remaining bounces as wavefront stages -- the hybrid of
                                   the paper's future work (Sec. 6.1).  Decided on the device, so the
                                   image is unchanged.  0 = off.  Ignored by the other entry points. */
} pt_render_opts;

typedef struct {
    uint64_t extension_rays;    /* closest-hit queries traced (device-counted) */
    uint64_t shadow_rays;       /* shadow (any-hit) queries traced */
    uint64_t paths;
    uint32_t bounces;           /* entries valid in active[] */
    uint32_t status;            /* device status word: 0 or a pt_status */
    uint64_t active[64];        /* wavefront: active paths entering each bounce (all waves) */
    /* PT_FLAG_PROFILE: total milliseconds per stage of the last profiled call, and launches
       (ms_megakernel includes the hybrid continuation kernel of a wavefront render).  A stage's
       interval runs from an event recorded before its first launch to the event that starts the
       next stage (or ends the call): consecutive stages share one event, and bookkeeping launches
       and launch gaps between two stages count toward the earlier one.  ms_adjoint spans the
       whole backward pass, which contains its replay's stages. */
    float ms_raygen, ms_extend, ms_sort, ms_shade, ms_shadow, ms_reduce, ms_megakernel, ms_adjoint;
    uint32_t launches_extend, launches_shadow, launches_total;
    float ms_total;
    /* PT_FLAG_COUNT_TRAVERSAL: internal BVH nodes visited and triangles tested by the closest-hit
       (extension) and any-hit (shadow) walks of the last call; 0 otherwise. */
    uint64_t nodes_closest, tris_closest, nodes_any, tris_any;
    uint64_t shadow_queued[64]; /* wavefront: shadow rays queued by shading at each bounce (all waves);
                                   entries [0, bounces) are valid and sum to shadow_rays */
    uint64_t group_walks[5];    /* walks (extension + shadow rays) that the fused trace stage traced
                                   with groups of 2, 4, 8, 16, 32 lanes per ray (launches with few
                                   walks, single-level scenes); the others took one lane each */
} pt_stats;

typedef struct pt_scene pt_scene;

/* Build a scene from host triangles (Sec. 3: scene data packed on the host into GPU-friendly
 * buffers and uploaded).  verts: host n_verts x 3 float; tris: host n_tris x 3 uint32 vertex
 * indices; tri_material: host n_tris uint32 (< n_mats); mats: host n_mats pt_material;
 * env_radiance: host 3 floats (radiance of rays that leave the scene).  Builds a binned-SAH BVH on
 * the host (multithreaded), packs 64-byte nodes and 48-byte triangle records, and uploads them
 * with cudaMemcpyAsync on `cuda_stream` (the call returns after the upload is enqueued and the host
 * staging is released, i.e. it synchronises that stream).  n_tris may be 0 (every ray misses).
 * Errors: PT_ERR_INVALID_ARG (NULL pointers with non-zero counts, index out of range, negative or
 * non-finite parameters, n_mats >= 2^28), PT_ERR_OOM, PT_ERR_CUDA.  The scene is owned by the library until
 * pt_scene_destroy. */
pt_status pt_scene_create(const float* verts, uint32_t n_verts, const uint32_t* tris, uint32_t n_tris,
                          const uint32_t* tri_material, const pt_material* mats, uint32_t n_mats,
                          const float env_radiance[3], void* cuda_stream, pt_scene** out);

/* One placed copy of a mesh in a two-level scene. */
#define PT_NO_MATERIAL 0xFFFFFFFFu
typedef struct {
    float xform[12];            /* object-to-world affine transform, row-major 3 x 4 [R | t]: world = R v + t
                                   (R invertible; any rotation, scale or shear) */
    uint32_t mesh;              /* index of the mesh */
    uint32_t material;          /* material of every triangle of this copy, or PT_NO_MATERIAL (the mesh's) */
    uint32_t reserved[2];       /* 0 */
} pt_instance;                  /* 64 bytes */

/* Build a two-level scene (the TLAS/BLAS acceleration structure of Sec. 2.3): n_meshes meshes in
 * object space (mesh m: host verts[m] n_verts[m] x 3 float, tris[m] n_tris[m] x 3 uint32,
 * tri_material[m] n_tris[m] uint32) and n_instances placed copies.  One binned-SAH BVH is built per
 * mesh and one over the instances' world boxes; rays are taken into each instance's object space
 * with the inverse transform, so a mesh is stored once however often it is placed.  Triangle ids
 * (returned by pt_trace_closest, used to break ties and in branch signatures) run over the
 * instances in order, each mesh's triangles in order.  The light list holds every instance's
 * triangles whose (instance or mesh) material emits at creation, placed in the world, ascending
 * id; its pmf is proportional to world area.  Renders, backward passes, progressive renders and
 * queries take the scene like any other; pt_render_batch and pt_autotune_batch reject it
 * (PT_ERR_UNSUPPORTED).  Errors: PT_ERR_INVALID_ARG (no mesh or instance, an empty mesh, NULL
 * arrays, out-of-range indices or materials, non-finite or singular transforms, n_mats >= 2^28,
 * >= 2^28 mesh triangles or >= 2^32 - 1 placed triangles), PT_ERR_OOM, PT_ERR_CUDA; the upload
 * synchronises cuda_stream. */
pt_status pt_scene_create_instanced(uint32_t n_meshes, const float* const* verts, const uint32_t* n_verts,
                                    const uint32_t* const* tris, const uint32_t* n_tris,
                                    const uint32_t* const* tri_material, const pt_instance* instances,
                                    uint32_t n_instances, const pt_material* mats, uint32_t n_mats,
                                    const float env_radiance[3], void* cuda_stream, pt_scene** out);

/* Replace per-material albedo (device n_mats x 3) and emission (device n_mats) -- the
 * differentiable parameters -- asynchronously on `stream`.  Either pointer may be NULL (kept).
 * The light list stays the one fixed at creation. */
pt_status pt_scene_set_materials(pt_scene* scene, const float* d_albedo, const float* d_emission, void* stream);

/* Render one image: W x H pixels, spp samples each, paths of at most max_depth vertices (Sec. 2.2
 * step 5), random numbers keyed by `seed`.  d_out_rgb: H x W x 3 float, host or device (host: the
 * library copies the result back and synchronises `stream`).  d_path_L_or_null: device N_p x 3
 * float per-path radiance (NULL to skip).  opts may be NULL (wavefront, RR from bounce 3, no
 * sort).  The image is img[p] = (1/spp) * sum over samples s = 0..spp-1 (in order) of L[p, s];
 * megakernel and wavefront produce the same image. */
pt_status pt_render(pt_scene* scene, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                    const pt_render_opts* opts, float* d_out_rgb, float* d_path_L_or_null, void* stream);

/* Progressive rendering (the running average of the accumulation stage, Sec. 2.3): render pixel
 * samples sample_offset .. sample_offset + spp - 1 (the random numbers of sample s are those of
 * sample s of a one-call render), add each pixel's samples in sample order to its running FP32 sum
 * in d_accum_rgb (device H x W x 3; zeroed first when sample_offset == 0, otherwise the caller's sums
 * of samples 0 .. sample_offset - 1, e.g. from an earlier call or a saved state), and write
 * sum / (sample_offset + spp) to d_out_rgb_or_null (device H x W x 3, or NULL).  Frames of k1, k2, ...
 * samples therefore give exactly the image of one pt_render call with k1 + k2 + ... samples, and a
 * render resumes from (sums, sample count).  Errors as pt_render, plus PT_ERR_INVALID_ARG for a NULL
 * or host d_accum_rgb, a host d_out_rgb_or_null, or sample_offset + spp >= 2^32. */
pt_status pt_render_progressive(pt_scene* scene, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                                uint32_t sample_offset, const pt_render_opts* opts, float* d_accum_rgb,
                                float* d_out_rgb_or_null, void* stream);

/* Path-replay adjoint: accumulate d(loss)/d(albedo) and d(loss)/d(emission) for the image that
 * pt_render produces with the same arguments, given d_grad_rgb = d(loss)/d(image) (H x W x 3,
 * host or device).  Paths are re-traced from the random numbers (no path storage between forward
 * and backward); Russian roulette probabilities are treated as constants.  opts->mode selects the
 * replay: PT_MODE_WAVEFRONT (default) re-runs the wavefront stages with shading that writes a
 * 64-byte record per path and vertex into a library workspace (waves are sized to keep it under
 * 8 GiB), then walks each path's records backward; PT_MODE_MEGAKERNEL replays each path in one
 * thread with the records in thread-local memory, and a thread whose path is done takes the next
 * one.  d_grad_albedo (device n_mats x 3) and
 * d_grad_emission (device n_mats) are ACCUMULATED into (the caller zeroes them).  max_depth <= 32
 * (else PT_ERR_UNSUPPORTED). */
pt_status pt_render_backward(pt_scene* scene, const pt_camera* cam, uint32_t spp, uint32_t max_depth,
                             uint64_t seed, const pt_render_opts* opts, const float* d_grad_rgb,
                             float* d_grad_albedo, float* d_grad_emission, void* stream);

/* Render n scenes in one persistent wavefront (batched mode): scenes[i] with cams[i] and spp[i]
 * into d_out[i] (device H_i x W_i x 3).  Same estimator and random numbers as pt_render, so each
 * image equals its standalone render.  The bounce loop is captured once in a CUDA graph and
 * replayed per wave; opts->queue_capacity bounds the paths in flight (0 = automatic). */
pt_status pt_render_batch(pt_scene* const* scenes, const pt_camera* cams, const uint32_t* spp, uint32_t n,
                          uint32_t max_depth, uint64_t seed, const pt_render_opts* opts, float* const* d_out,
                          void* stream);

/* Autotuner for pt_render_batch: times the batch under candidate {queue capacity, block size, sort
 * mode} settings on `stream` (synchronous) and writes the fastest into *best (mode = wavefront).
 * `base` supplies the remaining fields (may be NULL).  *best_ms receives its time (may be NULL). */
pt_status pt_autotune_batch(pt_scene* const* scenes, const pt_camera* cams, const uint32_t* spp, uint32_t n,
                            uint32_t max_depth, uint64_t seed, const pt_render_opts* base, float* const* d_out,
                            void* stream, pt_render_opts* best, float* best_ms);

/* Closest-hit query for n rays (the extend stage as a standalone call): d_rays device n x 8 float
 * (o.xyz, tmin(ignored, 0), d.xyz, pad); outputs d_t (n float, +inf on miss) and d_prim (n int32,
 * original triangle id or -1). */
pt_status pt_trace_closest(pt_scene* scene, const float* d_rays, uint32_t n, float* d_t, int32_t* d_prim,
                           void* stream);

/* Wavefront render that allocates nothing.  The paper has no counterpart: this is a deployment
 * variant of pt_render (mode = wavefront) for callers that cannot allocate device memory or let a
 * library do it -- an application whose own memory manager owns the whole device, or a real-time
 * loop that cannot absorb the implicit synchronisation of cudaMalloc/cudaFree.  Its queues live in
 * one 384 MiB file-scope device array, which a GPU holds from the first call on it (when CUDA loads
 * that part of the library) until the process exits; frames
 * are rendered in waves of whole pixels that fit it (2,236,954 paths per wave: a 1-spp 1920x1080
 * frame is one wave), with the
 * same kernels and random numbers, so the image equals pt_render's.  Arguments as for pt_render,
 * except: d_out_rgb (and opts->d_path_sig, if set) must be device memory (nothing is staged), there
 * is no per-path output, and of opts only rr_start, rr_fixed, sort_mode, block_size, d_path_sig and
 * the flags PT_FLAG_HALTON, PT_FLAG_MIS and PT_FLAG_SEPARATE_SHADOW are used (queue_capacity and the
 * other flags are ignored).  Device-side faults of the call (the traversal step cap, a queue overflow) are recorded
 * in a status word inside the array, which the call clears when it starts; they are not reported
 * (pt_get_stats does not see this call and keeps describing the scene's last pt_render call).
 * Errors: PT_ERR_INVALID_ARG also when one pixel's spp samples need more than the array
 * (spp x 180 bytes > 384 MiB), for opts->mode other than PT_MODE_WAVEFRONT and for a nonzero
 * opts->hybrid_threshold.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents: each call clears its own counters, and calls that
 * overlap on the GPU (other streams or threads without ordering between them) race. */
pt_status pt_render_wavefront_static(pt_scene* scene, const pt_camera* cam, uint32_t spp, uint32_t max_depth,
                                     uint64_t seed, const pt_render_opts* opts, float* d_out_rgb, void* stream);

/* Statistics of the last render/backward/batch call on this scene (synchronises the stream used by
 * that call).  status reports device-side faults. */
pt_status pt_get_stats(pt_scene* scene, pt_stats* out);

/* Random numbers exactly as the renderer draws them: out[i] = u(seed, pixel[i], sample[i],
 * bounce[i], dim[i]) in [0, 1) on a 2^-24 grid (device arrays, n entries). */
pt_status pt_debug_rng(uint64_t seed, const uint32_t* d_pixel, const uint32_t* d_sample, const uint32_t* d_bounce,
                       const uint32_t* d_dim, uint32_t n, float* d_out, void* stream);

/* Event logs of selected paths, traced by the megakernel's per-path code (testing aid: find the
 * first decision where two implementations of the estimator part ways).  d_path_ids: device n
 * uint64 path ids; d_events: device n x 64 x 2 uint32 pairs (bounce << 4 | kind, value) with kind
 * 0 = hit (value: triangle id, 0xFFFFFFFF = miss), 1 = NEE (light << 2 | cast << 1 | visible),
 * 2 = BSDF outcome code, 3 = roulette survival; d_payload: device n x 64 x 2 float diagnostics per
 * event (hit: t, throughput.x; NEE: the two cosines; BSDF: weight.x, direction.x; roulette: q, u);
 * d_n_events: device n uint32; d_path_L: device n x 3 float radiance. */
pt_status pt_debug_trace_paths(pt_scene* scene, const pt_camera* cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                               const pt_render_opts* opts, const uint64_t* d_path_ids, uint32_t n, uint32_t* d_events,
                               float* d_payload, uint32_t* d_n_events, float* d_path_L, void* stream);

/* Scene facts: triangle, node, light counts, total light area, device bytes held. */
pt_status pt_scene_info(const pt_scene* scene, uint64_t* n_tris, uint64_t* n_nodes, uint64_t* n_lights,
                        float* light_area, uint64_t* device_bytes);

const char* pt_status_string(pt_status status);
const char* pt_last_error(void);     /* thread-local message of the last failure on this thread */
void pt_scene_destroy(pt_scene* scene);

#ifdef __cplusplus
}
#endif
#endif /* PT_H */
