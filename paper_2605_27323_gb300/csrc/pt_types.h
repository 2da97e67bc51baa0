// pt_types.h -- plain structs shared by host code (pt_api.cpp) and device code: the device views
// of a scene, the camera, the render parameters and the wavefront buffers.
#pragma once
#include <cstdint>
#include <vector_types.h>

namespace pt {

// ------------------------------------------------------------------ scene views
struct DevMat {            // 32 bytes, mirrors pt_material
    uint32_t type;
    float ar, ag, ab;
    float emission;
    float roughness;
    float ior;
    uint32_t flags;
};

struct DevScene {
    const float4* __restrict__ nodes;      // 4 float4 per node (two child boxes + refs)
    const float4* __restrict__ tris;       // 3 float4 per triangle: v0|prim, e1|material, e2|is_light
    const DevMat* __restrict__ mats;
    const float4* __restrict__ lights;     // 3 float4 per light: p0|material, p1|-, p2|-
    const float* __restrict__ light_cdf;   // inclusive prefix of area / total area
    uint32_t n_lights;
    float light_area;
    float env_r, env_g, env_b;
    uint32_t n_mats;
    uint32_t* status;                      // device status word (atomicOr of fault bits)
    // two-level scenes: `nodes`/`tris` hold every mesh's BVH and object-space triangles, `tlas` the
    // top-level BVH over the instances, `inst` 8 float4 (128 bytes) per instance in top-level leaf
    // order: i0..i2 = world-to-object rows (A | b), i3 = (mesh root node, first triangle id of the
    // instance, material word, -), i4..i6 = object-to-world rotation/scale rows; the material word
    // is 0 (the mesh's materials) or (material + 1) | (material emitted at creation) << 31.
    const float4* __restrict__ tlas = nullptr;
    const float4* __restrict__ inst = nullptr;
    // traversal counters of the counting instantiations (PT_FLAG_COUNT_TRAVERSAL): [0] internal
    // nodes visited and [1] triangles tested by closest-hit walks, [2] and [3] by any-hit walks
    unsigned long long* trav = nullptr;
};

struct DevCamera {         // U = u * tan(fov/2) * aspect, V = v * tan(fov/2), Wd = w (view -> eye)
    float ex, ey, ez;
    float ux, uy, uz;
    float vx, vy, vz;
    float wx, wy, wz;
    uint32_t W, H;
};

struct RenderParams {
    uint64_t seed;
    uint64_t path_begin;   // first path id of this launch / wave
    uint32_t spp;
    uint32_t max_depth;
    uint32_t rr_start;
    float rr_fixed;
    uint32_t sample_offset = 0;   // sample index of a pixel's first path (progressive accumulation)
    uint32_t sampler = 0;         // pixel jitter: 0 PCG uniforms, 1 Halton (2,3) + Cranley-Patterson
    uint32_t mis = 0;             // 1: NEE and BSDF-sampled light hits combined by the power heuristic
    uint32_t short_stack = 0;     // 1: single-level walks keep their top stack entries in shared memory
    uint32_t count_trav = 0;      // 1: single-level walks count visited nodes and tested triangles
};

enum : uint32_t { MAT_LAMBERT = 0, MAT_GGX = 1, MAT_DIELECTRIC = 2 };
constexpr uint32_t SAMPLER_HALTON_ID = 1;   // RenderParams::sampler value of the Halton jitter
enum : uint32_t { ST_TRAVERSAL = 1u, ST_QUEUE = 2u, ST_TIMEOUT = 4u };

// Wavefront buffers of one wave (Sec. 2.3 / 3.1): ping-pong ray queues, hit records, sort
// scratch, the shadow-ray queue, per-path radiance, and the counters.  counts[0] = active paths of
// the current bounce, counts[1] = next bounce's count (filled by compaction), counts[2] = shadow
// rays; the prepare step promotes [1] to [0] and resets [1] and [2] (the two-slot count of
// Sec. 3.1).  The paper reuses one index buffer in place; here the two ray queues alternate, since
// on CUDA a block may append into a slot that a block not yet scheduled still has to read.
struct WfBuffers {
    float4* q_o[2];          // o.xyz | path index (wave-local) bits
    float4* q_d[2];          // d.xyz | flags (bit 0: previous vertex was delta)
    float4* q_tp[2];         // throughput.xyz | solid-angle density of the BSDF sample (MIS weights)
    float2* hit;             // per queue slot: t, reordered triangle bits (0xFFFFFFFF: miss)
    uint32_t* hit_inst;      // per queue slot: instance of the hit (two-level scenes only)
    uint32_t* keys;          // per queue slot: sort key
    uint32_t* perm;          // per sorted position: queue slot
    uint32_t* bucket;        // sort: per-key counts, then running offsets (up to kMaxSortKeys)
    float4* s_o;             // shadow ray: o.xyz | tmax
    float4* s_d;             // shadow ray: d.xyz | path index bits
    float4* s_c;             // shadow ray: contribution.rgb | light index bits
    float4* L;               // per path (wave-local): radiance.rgb | -
    uint32_t* counts;        // [0] active, [1] next, [2] shadow, [3] sort key count, [4] [5] work claims,
                             // [6] shadow rays pending for the fused trace launch
    unsigned long long* hist;  // kHistWords per-call totals (layout at kHistWords)
    uint32_t* sig;           // per path (global id) branch signature, or null
    uint32_t capacity;
};

// Device tables of a batched render (many scenes in one wavefront): per scene its view, camera,
// first global path id (off[n] = total), spp and output image; the current wave's first global path
// id lives in device memory so that one captured bounce loop serves every wave.
struct BatchTables {
    const DevScene* scenes;
    const DevCamera* cams;
    const unsigned long long* off;     // n + 1 entries
    const uint32_t* spp;
    float* const* out;
    uint32_t n;
    unsigned long long* wave_base;
    const unsigned long long* seed;    // device copy of the seed (graph replays stay valid across seeds)
};

// One run of whole or partial pixels of one scene inside a wave (batched accumulation).
struct BatchSegment {
    uint32_t scene;
    uint32_t pad;
    unsigned long long px_begin;
    unsigned long long px_count;
    unsigned long long flat_begin;     // prefix of px_count over the wave's segments
};

// Wavefront adjoint: one 64-byte record per path and vertex, bounce-major (rec[b * cap + pid]):
//   r0 = throughput arriving at the vertex | material,  r1 = continuation weight w | dw/dalbedo,
//   r2 = f G A of the NEE sample (times its MIS weight) | d(f G A Le)/dalbedo,
//   r3 = (Le * w_e, Le_light, w_e, flags | light material << 4) with w_e the emission term's weight;
// flags: 1 continues, 2 NEE visible, 4 emission counted, 8 shadow ray cast.  pend[pid] = number of
// vertices | (path ended in a miss) << 8.
struct AdjBuffers {
    float4* rec;
    uint32_t* pend;
};

constexpr uint32_t kMaxSortKeys = 4096;
constexpr uint32_t kMaxEvents = 64;     // event-log capacity per path (testing aid)

// Device bytes of one wave's records per path: two ping-pong ray queues of three float4 arrays, the
// hit record (float2), the hit instance, sort key and permutation (u32 each), the shadow queue (three
// float4 arrays) and the radiance (float4).
// Per-call device totals (64-bit words after the 256-byte count block): [b] extension rays of bounce
// b, [64 + b] shadow rays of bounce b, [128] [129] megakernel ray totals, [130] next path to start,
// [131] hybrid claim, [132, 136) traversal counters, [136, 141) walks the fused trace stage traced
// with groups of 2, 4, 8, 16, 32 lanes per ray.
constexpr int kHistWords = 144;
constexpr int kHistGroupWalks = 136;

constexpr size_t kWfBytesPerPath = 2 * 3 * 16 + 8 + 3 * 4 + 3 * 16 + 16;
static_assert(kWfBytesPerPath == 180, "wavefront record layout changed: update the documented sizes");

inline size_t wf_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carve the wavefront arrays of `cap` paths (and the sort buckets) out of `base` (null: only count);
// returns the bytes used.  The single layout of both the allocating entry points and the
// allocation-free one.
inline size_t carve_wavefront_at(char* base, uint64_t cap, WfBuffers& w) {
    size_t off = 0;
    auto take = [&](size_t n) {
        char* r = base ? base + off : nullptr;
        off += wf_align256(n);
        return r;
    };
    for (int i = 0; i < 2; ++i) {
        w.q_o[i] = reinterpret_cast<float4*>(take(cap * 16));
        w.q_d[i] = reinterpret_cast<float4*>(take(cap * 16));
        w.q_tp[i] = reinterpret_cast<float4*>(take(cap * 16));
    }
    w.hit = reinterpret_cast<float2*>(take(cap * 8));
    w.hit_inst = reinterpret_cast<uint32_t*>(take(cap * 4));
    w.keys = reinterpret_cast<uint32_t*>(take(cap * 4));
    w.perm = reinterpret_cast<uint32_t*>(take(cap * 4));
    w.bucket = reinterpret_cast<uint32_t*>(take(kMaxSortKeys * 4));
    w.s_o = reinterpret_cast<float4*>(take(cap * 16));
    w.s_d = reinterpret_cast<float4*>(take(cap * 16));
    w.s_c = reinterpret_cast<float4*>(take(cap * 16));
    w.L = reinterpret_cast<float4*>(take(cap * 16));
    return off;
}

inline size_t wavefront_bytes(uint64_t cap) {
    WfBuffers w{};
    return carve_wavefront_at(nullptr, cap, w);
}

}  // namespace pt
