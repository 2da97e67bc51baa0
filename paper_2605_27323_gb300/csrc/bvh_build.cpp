// bvh_build.cpp -- host construction of the traversal structure (the paper builds hardware
// acceleration structures on the host, Sec. 3; here a binned-SAH binary BVH, Wald 2007, "On fast
// Construction of SAH-based Bounding Volume Hierarchies").
//
// Output (see pt_trace.cuh for the layout): 64-byte internal nodes holding both children's boxes
// and child references, leaves of at most 8 triangles referenced from their parent, and the
// triangle order of the leaves.  The tree depth is capped below the traversal stack size by
// switching to median splits deep in the tree.  The top levels are built in parallel threads; the
// output is deterministic (subtrees are concatenated in a fixed order).
#include "bvh_build.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>

namespace pt {
namespace {

constexpr int kBins = 16;
constexpr uint32_t kMaxLeaf = 8;
constexpr int kMedianDepth = 32;      // below this depth: SAH; beyond: median splits (depth cap)
constexpr float kTravCost = 1.2f;     // cost of one node visit relative to one triangle test
constexpr uint32_t kParallelMin = 1u << 15;
constexpr int kParallelDepth = 4;

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::numeric_limits<float>::infinity();
            hi[k] = -std::numeric_limits<float>::infinity();
        }
    }
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow(const float* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    float area() const {
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        if (!(dx >= 0.f) || !(dy >= 0.f) || !(dz >= 0.f)) return 0.f;
        return 2.f * (dx * dy + dy * dz + dz * dx);
    }
};

struct BNode {
    Box box;
    int32_t left = -1, right = -1;   // local indices within the output vector
    uint32_t first = 0, count = 0;   // leaf range when count > 0
};

struct Builder {
    const std::vector<Box>* tri_box;
    const std::vector<float>* cen;   // 3 per triangle
    uint32_t* idx;
    uint32_t max_leaf = kMaxLeaf;

    void bounds(uint32_t first, uint32_t count, Box& b, Box& cb) const {
        b.reset();
        cb.reset();
        for (uint32_t i = first; i < first + count; ++i) {
            b.grow((*tri_box)[idx[i]]);
            cb.grow(&(*cen)[3 * (size_t)idx[i]]);
        }
    }

    // Median split along the widest centroid axis (always splits count >= 2).
    uint32_t median_split(uint32_t first, uint32_t count, const Box& cb) const {
        int axis = 0;
        for (int k = 1; k < 3; ++k)
            if (cb.hi[k] - cb.lo[k] > cb.hi[axis] - cb.lo[axis]) axis = k;
        uint32_t mid = first + count / 2;
        const std::vector<float>& c = *cen;
        std::nth_element(idx + first, idx + mid, idx + first + count, [&](uint32_t a, uint32_t b) {
            float ca = c[3 * (size_t)a + axis], cb2 = c[3 * (size_t)b + axis];
            return ca < cb2 || (ca == cb2 && a < b);
        });
        return mid;
    }

    // Binned SAH: returns the split position, or 0 when a leaf is cheaper (count <= max_leaf).
    uint32_t sah_split(uint32_t first, uint32_t count, const Box& b, const Box& cb) const {
        float best_cost = std::numeric_limits<float>::infinity();
        int best_axis = -1, best_bin = -1;
        const std::vector<float>& c = *cen;
        for (int axis = 0; axis < 3; ++axis) {
            float lo = cb.lo[axis], ext = cb.hi[axis] - cb.lo[axis];
            if (!(ext > 0.f)) continue;
            float scale = kBins / ext;
            Box bb[kBins];
            uint32_t bn[kBins] = {};
            for (int k = 0; k < kBins; ++k) bb[k].reset();
            for (uint32_t i = first; i < first + count; ++i) {
                int k = std::min(kBins - 1, (int)((c[3 * (size_t)idx[i] + axis] - lo) * scale));
                bn[k]++;
                bb[k].grow((*tri_box)[idx[i]]);
            }
            float right_area[kBins];
            uint32_t right_n[kBins];
            Box acc;
            acc.reset();
            uint32_t n = 0;
            for (int k = kBins - 1; k > 0; --k) {
                acc.grow(bb[k]);
                n += bn[k];
                right_area[k] = acc.area();
                right_n[k] = n;
            }
            acc.reset();
            n = 0;
            for (int k = 0; k < kBins - 1; ++k) {
                acc.grow(bb[k]);
                n += bn[k];
                if (n == 0 || right_n[k + 1] == 0) continue;
                float cost = acc.area() * n + right_area[k + 1] * right_n[k + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = axis;
                    best_bin = k;
                }
            }
        }
        float area = b.area();
        float leaf_cost = (float)count;
        float split_cost = area > 0.f ? kTravCost + best_cost / area : std::numeric_limits<float>::infinity();
        if (count <= max_leaf && leaf_cost <= split_cost) return 0;
        if (best_axis < 0) return median_split(first, count, cb);
        float lo = cb.lo[best_axis], scale = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
        uint32_t* mid = std::partition(idx + first, idx + first + count, [&](uint32_t t) {
            int k = std::min(kBins - 1, (int)((c[3 * (size_t)t + best_axis] - lo) * scale));
            return k <= best_bin;
        });
        uint32_t m = (uint32_t)(mid - idx);
        if (m == first || m == first + count) return median_split(first, count, cb);
        return m;
    }

    int32_t build(std::vector<BNode>& out, uint32_t first, uint32_t count, int depth) {
        int32_t id = (int32_t)out.size();
        out.emplace_back();
        Box b, cb;
        bounds(first, count, b, cb);
        out[id].box = b;
        uint32_t mid;
        if (count <= 1) {
            mid = 0;
        } else if (depth >= kMedianDepth) {
            mid = count <= max_leaf ? 0 : median_split(first, count, cb);
        } else {
            mid = sah_split(first, count, b, cb);
        }
        if (mid == 0) {
            out[id].first = first;
            out[id].count = count;
            return id;
        }
        uint32_t nl = mid - first, nr = count - nl;
        int32_t l, r;
        if (depth < kParallelDepth && count >= kParallelMin) {
            std::vector<BNode> right;
            std::thread th([&] { build(right, mid, nr, depth + 1); });
            l = build(out, first, nl, depth + 1);
            th.join();
            int32_t off = (int32_t)out.size();
            for (BNode& n : right) {
                if (n.count == 0) {
                    n.left += off;
                    n.right += off;
                }
                out.push_back(n);
            }
            r = off;
        } else {
            l = build(out, first, nl, depth + 1);
            r = build(out, mid, nr, depth + 1);
        }
        out[id].left = l;
        out[id].right = r;
        return id;
    }
};

float f32_bits(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

bool build_bvh(const float* verts, const uint32_t* tris, uint32_t n_tris, BvhOut& out, std::string& err,
               uint32_t max_leaf) {
    if (max_leaf < 1 || max_leaf > kMaxLeaf) {
        err = "max_leaf must be in [1, 8]";
        return false;
    }
    out.nodes.clear();
    out.order.clear();
    out.depth = 0;
    if (n_tris >= (1u << 28)) {
        err = "too many triangles for the leaf encoding (limit 2^28)";
        return false;
    }
    std::vector<Box> tri_box(n_tris);
    std::vector<float> cen(3 * (size_t)n_tris);
    std::vector<uint32_t> idx(n_tris);
    for (uint32_t i = 0; i < n_tris; ++i) {
        Box b;
        b.reset();
        for (int v = 0; v < 3; ++v) b.grow(verts + 3 * (size_t)tris[3 * (size_t)i + v]);
        tri_box[i] = b;
        for (int k = 0; k < 3; ++k) cen[3 * (size_t)i + k] = 0.5f * (b.lo[k] + b.hi[k]);
        idx[i] = i;
    }
    std::vector<BNode> bn;
    bn.reserve(2 * (size_t)n_tris + 1);
    if (n_tris > 0) {
        Builder B{&tri_box, &cen, idx.data(), max_leaf};
        B.build(bn, 0, n_tris, 0);
    }
    // Convert: GPU nodes are the internal build nodes in depth-first order; a leaf lives in its
    // parent's child slot.  A root that is a leaf gets a synthetic root whose two slots both hold it
    // (the second visit finds the same hits); an empty scene gets a root whose slots reference one
    // all-zero triangle record, which no ray can hit (its determinant is 0).  No slot is ever left
    // with an inverted box: the slab test does not reject those.
    Box zero;
    for (int k = 0; k < 3; ++k) zero.lo[k] = zero.hi[k] = 0.f;
    auto leaf_ref = [&](const BNode& n) { return 0x80000000u | (n.first << 3) | (n.count - 1u); };
    std::vector<int32_t> gpu_id(bn.size(), -1);
    int32_t n_int = 0;
    for (size_t i = 0; i < bn.size(); ++i)
        if (bn[i].count == 0) gpu_id[i] = n_int++;
    auto emit = [&](const Box& b0, uint32_t r0, const Box& b1, uint32_t r1) {
        float f[16];
        for (int k = 0; k < 3; ++k) {      // row k: (c0.lo, c1.lo, c0.hi, c1.hi) of axis k
            f[4 * k] = b0.lo[k];
            f[4 * k + 1] = b1.lo[k];
            f[4 * k + 2] = b0.hi[k];
            f[4 * k + 3] = b1.hi[k];
        }
        f[12] = f32_bits(r0);
        f[13] = f32_bits(r1);
        f[14] = 0.f;
        f[15] = 0.f;
        out.nodes.insert(out.nodes.end(), f, f + 16);
    };
    if (bn.empty() || bn[0].count > 0) {
        if (bn.empty()) emit(zero, 0x80000000u, zero, 0x80000000u);
        else emit(bn[0].box, leaf_ref(bn[0]), bn[0].box, leaf_ref(bn[0]));
        out.depth = 1;
    } else {
        // depth-first order of internal nodes == build order (children follow their parent)
        std::vector<int> depth(bn.size(), 0);
        for (size_t i = 0; i < bn.size(); ++i) {
            const BNode& n = bn[i];
            if (n.count > 0) continue;
            const BNode& a = bn[n.left];
            const BNode& b = bn[n.right];
            depth[n.left] = depth[n.right] = depth[i] + 1;
            out.depth = std::max(out.depth, depth[i] + 2);
            if (a.count > 0 && a.count > 8) {
                err = "internal error: leaf larger than 8 triangles";
                return false;
            }
            uint32_t ra = a.count > 0 ? leaf_ref(a) : (uint32_t)gpu_id[n.left];
            uint32_t rb = b.count > 0 ? leaf_ref(b) : (uint32_t)gpu_id[n.right];
            emit(a.box, ra, b.box, rb);
        }
    }
    out.order = std::move(idx);
    out.n_internal = (uint32_t)(out.nodes.size() / 16);
    if (out.depth >= 64) {
        err = "BVH deeper than the traversal stack";
        return false;
    }
    return true;
}

}  // namespace pt
