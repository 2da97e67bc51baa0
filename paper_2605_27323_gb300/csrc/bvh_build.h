// bvh_build.h -- host BVH construction (binned SAH) into the 64-byte node layout of pt_trace.cuh.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pt {

struct BvhOut {
    std::vector<float> nodes;      // 16 floats per internal node (4 x float4 rows)
    std::vector<uint32_t> order;   // leaf order: position -> original triangle id
    uint32_t n_internal = 0;
    int depth = 0;                 // levels of internal nodes plus the leaf level
};

// verts: n_verts x 3; tris: n_tris x 3 indices (already validated).  Returns false with a message
// when the input cannot be encoded.
// max_leaf: most primitives per leaf (1 for the top level of a two-level scene, so that each
// instance's box is tested in its parent before the ray is transformed).
bool build_bvh(const float* verts, const uint32_t* tris, uint32_t n_tris, BvhOut& out, std::string& err,
               uint32_t max_leaf = 8);

}  // namespace pt
