// Host BVH builder interface (see pb_bvh.cpp for the node layout).
#pragma once
#include <cstdint>
#include <vector>

struct PbBvh {
    std::vector<float> nodes;      // 16 floats per node
    std::vector<int32_t> parent;   // per node, -1 for the root
    std::vector<int32_t> sibling;  // per internal node: the other internal child of its parent, or -1
    std::vector<int32_t> order;    // leaf-ordered triangle indices
};

// Returns the node count.
int pb_bvh_build(const float *verts, int nv, const int32_t *tris, int nt, PbBvh *out);
