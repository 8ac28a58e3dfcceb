// wos_mesh.h -- host BVH build for triangle-mesh boundaries (see wos_mesh.cpp).
#pragma once

#include <stdint.h>

#include <vector>

namespace wos {

// 32-byte node: bounds, then `left` (first child, or first triangle of a leaf)
// and `count` (0 for an interior node, else the leaf's triangle count)
struct MeshNode {
  float lo[3];
  int32_t left;
  float hi[3];
  int32_t count;
};
static_assert(sizeof(MeshNode) == 32, "MeshNode must be two float4");

// Build the BVH of a closed triangle mesh (host arrays).  tri_data receives 12
// floats per triangle in leaf order: v0.xyz, -, v1.xyz, -, v2.xyz, -.
// Returns 0, or -1 for invalid input (out-of-range index, non-finite vertex).
int mesh_build_bvh(const float* verts, int64_t nverts, const int32_t* tris, int64_t ntris,
                   std::vector<MeshNode>* nodes, std::vector<float>* tri_data, int* depth);

}  // namespace wos
