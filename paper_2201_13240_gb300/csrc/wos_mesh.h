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

// 128-byte 4-wide node (one cache line), the layout the device traverses: the four
// children's boxes as structure of arrays, then per child `child` (a 4-wide node index,
// or the first triangle of a leaf) and `count` (0: interior, > 0: a leaf's triangle
// count, -1: empty slot, whose box is empty: lo = +inf, hi = -inf).
struct MeshNode4 {
  float lox[4], loy[4], loz[4];
  float hix[4], hiy[4], hiz[4];
  int32_t child[4];
  int32_t count[4];
};
static_assert(sizeof(MeshNode4) == 128, "MeshNode4 must be one 128-byte line");

// Collapse a binary BVH (as built below) into 4-wide nodes: each wide node holds the
// grandchildren of a binary node (or a child that is a leaf).  depth: levels of the
// wide tree.  Wide node 0 is the root.
void mesh_collapse4(const std::vector<MeshNode>& bin, std::vector<MeshNode4>* wide, int* depth);

// Nodes of the wide tree's top `levels` levels (the root is level 1), placed first in
// breadth-first order; the other nodes keep their order after them and every child index
// is renumbered.  Returns how many nodes come first (the kernels stage them in shared
// memory: every query starts at the root).
constexpr int kMeshTopLevels = 3;  // at most 1 + 4 + 16 = 21 nodes, 2.7 KB
int mesh_top_first(std::vector<MeshNode4>* wide, int levels);

// Build the BVH of a closed triangle mesh (host arrays).  tri_data receives 12
// floats per triangle in leaf order: v0.xyz, -, v1.xyz, -, v2.xyz, -.
// Returns 0, or -1 for invalid input (out-of-range index, non-finite vertex).
int mesh_build_bvh(const float* verts, int64_t nverts, const int32_t* tris, int64_t ntris,
                   std::vector<MeshNode>* nodes, std::vector<float>* tri_data, int* depth);

}  // namespace wos
