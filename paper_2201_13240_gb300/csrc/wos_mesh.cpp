// wos_mesh.cpp -- host construction of the bounding volume hierarchy that
// accelerates closest-point queries on a triangle-mesh boundary (Sec. 7.1: the
// distance query, the main cost of walk on spheres, uses a BVH).
//
// Binned surface-area-heuristic build over triangle centroids (16 bins per
// axis, leaves of at most 4 triangles).  Output, ready to upload:
//   nodes:  2 x float4 per node: (min.xyz, left) and (max.xyz, count) with the
//           int fields stored bit-for-bit; count == 0 marks an interior node
//           whose children are nodes `left` and `left + 1`; a leaf holds
//           triangles first = left .. left + count - 1 of the reordered list.
//   tris:   3 x float4 per triangle in leaf order: (v0, v1, v2), w unused.
// Node 0 is the root.  The build is deterministic.  mesh_collapse4 turns the binary
// tree into the 4-wide nodes the device traverses.
#include "wos_mesh.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace wos {
namespace {

struct Box {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const float* p) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], p[d]);
      hi[d] = std::max(hi[d], p[d]);
    }
  }
  void grow(const Box& b) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], b.lo[d]);
      hi[d] = std::max(hi[d], b.hi[d]);
    }
  }
  float area() const {
    float e[3];
    for (int d = 0; d < 3; ++d) e[d] = std::max(0.0f, hi[d] - lo[d]);
    return 2.0f * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
  }
};

struct Prim {
  Box box;
  float c[3];
  int64_t tri;
};

struct Builder {
  std::vector<Prim> prims;
  std::vector<MeshNode> nodes;
  static constexpr int kBins = 16;
  static constexpr int kLeaf = 4;

  void build(int64_t node, int64_t first, int64_t count, int depth) {
    Box nb, cb;
    for (int64_t i = first; i < first + count; ++i) {
      nb.grow(prims[i].box);
      cb.grow(prims[i].c);
    }
    MeshNode& N = nodes[node];
    std::memcpy(N.lo, nb.lo, sizeof(N.lo));
    std::memcpy(N.hi, nb.hi, sizeof(N.hi));
    if (count <= kLeaf || depth >= 28) {  // depth <= 29: the traversal stack holds 32 entries
      N.left = first;
      N.count = count;
      return;
    }
    // binned SAH over the centroid box
    int best_axis = -1, best_split = -1;
    float best_cost = INFINITY;
    for (int ax = 0; ax < 3; ++ax) {
      float ext = cb.hi[ax] - cb.lo[ax];
      if (!(ext > 0.0f)) continue;
      Box bin_box[kBins];
      int64_t bin_n[kBins] = {0};
      float scale = kBins / ext;
      for (int64_t i = first; i < first + count; ++i) {
        int b = std::min(kBins - 1, (int)((prims[i].c[ax] - cb.lo[ax]) * scale));
        bin_n[b]++;
        bin_box[b].grow(prims[i].box);
      }
      float left_area[kBins];
      int64_t left_n[kBins];
      Box acc;
      int64_t n = 0;
      for (int b = 0; b < kBins - 1; ++b) {
        acc.grow(bin_box[b]);
        n += bin_n[b];
        left_area[b] = acc.area();
        left_n[b] = n;
      }
      Box racc;
      int64_t rn = 0;
      for (int b = kBins - 1; b > 0; --b) {
        racc.grow(bin_box[b]);
        rn += bin_n[b];
        int64_t ln = left_n[b - 1];
        if (ln == 0 || rn == 0) continue;
        float cost = left_area[b - 1] * (float)ln + racc.area() * (float)rn;
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = ax;
          best_split = b;
        }
      }
    }
    int64_t mid;
    if (best_axis < 0) {
      // all centroids coincide: split the list in half
      mid = first + count / 2;
    } else {
      float ext = cb.hi[best_axis] - cb.lo[best_axis];
      float scale = kBins / ext;
      auto it = std::partition(prims.begin() + first, prims.begin() + first + count, [&](const Prim& p) {
        int b = std::min(kBins - 1, (int)((p.c[best_axis] - cb.lo[best_axis]) * scale));
        return b < best_split;
      });
      mid = it - prims.begin();
      if (mid == first || mid == first + count) mid = first + count / 2;
    }
    int64_t left = (int64_t)nodes.size();
    nodes.emplace_back();
    nodes.emplace_back();
    nodes[node].left = left;
    nodes[node].count = 0;
    build(left, first, mid - first, depth + 1);
    build(left + 1, mid, first + count - mid, depth + 1);
  }
};

int collapse(const std::vector<MeshNode>& bin, int64_t n, std::vector<MeshNode4>* wide, int level, int* depth) {
  const int idx = (int)wide->size();
  wide->emplace_back();
  *depth = std::max(*depth, level);
  int64_t slot[4];
  int ns = 0;
  if (bin[n].count > 0) {
    slot[ns++] = n;  // a root that is a leaf
  } else {
    for (int64_t c = bin[n].left; c < bin[n].left + 2; ++c) {
      if (bin[c].count == 0) {
        slot[ns++] = bin[c].left;
        slot[ns++] = bin[c].left + 1;
      } else {
        slot[ns++] = c;
      }
    }
  }
  int32_t child[4], count[4];
  for (int i = 0; i < 4; ++i) {
    if (i >= ns) {
      child[i] = 0;
      count[i] = -1;
    } else if (bin[slot[i]].count > 0) {
      child[i] = bin[slot[i]].left;
      count[i] = bin[slot[i]].count;
    } else {
      child[i] = collapse(bin, slot[i], wide, level + 1, depth);
      count[i] = 0;
    }
  }
  MeshNode4& w = (*wide)[idx];  // after the recursion: the vector may have moved
  for (int i = 0; i < 4; ++i) {
    const bool on = i < ns;
    w.lox[i] = on ? bin[slot[i]].lo[0] : INFINITY;
    w.loy[i] = on ? bin[slot[i]].lo[1] : INFINITY;
    w.loz[i] = on ? bin[slot[i]].lo[2] : INFINITY;
    w.hix[i] = on ? bin[slot[i]].hi[0] : -INFINITY;
    w.hiy[i] = on ? bin[slot[i]].hi[1] : -INFINITY;
    w.hiz[i] = on ? bin[slot[i]].hi[2] : -INFINITY;
    w.child[i] = child[i];
    w.count[i] = count[i];
  }
  return idx;
}

}  // namespace

void mesh_collapse4(const std::vector<MeshNode>& bin, std::vector<MeshNode4>* wide, int* depth) {
  wide->clear();
  wide->reserve(bin.size() / 2 + 1);
  int d = 0;
  collapse(bin, 0, wide, 1, &d);
  if (depth) *depth = d;
}

int mesh_top_first(std::vector<MeshNode4>* wide, int levels) {
  std::vector<MeshNode4>& w = *wide;
  const int n = (int)w.size();
  std::vector<int> order;  // new position -> old index
  std::vector<int> level_of(n, 0);
  std::vector<char> top(n, 0);
  order.reserve(n);
  // breadth-first over the interior children down to `levels`
  std::vector<int> queue = {0};
  level_of[0] = 1;
  for (size_t q = 0; q < queue.size(); ++q) {
    const int v = queue[q];
    top[v] = 1;
    order.push_back(v);
    if (level_of[v] >= levels) continue;
    for (int i = 0; i < 4; ++i)
      if (w[v].count[i] == 0) {
        level_of[w[v].child[i]] = level_of[v] + 1;
        queue.push_back(w[v].child[i]);
      }
  }
  const int ntop = (int)order.size();
  for (int v = 0; v < n; ++v)
    if (!top[v]) order.push_back(v);
  std::vector<int> pos(n);
  for (int i = 0; i < n; ++i) pos[order[i]] = i;
  std::vector<MeshNode4> out(n);
  for (int i = 0; i < n; ++i) {
    out[i] = w[order[i]];
    for (int c = 0; c < 4; ++c)
      if (out[i].count[c] == 0) out[i].child[c] = pos[out[i].child[c]];
  }
  w.swap(out);
  return ntop;
}

int mesh_build_bvh(const float* verts, int64_t nverts, const int32_t* tris, int64_t ntris,
                   std::vector<MeshNode>* nodes, std::vector<float>* tri_data, int* depth_out) {
  if (!verts || !tris || nverts < 3 || ntris < 1 || ntris > (int64_t)1 << 30) return -1;
  for (int64_t i = 0; i < 3 * ntris; ++i)
    if (tris[i] < 0 || tris[i] >= nverts) return -1;
  for (int64_t i = 0; i < 3 * nverts; ++i)
    if (!std::isfinite(verts[i])) return -1;
  Builder B;
  B.prims.resize(ntris);
  for (int64_t t = 0; t < ntris; ++t) {
    Prim& p = B.prims[t];
    for (int k = 0; k < 3; ++k) p.box.grow(verts + 3 * (int64_t)tris[3 * t + k]);
    for (int d = 0; d < 3; ++d) {
      float s = 0.0f;
      for (int k = 0; k < 3; ++k) s += verts[3 * (int64_t)tris[3 * t + k] + d];
      p.c[d] = s / 3.0f;
    }
    p.tri = t;
  }
  B.nodes.reserve(2 * (size_t)ntris);
  B.nodes.emplace_back();
  B.build(0, 0, ntris, 0);
  *nodes = B.nodes;
  tri_data->assign((size_t)ntris * 12, 0.0f);
  for (int64_t i = 0; i < ntris; ++i) {
    const int32_t* t = tris + 3 * B.prims[i].tri;
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) (*tri_data)[(size_t)i * 12 + 4 * k + d] = verts[3 * (int64_t)t[k] + d];
  }
  // depth of the tree (for the traversal stack bound)
  std::vector<std::pair<int64_t, int>> st = {{0, 1}};
  int depth = 0;
  while (!st.empty()) {
    auto [n, dpt] = st.back();
    st.pop_back();
    depth = std::max(depth, dpt);
    if ((*nodes)[n].count == 0) {
      st.push_back({(*nodes)[n].left, dpt + 1});
      st.push_back({(*nodes)[n].left + 1, dpt + 1});
    }
  }
  if (depth_out) *depth_out = depth;
  return 0;
}

}  // namespace wos
