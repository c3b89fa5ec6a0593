// scene_build.cpp -- host-side scene preparation for libsdd: the subdomain split and one
// binned-SAH BVH per subdomain.
//
// Sec. 5 of arXiv:1912.05494: the global geometry is split into sub-domains once and the
// split is reused for every run; each sub-domain keeps its own acceleration structure.
// Here the sub-domains are S slabs of equal length along one axis (the nave's length),
// the outer two extending to infinity.  A triangle is referenced by every slab its
// bounding box overlaps (widened by `slop`), with its box clipped to the slab so that
// the BVH of a slab bounds only the part of the geometry that lies in it.  A hit inside a
// slab's ray interval therefore always lies inside that slab's BVH.
//
// The BVH is built binary, top-down with 16-bin SAH, then collapsed to a 4-wide tree (each
// node takes the two children of a binary node and opens the largest inner child until it
// holds four), stored in breadth-first order (so that the top levels form one contiguous
// block) as 128-byte nodes holding the four children's boxes, and 48-byte triangle records
// (three float4 vertices).  A walk step then fetches one node for four boxes, halving the
// chain of dependent node fetches that bounds the traversal.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#include "sdd_internal.h"
#include "scene_build.h"

namespace sdd {
namespace {

struct Box3 {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const Box3& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  void grow_pt(const float* p) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p[a]);
      hi[a] = std::max(hi[a], p[a]);
    }
  }
  bool empty() const { return !(lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2]); }
  float area() const {
    if (empty()) return 0.f;
    float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.f * (dx * dy + dy * dz + dz * dx);
  }
  float cen(int a) const { return 0.5f * (lo[a] + hi[a]); }
};

struct Ref {
  Box3 box;
  int prim;
};

struct TmpNode {
  Box3 box;
  int left = -1, right = -1;  // children (tmp indices) for inner nodes
  int first = 0, count = 0;   // refs for leaves
};

constexpr int kBins = 16;
// Ranges of at most kLeafMax references become leaves (up to 2 kLeafMax when no split is
// cheaper).  A triangle test costs the walk about as much as a node step, so small leaves win:
// on the nave bench frame (binary tree, bundles of 14), closest-hit passes 109.6 ms and shadow
// passes 53.8 ms with 2, against 124.2 / 60.7 ms with 4, 160.2 / 73.7 ms with 8 and 112.8 /
// 53.8 ms with 1; on the 4-wide tree (bundles of 41) the frame takes 96.1 ms with 2 or 3,
// 98.9 with 1 and 102.0 with 4.
constexpr int kLeafMax = 2;
constexpr int kDepthLimit = 60;  // binary levels; the 4-wide walk pushes at most 3 per node

struct Builder {
  std::vector<Ref>& refs;
  std::vector<TmpNode> nodes;
  int max_depth = 0;
  explicit Builder(std::vector<Ref>& r) : refs(r) {}

  int make_leaf(int first, int count, const Box3& box) {
    TmpNode n;
    n.box = box;
    n.first = first;
    n.count = count;
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }

  int build(int first, int count, int depth) {
    max_depth = std::max(max_depth, depth);
    Box3 box, cb;
    for (int i = first; i < first + count; ++i) {
      box.grow(refs[i].box);
      float c[3] = {refs[i].box.cen(0), refs[i].box.cen(1), refs[i].box.cen(2)};
      cb.grow_pt(c);
    }
    if (count <= kLeafMax || depth >= kDepthLimit) return make_leaf(first, count, box);

    int best_axis = -1, best_split = -1;
    float best_cost = INFINITY;
    for (int a = 0; a < 3; ++a) {
      float ext = cb.hi[a] - cb.lo[a];
      if (!(ext > 0.f)) continue;
      Box3 bb[kBins];
      int bc[kBins] = {0};
      float scale = kBins / ext;
      for (int i = first; i < first + count; ++i) {
        int b = std::min(kBins - 1, (int)((refs[i].box.cen(a) - cb.lo[a]) * scale));
        bb[b].grow(refs[i].box);
        bc[b]++;
      }
      float right_area[kBins];
      int right_count[kBins];
      Box3 acc;
      int cnt = 0;
      for (int b = kBins - 1; b > 0; --b) {
        acc.grow(bb[b]);
        cnt += bc[b];
        right_area[b] = acc.area();
        right_count[b] = cnt;
      }
      Box3 lacc;
      int lcnt = 0;
      for (int b = 0; b < kBins - 1; ++b) {
        lacc.grow(bb[b]);
        lcnt += bc[b];
        if (lcnt == 0 || right_count[b + 1] == 0) continue;
        float cost = lacc.area() * lcnt + right_area[b + 1] * right_count[b + 1];
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = a;
          best_split = b;
        }
      }
    }
    int mid;
    if (best_axis < 0) {
      // all centroids coincide: split by count
      mid = first + count / 2;
    } else {
      float leaf_cost = box.area() * count;
      if (count <= 2 * kLeafMax && best_cost >= leaf_cost) return make_leaf(first, count, box);
      float scale = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
      auto it = std::partition(refs.begin() + first, refs.begin() + first + count, [&](const Ref& r) {
        int b = std::min(kBins - 1, (int)((r.box.cen(best_axis) - cb.lo[best_axis]) * scale));
        return b <= best_split;
      });
      mid = (int)(it - refs.begin());
      if (mid == first || mid == first + count) mid = first + count / 2;
    }
    int me = (int)nodes.size();
    nodes.push_back(TmpNode{});
    nodes[me].box = box;
    int l = build(first, mid - first, depth + 1);
    int r = build(mid, first + count - mid, depth + 1);
    nodes[me].left = l;
    nodes[me].right = r;
    return me;
  }
};

void set_child(Node& n, int c, const Box3& b, int link, int count) {
  reinterpret_cast<float*>(&n.lox)[c] = b.lo[0];
  reinterpret_cast<float*>(&n.hix)[c] = b.hi[0];
  reinterpret_cast<float*>(&n.loy)[c] = b.lo[1];
  reinterpret_cast<float*>(&n.hiy)[c] = b.hi[1];
  reinterpret_cast<float*>(&n.loz)[c] = b.lo[2];
  reinterpret_cast<float*>(&n.hiz)[c] = b.hi[2];
  reinterpret_cast<int*>(&n.link)[c] = link;
  reinterpret_cast<int*>(&n.cnt)[c] = count;
}

// Children of the 4-wide node made from binary inner node t: t's two children, then the inner
// child of largest surface area replaced by its own two children until there are four (or
// only leaves are left).  Returns how many.
int wide_children(const Builder& bld, int t, int ch[kBvhWidth]) {
  int k = 2;
  ch[0] = bld.nodes[t].left;
  ch[1] = bld.nodes[t].right;
  while (k < kBvhWidth) {
    int open = -1;
    float area = -1.f;
    for (int j = 0; j < k; ++j) {
      const TmpNode& c = bld.nodes[ch[j]];
      if (c.left >= 0 && c.box.area() > area) {
        open = j;
        area = c.box.area();
      }
    }
    if (open < 0) break;
    const int c = ch[open];
    ch[open] = bld.nodes[c].left;
    ch[k++] = bld.nodes[c].right;
  }
  return k;
}

// Flatten one tmp tree into BFS-ordered 4-wide Nodes appended to `out`, triangle records to
// `tris`.
int flatten(const Builder& bld, int tmp_root, const std::vector<Ref>& refs, const float* verts,
            const uint32_t* idx, std::vector<Node>& out, std::vector<TriRec>& tris, int* stack_need) {
  const int base = (int)out.size();
  const Box3 none;  // inverted box (and link -1): never entered
  // tmp inner node of every output node (-1: a synthetic root over a subdomain that is one
  // leaf) and its children, in breadth-first order
  std::vector<int> order;
  std::vector<std::array<int, kBvhWidth>> kids;
  std::vector<int> n_kids;
  std::vector<int> out_index(bld.nodes.size(), -1);
  order.push_back(bld.nodes[tmp_root].left < 0 ? -1 : tmp_root);
  for (size_t q = 0; q < order.size(); ++q) {
    std::array<int, kBvhWidth> ch{};
    int k = 0;
    if (order[q] < 0) {
      ch[k++] = tmp_root;
    } else {
      k = wide_children(bld, order[q], ch.data());
      for (int j = 0; j < k; ++j)
        if (bld.nodes[ch[j]].left >= 0) {
          out_index[ch[j]] = base + (int)order.size();
          order.push_back(ch[j]);
        }
    }
    kids.push_back(ch);
    n_kids.push_back(k);
  }
  out.resize(base + order.size());
  auto emit_leaf = [&](const TmpNode& lf) -> int {
    int first = (int)tris.size();
    for (int i = lf.first; i < lf.first + lf.count; ++i) {
      int p = refs[i].prim;
      TriRec r;
      const float* a = verts + 3 * idx[3 * p + 0];
      const float* b = verts + 3 * idx[3 * p + 1];
      const float* c = verts + 3 * idx[3 * p + 2];
      float pid;
      uint32_t up = (uint32_t)p;
      std::memcpy(&pid, &up, 4);
      r.v0 = make_float4(a[0], a[1], a[2], pid);
      r.v1 = make_float4(b[0], b[1], b[2], 0.f);
      r.v2 = make_float4(c[0], c[1], c[2], 0.f);
      tris.push_back(r);
    }
    return first;
  };
  for (size_t q = 0; q < order.size(); ++q) {
    Node n;
    std::memset(&n, 0, sizeof(n));
    for (int w = 0; w < kBvhWidth; ++w) {
      if (w >= n_kids[q]) {
        set_child(n, w, none, -1, 0);
        continue;
      }
      const TmpNode& c = bld.nodes[kids[q][w]];
      if (c.left >= 0) {
        set_child(n, w, c.box, out_index[kids[q][w]], 0);
      } else if (c.count > 0) {
        set_child(n, w, c.box, emit_leaf(c), c.count);
      } else {
        set_child(n, w, none, -1, 0);
      }
    }
    out[base + q] = n;
  }
  // deepest traversal stack a walk of this tree can need: at a node whose k inner children
  // are all entered the walk descends into one and pushes k - 1
  std::vector<int> need(order.size(), 0);
  for (size_t q = order.size(); q-- > 0;) {
    int k_in = 0, below = 0;
    for (int w = 0; w < n_kids[q]; ++w) {
      const int c = kids[q][w];
      if (bld.nodes[c].left >= 0) {
        ++k_in;
        below = std::max(below, need[out_index[c] - base]);
      }
    }
    need[q] = k_in > 0 ? k_in - 1 + below : 0;
  }
  *stack_need = std::max(*stack_need, need[0]);
  return base;
}

}  // namespace

void build_scene_bvh(const BuildInput& in, HostBVH& out) {
  out.nodes.clear();
  out.tris.clear();
  out.root.assign(in.n_sub, 0);
  out.n_nodes.assign(in.n_sub, 0);
  out.max_depth = 0;
  out.stack_need = 0;
  out.n_refs = 0;
  // triangle boxes
  std::vector<Box3> tbox(in.n_tris);
  for (int t = 0; t < in.n_tris; ++t)
    for (int c = 0; c < 3; ++c) tbox[t].grow_pt(in.verts + 3 * in.idx[3 * t + c]);
  for (int s = 0; s < in.n_sub; ++s) {
    float lo = in.planes[s] - in.slop, hi = in.planes[s + 1] + in.slop;
    std::vector<Ref> refs;
    for (int t = 0; t < in.n_tris; ++t) {
      const Box3& b = tbox[t];
      if (b.hi[in.axis] < lo || b.lo[in.axis] > hi) continue;
      Ref r;
      r.box = b;
      r.box.lo[in.axis] = std::max(b.lo[in.axis], lo);
      r.box.hi[in.axis] = std::min(b.hi[in.axis], hi);
      r.prim = t;
      refs.push_back(r);
    }
    out.n_refs += (int64_t)refs.size();
    Builder bld(refs);
    int root;
    if (refs.empty()) {
      TmpNode n;  // empty leaf
      bld.nodes.push_back(n);
      root = 0;
    } else {
      root = bld.build(0, (int)refs.size(), 0);
    }
    out.max_depth = std::max(out.max_depth, bld.max_depth);
    int before = (int)out.nodes.size();
    out.root[s] = flatten(bld, root, refs, in.verts, in.idx, out.nodes, out.tris, &out.stack_need);
    out.n_nodes[s] = (int)out.nodes.size() - before;
  }
}

}  // namespace sdd
