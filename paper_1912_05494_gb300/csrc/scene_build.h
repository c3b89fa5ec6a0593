// scene_build.h -- host-side subdomain split and BVH construction (see scene_build.cpp).
#pragma once

#include <stdint.h>

#include <vector>

#include "sdd_internal.h"

namespace sdd {

struct BuildInput {
  const float* verts;
  const uint32_t* idx;
  int n_tris;
  int n_sub;
  int axis;
  float planes[kMaxSubdomains + 1];
  float slop;  // references extend this far past each slab boundary
};

struct HostBVH {
  std::vector<Node> nodes;  // every subdomain's BVH, concatenated, absolute links
  std::vector<TriRec> tris; // triangle records referenced by the leaves
  std::vector<int> root, n_nodes;
  int max_depth = 0;   // binary levels before the collapse to 4-wide nodes
  int stack_need = 0;  // deepest traversal stack a walk of any subdomain's tree can need
  int64_t n_refs = 0;
};

void build_scene_bvh(const BuildInput& in, HostBVH& out);

}  // namespace sdd
