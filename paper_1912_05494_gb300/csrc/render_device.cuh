// render_device.cuh -- per-ray device functions of the wavefront path, shared by the
// host-driven kernels (render_kernels.cu) and the persistent drain kernel (persistent.cu).
//
// One generation of rays is processed by:
//   dev_traverse_warp  closest hit per subdomain queue (Sec. 3.1: the cost of ray tracing
//                 lies in the intersectors) as a warp-uniform BVH walk; a ray that leaves its
//                 slab without a hit is handed, unchanged, to the neighbouring slab's queue
//                 (Sec. 5: interface conditions keep the ray properties continuous)
//   dev_shade     per-wavelength shading: complex Fresnel, Snell, Beer-Lambert (Eq. 1),
//                 thin-slab series, Lambertian walls with a shadow ray to the sun (Eq. 3),
//                 deterministic splitting (Sec. 3.1) or Philox-driven choices (Sec. 3.2);
//                 children are compacted into the next generation and binned by subdomain
//   dev_shadow    any-hit transmittance toward the sun per subdomain queue, with hand-off
//                 (per-lane walk; dev_shadow_warp: warp-uniform, used with brute-force tiles)
// Queue appends are warp-aggregated: one atomic per distinct target queue per warp (ballot /
// match_any / popc).  Every function that appends must be called by all 32 lanes of a warp.
#pragma once

#include <math_constants.h>

#include "device_math.cuh"
#include "photon_device.cuh"
#include "render_kernels.cuh"
#include "tile_device.cuh"

namespace sdd {

namespace {

constexpr float kInvPi = 0.31830988618379067f;
constexpr int kBlock = 128;
static_assert(kBlock == kShadeThreads, "bundle shading rows are sized for kShadeThreads threads");

enum Event : uint32_t {
  EV_REFLECT = 0, EV_TRANSMIT = 1, EV_DIFFUSE = 2, EV_ABSORB = 3, EV_RR_KILL = 4,
  EV_DEPTH_CAP = 5, EV_ESCAPE = 6, EV_SHADOW_BLOCKED = 7, EV_SHADOW_OPEN = 8
};

__device__ __forceinline__ uint32_t fnv_byte(uint32_t h, uint32_t b) { return (h ^ (b & 0xFFu)) * 0x01000193u; }
__device__ __forceinline__ uint32_t fnv_word(uint32_t h, uint32_t w) {
  h = fnv_byte(h, w);
  h = fnv_byte(h, w >> 8);
  h = fnv_byte(h, w >> 16);
  return fnv_byte(h, w >> 24);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated append.  Every lane of the warp calls it (converged); lanes with `want`
// get consecutive slots of counters[key], one atomicAdd per distinct key in the warp.
__device__ __forceinline__ int warp_append(int* counters, int key, bool want) {
  unsigned act = __ballot_sync(0xffffffffu, want);
  int pos = -1;
  if (want) {
    unsigned peers = __match_any_sync(act, key);
    int leader = __ffs(peers) - 1;
    int base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&counters[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    pos = base + __popc(peers & lanemask_lt());
  }
  return pos;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int subdomain_of(const DevScene& sc, float3 o) {
  float x = comp3(o, sc.axis);
  int s = 0;
  for (int i = 1; i < sc.n_sub; ++i) s += (x >= sc.planes[i]) ? 1 : 0;
  return s;
}

// The part of the ray inside slab s: t in (t0, t1]; `next` is the slab it enters at t1
// (-1 when it leaves the outermost slab, i.e. it escapes).
__device__ __forceinline__ void slab_interval(const DevScene& sc, int s, float3 o, float3 d, float* t0, float* t1,
                                              int* next) {
  float oa = comp3(o, sc.axis), da = comp3(d, sc.axis);
  *t0 = 0.f;
  *t1 = CUDART_INF_F;
  *next = -1;
  if (da > 0.f) {
    if (s + 1 < sc.n_sub) {
      *t1 = (sc.planes[s + 1] - oa) / da;
      *next = s + 1;
    }
    if (s > 0) *t0 = fmaxf(0.f, (sc.planes[s] - oa) / da);
  } else if (da < 0.f) {
    if (s > 0) {
      *t1 = (sc.planes[s] - oa) / da;
      *next = s - 1;
    }
    if (s + 1 < sc.n_sub) *t0 = fmaxf(0.f, (sc.planes[s + 1] - oa) / da);
  }
}

// A node as one ray sees it: per axis the child planes the ray enters through (near) and
// leaves through (far), picked once per walk from the signs of its direction, so that a slab
// test takes no min / max per axis (the values equal the min / max of the two plane
// distances: t(plane) is monotonic in the plane, increasing for a positive component).
struct NodeView {
  float4 nx, fx, ny, fy, nz, fz;
  int4 link, cnt;
};
// Node fields of the near planes for the ray's octant: 1 where the direction component is
// negative (the near plane is then the upper bound).
struct Octant {
  int ox, oy, oz;
};
__device__ __forceinline__ Octant octant_of(const RayPre& rp) {
  return Octant{rp.inv.x < 0.f ? 1 : 0, rp.inv.y < 0.f ? 1 : 0, rp.inv.z < 0.f ? 1 : 0};
}

__device__ __forceinline__ NodeView load_view(const Node* __restrict__ g, const Node* s_nodes, int idx, int root,
                                              int n_staged, const Octant& o) {
  const int local = idx - root;
  NodeView v;
  if (local >= 0 && local < n_staged) {
    const float4* p = reinterpret_cast<const float4*>(s_nodes + local);
    v.nx = p[o.ox];
    v.fx = p[1 - o.ox];
    v.ny = p[2 + o.oy];
    v.fy = p[3 - o.oy];
    v.nz = p[4 + o.oz];
    v.fz = p[5 - o.oz];
    v.link = reinterpret_cast<const int4*>(p)[6];
    v.cnt = reinterpret_cast<const int4*>(p)[7];
    return v;
  }
  const float4* p = reinterpret_cast<const float4*>(g + idx);
  v.nx = __ldg(p + o.ox);
  v.fx = __ldg(p + 1 - o.ox);
  v.ny = __ldg(p + 2 + o.oy);
  v.fy = __ldg(p + 3 - o.oy);
  v.nz = __ldg(p + 4 + o.oz);
  v.fz = __ldg(p + 5 - o.oz);
  v.link = __ldg(reinterpret_cast<const int4*>(p + 6));
  v.cnt = __ldg(reinterpret_cast<const int4*>(p + 7));
  return v;
}

// Stage the first `want` nodes (the top BVH levels, stored breadth-first) of subdomain s.
__device__ __forceinline__ int stage_top(const DevScene& sc, Node* s_nodes, int s, int want) {
  constexpr int kVec = (int)(sizeof(Node) / sizeof(float4));
  int n = min(want, sc.n_nodes_sub[s]);
  const float4* src = reinterpret_cast<const float4*>(sc.nodes + sc.root[s]);
  float4* dst = reinterpret_cast<float4*>(s_nodes);
  for (int i = threadIdx.x; i < kVec * n; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  return n;
}

// Component c of a node field (c is a constant after unrolling, else a select chain).
__device__ __forceinline__ float comp4(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__device__ __forceinline__ int comp4(const int4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Slab tests of a node's children against (t0, t1]: bit c is set when child c exists and its
// box meets the interval; tn[c] is its entry distance.  The exit distance is widened by
// Ize's 1 + 2 gamma(3) so that rounding cannot produce a false miss.
__device__ __forceinline__ unsigned child_hits(const RayPre& rp, const NodeView& n, float t0, float t1,
                                               float (&tn)[kBvhWidth]) {
  unsigned m = 0u;
#pragma unroll
  for (int c = 0; c < kBvhWidth; ++c) {
    const float tnx = fmaf(comp4(n.nx, c), rp.inv.x, -rp.oinv.x), tfx = fmaf(comp4(n.fx, c), rp.inv.x, -rp.oinv.x);
    const float tny = fmaf(comp4(n.ny, c), rp.inv.y, -rp.oinv.y), tfy = fmaf(comp4(n.fy, c), rp.inv.y, -rp.oinv.y);
    const float tnz = fmaf(comp4(n.nz, c), rp.inv.z, -rp.oinv.z), tfz = fmaf(comp4(n.fz, c), rp.inv.z, -rp.oinv.z);
    const float tmin = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, t0));
    const float tmax = fminf(fminf(tfx, tfy), fminf(tfz, t1));
    tn[c] = tmin;
    if (tmin <= tmax * 1.0000004f && comp4(n.link, c) >= 0) m |= 1u << c;
  }
  return m;
}

// Children of a node that are leaves (bit c: child c holds triangle records).
__device__ __forceinline__ unsigned leaf_mask(const NodeView& n) {
  return (n.cnt.x > 0 ? 1u : 0u) | (n.cnt.y > 0 ? 2u : 0u) | (n.cnt.z > 0 ? 4u : 0u) | (n.cnt.w > 0 ? 8u : 0u);
}

__device__ __forceinline__ TileDev tile_of(const TileSetDev& ts, int t) {
  TileDev g;
  g.h = ts.heights + (size_t)t * (ts.G + 1) * (ts.G + 1);
  g.hmin = __ldg(ts.hmin + t);
  g.hmax = __ldg(ts.hmax + t);
  g.rho = __ldg(ts.rho + t);
  g.G = ts.G;
  g.L = ts.L;
  return g;
}

// Tile frame of a hit: front face on the +n side of the geometric normal, (t1, t2) its Duff
// basis, positions wrapped with the tile period.
__device__ __forceinline__ void tile_frame(float L, float3 p, float3 n, float3 d, float* x, float* y, float3* dl,
                                           float3* t1, float3* t2) {
  onb(n, t1, t2);
  float a = dot3(p, *t1), b = dot3(p, *t2);
  *x = a - L * floorf(a / L);
  *y = b - L * floorf(b / L);
  *dl = make_float3(dot3(d, *t1), dot3(d, *t2), dot3(d, n));
}

constexpr float kCos1Deg = 0.99984769515639124f;
// Node steps of one warp-uniform walk beyond which it is abandoned with the stack-overflow
// error (a walk visits each node at most once; the largest trees have ~2M nodes).
constexpr int kMaxTraversalSteps = 1 << 22;
constexpr int kTileEvents = 64;

struct ShadowKey {
  uint32_t pixel, sample, bounce;
  uint64_t seed;
  uint32_t word;  // wavelength word of the draws: the wavelength index, or its bundle's index
};

// A surface met by a shadow ray of wavelength lam at distance t: multiplies *T by its
// transmittance and returns false (thin-slab tiles; heterogeneous tiles through the network's
// table or one brute-force ray through the tile), or returns true when it blocks the ray.
// kTM: heterogeneous-tile mode of the scene: 0 none, 1 brute-force tile tracing, 2 network.
template <int kTM>
__device__ __forceinline__ bool shadow_surface(const RenderParams& p, const DevSpectral& sp, int lam, float lambda_nm,
                                               const ShadowKey& key, const RayPre& rp, float3 d, float t,
                                               uint32_t prim, float* T) {
  float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
  int mat = __float_as_int(nm.w);
  int kind = __ldg(sp.mat_kind + mat);
  size_t mi = (size_t)mat * sp.n_lambda + lam;
  if (kind == MAT_SLAB) {
    float cos_i = fabsf(dot3(d, f3(nm)));
    float Rs, Ts;
    slab_RT(cos_i, __ldg(sp.mat_n + mi), __ldg(sp.mat_k + mi), __ldg(sp.mat_thick + mat), lambda_nm, &Rs, &Ts,
            sp.slab_pol);
    *T *= Ts;
    return false;
  }
  if (kTM == 2 && kind == MAT_TILE) {
    *T *= __ldg(p.tile_sun_T + mi);  // network: transmittance x ballistic fraction
    return false;
  }
  if (kTM == 1 && kind == MAT_TILE) {
    // one brute-force ray through the tile: counts if it leaves on the far side within 1
    // degree of the shadow direction
    float x, y;
    float3 dl, t1v, t2v;
    tile_frame(p.tiles.L, rp.o + t * d, f3(nm), d, &x, &y, &dl, &t1v, &t2v);
    TileOut r = tile_trace(tile_of(p.tiles, __ldg(p.mat_tile + mat)), x, y, dl, __ldg(sp.mat_n + mi),
                           __ldg(sp.mat_k + mi), lambda_nm, key.pixel, key.sample, key.bounce, key.word, key.seed,
                           kTileEvents, STREAM_SHADOW_TILE);
    if (r.side == 1 && dot3(r.dir, dl) > kCos1Deg) {
      *T *= r.w;
      return false;
    }
  }
  return true;
}

// Any-hit walk of subdomain s's BVH over (t0, t1] for one lane: `hit(t, prim)` is called for
// every triangle the ray meets (in walk order) and returns true when that surface blocks the
// ray, which ends the walk.  Returns true when the ray was blocked.
template <bool kStats, class Hit>
__device__ __forceinline__ bool any_hit_walk(const DevScene& sc, const Node* s_nodes, int n_staged, int s,
                                             const RayPre& rp, float t0, float t1, uint32_t* n_nodes,
                                             uint32_t* n_tris, bool* overflow, Hit& hit) {
  int stack[kStackSize];
  int spn = 0;
  const int root = sc.root[s];
  int node = root;
  const Octant oct = octant_of(rp);
  for (;;) {
    const NodeView n = load_view(sc.nodes, s_nodes, node, root, n_staged, oct);
    if (kStats) ++*n_nodes;
    float tn[kBvhWidth];
    const unsigned hm = child_hits(rp, n, t0, t1, tn);
    const unsigned leaf = leaf_mask(n);
    for (unsigned lm = hm & leaf; lm; lm &= lm - 1u) {
      const int c = __ffs(lm) - 1;
      const int first = comp4(n.link, c), cnt = comp4(n.cnt, c);
      for (int i = first; i < first + cnt; ++i) {
        const float4* tp = reinterpret_cast<const float4*>(sc.tris + i);
        float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        if (kStats) ++*n_tris;
        float t = tri_hit(rp, v0, v1, v2, t0, t1);
        if (t >= 0.f && hit(t, __float_as_uint(v0.w))) return true;
      }
    }
    // entered inner children: descend into the first, push the others
    const unsigned im = hm & ~leaf;
    int next = -1;
#pragma unroll
    for (int c = 0; c < kBvhWidth; ++c) {
      if ((im >> c) & 1u) {
        const int l = comp4(n.link, c);
        if (next < 0) {
          next = l;
        } else if (spn < kStackSize) {
          stack[spn++] = l;
        } else {
          *overflow = true;
        }
      }
    }
    if (next >= 0) {
      node = next;
    } else {
      if (spn == 0) break;
      node = stack[--spn];
    }
  }
  return false;
}

// Transmittance of a shadow ray of wavelength lam across subdomain s over (t0, t1] (0 when
// blocked), as a per-lane walk.
template <bool kStats, int kTM>
__device__ __forceinline__ float shadow_T(const RenderParams& p, const DevScene& sc, const DevSpectral& sp, int lam,
                                          float lambda_nm, const ShadowKey& key, const Node* s_nodes, int n_staged,
                                          int s, const RayPre& rp, float3 d, float t0, float t1, uint32_t* n_nodes,
                                          uint32_t* n_tris, bool* overflow) {
  float T = 1.f;
  auto hit = [&](float t, uint32_t prim) {
    return shadow_surface<kTM>(p, sp, lam, lambda_nm, key, rp, d, t, prim, &T);
  };
  return any_hit_walk<kStats>(sc, s_nodes, n_staged, s, rp, t0, t1, n_nodes, n_tris, overflow, hit) ? 0.f : T;
}

// Closest hit in (t0, t1] against subdomain s's BVH as a warp-uniform walk; ties in t go to
// the lower primitive.  The lanes must enter converged (the host-driven traversal kernel,
// whose subdomain is the block's, and the persistent kernel's subdomain-aligned chunks).
// Every lane of the warp calls it (live = false for lanes without a ray).  Each iteration every lane still traversing takes one node
// step (box tests of its four children, the triangles of any leaf child, then push / pop) and
// the warp reconverges at the vote that ends the step.  A data-dependent loop per lane lets
// the warp split into groups that each iterate on their own: on incoherent rays of large
// scenes only ~3 of 32 lanes then issue together.
template <bool kStats>
__device__ __forceinline__ uint32_t closest_hit_warp(const DevScene& sc, const Node* s_nodes, int n_staged, int s,
                                                const RayPre& rp, float t0, float t1, bool live, float* t_out,
                                                uint32_t* n_nodes, uint32_t* n_tris, bool* overflow) {
  int stack[kStackSize];
  int sp = 0;
  const int root = sc.root[s];
  int node = root;
  const Octant oct = octant_of(rp);
  float tbest = t1;
  uint32_t best = kMissPrim;
  bool done = !live;
  int steps = 0;
  // One vote per step, executed by all 32 lanes at the same instruction (no lane skips to
  // it by another path): finished lanes only wait at the bottom of the loop.
  bool any = __any_sync(0xffffffffu, !done);
  while (any) {
   if (!done && ++steps > kMaxTraversalSteps) {
    *overflow = true;  // a tree walk never takes this many steps: report it and stop
    done = true;
   }
   if (!done) {
    const NodeView n = load_view(sc.nodes, s_nodes, node, root, n_staged, oct);
    if (kStats) ++*n_nodes;
    float tn[kBvhWidth];
    const unsigned hm = child_hits(rp, n, t0, tbest, tn);
    const unsigned leaf = leaf_mask(n);
    for (unsigned lm = hm & leaf; lm; lm &= lm - 1u) {
      const int c = __ffs(lm) - 1;
      const int first = comp4(n.link, c), cnt = comp4(n.cnt, c);
      for (int i = first; i < first + cnt; ++i) {
        const float4* tp = reinterpret_cast<const float4*>(sc.tris + i);
        float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        if (kStats) ++*n_tris;
        float t = tri_hit(rp, v0, v1, v2, t0, tbest);
        if (t >= 0.f) {
          uint32_t prim = __float_as_uint(v0.w);
          if (t < tbest || prim < best) {
            tbest = t;
            best = prim;
          }
        }
      }
    }
    // entered inner children, nearest first; one whose box is entered beyond the closest hit
    // found in this step cannot hold a closer one (same slack as the box test)
    const unsigned im = hm & ~leaf;
    const float cut = tbest * 1.0000004f;
    float k[kBvhWidth];
    int l[kBvhWidth];
#pragma unroll
    for (int c = 0; c < kBvhWidth; ++c) {
      k[c] = (((im >> c) & 1u) && tn[c] <= cut) ? tn[c] : CUDART_INF_F;
      l[c] = comp4(n.link, c);
    }
    auto order = [&](int a, int b) {
      if (k[b] < k[a]) {
        const float tk = k[a];
        k[a] = k[b];
        k[b] = tk;
        const int tl = l[a];
        l[a] = l[b];
        l[b] = tl;
      }
    };
    order(0, 1);
    order(2, 3);
    order(0, 2);
    order(1, 3);
    order(1, 2);
    if (k[0] < CUDART_INF_F) {
      node = l[0];
#pragma unroll
      for (int c = kBvhWidth - 1; c >= 1; --c) {
        if (k[c] < CUDART_INF_F) {
          if (sp < kStackSize) stack[sp++] = l[c];
          else *overflow = true;
        }
      }
    } else if (sp == 0) {
      done = true;
    } else {
      node = stack[--sp];
    }
   }
    any = __any_sync(0xffffffffu, !done);
  }
  *t_out = tbest;
  return best;
}

// any_hit_walk as a warp-uniform walk (see closest_hit_warp); every lane of the warp calls it
// (live = false for lanes without a ray).  A walk that exceeds kMaxTraversalSteps raises
// *overflow and counts as blocked.
template <bool kStats, class Hit>
__device__ __forceinline__ bool any_hit_walk_warp(const DevScene& sc, const Node* s_nodes, int n_staged, int s,
                                                  const RayPre& rp, float t0, float t1, bool live, uint32_t* n_nodes,
                                                  uint32_t* n_tris, bool* overflow, Hit& hit) {
  int stack[kStackSize];
  int spn = 0;
  const int root = sc.root[s];
  int node = root;
  const Octant oct = octant_of(rp);
  bool done = !live, res = false;
  int steps = 0;
  bool any = __any_sync(0xffffffffu, !done);
  while (any) {
   if (!done && ++steps > kMaxTraversalSteps) {
    *overflow = true;
    res = true;
    done = true;
   }
   if (!done) {
    const NodeView n = load_view(sc.nodes, s_nodes, node, root, n_staged, oct);
    if (kStats) ++*n_nodes;
    float tn[kBvhWidth];
    const unsigned hm = child_hits(rp, n, t0, t1, tn);
    const unsigned leaf = leaf_mask(n);
    bool blocked = false;
    for (unsigned lm = hm & leaf; lm && !blocked; lm &= lm - 1u) {
      const int c = __ffs(lm) - 1;
      const int first = comp4(n.link, c), cnt = comp4(n.cnt, c);
      for (int i = first; i < first + cnt && !blocked; ++i) {
        const float4* tp = reinterpret_cast<const float4*>(sc.tris + i);
        float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        if (kStats) ++*n_tris;
        float t = tri_hit(rp, v0, v1, v2, t0, t1);
        if (t >= 0.f) blocked = hit(t, __float_as_uint(v0.w));
      }
    }
    const unsigned im = hm & ~leaf;
    int next = -1;
    if (!blocked) {
#pragma unroll
      for (int c = 0; c < kBvhWidth; ++c) {
        if ((im >> c) & 1u) {
          const int l = comp4(n.link, c);
          if (next < 0) {
            next = l;
          } else if (spn < kStackSize) {
            stack[spn++] = l;
          } else {
            *overflow = true;
          }
        }
      }
    }
    if (blocked) {
      res = true;
      done = true;
    } else if (next >= 0) {
      node = next;
    } else if (spn == 0) {
      done = true;
    } else {
      node = stack[--spn];
    }
   }
    any = __any_sync(0xffffffffu, !done);
  }
  return res;
}

// shadow_T as a warp-uniform walk; every lane of the warp calls it.
template <bool kStats, int kTM>
__device__ __forceinline__ float shadow_T_warp(const RenderParams& p, const DevScene& sc, const DevSpectral& sp, int lam,
                                          float lambda_nm, const ShadowKey& key, const Node* s_nodes, int n_staged,
                                          int s, const RayPre& rp, float3 d, float t0, float t1, bool live,
                                          uint32_t* n_nodes, uint32_t* n_tris, bool* overflow) {
  float T = 1.f;
  auto hit = [&](float t, uint32_t prim) {
    return shadow_surface<kTM>(p, sp, lam, lambda_nm, key, rp, d, t, prim, &T);
  };
  return any_hit_walk_warp<kStats>(sc, s_nodes, n_staged, s, rp, t0, t1, live, n_nodes, n_tris, overflow, hit) ? 0.f
                                                                                                                : T;
}

__device__ __forceinline__ float3 offset_point(float3 p, float3 ng, float3 dir, float eps) {
  return dot3(dir, ng) >= 0.f ? p + eps * ng : p - eps * ng;
}
__device__ __forceinline__ float seg0_of(float3 ng, float3 dir, float eps) {
  return eps / fmaxf(fabsf(dot3(ng, dir)), 1e-6f);
}
__device__ __forceinline__ float3 reflect3(float3 d, float3 n) { return d - (2.f * dot3(d, n)) * n; }

struct PathId {
  uint32_t sample, cell, px_i, lam, pixel;
};
__device__ __forceinline__ PathId path_id(const RenderParams& p, const WaveDesc& w, uint32_t path) {
  PathId r;
  uint32_t ls = path / w.nc;
  uint32_t lc = path - ls * w.nc;
  r.sample = w.s0 + ls;
  r.cell = w.c0 + lc;
  r.px_i = r.cell / (uint32_t)p.sp.n_lambda;
  r.lam = r.cell - r.px_i * (uint32_t)p.sp.n_lambda;
  r.pixel = p.pixel_list ? (uint32_t)p.pixel_list[r.px_i] : r.px_i;
  return r;
}

__device__ __forceinline__ float escape_radiance(const DevSpectral& sp, float3 d, int lam, bool sun_counted) {
  float L = (sp.sky_mode == 0 || d.z > 0.f) ? __ldg(sp.sky + lam) : 0.f;
  if (!sun_counted && sp.sun_h > 0.f) {
    float3 c = d - sp.sun_dir;
    if (dot3(c, c) <= 2.f * sp.sun_h) L += __ldg(sp.sun + lam);
  }
  return L;
}

// Append a ray to the next generation and bin it by the subdomain of its origin.
__device__ __forceinline__ void emit_ray(bool want, const DevScene& sc, RayBuf nb, int* next_count, uint32_t* q,
                                         int* q_count, int qcap, float3 o, float seg0, float3 d, float thr,
                                         uint32_t path, uint32_t meta, Control* ctl) {
  int pos = warp_append(next_count, 0, want);
  bool ok = want && pos < nb.cap;
  if (want && !ok) atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  if (ok) {
    nb.o[pos] = make_float4(o.x, o.y, o.z, seg0);
    nb.d[pos] = make_float4(d.x, d.y, d.z, thr);
    nb.info[pos] = make_uint2(path, meta);
  }
  int s = ok ? subdomain_of(sc, o) : 0;
  int qpos = warp_append(q_count, s, ok);
  if (ok) {
    if (qpos < qcap) q[(size_t)s * qcap + qpos] = (uint32_t)pos;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
}

}  // namespace

// ------------------------------------------------------------------------------ raygen
// Camera ray through pixel `pixel` offset by (xi, yi) pixels from its centre.
__device__ __forceinline__ void primary_ray(const RenderParams& p, uint32_t pixel, float xi, float yi, float3* o,
                                            float3* d) {
  int px = (int)(pixel % (uint32_t)p.cam.width), py = (int)(pixel / (uint32_t)p.cam.width);
  float sx = ((px + 0.5f + xi) / p.cam.width) * 2.f - 1.f;
  float sy = 1.f - ((py + 0.5f + yi) / p.cam.height) * 2.f;
  if (p.cam.ortho) {
    *o = p.cam.pos + (sx * p.cam.ortho_half * p.cam.aspect) * p.cam.right + (sy * p.cam.ortho_half) * p.cam.up;
    *d = p.cam.fwd;
  } else {
    *o = p.cam.pos;
    *d = normalize3(p.cam.fwd + (sx * p.cam.tan_half * p.cam.aspect) * p.cam.right + (sy * p.cam.tan_half) * p.cam.up);
  }
}

// One primary ray per wave-local path i (every lane of the warp calls this).
__device__ __forceinline__ void dev_raygen(const RenderParams& p, const WaveDesc& w, uint32_t i, bool active,
                                           RayBuf rb, uint32_t* q, int* q_count, int qcap, Control* ctl) {
  float3 o = make_float3(0.f, 0.f, 0.f), d = o;
  if (active) {
    PathId id = path_id(p, w, i);
    float xi = 0.f, yi = 0.f;
    if (p.mode == 1) {
      float4 u = draw4(id.pixel, id.sample, 0, STREAM_PATH, 0, id.lam, p.seed);
      xi = u.x - 0.5f;
      yi = u.y - 0.5f;
    }
    primary_ray(p, id.pixel, xi, yi, &o, &d);
    rb.o[i] = make_float4(o.x, o.y, o.z, 0.f);
    rb.d[i] = make_float4(d.x, d.y, d.z, 1.f);
    rb.info[i] = make_uint2(i, (1u << 16));  // depth 0, no flags, tree code 1
    if (p.path_hash) p.path_hash[i] = 0x811C9DC5u;
  }
  int s = active ? subdomain_of(p.sc, o) : 0;
  int pos = warp_append(q_count, s, active);
  if (active) {
    if (pos < qcap) q[(size_t)s * qcap + pos] = i;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
}


// ------------------------------------------------------------------------------ traverse
// Closest hit of queue entry i of subdomain s (every lane of the warp calls this, the lanes
// converged): writes the hit record, or hands the ray to the neighbouring subdomain's queue.
template <bool kStats>
__device__ __forceinline__ void dev_traverse_warp(const RenderParams& p, int s, int i, bool active, const Node* s_nodes,
                                             int n_staged, QueuePair qp, RayBuf rb, float2* hits, Control* ctl) {
  uint32_t r = active ? qp.in[(size_t)s * qp.cap + i] : 0u;
  bool cross = false;
  int next = -1;
  uint32_t nn = 0, nt = 0;
  float t0 = 0.f, t1 = 0.f;
  float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
  if (active) {
    float4 O = rb.o[r], D = rb.d[r];
    o = f3(O);
    d = f3(D);
    slab_interval(p.sc, s, o, d, &t0, &t1, &next);
  }
  const bool live = active && t1 > t0;
  float t = t1;
  bool ovf = false;
  const RayPre rp = ray_pre(o, d);
  const uint32_t prim = closest_hit_warp<kStats>(p.sc, s_nodes, n_staged, s, rp, t0, t1, live, &t, &nn, &nt, &ovf);
  if (active) {
    if (ovf) atomicOr(&ctl->error, ERR_STACK_OVERFLOW);
    cross = prim == kMissPrim && next >= 0;
    if (!cross) hits[r] = make_float2(prim == kMissPrim ? CUDART_INF_F : t, __uint_as_float(prim));
  }
  int pos = warp_append(qp.out_count, cross ? next : 0, cross);
  if (cross) {
    if (pos < qp.cap) qp.out[(size_t)next * qp.cap + pos] = r;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
  if (kStats) {
    unsigned long long a = warp_sum<unsigned long long>(active ? 1ull : 0ull);
    unsigned long long c = warp_sum<unsigned long long>(cross ? 1ull : 0ull);
    unsigned long long n1 = warp_sum<unsigned long long>(nn);
    unsigned long long n2 = warp_sum<unsigned long long>(nt);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctl->rays_closest, a);
      atomicAdd(&ctl->crossings, c);
      atomicAdd(&ctl->node_visits, n1);
      atomicAdd(&ctl->tri_tests, n2);
    }
  }
}


// ------------------------------------------------------------------------------ shade
// Shade ray r of the current generation (every lane of the warp calls this): adds escape
// and NEE radiance, appends the children to `next` (counter *next_count) and the subdomain
// queues q, and the shadow ray to sb (counter *shadow_count) and the shadow queues sq.
// kPM: with photon maps (Sec. 3.2) the first diffuse vertex of a path adds albedo / pi times
// the maps' caustic and indirect irradiance beside its sun NEE; after it the path carries
// FLAG_PHOTON_DONE and takes sky light only (no NEE, no sun disc on escape).
template <int kTM, bool kPM = false>
__device__ __forceinline__ void dev_shade(const RenderParams& p, const WaveDesc& w, int r, bool active, RayBuf cur,
                                          const float2* __restrict__ hits, RayBuf next, int* next_count, uint32_t* q,
                                          int* q_count, int qcap, ShadowBuf sb, int* shadow_count, uint32_t* sq,
                                          int* sq_count, float* path_L, Control* ctl) {
  const bool mc = p.mode == 1;
  const float eps = p.sc.eps;
  bool e0 = false, e1 = false, esh = false;
  float3 o0 = make_float3(0.f, 0.f, 0.f), d0 = o0, o1 = o0, d1 = o0, osh = o0, dsh = o0;
  float thr0 = 0.f, thr1 = 0.f, s00 = 0.f, s01 = 0.f, csh = 0.f;
  uint32_t meta0 = 0, meta1 = 0, path = 0, slot_sh = 0, bounce_sh = 0;
  bool tile_q = false;  // tile hit deferred to the BTDF network
  if (active) {
    float4 O = cur.o[r], D = cur.d[r];
    uint2 inf = cur.info[r];
    float2 H = hits[r];
    path = inf.x;
    uint32_t depth = inf.y & 0xFFu, flags = (inf.y >> 8) & 0xFFu, code = inf.y >> 16;
    float thr = D.w, seg0 = O.w;
    float3 o = f3(O), d = f3(D);
    PathId id = path_id(p, w, path);
    const int lam = (int)id.lam;
    const float lambda = __ldg(p.sp.lambda_nm + lam);
    const uint32_t slot = path * (uint32_t)p.n_slots + (mc ? 0u : code);
    uint32_t hsh = p.path_hash ? p.path_hash[path] : 0u;
    uint32_t prim = __float_as_uint(H.y);
    if (prim != kMissPrim && prim >= (uint32_t)p.sc.n_prims) {
      // a ray dropped by a full queue was never traced and its hit record is stale: the frame
      // already carries the overflow error; nothing is read through the stale index
      atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
    } else if (prim == kMissPrim) {
      path_L[slot] += thr * escape_radiance(p.sp, d, lam, (flags & (FLAG_SUN_COUNTED | FLAG_PHOTON_DONE)) != 0u);
      hsh = fnv_byte(fnv_word(hsh, 0xFFFFFFFFu), EV_ESCAPE);
    } else {
      hsh = fnv_word(hsh, prim);
      uint32_t v = depth + 1;
      if ((int)v > p.max_depth) {
        hsh = fnv_byte(hsh, EV_DEPTH_CAP);
      } else {
        float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
        float3 ng = f3(nm);
        int mat = __float_as_int(nm.w);
        int kind = __ldg(p.sp.mat_kind + mat);
        size_t mi = (size_t)mat * p.sp.n_lambda + lam;
        float3 pt = o + H.x * d;
        float cos_n = dot3(d, ng);
        float3 nf = cos_n < 0.f ? ng : -1.f * ng;
        float cos_i = fabsf(cos_n);
        float4 u = mc ? draw4(id.pixel, id.sample, v, STREAM_PATH, 0, lam, p.seed) : make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t base_meta = v;  // depth v, flags and code filled per child
        if (kind == MAT_SOLID) {
          bool inside = cos_n > 0.f;
          float nre = __ldg(p.sp.mat_n + mi), kk = __ldg(p.sp.mat_k + mi);
          if (inside) thr *= beer_lambert(kk, H.x + seg0, lambda);
          float n1 = inside ? nre : 1.f;
          float n2re = inside ? 1.f : nre, n2im = inside ? 0.f : kk;
          float R = fresnel_R(cos_i, n1, n2re, n2im);
          float eta = n1 / n2re;
          float c2 = 1.f - eta * eta * (1.f - cos_i * cos_i);
          float3 dr = reflect3(d, nf);
          float3 dt = c2 > 0.f ? normalize3(eta * d + (eta * cos_i - sqrtf(c2)) * nf) : dr;
          uint32_t fl = flags & ~FLAG_SUN_COUNTED;
          if (!mc) {
            e0 = true;
            d0 = dr;
            thr0 = thr * R;
            meta0 = base_meta | (fl << 8) | ((code * 2u) << 16);
            e1 = c2 > 0.f && R < 1.f;
            d1 = dt;
            thr1 = thr * (1.f - R);
            meta1 = base_meta | (fl << 8) | ((code * 2u + 1u) << 16);
          } else {
            bool refl = u.x < R || c2 <= 0.f;
            hsh = fnv_byte(hsh, refl ? EV_REFLECT : EV_TRANSMIT);
            e0 = true;
            d0 = refl ? dr : dt;
            thr0 = thr;
            meta0 = base_meta | (fl << 8);
          }
        } else if (kind == MAT_SLAB) {
          float Rs, Ts;
          slab_RT(cos_i, __ldg(p.sp.mat_n + mi), __ldg(p.sp.mat_k + mi), __ldg(p.sp.mat_thick + mat), lambda, &Rs,
                  &Ts, p.sp.slab_pol);
          float3 dr = reflect3(d, nf);
          uint32_t fl_r = flags & ~FLAG_SUN_COUNTED;
          if (!mc) {
            e0 = true;
            d0 = dr;
            thr0 = thr * Rs;
            meta0 = base_meta | (fl_r << 8) | ((code * 2u) << 16);
            e1 = true;
            d1 = d;
            thr1 = thr * Ts;
            meta1 = base_meta | (flags << 8) | ((code * 2u + 1u) << 16);
          } else {
            float P = Rs / (Rs + Ts);
            bool refl = u.x < P;
            hsh = fnv_byte(hsh, refl ? EV_REFLECT : EV_TRANSMIT);
            e0 = true;
            d0 = refl ? dr : d;
            thr0 = thr * (Rs + Ts);
            meta0 = base_meta | ((refl ? fl_r : flags) << 8);
          }
        } else if (kind == MAT_DIFFUSE) {
          float alb = __ldg(p.sp.mat_albedo + mi);
          if (mc) hsh = fnv_byte(hsh, EV_DIFFUSE);
          const bool photon_done = kPM && (flags & FLAG_PHOTON_DONE) != 0u;
          if (kPM && !photon_done) {
            const float2 E = photon_irradiance(p.pm, pt, nf, lam);
            path_L[slot] += thr * alb * kInvPi * (E.x + E.y);
          }
          if (p.sp.sun_h > 0.f && !photon_done) {
            float3 wl = p.sp.sun_dir;
            if (mc) {
              float4 un = draw4(id.pixel, id.sample, v, STREAM_NEE, 0, lam, p.seed);
              wl = cone_dir(p.sp.sun_dir, p.sp.sun_h, un.x, un.y);
            }
            float cl = dot3(nf, wl);
            if (cl > 0.f) {
              esh = true;
              osh = offset_point(pt, ng, wl, eps);
              dsh = wl;
              csh = thr * alb * kInvPi * cl * __ldg(p.sp.sun + lam) * p.sp.sun_omega;
              slot_sh = mc ? 0u : code;
              bounce_sh = v;
            }
          }
          if (mc) {
            e0 = true;
            d0 = cosine_dir(nf, u.y, u.z);
            thr0 = thr * alb;
            meta0 = base_meta | ((flags | FLAG_SUN_COUNTED | (kPM ? FLAG_PHOTON_DONE : 0u)) << 8);
          }
        } else if (kTM == 1 && kind == MAT_TILE && mc) {
          // heterogeneous tile: one brute-force ray through it on the tile stream
          float x, y;
          float3 dl, t1v, t2v;
          tile_frame(p.tiles.L, pt, ng, d, &x, &y, &dl, &t1v, &t2v);
          TileOut r = tile_trace(tile_of(p.tiles, __ldg(p.mat_tile + mat)), x, y, dl, __ldg(p.sp.mat_n + mi),
                                 __ldg(p.sp.mat_k + mi), lambda, id.pixel, id.sample, v, lam, p.seed, kTileEvents,
                                 STREAM_TILE);
          if (r.side == 2) {
            hsh = fnv_byte(hsh, EV_ABSORB);
          } else {
            hsh = fnv_byte(hsh, r.side == 0 ? EV_REFLECT : EV_TRANSMIT);
            e0 = true;
            d0 = normalize3(r.dir.x * t1v + r.dir.y * t2v + r.dir.z * ng);
            thr0 = thr * r.w;
            bool keep = r.side == 1 && dot3(r.dir, dl) > kCos1Deg;
            meta0 = base_meta | ((keep ? flags : (flags & ~FLAG_SUN_COUNTED)) << 8);
          }
        } else if (kTM == 2 && kind == MAT_TILE && mc) {
          tile_q = true;  // surrogate form: shaded after the network has run on all tile hits
        } else {
          if (mc) hsh = fnv_byte(hsh, EV_ABSORB);
        }
        if (mc && e0 && (int)v >= p.rr_start) {
          float qs = fminf(0.95f, thr0);
          if (u.w >= qs) {
            e0 = false;
            hsh = fnv_byte(hsh, EV_RR_KILL);
          } else {
            thr0 = thr0 / qs;
          }
        }
        if (e0) {
          o0 = offset_point(pt, ng, d0, eps);
          s00 = seg0_of(ng, d0, eps);
        }
        if (e1) {
          o1 = offset_point(pt, ng, d1, eps);
          s01 = seg0_of(ng, d1, eps);
        }
      }
    }
    if (p.path_hash) p.path_hash[path] = hsh;
  }
  emit_ray(e0, p.sc, next, next_count, q, q_count, qcap, o0, s00, d0, thr0, path, meta0, ctl);
  emit_ray(e1, p.sc, next, next_count, q, q_count, qcap, o1, s01, d1, thr1, path, meta1, ctl);
  // shadow ray toward the sun
  int pos = warp_append(shadow_count, 0, esh);
  bool ok = esh && pos < sb.cap;
  if (esh && !ok) atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  if (ok) {
    sb.o[pos] = make_float4(osh.x, osh.y, osh.z, 0.f);
    sb.d[pos] = make_float4(dsh.x, dsh.y, dsh.z, csh);
    sb.info[pos] = make_uint2(path, slot_sh | (bounce_sh << 16));
  }
  int ss = ok ? subdomain_of(p.sc, osh) : 0;
  int qpos = warp_append(sq_count, ss, ok);
  if (ok) {
    if (qpos < qcap) sq[(size_t)ss * qcap + qpos] = (uint32_t)pos;
    else atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  }
  if (kTM == 2) {
    int tpos = warp_append(p.tile_count, 0, tile_q);
    if (tile_q) {
      if (tpos < p.tile_cap) p.tile_queue[tpos] = (uint32_t)r;
      else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
    }
  }
}


// ------------------------------------------------------------------------------ shadow
// Transmittance of shadow-queue entry i of subdomain s toward the sun (every lane of the
// warp calls this): blocked, handed on to the neighbouring subdomain, or added to its path.
template <bool kStats, int kTM>
__device__ __forceinline__ void dev_shadow(const RenderParams& p, const WaveDesc& w, int s, int i, bool active,
                                           const Node* s_nodes, int n_staged, QueuePair qp, ShadowBuf sb,
                                           float* path_L, Control* ctl) {
  uint32_t r = active ? qp.in[(size_t)s * qp.cap + i] : 0u;
  bool cross = false;
  int next = -1;
  uint32_t nn = 0, nt = 0;
  if (active) {
    float4 O = sb.o[r], D = sb.d[r];
    uint2 inf = sb.info[r];
    float3 o = f3(O), d = f3(D);
    PathId id = path_id(p, w, inf.x);
    float t0, t1;
    slab_interval(p.sc, s, o, d, &t0, &t1, &next);
    float T = 1.f;
    bool ovf = false;
    if (t1 > t0) {
      RayPre rp = ray_pre(o, d);
      ShadowKey key{id.pixel, id.sample, inf.y >> 16, p.seed, id.lam};
      T = shadow_T<kStats, kTM>(p, p.sc, p.sp, (int)id.lam, __ldg(p.sp.lambda_nm + id.lam), key, s_nodes, n_staged, s, rp,
                           d, t0, t1, &nn, &nt, &ovf);
    }
    if (ovf) atomicOr(&ctl->error, ERR_STACK_OVERFLOW);
    bool blocked = !(T > 0.f);
    float contrib = D.w * T;
    cross = !blocked && next >= 0;
    if (cross) {
      sb.d[r].w = contrib;
    } else {
      if (!blocked) path_L[inf.x * (uint32_t)p.n_slots + (inf.y & 0xFFFFu)] += contrib;
      if (p.path_hash && p.mode == 1)
        p.path_hash[inf.x] = fnv_byte(p.path_hash[inf.x], blocked ? EV_SHADOW_BLOCKED : EV_SHADOW_OPEN);
    }
  }
  int pos = warp_append(qp.out_count, cross ? next : 0, cross);
  if (cross) {
    if (pos < qp.cap) qp.out[(size_t)next * qp.cap + pos] = r;
    else atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  }
  if (kStats) {
    unsigned long long a = warp_sum<unsigned long long>(active ? 1ull : 0ull);
    unsigned long long n1 = warp_sum<unsigned long long>(nn);
    unsigned long long n2 = warp_sum<unsigned long long>(nt);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctl->rays_shadow, a);
      atomicAdd(&ctl->shadow_node_visits, n1);
      atomicAdd(&ctl->shadow_tri_tests, n2);
    }
  }
}


// dev_shadow with the warp-uniform walk (host-driven shadow kernel).
template <bool kStats, int kTM>
__device__ __forceinline__ void dev_shadow_warp(const RenderParams& p, const WaveDesc& w, int s, int i, bool active,
                                           const Node* s_nodes, int n_staged, QueuePair qp, ShadowBuf sb,
                                           float* path_L, Control* ctl) {
  uint32_t r = active ? qp.in[(size_t)s * qp.cap + i] : 0u;
  bool cross = false;
  int next = -1;
  uint32_t nn = 0, nt = 0;
  float4 O = make_float4(0.f, 0.f, 0.f, 0.f), D = make_float4(0.f, 0.f, 1.f, 0.f);
  uint2 inf = make_uint2(0u, 0u);
  float t0 = 0.f, t1 = 0.f;
  if (active) {
    O = sb.o[r];
    D = sb.d[r];
    inf = sb.info[r];
    slab_interval(p.sc, s, f3(O), f3(D), &t0, &t1, &next);
  }
  const float3 o = f3(O), d = f3(D);
  const PathId id = path_id(p, w, inf.x);
  const ShadowKey key{id.pixel, id.sample, inf.y >> 16, p.seed, id.lam};
  const bool live = active && t1 > t0;
  bool ovf = false;
  const RayPre rp = ray_pre(o, d);
  const float T = shadow_T_warp<kStats, kTM>(p, p.sc, p.sp, (int)id.lam, __ldg(p.sp.lambda_nm + id.lam), key,
                                             s_nodes, n_staged, s, rp, d, t0, t1, live, &nn, &nt, &ovf);
  if (active) {
    if (ovf) atomicOr(&ctl->error, ERR_STACK_OVERFLOW);
    bool blocked = !(T > 0.f);
    float contrib = D.w * T;
    cross = !blocked && next >= 0;
    if (cross) {
      sb.d[r].w = contrib;
    } else {
      if (!blocked) path_L[inf.x * (uint32_t)p.n_slots + (inf.y & 0xFFFFu)] += contrib;
      if (p.path_hash && p.mode == 1)
        p.path_hash[inf.x] = fnv_byte(p.path_hash[inf.x], blocked ? EV_SHADOW_BLOCKED : EV_SHADOW_OPEN);
    }
  }
  int pos = warp_append(qp.out_count, cross ? next : 0, cross);
  if (cross) {
    if (pos < qp.cap) qp.out[(size_t)next * qp.cap + pos] = r;
    else atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  }
  if (kStats) {
    unsigned long long a = warp_sum<unsigned long long>(active ? 1ull : 0ull);
    unsigned long long n1 = warp_sum<unsigned long long>(nn);
    unsigned long long n2 = warp_sum<unsigned long long>(nt);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctl->rays_shadow, a);
      atomicAdd(&ctl->shadow_node_visits, n1);
      atomicAdd(&ctl->shadow_tri_tests, n2);
    }
  }
}

}  // namespace sdd
