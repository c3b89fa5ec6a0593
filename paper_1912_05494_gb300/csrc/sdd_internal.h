// sdd_internal.h -- device-side data layout shared by the host driver and the kernels of
// libsdd.  Nothing here is part of the public C ABI (include/sdd.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tileset.h"

namespace sdd {

constexpr int kMaxSubdomains = 64;
constexpr int kMaxBundle = 64;            // wavelengths per spectral bundle (member mask bits)
constexpr int kBvhWidth = 4;              // children per BVH node
constexpr int kStackSize = 64;            // BVH traversal stack entries per ray
constexpr uint32_t kMissPrim = 0xFFFFFFFFu;

enum MatKind : int { MAT_SOLID = 0, MAT_SLAB = 1, MAT_TILE = 2, MAT_DIFFUSE = 3, MAT_OPAQUE = 4 };

// Error bits raised by kernels into Control::error.
enum ErrBits : uint32_t {
  ERR_QUEUE_OVERFLOW = 1u,
  ERR_STACK_OVERFLOW = 2u,
  ERR_TIMEOUT = 4u,
  ERR_SHADOW_OVERFLOW = 8u,
};

// BVH node, 128 bytes (one L1 line): the bounds of up to four children as structure of
// arrays (child c in component c) and their links, as int bits:
//   cnt[c] > 0  -> leaf: triangle records [link[c], link[c] + cnt[c])
//   cnt[c] == 0 -> inner node index link[c] (absolute), or no child when link[c] < 0
struct alignas(16) Node {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 link, cnt;
};
static_assert(sizeof(Node) == 128, "a BVH node fills one 128-byte line");

// Triangle record, 48 bytes: the three vertices; v0.w holds the global primitive id bits.
struct alignas(16) TriRec {
  float4 v0, v1, v2;
};

// Everything the kernels read about the scene (device pointers).
struct DevScene {
  const Node* nodes;
  const TriRec* tris;
  const float4* prim_nrm_mat;   // per global primitive: unit normal xyz, material id in w bits
  int n_prims;
  int n_sub;
  int axis;
  float planes[kMaxSubdomains + 1];  // slab boundaries (planes[0] = -inf, planes[n_sub] = +inf)
  int root[kMaxSubdomains];          // root node of each subdomain's BVH
  int n_nodes_sub[kMaxSubdomains];   // nodes of each subdomain's BVH (BFS order from root)
  float eps;                         // spawn offset along the normal
};

// Per-render spectral tables (device pointers) and illuminant.
struct DevSpectral {
  int n_lambda;
  const float* lambda_nm;    // [L]
  const int* mat_kind;       // [M]
  const float* mat_thick;    // [M]
  const float* mat_n;        // [M][L]
  const float* mat_k;        // [M][L]
  const float* mat_albedo;   // [M][L]
  const float* sky;          // [L]
  const float* sun;          // [L]
  int sky_mode;
  float3 sun_dir;
  float sun_h;               // 1 - cos(half angle); 0 = no sun
  float sun_omega;           // solid angle of the disc
  int slab_pol;              // thin-slab series: 0 on the unpolarised R, 1 per polarisation
};

struct DevCamera {
  float3 pos, fwd, right, up;
  float tan_half, aspect, ortho_half;
  int width, height, ortho;
};

// Threads per block of the shading kernels (host-driven, graph form and persistent).
constexpr int kShadeThreads = 128;
// Dynamic shared memory of a kernel that shades spectral-bundle rays: per thread a row of its
// ray's B member throughputs and a staging row of B child values.
inline size_t bundle_shade_smem(int bundle) {
  return bundle > 1 ? 2u * (size_t)kShadeThreads * (size_t)bundle * sizeof(float) : 0u;
}
// Lets kernel fn take `bytes` of dynamic shared memory (above 48 KB a kernel must opt in).
inline cudaError_t allow_dynamic_smem(const void* fn, size_t bytes) {
  return bytes > 48u * 1024u ? cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                             : cudaSuccess;
}

// Ray state, structure of arrays with capacity `cap`.
struct RayBuf {
  float4* o;      // origin xyz, w = seg0 (distance back to the previous surface plane)
  float4* d;      // direction xyz, w = throughput (unused with spectral bundles)
  uint2* info;    // x = wave-local path id, y = depth(8) | flags(8) << 8 | code(16) << 16
                  // (the code is unused with spectral bundles)
  int cap;
  float* w;       // spectral bundles: per-member throughput [cap][bundle], else unused
  unsigned long long* m;  // spectral bundles: the members that follow the ray [cap], else unused
};

struct ShadowBuf {
  float4* o;      // origin xyz, w unused
  float4* d;      // direction xyz, w = contribution carried so far (unused with bundles)
  uint2* info;    // x = wave-local path id, y = contribution slot (deterministic mode, low 16
                  // bits) | bounce of the vertex that cast it << 16
  int cap;
  float* c;       // spectral bundles: per-member contribution [cap][bundle], else unused
  unsigned long long* m;  // spectral bundles: the members still carried [cap], else unused
};

// Device control block: queue counters and error word, read back by the host.
struct Control {
  int q_count[2][kMaxSubdomains];       // closest-hit queues (current / crossing)
  int sq_count[2][kMaxSubdomains];      // shadow queues
  int next_rays;                        // rays written into the next generation buffer
  int next_shadow;                      // shadow rays written this generation
  uint32_t error;
  int tile_hits;                        // tile hits queued for the network this generation
  int gen_rays[2];                      // graph form: rays of the current / next generation
  int loop_iter;                        // graph form: iterations of the running pass loop
  int work[2];                          // graph form: chunk counters of a loop's two passes
  unsigned long long node_visits, tri_tests, shadow_node_visits, shadow_tri_tests;
  unsigned long long rays_closest, rays_shadow, crossings;
  unsigned long long tile_shaded;       // tile hits shaded by the network (profiling level >= 2)
  unsigned long long graph_passes[2];   // graph form: closest-hit / shadow pass launches
};

// Ray flags: the sun's direct light was counted by a diffuse vertex's NEE; with photon maps,
// the sun's light was taken from the maps at a diffuse vertex (later vertices: sky only).
enum RayFlags : uint32_t { FLAG_SUN_COUNTED = 1u, FLAG_PHOTON_DONE = 2u };

// Photon maps on the device (Sec. 3.2): per map (0 caustic, 1 global) the stored photons
// sorted into the buckets of a hashed uniform grid of cell edge 2 r.
struct PhotonMapDev {
  const float4* pos_pw[2];        // position xyz, power
  const float4* nrm_lam[2];       // normal facing the photon's arrival xyz, wavelength index (int bits)
  const uint32_t* start[2];       // [table + 1] first photon of each bucket
  uint32_t mask;                  // table size - 1 (a power of two)
  float inv_cell, radius;        // 1 / cell edge (cell edge 2 r), gather radius
};

struct WaveDesc {
  uint32_t s0, ns;        // samples [s0, s0 + ns)
  uint32_t c0, nc;        // cells [c0, c0 + nc) with cell = pixel_index * L + lambda, or with
                          // spectral bundles cell = pixel_index * n_bundles + bundle
  uint32_t n_paths;       // ns * nc
};

struct RenderParams {
  DevScene sc;
  DevSpectral sp;
  DevCamera cam;
  const int32_t* pixel_list;   // device, or nullptr for all pixels
  int n_px;
  int spp;
  uint64_t seed;
  int max_depth;
  int mode;                    // 0 deterministic, 1 Monte Carlo
  int rr_start;
  int n_slots;                 // contribution slots per path (deterministic: 2^(max_depth+1))
  int stats;                   // profiling level
  uint32_t* path_hash;         // wave-local hash per path or nullptr
  // heterogeneous tiles
  TileSetDev tiles;            // tile set (heights, ranges, densities), or n_tiles = 0
  const int* mat_tile;         // [M] tile index of HETERO_TILE materials, -1 otherwise
  int use_surrogate;           // 1: tile hits are queued for the BTDF network
  const float* tile_sun_T;     // [M][L] network transmittance x ballistic fraction toward the sun
  uint32_t* tile_queue;        // ray slots of the generation's tile hits (surrogate form)
  int* tile_count;
  int tile_cap;
  // spectral bundles (Monte Carlo): `bundle` consecutive wavelengths share one ray while their
  // chains agree; 1 = every wavelength is its own path
  int bundle;
  int n_bundles;               // ceil(L / bundle)
  // photon maps: the first diffuse vertex of a path takes the sun's caustic and indirect light
  // from them (host-driven form, one wavelength per path)
  int use_photons;
  PhotonMapDev pm;
};

// Heterogeneous-tile mode compiled into the shading and shadow kernels: 0 the scene has no
// such tiles, 1 brute-force tracing through them, 2 the BTDF network.
inline int tile_mode(const RenderParams& p) { return p.tiles.n_tiles > 0 ? (p.use_surrogate ? 2 : 1) : 0; }

}  // namespace sdd
