// bundle_kernels.cu -- host-driven wavefront kernels of the spectral-bundle path
// (bundle_device.cuh): raygen, shading, shadow rays and film accumulation.  Closest-hit
// traversal is the same kernel as without bundles: it reads only origins and directions.
#include "bundle_device.cuh"

namespace sdd {

__global__ void __launch_bounds__(kBlock) k_raygen_bundle(RenderParams p, WaveDesc w, RayBuf rb, uint32_t* q,
                                                          int* q_count, int qcap, Control* ctl) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  dev_raygen_bundle(p, w, i, i < w.n_paths, rb, q, q_count, qcap, ctl);
}

// Resident blocks per SM as in the graph form's bundle shading (a register cap that keeps more
// warps in flight for the shading's memory latency: 5, 6 with the network's tile queue);
// brute-force tiles keep their registers.
template <int kTM, bool kPM = false>
__global__ void __launch_bounds__(kBlock, kTM == 1 ? 1 : (kTM == 2 ? 6 : 5)) k_shade_bundle(RenderParams p, WaveDesc w, int n_rays, RayBuf cur,
                                                         const float2* __restrict__ hits, RayBuf next, uint32_t* q,
                                                         int* q_count, int qcap, ShadowBuf sb, uint32_t* sq,
                                                         int* sq_count, float* path_L, Control* ctl) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  dev_shade_bundle<kTM, kPM>(p, w, r, r < n_rays, cur, hits, next, &ctl->next_rays, q, q_count, qcap, sb,
                             &ctl->next_shadow, sq, sq_count, path_L, ctl);
}

// Blocks grouped by subdomain as in the traversal kernel; the per-lane walk without
// brute-force tiles, the warp-uniform one with them (as without bundles).
template <bool kStats, int kTM>
__device__ __forceinline__ void shadow_bundle_entry(const RenderParams& p, const WaveDesc& w, const Sched& sch,
                                                    int top_nodes, const QueuePair& qp, const ShadowBuf& sb,
                                                    float* path_L, Control* ctl) {
  extern __shared__ Node s_nodes[];
  int b = blockIdx.x;
  int s = 0;
  while (s + 1 < sch.n_sub && sch.blk_start[s + 1] <= b) ++s;
  int n_staged = top_nodes > 0 ? stage_top(p.sc, s_nodes, s, top_nodes) : 0;
  int i = (b - sch.blk_start[s]) * blockDim.x + threadIdx.x;
  dev_shadow_bundle<kStats, kTM, kTM == 1>(p, w, s, i, i < sch.count[s], s_nodes, n_staged, qp, sb, path_L, ctl);
}

template <bool kStats, int kB, int kTM>
__global__ void __launch_bounds__(kB, kTM == 1 ? 1 : 6 * 128 / kB)
    k_shadow_bundle(RenderParams p, WaveDesc w, Sched sch, int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L,
                    Control* ctl) {
  shadow_bundle_entry<kStats, kTM>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
}

// Adds every member's radiance into the FP64 film, samples in order: one thread per
// (cell, member), so no two threads touch the same film entry.
__global__ void k_film_accum_bundle(RenderParams p, WaveDesc w, const float* __restrict__ path_L, double* film,
                                    float* path_rad_out, uint32_t* path_hash_out) {
  const uint32_t B = (uint32_t)p.bundle;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w.nc * B) return;
  const uint32_t lc = t / B, b = t - lc * B;
  const uint32_t cell = w.c0 + lc;
  const uint32_t L = (uint32_t)p.sp.n_lambda;
  const uint32_t px_i = cell / (uint32_t)p.n_bundles, j = cell - px_i * (uint32_t)p.n_bundles;
  const uint32_t lam = j * B + b;
  if (lam >= L) return;
  // the wave's samples, in sample order, summed exactly as a double-float pair (GB300's FP64
  // rate made one FP64 add per sample the kernel's limit), added once to the FP64 film;
  // values are loaded kS at a time
  constexpr uint32_t kS = 8;
  const size_t stride = (size_t)w.nc * B;
  const size_t slot0 = (size_t)lc * B + b;
  float hi = 0.f, lo = 0.f;
  for (uint32_t s0 = 0; s0 < w.ns; s0 += kS) {
    const uint32_t m = min(kS, w.ns - s0);
    float v[kS];
#pragma unroll
    for (uint32_t u = 0; u < kS; ++u) v[u] = u < m ? path_L[slot0 + (size_t)(s0 + u) * stride] : 0.f;
#pragma unroll
    for (uint32_t u = 0; u < kS; ++u) {
      if (u >= m) break;
      two_sum_add(hi, lo, v[u]);
      const size_t out = ((size_t)px_i * p.spp + (w.s0 + s0 + u)) * L + lam;
      if (path_rad_out) path_rad_out[out] = v[u];
      if (path_hash_out && p.path_hash) path_hash_out[out] = p.path_hash[slot0 + (size_t)(s0 + u) * stride];
    }
  }
  film[(size_t)px_i * L + lam] += (double)hi + (double)lo;
}

// ------------------------------------------------------------------------------ launchers
static inline int blocks_for(long long n, int b) { return (int)((n + b - 1) / b); }

void launch_raygen_bundle(const RenderParams& p, const WaveDesc& w, RayBuf rb, uint32_t* q, int* q_count, int qcap,
                          Control* ctl, cudaStream_t st) {
  if (w.n_paths == 0) return;
  k_raygen_bundle<<<blocks_for(w.n_paths, kBlock), kBlock, 0, st>>>(p, w, rb, q, q_count, qcap, ctl);
}

template <int kTM, bool kPM>
static void launch_shade_bundle_t(const RenderParams& p, const WaveDesc& w, int n_rays, RayBuf cur, const float2* hits,
                                  RayBuf next, uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq,
                                  int* sq_count, float* path_L, Control* ctl, cudaStream_t st) {
  const size_t smem = bundle_shade_smem(p.bundle);
  if (allow_dynamic_smem((const void*)k_shade_bundle<kTM, kPM>, smem) != cudaSuccess) return;  // reported at the
                                                                                                 // next error check
  k_shade_bundle<kTM, kPM><<<blocks_for(n_rays, kBlock), kBlock, smem, st>>>(p, w, n_rays, cur, hits, next, q, q_count,
                                                                           qcap, sb, sq, sq_count, path_L, ctl);
}

void launch_shade_bundle(const RenderParams& p, const WaveDesc& w, int n_rays, RayBuf cur, const float2* hits,
                         RayBuf next, uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count,
                         float* path_L, Control* ctl, cudaStream_t st) {
  if (n_rays <= 0) return;
  if (p.use_photons) {  // photon maps: brute-force tiles or none
    if (tile_mode(p) == 1)
      launch_shade_bundle_t<1, true>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
    else
      launch_shade_bundle_t<0, true>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
    return;
  }
  if (tile_mode(p) == 1)
    launch_shade_bundle_t<1, false>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
  else if (tile_mode(p) == 2)
    launch_shade_bundle_t<2, false>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
  else
    launch_shade_bundle_t<0, false>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
}

template <int kB, int kTM>
static void launch_shadow_bundle_b(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks,
                                   int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl,
                                   cudaStream_t st) {
  size_t smem = (size_t)top_nodes * sizeof(Node);
  if (p.stats >= 2)
    k_shadow_bundle<true, kB, kTM><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
  else
    k_shadow_bundle<false, kB, kTM><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
}

template <int kTM>
static void launch_shadow_bundle_m(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks,
                                   int block, int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl,
                                   cudaStream_t st) {
  if (block == 64) launch_shadow_bundle_b<64, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
  else if (block == 256) launch_shadow_bundle_b<256, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
  else launch_shadow_bundle_b<128, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
}

void launch_shadow_bundle(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks, int block,
                          int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st) {
  if (tile_mode(p) == 1)
    launch_shadow_bundle_m<1>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
  else if (tile_mode(p) == 2)
    launch_shadow_bundle_m<2>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
  else
    launch_shadow_bundle_m<0>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
}

void launch_film_accum_bundle(const RenderParams& p, const WaveDesc& w, const float* path_L, double* film,
                              float* path_rad_out, uint32_t* path_hash_out, cudaStream_t st) {
  k_film_accum_bundle<<<blocks_for((long long)w.nc * p.bundle, 256), 256, 0, st>>>(p, w, path_L, film, path_rad_out,
                                                                                   path_hash_out);
}

}  // namespace sdd
