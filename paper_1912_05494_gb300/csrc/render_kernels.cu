// render_kernels.cu -- the wavefront kernels of the GB300 spectral glass renderer.
//
// One generation of rays is processed by:
//   k_traverse  closest hit per subdomain queue (Sec. 3.1: "the complexity of ray tracers
//               is mostly contained in the intersectors"); a ray that leaves its slab
//               without a hit is handed, unchanged, to the neighbouring slab's queue
//               (Sec. 5: interface conditions keep the ray properties continuous)
//   k_shade     per-wavelength shading: complex Fresnel, Snell, Beer-Lambert (Eq. 1),
//               thin-slab series, Lambertian walls with a shadow ray to the sun (Eq. 3),
//               deterministic splitting (Sec. 3.1) or Philox-driven choices (Sec. 3.2);
//               children are compacted into the next generation and binned by subdomain
//   k_shadow    any-hit transmittance toward the sun per subdomain queue, with hand-off
// and, once per wave, k_film_accum adds every path's radiance into the FP64 film in
// sample order.  Queue appends are warp-aggregated: one atomic per distinct target queue
// per warp (ballot / match_any / popc).
#include "render_device.cuh"

namespace sdd {

__global__ void __launch_bounds__(kBlock) k_raygen(RenderParams p, WaveDesc w, RayBuf rb, uint32_t* q, int* q_count,
                                                   int qcap, Control* ctl) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  dev_raygen(p, w, i, i < w.n_paths, rb, q, q_count, qcap, ctl);
}

// Resident blocks per SM: 7 x 128 threads for traversal (4-wide nodes seen by the ray's
// octant, 72 registers), 6 x 128 for shadow rays without brute-force tiles (80 registers).
template <bool kStats, int kB>
__global__ void __launch_bounds__(kB, 7 * 128 / kB) k_traverse(RenderParams p, Sched sch, int top_nodes, QueuePair qp,
                                                     RayBuf rb, float2* hits, Control* ctl) {
  extern __shared__ Node s_nodes[];
  int b = blockIdx.x;
  int s = 0;
  while (s + 1 < sch.n_sub && sch.blk_start[s + 1] <= b) ++s;
  int n_staged = top_nodes > 0 ? stage_top(p.sc, s_nodes, s, top_nodes) : 0;
  int i = (b - sch.blk_start[s]) * blockDim.x + threadIdx.x;
  dev_traverse_warp<kStats>(p, s, i, i < sch.count[s], s_nodes, n_staged, qp, rb, hits, ctl);
}

template <int kTM, bool kPM = false>
__global__ void __launch_bounds__(kBlock) k_shade(RenderParams p, WaveDesc w, int n_rays, RayBuf cur,
                                                  const float2* __restrict__ hits, RayBuf next, uint32_t* q,
                                                  int* q_count, int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count,
                                                  float* path_L, Control* ctl) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  dev_shade<kTM, kPM>(p, w, r, r < n_rays, cur, hits, next, &ctl->next_rays, q, q_count, qcap, sb, &ctl->next_shadow,
                      sq, sq_count, path_L, ctl);
}

template <bool kStats, int kTM>
__device__ __forceinline__ void shadow_entry(const RenderParams& p, const WaveDesc& w, const Sched& sch,
                                             int top_nodes, const QueuePair& qp, const ShadowBuf& sb, float* path_L,
                                             Control* ctl) {
  extern __shared__ Node s_nodes[];
  int b = blockIdx.x;
  int s = 0;
  while (s + 1 < sch.n_sub && sch.blk_start[s + 1] <= b) ++s;
  int n_staged = top_nodes > 0 ? stage_top(p.sc, s_nodes, s, top_nodes) : 0;
  int i = (b - sch.blk_start[s]) * blockDim.x + threadIdx.x;
  // Any-hit rays without brute-force tiles are short and end early: the per-lane walk is
  // faster for them; with brute-force tile tracing inside the walk the warp-uniform one is.
  if constexpr (kTM == 1) {
    dev_shadow_warp<kStats, kTM>(p, w, s, i, i < sch.count[s], s_nodes, n_staged, qp, sb, path_L, ctl);
  } else {
    dev_shadow<kStats, kTM>(p, w, s, i, i < sch.count[s], s_nodes, n_staged, qp, sb, path_L, ctl);
  }
}

// Shadow rays of scenes without brute-force tiles: 8 x 128-thread blocks per SM.
template <bool kStats, int kB, int kTM>
__global__ void __launch_bounds__(kB, 6 * 128 / kB) k_shadow(RenderParams p, WaveDesc w, Sched sch, int top_nodes,
                                                             QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl) {
  shadow_entry<kStats, kTM>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
}

// Shadow rays through brute-force tiles: no occupancy bound.  The tile tracer is also
// compiled into the persistent kernel, and the two forms give bit-identical paths with the
// register budgets both kernels had when that was verified.
template <bool kStats, int kB>
__global__ void __launch_bounds__(kB) k_shadow_bf(RenderParams p, WaveDesc w, Sched sch, int top_nodes, QueuePair qp,
                                                  ShadowBuf sb, float* path_L, Control* ctl) {
  shadow_entry<kStats, 1>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
}

// ------------------------------------------------------------------------------ film
// Adds each path's radiance (its slots summed in order) into the FP64 film, samples in
// order; cells of one wave are distinct, so no two threads touch the same cell.
__global__ void k_film_accum(RenderParams p, WaveDesc w, const float* __restrict__ path_L, double* film,
                             float* path_rad_out, uint32_t* path_hash_out) {
  uint32_t lc = blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= w.nc) return;
  uint32_t cell = w.c0 + lc;
  uint32_t L = (uint32_t)p.sp.n_lambda;
  uint32_t px_i = cell / L, lam = cell - px_i * L;
  if (p.n_slots == 1) {
    // one slot per path: the wave's samples, in sample order, summed exactly as a
    // double-float pair and added once to the FP64 film (as k_film_accum_bundle)
    constexpr uint32_t kS = 8;
    float hi = 0.f, lo = 0.f;
    for (uint32_t s0 = 0; s0 < w.ns; s0 += kS) {
      const uint32_t m = min(kS, w.ns - s0);
      float v[kS];
#pragma unroll
      for (uint32_t u = 0; u < kS; ++u) v[u] = u < m ? path_L[(size_t)(s0 + u) * w.nc + lc] : 0.f;
#pragma unroll
      for (uint32_t u = 0; u < kS; ++u) {
        if (u >= m) break;
        two_sum_add(hi, lo, v[u]);
        const size_t out = ((size_t)px_i * p.spp + (w.s0 + s0 + u)) * L + lam;
        if (path_rad_out) path_rad_out[out] = v[u];
        if (path_hash_out && p.path_hash) path_hash_out[out] = p.path_hash[(size_t)(s0 + u) * w.nc + lc];
      }
    }
    film[cell] += (double)hi + (double)lo;
    return;
  }
  double acc = film[cell];
  for (uint32_t ls = 0; ls < w.ns; ++ls) {
    uint32_t path = ls * w.nc + lc;
    double v = 0.0;
    const float* sl = path_L + (size_t)path * p.n_slots;
    for (int k = 0; k < p.n_slots; ++k) v += (double)sl[k];
    acc += v;
    size_t out = ((size_t)px_i * p.spp + (w.s0 + ls)) * L + lam;
    if (path_rad_out) path_rad_out[out] = (float)v;
    if (path_hash_out && p.path_hash) path_hash_out[out] = p.path_hash[path];
  }
  film[cell] = acc;
}

__global__ void k_film_finalize(RenderParams p, const double* __restrict__ film, const double* __restrict__ cmf_w,
                                float* spectral_out, float* xyz_out) {
  int px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= p.n_px) return;
  int L = p.sp.n_lambda;
  double inv = 1.0 / p.spp, X = 0.0, Y = 0.0, Z = 0.0;
  for (int l = 0; l < L; ++l) {
    double v = film[(size_t)px * L + l] * inv;
    if (spectral_out) spectral_out[(size_t)px * L + l] = (float)v;
    X += v * cmf_w[3 * l];
    Y += v * cmf_w[3 * l + 1];
    Z += v * cmf_w[3 * l + 2];
  }
  if (xyz_out) {
    xyz_out[3 * px] = (float)X;
    xyz_out[3 * px + 1] = (float)Y;
    xyz_out[3 * px + 2] = (float)Z;
  }
}

// CIE 1931 colour matching functions by the multi-lobe piecewise-Gaussian fit of Wyman,
// Sloan and Shirley (JCGT 2013), weighted by the trapezoid rule over the render grid and
// normalised so that a flat spectrum of radiance 1 has Y = 1.
__device__ double pwg(double x, double mu, double s1, double s2) {
  double t = (x - mu) / (x < mu ? s1 : s2);
  return exp(-0.5 * t * t);
}
__global__ void k_cmf_table(int L, const float* lambda_nm, double* cmf_w) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ysum = 0.0;
  for (int l = 0; l < L; ++l) {
    double lam = lambda_nm[l];
    double w = 1.0;
    if (L > 1) {
      double lo = lambda_nm[l > 0 ? l - 1 : l], hi = lambda_nm[l + 1 < L ? l + 1 : l];
      w = 0.5 * (hi - lo);
    }
    double x = 1.056 * pwg(lam, 599.8, 37.9, 31.0) + 0.362 * pwg(lam, 442.0, 16.0, 26.7) -
               0.065 * pwg(lam, 501.1, 20.4, 26.2);
    double y = 0.821 * pwg(lam, 568.8, 46.9, 40.5) + 0.286 * pwg(lam, 530.9, 16.3, 31.1);
    double z = 1.217 * pwg(lam, 437.0, 11.8, 36.0) + 0.681 * pwg(lam, 459.0, 26.0, 13.8);
    cmf_w[3 * l] = x * w;
    cmf_w[3 * l + 1] = y * w;
    cmf_w[3 * l + 2] = z * w;
    ysum += y * w;
  }
  for (int i = 0; i < 3 * L; ++i) cmf_w[i] /= ysum;
}

// ------------------------------------------------------------------------------ utilities
__global__ void k_rays_from_arrays(int n, const float* org, const float* dir, DevScene sc, RayBuf rb, uint32_t* q,
                                   int* q_count, int qcap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool active = i < n;
  float3 o = make_float3(0.f, 0.f, 0.f);
  if (active) {
    o = make_float3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
    rb.o[i] = make_float4(o.x, o.y, o.z, 0.f);
    rb.d[i] = make_float4(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2], 1.f);
    rb.info[i] = make_uint2((uint32_t)i, 0u);
  }
  int s = active ? subdomain_of(sc, o) : 0;
  int pos = warp_append(q_count, s, active);
  if (active && pos < qcap) q[(size_t)s * qcap + pos] = (uint32_t)i;
}

__global__ void k_hits_to_arrays(int n, const float2* hits, float* t_out, int32_t* prim_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 h = hits[i];
  uint32_t prim = __float_as_uint(h.y);
  t_out[i] = prim == kMissPrim ? CUDART_INF_F : h.x;
  prim_out[i] = prim == kMissPrim ? -1 : (int32_t)prim;
}

__global__ void k_eval_optics(int n, const float* cos_i, const float* n_re, const float* k, const float* d,
                              const float* lam, int pol, float* R, float* Rs, float* Ts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a, b;
  slab_RT(cos_i[i], n_re[i], k[i], d[i], lam[i], &a, &b, pol);
  R[i] = fresnel_R(cos_i[i], 1.f, n_re[i], k[i]);
  Rs[i] = a;
  Ts[i] = b;
}

__global__ void k_philox(int n, const uint4* ctr, uint64_t key, uint4* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = philox4x32_10(ctr[i], (uint32_t)key, (uint32_t)(key >> 32));
}

// ------------------------------------------------------------------------------ launchers
static inline int blocks_for(long long n, int b) { return (int)((n + b - 1) / b); }

void launch_raygen(const RenderParams& p, const WaveDesc& w, RayBuf rb, uint32_t* q, int* q_count, int qcap,
                   Control* ctl, cudaStream_t st) {
  if (p.bundle > 1) return launch_raygen_bundle(p, w, rb, q, q_count, qcap, ctl, st);
  if (w.n_paths == 0) return;
  k_raygen<<<blocks_for(w.n_paths, kBlock), kBlock, 0, st>>>(p, w, rb, q, q_count, qcap, ctl);
}

template <int kB>
static void launch_traverse_b(const RenderParams& p, const Sched& sch, int total_blocks, int top_nodes, QueuePair qp,
                              RayBuf rb, float2* hits, Control* ctl, cudaStream_t st) {
  size_t smem = (size_t)top_nodes * sizeof(Node);
  if (p.stats >= 2)
    k_traverse<true, kB><<<total_blocks, kB, smem, st>>>(p, sch, top_nodes, qp, rb, hits, ctl);
  else
    k_traverse<false, kB><<<total_blocks, kB, smem, st>>>(p, sch, top_nodes, qp, rb, hits, ctl);
}

void launch_traverse(const RenderParams& p, const Sched& sch, int total_blocks, int block, int top_nodes,
                     QueuePair qp, RayBuf rb, float2* hits, Control* ctl, cudaStream_t st) {
  if (block == 64) launch_traverse_b<64>(p, sch, total_blocks, top_nodes, qp, rb, hits, ctl, st);
  else if (block == 256) launch_traverse_b<256>(p, sch, total_blocks, top_nodes, qp, rb, hits, ctl, st);
  else launch_traverse_b<128>(p, sch, total_blocks, top_nodes, qp, rb, hits, ctl, st);
}

void launch_shade(const RenderParams& p, const WaveDesc& w, int n_rays, RayBuf cur, const float2* hits, RayBuf next,
                  uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count, float* path_L,
                  Control* ctl, cudaStream_t st) {
  if (p.bundle > 1)
    return launch_shade_bundle(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq, sq_count, path_L, ctl, st);
  if (n_rays <= 0) return;
  const int tm = tile_mode(p);
  if (p.use_photons) {  // photon maps: brute-force tiles or none
    if (tm == 1)
      k_shade<1, true><<<blocks_for(n_rays, kBlock), kBlock, 0, st>>>(p, w, n_rays, cur, hits, next, q, q_count, qcap,
                                                                      sb, sq, sq_count, path_L, ctl);
    else
      k_shade<0, true><<<blocks_for(n_rays, kBlock), kBlock, 0, st>>>(p, w, n_rays, cur, hits, next, q, q_count, qcap,
                                                                      sb, sq, sq_count, path_L, ctl);
    return;
  }
  if (tm == 1)
    k_shade<1><<<blocks_for(n_rays, kBlock), kBlock, 0, st>>>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq,
                                                              sq_count, path_L, ctl);
  else if (tm == 2)
    k_shade<2><<<blocks_for(n_rays, kBlock), kBlock, 0, st>>>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq,
                                                              sq_count, path_L, ctl);
  else
    k_shade<0><<<blocks_for(n_rays, kBlock), kBlock, 0, st>>>(p, w, n_rays, cur, hits, next, q, q_count, qcap, sb, sq,
                                                              sq_count, path_L, ctl);
}

template <int kB, int kTM>
static void launch_shadow_b(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks,
                            int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st) {
  size_t smem = (size_t)top_nodes * sizeof(Node);
  if constexpr (kTM == 1) {
    if (p.stats >= 2)
      k_shadow_bf<true, kB><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
    else
      k_shadow_bf<false, kB><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
  } else {
    if (p.stats >= 2)
      k_shadow<true, kB, kTM><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
    else
      k_shadow<false, kB, kTM><<<total_blocks, kB, smem, st>>>(p, w, sch, top_nodes, qp, sb, path_L, ctl);
  }
}

template <int kTM>
static void launch_shadow_m(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks, int block,
                            int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st) {
  if (block == 64) launch_shadow_b<64, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
  else if (block == 256) launch_shadow_b<256, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
  else launch_shadow_b<128, kTM>(p, w, sch, total_blocks, top_nodes, qp, sb, path_L, ctl, st);
}

void launch_shadow(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks, int block,
                   int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st) {
  if (p.bundle > 1)
    return launch_shadow_bundle(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
  const int tm = tile_mode(p);
  if (tm == 1) launch_shadow_m<1>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
  else if (tm == 2) launch_shadow_m<2>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
  else launch_shadow_m<0>(p, w, sch, total_blocks, block, top_nodes, qp, sb, path_L, ctl, st);
}

void launch_film_accum(const RenderParams& p, const WaveDesc& w, const float* path_L, double* film,
                       float* path_rad_out, uint32_t* path_hash_out, cudaStream_t st) {
  if (p.bundle > 1) return launch_film_accum_bundle(p, w, path_L, film, path_rad_out, path_hash_out, st);
  k_film_accum<<<blocks_for(w.nc, 256), 256, 0, st>>>(p, w, path_L, film, path_rad_out, path_hash_out);
}

void launch_film_finalize(const RenderParams& p, const double* film, const double* cmf_w, float* spectral_out,
                          float* xyz_out, cudaStream_t st) {
  k_film_finalize<<<blocks_for(p.n_px, 256), 256, 0, st>>>(p, film, cmf_w, spectral_out, xyz_out);
}

void launch_cmf_table(int n_lambda, const float* lambda_nm, double* cmf_w, cudaStream_t st) {
  k_cmf_table<<<1, 32, 0, st>>>(n_lambda, lambda_nm, cmf_w);
}

void launch_rays_from_arrays(int n, const float* org, const float* dir, const DevScene sc, RayBuf rb, uint32_t* q,
                             int* q_count, int qcap, cudaStream_t st) {
  k_rays_from_arrays<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, org, dir, sc, rb, q, q_count, qcap);
}

void launch_hits_to_arrays(int n, const float2* hits, float* t_out, int32_t* prim_out, cudaStream_t st) {
  k_hits_to_arrays<<<blocks_for(n, 256), 256, 0, st>>>(n, hits, t_out, prim_out);
}

void launch_eval_optics(int n, const float* cos_i, const float* n_re, const float* k, const float* d,
                        const float* lam, int pol, float* R, float* Rs, float* Ts, cudaStream_t st) {
  k_eval_optics<<<blocks_for(n, 256), 256, 0, st>>>(n, cos_i, n_re, k, d, lam, pol, R, Rs, Ts);
}

void launch_philox(int n, const uint32_t* ctr, uint64_t key, uint32_t* out, cudaStream_t st) {
  k_philox<<<blocks_for(n, 256), 256, 0, st>>>(n, reinterpret_cast<const uint4*>(ctr), key,
                                                reinterpret_cast<uint4*>(out));
}

}  // namespace sdd
