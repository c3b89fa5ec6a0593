// tile.cu -- heterogeneous glass tiles on the GPU: the tile set (height fields built on the
// device from each tile's parameters), per-ray brute-force tracing, and per-sample
// statistics of many rays (the training data of the BTDF surrogate).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "sdd_internal.h"
#include "tile_device.cuh"
#include "tileset.h"

namespace sdd {
sdd_status set_last_error(sdd_status st, const char* msg);
}
using namespace sdd;

namespace {

__global__ void k_tile_heights(int n_tiles, int G, float L, const float* d_mean, const float* amp, const uint32_t* seed,
                               float* h) {
  const int W = G + 1;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_tiles * W * W) return;
  int t = (int)(idx / (W * W));
  int v = (int)(idx - (long long)t * W * W);
  int j = v / W, i = v - j * W;
  h[idx] = tile_thickness(seed[t], d_mean[t], amp[t], i * L / G, j * L / G, L);
}

__device__ __forceinline__ TileDev tile_view(const TileSetDev& ts, int t) {
  TileDev g;
  g.h = ts.heights + (size_t)t * (ts.G + 1) * (ts.G + 1);
  g.hmin = ts.hmin[t];
  g.hmax = ts.hmax[t];
  g.rho = ts.rho[t];
  g.G = ts.G;
  g.L = ts.L;
  return g;
}

__global__ void k_tile_trace_rays(TileSetDev ts, int tile, int n, const float* xy, const float* dir, float n_re, float k,
                                  float lambda_nm, const uint32_t* px, const uint32_t* sample, uint32_t bounce,
                                  uint32_t lam, uint64_t seed, int max_events, int32_t* side, float* w, float* dout,
                                  int32_t* bubbles, int32_t* events) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TileDev g = tile_view(ts, tile);
  TileOut r = tile_trace(g, xy[2 * i], xy[2 * i + 1], make_float3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]), n_re, k,
                         lambda_nm, px[i], sample[i], bounce, lam, seed, max_events);
  side[i] = r.side;
  w[i] = r.w;
  dout[3 * i] = r.dir.x;
  dout[3 * i + 1] = r.dir.y;
  dout[3 * i + 2] = r.dir.z;
  bubbles[i] = r.bubbles;
  events[i] = r.events;
}

template <typename T>
__device__ __forceinline__ T warp_sum_all(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deflection-angle bin of the statistics from the cosine c of the angle: edges 0, 1, 2, 4, 8,
// 16, 32, 64, 180 degrees (cosines of the inner edges below).
__device__ __forceinline__ int deflection_bin(float c) {
  const float ce[kTileBins - 1] = {0.99984769515639124f, 0.99939082701909576f, 0.99756405025982420f,
                                   0.99026806874157036f, 0.96126169593831889f, 0.84804809615642596f,
                                   0.43837114678907746f};
  int b = 0;
#pragma unroll
  for (int j = 0; j < kTileBins - 1; ++j) b += c < ce[j] ? 1 : 0;
  return b;
}

// One warp per sample; lane l traces rays l, l + 32, ...; statistics reduced across the warp.
__global__ void k_tile_samples(TileSetDev ts, int n_samples, const float* cos_in, const float* phi_in,
                               const float* lambda_nm, const float* n_re, const float* k, const int32_t* tile, int rays,
                               uint64_t seed, int max_events, float* out) {
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= n_samples) return;  // whole warps leave together
  const int s = warp;
  TileDev g = tile_view(ts, tile[s]);
  const float ci = cos_in[s];  // < 0: enters through the rough back face
  const float st = sqrtf(fmaxf(0.f, 1.f - ci * ci));
  float sp, cp;
  sincosf(phi_in[s], &sp, &cp);
  const float3 d = make_float3(st * cp, st * sp, -ci);
  const float3 dm = make_float3(d.x, d.y, -d.z);
  float T = 0.f, R = 0.f, A = 0.f, bub = 0.f, hT[kTileBins], hR[kTileBins];
#pragma unroll
  for (int b = 0; b < kTileBins; ++b) hT[b] = hR[b] = 0.f;
  for (int r = lane; r < rays; r += 32) {
    float4 ue = draw4((uint32_t)s, (uint32_t)r, 0, STREAM_TILE, 0, 0, seed);
    TileOut tr = tile_trace(g, ue.x * g.L, ue.y * g.L, d, n_re[s], k[s], lambda_nm[s], (uint32_t)s, (uint32_t)r, 1, 0,
                            seed, max_events);
    bub += (float)tr.bubbles;
    if (tr.side == 1) {
      T += tr.w;
      const int b = deflection_bin(dot3(tr.dir, d));
#pragma unroll
      for (int j = 0; j < kTileBins; ++j) hT[j] += j == b ? tr.w : 0.f;
    } else if (tr.side == 0) {
      R += tr.w;
      const int b = deflection_bin(dot3(tr.dir, dm));
#pragma unroll
      for (int j = 0; j < kTileBins; ++j) hR[j] += j == b ? tr.w : 0.f;
    } else {
      A += tr.w;
    }
  }
  T = warp_sum_all(T);
  R = warp_sum_all(R);
  A = warp_sum_all(A);
  bub = warp_sum_all(bub);
#pragma unroll
  for (int b = 0; b < kTileBins; ++b) {
    hT[b] = warp_sum_all(hT[b]);
    hR[b] = warp_sum_all(hR[b]);
  }
  if (lane == 0) {
    float* o = out + kTileStatCols * (size_t)s;
    o[0] = T / rays;
    o[1] = R / rays;
    o[2] = A / rays;
    o[3] = bub / rays;
#pragma unroll
    for (int b = 0; b < kTileBins; ++b) {
      o[4 + b] = T > 0.f ? hT[b] / T : 0.f;
      o[4 + kTileBins + b] = R > 0.f ? hR[b] / R : 0.f;
    }
  }
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

struct sdd_tileset {
  TileSetDev dev{};
  float* d_mean = nullptr;
  float* d_amp = nullptr;
  uint32_t* d_seed = nullptr;
  ~sdd_tileset() {
    cudaFree((void*)dev.heights);
    cudaFree((void*)dev.hmin);
    cudaFree((void*)dev.hmax);
    cudaFree((void*)dev.rho);
    cudaFree(d_mean);
    cudaFree(d_amp);
    cudaFree(d_seed);
  }
};

namespace sdd {
const TileSetDev* tileset_device_view(const sdd_tileset* t) { return &t->dev; }
}

extern "C" {

sdd_status sdd_tileset_create(const sdd_tileset_desc* d, sdd_tileset** out) {
  if (!d || !out) return set_last_error(SDD_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (d->n_tiles < 1 || !d->d_mean_m || !d->amplitude_m || !d->bubble_density_m3 || !d->seed)
    return set_last_error(SDD_ERR_ARG, "tile set needs n_tiles >= 1 and all four parameter arrays");
  if (d->grid < 1 || d->grid > 1024) return set_last_error(SDD_ERR_ARG, "grid must be in [1, 1024]");
  if (!(d->tile_size_m > 0.f)) return set_last_error(SDD_ERR_ARG, "tile_size_m must be > 0");
  for (int t = 0; t < d->n_tiles; ++t) {
    if (!(d->d_mean_m[t] > 0.f) || !(d->amplitude_m[t] >= 0.f) || !(d->bubble_density_m3[t] >= 0.f))
      return set_last_error(SDD_ERR_ARG, ("tile " + std::to_string(t) + ": bad thickness, amplitude or density").c_str());
  }
  sdd_tileset* ts = new sdd_tileset;
  const int G = d->grid, W = G + 1, n = d->n_tiles;
  std::vector<float> mean(d->d_mean_m, d->d_mean_m + n), amp(d->amplitude_m, d->amplitude_m + n),
      rho(d->bubble_density_m3, d->bubble_density_m3 + n);
  std::vector<uint32_t> seed(d->seed, d->seed + n);
  float* heights = nullptr;
  cudaError_t e;
  if ((e = upload(&ts->d_mean, mean)) != cudaSuccess || (e = upload(&ts->d_amp, amp)) != cudaSuccess ||
      (e = upload(&ts->d_seed, seed)) != cudaSuccess ||
      (e = cudaMalloc(&heights, sizeof(float) * (size_t)n * W * W)) != cudaSuccess) {
    delete ts;
    return set_last_error(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  ts->dev.heights = heights;
  long long total = (long long)n * W * W;
  k_tile_heights<<<(unsigned)((total + 255) / 256), 256>>>(n, G, d->tile_size_m, ts->d_mean, ts->d_amp, ts->d_seed,
                                                            heights);
  std::vector<float> h((size_t)total), hmin(n), hmax(n);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpy(h.data(), heights, sizeof(float) * total, cudaMemcpyDeviceToHost)) != cudaSuccess) {
    delete ts;
    return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int t = 0; t < n; ++t) {
    auto b = h.begin() + (size_t)t * W * W;
    hmin[t] = *std::min_element(b, b + W * W);
    hmax[t] = *std::max_element(b, b + W * W);
  }
  float *dmin = nullptr, *dmax = nullptr, *drho = nullptr;
  if ((e = upload(&dmin, hmin)) != cudaSuccess || (e = upload(&dmax, hmax)) != cudaSuccess ||
      (e = upload(&drho, rho)) != cudaSuccess) {
    ts->dev.hmin = dmin;
    ts->dev.hmax = dmax;
    ts->dev.rho = drho;
    delete ts;
    return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  ts->dev.hmin = dmin;
  ts->dev.hmax = dmax;
  ts->dev.rho = drho;
  ts->dev.d_mean = ts->d_mean;
  ts->dev.n_tiles = n;
  ts->dev.G = G;
  ts->dev.L = d->tile_size_m;
  *out = ts;
  return SDD_OK;
}

void sdd_tileset_destroy(sdd_tileset* t) { delete t; }

sdd_status sdd_tileset_heights(const sdd_tileset* t, int tile, float* out_host) {
  if (!t || !out_host || tile < 0 || tile >= t->dev.n_tiles) return set_last_error(SDD_ERR_ARG, "bad arguments");
  size_t W = t->dev.G + 1;
  cudaError_t e = cudaMemcpy(out_host, t->dev.heights + (size_t)tile * W * W, sizeof(float) * W * W,
                             cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SDD_OK : set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
}

sdd_status sdd_tile_trace_rays(sdd_tileset* t, int tile, int n, const float* xy, const float* dir, float n_re, float k,
                               float lambda_nm, const uint32_t* px, const uint32_t* sample, uint32_t bounce,
                               uint32_t lam, uint64_t seed, int max_events, int32_t* side, float* w, float* dir_out,
                               int32_t* bubbles, int32_t* events, void* stream) {
  if (!t || tile < 0 || tile >= t->dev.n_tiles || n < 0 || max_events < 1 || max_events > 256)
    return set_last_error(SDD_ERR_ARG, "bad arguments (tile index, n, or max_events outside 1..256)");
  if (n == 0) return SDD_OK;
  if (!xy || !dir || !px || !sample || !side || !w || !dir_out || !bubbles || !events)
    return set_last_error(SDD_ERR_ARG, "NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  k_tile_trace_rays<<<(n + 127) / 128, 128, 0, st>>>(t->dev, tile, n, xy, dir, n_re, k, lambda_nm, px, sample, bounce,
                                                     lam, seed, max_events, side, w, dir_out, bubbles, events);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SDD_OK : set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
}

sdd_status sdd_tile_generate(sdd_tileset* t, int n_samples, const float* cos_in, const float* phi_in,
                             const float* lambda_nm, const float* n_re, const float* k, const int32_t* tile,
                             int rays_per_sample, uint64_t seed, int max_events, float* out, void* stream) {
  if (!t || n_samples < 0 || rays_per_sample < 1 || max_events < 1 || max_events > 256)
    return set_last_error(SDD_ERR_ARG, "bad arguments (n_samples, rays_per_sample, or max_events outside 1..256)");
  if (n_samples == 0) return SDD_OK;
  if (!cos_in || !phi_in || !lambda_nm || !n_re || !k || !tile || !out) return set_last_error(SDD_ERR_ARG, "NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  long long threads = (long long)n_samples * 32;
  k_tile_samples<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(t->dev, n_samples, cos_in, phi_in, lambda_nm, n_re,
                                                                    k, tile, rays_per_sample, seed, max_events, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SDD_OK : set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
