// photon_device.cuh -- density estimation on the photon maps (Sec. 3.2), shared by the
// renderer's shading and the gather entry point.
#pragma once

#include "device_math.cuh"
#include "sdd_internal.h"

namespace sdd {

constexpr float kPhotonPi = 3.14159265358979323846f;

// Bucket of grid cell (ix, iy, iz) in a table of mask + 1 buckets.
__host__ __device__ __forceinline__ uint32_t photon_bucket(int ix, int iy, int iz, uint32_t mask) {
  return ((uint32_t)ix * 73856093u ^ (uint32_t)iy * 19349663u ^ (uint32_t)iz * 83492791u) & mask;
}

__device__ __forceinline__ int photon_cell(float c, float inv_cell) { return (int)floorf(c * inv_cell); }

// Irradiance estimate of a map at x on a surface with normal n, wavelength index lam: the
// power of the photons within the radius that arrived on the same side, over pi r^2.  The
// disc of radius r around x lies in the cells [floor((x - r) / c), floor((x + r) / c)] per
// axis (cell edge c = 2 r: two cells); a photon counts only while its own cell is visited,
// so cells that share a bucket never count a photon twice.  The powers are summed in FP32 with
// Neumaier's compensation (error ~1 ulp of the sum whatever the photon count); an FP64 sum
// would run on the GPU's narrow FP64 pipe, which bounded this lookup at 82 % busy.
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
  const float t = s + x;
  c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

// One map's estimate (the sum before the division by pi r^2).
__device__ __forceinline__ float photon_power_within(const PhotonMapDev& pm, int map, float3 x, float3 n, int lam) {
  const float r = pm.radius, inv = pm.inv_cell;
  // first cell and extra cells (0..2) per axis; the loops are bounded for any input
  const int x0 = photon_cell(x.x - r, inv), y0 = photon_cell(x.y - r, inv), z0 = photon_cell(x.z - r, inv);
  const int nx = (int)min(max((long long)photon_cell(x.x + r, inv) - x0, 0ll), 2ll);
  const int ny = (int)min(max((long long)photon_cell(x.y + r, inv) - y0, 0ll), 2ll);
  const int nz = (int)min(max((long long)photon_cell(x.z + r, inv) - z0, 0ll), 2ll);
  float sum = 0.f, comp = 0.f;
  const float r2 = r * r;
  for (int c = 0; c <= nz; ++c)
    for (int b = 0; b <= ny; ++b)
      for (int a = 0; a <= nx; ++a) {
        const int ix = (int)((unsigned)x0 + a), iy = (int)((unsigned)y0 + b), iz = (int)((unsigned)z0 + c);
        const uint32_t bk = photon_bucket(ix, iy, iz, pm.mask);
        const uint32_t e = __ldg(pm.start[map] + bk + 1);
        for (uint32_t k = __ldg(pm.start[map] + bk); k < e; ++k) {
          const float4 ps = __ldg(pm.pos_pw[map] + k);
          if (photon_cell(ps.x, inv) != ix || photon_cell(ps.y, inv) != iy || photon_cell(ps.z, inv) != iz) continue;
          const float dx = ps.x - x.x, dy = ps.y - x.y, dz = ps.z - x.z;
          if (dx * dx + dy * dy + dz * dz >= r2) continue;
          const float4 q = __ldg(pm.nrm_lam[map] + k);
          if (__float_as_int(q.w) != lam || q.x * n.x + q.y * n.y + q.z * n.z <= 0.f) continue;
          neumaier_add(sum, comp, ps.w);
        }
      }
  return sum + comp;
}

// Irradiance estimates of both maps (x: caustic, y: global) at x, normal n, wavelength lam.
// (Fetching the 16 bucket ranges of both maps before any photon, to overlap their
// latencies, measured slower: 64 registers and more divergent lanes.)
__device__ __forceinline__ float2 photon_irradiance(const PhotonMapDev& pm, float3 x, float3 n, int lam) {
  const float area = kPhotonPi * pm.radius * pm.radius;
  return make_float2(photon_power_within(pm, 0, x, n, lam) / area, photon_power_within(pm, 1, x, n, lam) / area);
}

}  // namespace sdd
