// photon.cuh -- photon-map kernels (Sec. 3.2): launchers and their argument blocks.
#pragma once

#include <cuda_runtime.h>

#include "sdd_internal.h"

namespace sdd {

// Emitter disc of the sun's photons: centre origin (= C + D s), radius; power_scale =
// Omega pi R^2 / N (a photon's power is L_sun(l) (s . w) power_scale); photons
// [j0, j0 + n) of the n_lambda * n_per_lambda, photon j = l * n_per_lambda + i.
struct PhotonEmit {
  float3 origin;
  float radius;
  float power_scale;
  int n_per_lambda;
  uint32_t j0;
};

// Append buffers of the stored photons, per map (0 caustic, 1 global); count[map] keeps
// counting past cap (entries beyond cap are dropped, and the caller grows cap and repeats).
struct PhotonStore {
  float4* pos_pw[2];    // position xyz, power
  float4* nrm_lam[2];   // normal facing the arrival xyz, wavelength index (int bits)
  uint2* id_seq[2];     // photon index i within its wavelength, diffuse surfaces met before
  int* count;           // [2]
  int cap;
};

void launch_photon_emit(const RenderParams& p, const PhotonEmit& pe, int n, RayBuf rb, uint32_t* q, int* q_count,
                        int qcap, Control* ctl, cudaStream_t st);
void launch_photon_shade(const RenderParams& p, const PhotonEmit& pe, int n_rays, RayBuf cur, const float2* hits,
                         RayBuf next, int* next_count, uint32_t* q, int* q_count, int qcap, const PhotonStore& s,
                         Control* ctl, cudaStream_t st);
// Sorts n photons into the buckets of a table of mask + 1 entries (a power of two, >= 1024),
// cells of edge 1 / inv_cell: start [mask + 2], scratch [(mask + 1) + (mask + 1) / 1024] words.
cudaError_t build_photon_grid(int n, const float4* pos, const float4* nrm, float inv_cell, uint32_t mask, uint32_t* start,
                              uint32_t* scratch, float4* out_pos, float4* out_nrm, cudaStream_t st);
void launch_photon_gather(const PhotonMapDev& pm, int n, const float* x, const float* nrm, const int32_t* lam,
                          float* ec, float* eg, cudaStream_t st);

}  // namespace sdd
