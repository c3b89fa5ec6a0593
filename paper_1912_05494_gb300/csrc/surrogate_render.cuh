// surrogate_render.cuh -- launchers of the network-form tile kernels (surrogate_render.cu).
#pragma once

#include "sdd_internal.h"

struct sdd_surrogate;

namespace sdd {

struct PersistBuffers;
struct PersistCtl;

// Fused shading of the generation's queued tile hits (count read from p.tile_count on the
// device): network inputs gathered from the ray state, the network, exit sampling, and the
// append of the exit rays to the next generation and its closest-hit queues.
cudaError_t launch_tile_shade(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits, RayBuf next,
                              int* next_count, uint32_t* q, int* q_count, int qcap, Control* ctl,
                              const sdd_surrogate* net, cudaStream_t st);
// The same between the two persistent segments of a generation (buffers from pc's state).
cudaError_t launch_tile_shade_persistent(const RenderParams& p, const WaveDesc& w, const PersistBuffers& b,
                                         PersistCtl* pc, Control* ctl, const sdd_surrogate* net, cudaStream_t st);
void launch_sun_queries(const RenderParams& p, const int* mats, const float3* mat_normal, int n_mats, float* raw,
                        cudaStream_t st);
void launch_sun_table(const int* mats, int n_mats, int L, const float* pred, float* table, cudaStream_t st);
// Predictions [n][8] for raw inputs [n][7]; with n_dev the count is read on the device.
cudaError_t surrogate_predict(sdd_surrogate* s, int n, const float* raw, float* out, cudaStream_t st,
                              const int* n_dev = nullptr);
unsigned surrogate_version(const sdd_surrogate* s);

}  // namespace sdd
