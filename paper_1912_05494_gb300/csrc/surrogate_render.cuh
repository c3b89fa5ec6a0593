// surrogate_render.cuh -- launchers of the surrogate-form tile kernels (surrogate_render.cu).
#pragma once

#include "sdd_internal.h"

struct sdd_surrogate;

namespace sdd {

void launch_tile_inputs(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits,
                        const uint32_t* queue, int n, float* raw, cudaStream_t st);
void launch_tile_apply(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits,
                       const uint32_t* queue, int n, const float* pred, RayBuf next, int* next_count, uint32_t* q,
                       int* q_count, int qcap, Control* ctl, cudaStream_t st);
void launch_sun_queries(const RenderParams& p, const int* mats, const float3* mat_normal, int n_mats, float* raw,
                        cudaStream_t st);
void launch_sun_table(const int* mats, int n_mats, int L, const float* pred, float* table, cudaStream_t st);
cudaError_t surrogate_predict(sdd_surrogate* s, int n, const float* raw, float* out, cudaStream_t st);
unsigned surrogate_version(const sdd_surrogate* s);

}  // namespace sdd
