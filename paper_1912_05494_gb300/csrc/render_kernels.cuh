// render_kernels.cuh -- launch wrappers of the wavefront kernels (render_kernels.cu).
#pragma once

#include "sdd_internal.h"

namespace sdd {

// Blocks of one traversal launch, grouped by subdomain: subdomain s owns blocks
// [blk_start[s], blk_start[s+1]) and count[s] queue entries.
struct Sched {
  int n_sub;
  int blk_start[kMaxSubdomains + 1];
  int count[kMaxSubdomains];
};

struct QueuePair {
  const uint32_t* in;   // [n_sub][cap]
  uint32_t* out;        // [n_sub][cap] rays handed to a neighbour
  int* out_count;       // [n_sub]
  int cap;
};

void launch_raygen(const RenderParams& p, const WaveDesc& w, RayBuf rb, uint32_t* q, int* q_count, int qcap,
                   Control* ctl, cudaStream_t st);
void launch_traverse(const RenderParams& p, const Sched& sch, int total_blocks, int block, int top_nodes,
                     QueuePair qp, RayBuf rb, float2* hits, Control* ctl, cudaStream_t st);
void launch_shade(const RenderParams& p, const WaveDesc& w, int n_rays, RayBuf cur, const float2* hits, RayBuf next,
                  uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count, float* path_L,
                  Control* ctl, cudaStream_t st);
void launch_shadow(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks, int block,
                   int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st);
void launch_film_accum(const RenderParams& p, const WaveDesc& w, const float* path_L, double* film,
                       float* path_rad_out, uint32_t* path_hash_out, cudaStream_t st);
void launch_film_finalize(const RenderParams& p, const double* film, const double* cmf_w, float* spectral_out,
                          float* xyz_out, cudaStream_t st);
// Spectral-bundle variants (bundle_kernels.cu); the launchers above forward to them when
// p.bundle > 1.
void launch_raygen_bundle(const RenderParams& p, const WaveDesc& w, RayBuf rb, uint32_t* q, int* q_count, int qcap,
                          Control* ctl, cudaStream_t st);
void launch_shade_bundle(const RenderParams& p, const WaveDesc& w, int n_rays, RayBuf cur, const float2* hits,
                         RayBuf next, uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count,
                         float* path_L, Control* ctl, cudaStream_t st);
void launch_shadow_bundle(const RenderParams& p, const WaveDesc& w, const Sched& sch, int total_blocks, int block,
                          int top_nodes, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st);
void launch_film_accum_bundle(const RenderParams& p, const WaveDesc& w, const float* path_L, double* film,
                              float* path_rad_out, uint32_t* path_hash_out, cudaStream_t st);
void launch_cmf_table(int n_lambda, const float* lambda_nm, double* cmf_w, cudaStream_t st);
void launch_rays_from_arrays(int n, const float* org, const float* dir, const DevScene sc, RayBuf rb, uint32_t* q,
                             int* q_count, int qcap, cudaStream_t st);
void launch_hits_to_arrays(int n, const float2* hits, float* t_out, int32_t* prim_out, cudaStream_t st);
void launch_eval_optics(int n, const float* cos_i, const float* n_re, const float* k, const float* d,
                        const float* lam, int pol, float* R, float* Rs, float* Ts, cudaStream_t st);
void launch_philox(int n, const uint32_t* ctr, uint64_t key, uint32_t* out, cudaStream_t st);

}  // namespace sdd
