// graph_form.h -- launchers of the graph form's kernels (graph_kernels.cu).
#pragma once

#include "render_kernels.cuh"

namespace sdd {

// Fixed grids (SMs x resident blocks) of one render's traversal, shading and shadow kernels;
// query them before a stream capture begins.
struct GraphGrids {
  int traverse, shade, shadow;
  int top_nodes;     // BVH nodes per subdomain the traversal stages in shared memory (0: none)
  int block_chunks;  // bit 0 closest-hit, bit 1 shadow passes: 128-ray chunks per block (else 32 per warp)
};
GraphGrids graph_grids(const RenderParams& p, int top_nodes, int block_chunks);

// work: the pass's chunk counter, zero before the pass
cudaError_t launch_traverse_g(const RenderParams& p, const GraphGrids& g, const int* counts_in, int* work,
                              QueuePair qp, RayBuf rb, float2* hits, Control* ctl, cudaStream_t st);
cudaError_t launch_shade_g(const RenderParams& p, const GraphGrids& g, const WaveDesc& w, const int* n_in,
                           RayBuf cur, const float2* hits, RayBuf next, int* next_count, uint32_t* q, int* q_count,
                           int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count, float* path_L, Control* ctl,
                           cudaStream_t st);
cudaError_t launch_shadow_g(const RenderParams& p, const GraphGrids& g, const WaveDesc& w, const int* counts_in,
                            int* work, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st);
void launch_set_int(int* dst, int v, cudaStream_t st);
void launch_loop_cond(cudaGraphConditionalHandle h, const int* counts, int n_sub, int max_iter, int kind,
                      Control* ctl, cudaStream_t st);
void launch_check_drained(const int* counts, int n_sub, Control* ctl, cudaStream_t st);

}  // namespace sdd
