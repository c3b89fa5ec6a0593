// graph_kernels.cu -- kernels of the graph form of the wavefront.
//
// The host-driven form sizes every traversal launch from queue counts it reads back, one
// round trip per subdomain pass; the persistent form removes the round trips but runs every
// step at the one occupancy its register budget allows.  The graph form keeps one kernel per
// step, each at its own occupancy, and reads the counts on the device instead: every launch
// has a fixed grid (SMs x resident blocks) whose blocks take subdomain-aligned 128-ray chunks
// of the queues from a work counter (traversal) or stride over the generation's rays
// (shading).  A generation is the
// closest-hit passes, shading, the shadow passes; the passes run in conditional 'while' nodes
// of the frame's CUDA graph whose condition kernel (k_loop_cond) reads the queue counts, so a
// whole frame is captured once and replayed with no host round trip and no empty passes
// beyond the second of a loop iteration (a ray crosses each slab at most once, Sec. 5
// hand-off, which bounds the iterations).  The per-ray work is the same device code as the
// other forms (render_device.cuh, bundle_device.cuh).
#include "bundle_device.cuh"
#include "chunk_sched.cuh"
#include "graph_form.h"

#include <mutex>
#include <unordered_map>

namespace sdd {

namespace {

constexpr int kWarpChunk = 32;  // rays a warp takes from the pass's work counter at a time

// Next 32-ray chunk of a pass for this warp from the pass's work counter (zeroed before the
// pass): warps take chunks as they finish, each on its own (no block barrier, so a warp
// never waits for the slowest warp of its block), and the pass's cost balances over the
// grid.  The per-subdomain layout is padded to 128-ray chunks, so a 32-ray chunk never
// straddles two subdomains and the warp enters the walk converged.  Returns a value >= total
// when the pass is done.
__device__ __forceinline__ int next_warp_chunk(int* work) {
  int c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(work, kWarpChunk);
  return __shfl_sync(0xFFFFFFFFu, c, 0);
}
// The block-wide alternative: the block takes a 128-ray chunk (one per thread) at a time,
// which keeps a block's warps on consecutive queue entries but makes them wait for each other.
__device__ __forceinline__ int next_block_chunk(int* work) {
  __shared__ int s_chunk;
  __syncthreads();
  if (threadIdx.x == 0) s_chunk = atomicAdd(work, kChunk);
  __syncthreads();
  return s_chunk;
}

// Closest-hit pass over the queues whose counts are counts_in.  With top_nodes > 0 every
// block first stages the top_nodes first (breadth-first: top-level) nodes of every
// subdomain's BVH in shared memory (Sec. 5: the top of the hierarchy first).  Seven resident
// blocks per SM (73 registers) hold a 4-wide node as the ray's octant sees it (nave frame:
// closest-hit passes 28.0 ms at 7 blocks, 29.5 at 6; before the octant view, 28.8 at 6, 29.1
// at 8 with 48 B of spills and 39.6 at 10).
template <bool kStats>
__global__ void __launch_bounds__(kChunk, 7) k_traverse_g(RenderParams p, const int* counts_in, int* work,
                                                           int top_nodes, int block_chunks, QueuePair qp, RayBuf rb,
                                                           float2* hits, Control* ctl) {
  __shared__ int s_prefix[kMaxSubdomains + 1];
  __shared__ int s_count[kMaxSubdomains];
  extern __shared__ Node s_top[];
  const int n_sub = p.sc.n_sub;
  const int total = load_prefix(counts_in, n_sub, qp.cap, s_prefix, s_count);
  if (total == 0) return;
  if (top_nodes > 0) {
    for (int s = 0; s < n_sub; ++s) {
      const int n = min(top_nodes, p.sc.n_nodes_sub[s]);
      const float4* src = reinterpret_cast<const float4*>(p.sc.nodes + p.sc.root[s]);
      float4* dst = reinterpret_cast<float4*>(s_top + (size_t)s * top_nodes);
      for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
  }
  const int lane = block_chunks ? (int)threadIdx.x : ((int)threadIdx.x & 31);
  for (int c0 = block_chunks ? next_block_chunk(work) : next_warp_chunk(work); c0 < total;
       c0 = block_chunks ? next_block_chunk(work) : next_warp_chunk(work)) {
    const int s = find_subdomain(s_prefix, n_sub, c0);  // the whole chunk's subdomain
    const int i = c0 - s_prefix[s] + lane;
    const int n_staged = top_nodes > 0 ? min(top_nodes, p.sc.n_nodes_sub[s]) : 0;
    dev_traverse_warp<kStats>(p, s, i, i < s_count[s], s_top + (size_t)s * top_nodes, n_staged, qp, rb, hits, ctl);
  }
}

// Shading of the generation's *n_in rays (children counted in *next_count).
template <int kTM, bool kPM>
__global__ void __launch_bounds__(kBlock) k_shade_g(RenderParams p, WaveDesc w, const int* n_in, RayBuf cur,
                                                    const float2* __restrict__ hits, RayBuf next, int* next_count,
                                                    uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq,
                                                    int* sq_count, float* path_L, Control* ctl) {
  // a count above the capacity was already reported by the append that overflowed
  const int n = min(*(volatile const int*)n_in, qcap);
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int r = base + (int)threadIdx.x;
    dev_shade<kTM, kPM>(p, w, r, r < n, cur, hits, next, next_count, q, q_count, qcap, sb, &ctl->next_shadow, sq,
                        sq_count, path_L, ctl);
  }
}

// The same for bundle rays.  Resident blocks per SM: a register cap that keeps more warps in
// flight for the shading's memory latency.  Measured on the nave frame (shading per frame):
// bundles of 14: no cap 63.2 ms, 4 blocks 52.6, 5 blocks 51.6, 6 blocks 49.5; bundles of 41,
// whose 42 KB of member rows per block allow 5: 4 blocks 37.2, 5 blocks 37.0, 6 blocks (5
// resident) 38.9.  With the network's tile queue (the large frame, bundles of 14) 6 blocks:
// 338 ms per frame against 457 ms with 5.  Brute-force tiles keep their registers.
template <int kTM>
constexpr int shade_blocks() { return kTM == 1 ? 1 : (kTM == 2 ? 6 : 5); }
template <int kTM, bool kPM>
__global__ void __launch_bounds__(kBlock, shade_blocks<kTM>())
    k_shade_bundle_g(RenderParams p, WaveDesc w, const int* n_in, RayBuf cur, const float2* __restrict__ hits,
                     RayBuf next, int* next_count, uint32_t* q, int* q_count, int qcap, ShadowBuf sb, uint32_t* sq,
                     int* sq_count, float* path_L, Control* ctl) {
  const int n = min(*(volatile const int*)n_in, qcap);
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int r = base + (int)threadIdx.x;
    dev_shade_bundle<kTM, kPM>(p, w, r, r < n, cur, hits, next, next_count, q, q_count, qcap, sb, &ctl->next_shadow,
                               sq, sq_count, path_L, ctl);
  }
}

// Shadow pass over the queues whose counts are counts_in (walk choice as in the other forms).
template <bool kStats, int kTM, bool kBund>
__global__ void __launch_bounds__(kChunk, kTM == 1 ? 1 : 6) k_shadow_g(RenderParams p, WaveDesc w,
                                                                      const int* counts_in, int* work,
                                                                      int block_chunks, QueuePair qp, ShadowBuf sb,
                                                                      float* path_L, Control* ctl) {
  __shared__ int s_prefix[kMaxSubdomains + 1];
  __shared__ int s_count[kMaxSubdomains];
  const int n_sub = p.sc.n_sub;
  const int total = load_prefix(counts_in, n_sub, qp.cap, s_prefix, s_count);
  const int lane = block_chunks ? (int)threadIdx.x : ((int)threadIdx.x & 31);
  for (int c0 = block_chunks ? next_block_chunk(work) : next_warp_chunk(work); c0 < total;
       c0 = block_chunks ? next_block_chunk(work) : next_warp_chunk(work)) {
    const int s = find_subdomain(s_prefix, n_sub, c0);
    const int i = c0 - s_prefix[s] + lane;
    const bool act = i < s_count[s];
    if constexpr (kBund) {
      dev_shadow_bundle<kStats, kTM, kTM == 1>(p, w, s, i, act, nullptr, 0, qp, sb, path_L, ctl);
    } else if constexpr (kTM == 1) {
      dev_shadow_warp<kStats, kTM>(p, w, s, i, act, nullptr, 0, qp, sb, path_L, ctl);
    } else {
      dev_shadow<kStats, kTM>(p, w, s, i, act, nullptr, 0, qp, sb, path_L, ctl);
    }
  }
}

__global__ void k_set_int(int* dst, int v) { *dst = v; }

// Condition of a pass loop (a conditional 'while' node whose body runs two passes): go on
// while rays remain in the queues the second pass wrote, for at most max_iter iterations
// (then the timeout bit).  kind 0 counts closest-hit passes, 1 shadow passes.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* counts, int n_sub, int max_iter, int kind,
                            Control* ctl) {
  int any = 0;
  for (int s = 0; s < n_sub; ++s) any |= counts[s] > 0;
  const int it = ++ctl->loop_iter;
  ctl->graph_passes[kind] += 2;
  if (any && it >= max_iter) atomicOr(&ctl->error, ERR_TIMEOUT);
  cudaGraphSetConditional(h, (any && it < max_iter) ? 1u : 0u);
}

// Rays left in a queue after the last pass of a generation: raise the timeout bit.
__global__ void k_check_drained(const int* counts, int n_sub, Control* ctl) {
  const int s = threadIdx.x;
  if (s < n_sub && counts[s] > 0) atomicOr(&ctl->error, ERR_TIMEOUT);
}

// Resident blocks x SMs of a kernel at a dynamic shared-memory size, queried once each.
int grid_of(const void* fn, int block, size_t smem = 0) {
  static std::mutex m;
  static std::unordered_map<const void*, std::unordered_map<size_t, int>> cache;
  std::lock_guard<std::mutex> lk(m);
  auto& c = cache[fn];
  auto it = c.find(smem);
  if (it != c.end()) return it->second;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
  const int g = std::max(1, sms * per_sm);
  c[smem] = g;
  return g;
}

// Shared memory of the staged top nodes: top_nodes per subdomain, within the 48 KB a block
// may take without opting in (fewer nodes per subdomain when there are many subdomains).
int staged_nodes(int n_sub, int top_nodes) {
  const int cap = (48 * 1024) / (std::max(n_sub, 1) * (int)sizeof(Node));
  return std::max(0, std::min(top_nodes, cap));
}

// The kernel of each step for a render's parameters.
const void* traverse_fn(const RenderParams& p) {
  return p.stats >= 2 ? (const void*)k_traverse_g<true> : (const void*)k_traverse_g<false>;
}

template <int kTM, bool kPM>
const void* shade_fn_t(bool b) {
  return b ? (const void*)k_shade_bundle_g<kTM, kPM> : (const void*)k_shade_g<kTM, kPM>;
}
const void* shade_fn(const RenderParams& p) {
  const bool b = p.bundle > 1;
  if (p.use_photons)  // photon maps: brute-force tiles or none
    return tile_mode(p) == 1 ? shade_fn_t<1, true>(b) : shade_fn_t<0, true>(b);
  switch (tile_mode(p)) {
    case 1: return shade_fn_t<1, false>(b);
    case 2: return shade_fn_t<2, false>(b);
    default: return shade_fn_t<0, false>(b);
  }
}

template <bool kStats, int kTM>
const void* shadow_fn_t(bool b) {
  return b ? (const void*)k_shadow_g<kStats, kTM, true> : (const void*)k_shadow_g<kStats, kTM, false>;
}
const void* shadow_fn(const RenderParams& p) {
  const bool b = p.bundle > 1, st = p.stats >= 2;
  switch (tile_mode(p)) {
    case 1: return st ? shadow_fn_t<true, 1>(b) : shadow_fn_t<false, 1>(b);
    case 2: return st ? shadow_fn_t<true, 2>(b) : shadow_fn_t<false, 2>(b);
    default: return st ? shadow_fn_t<true, 0>(b) : shadow_fn_t<false, 0>(b);
  }
}

cudaError_t launch_fn(const void* fn, int grid, int block, void** args, cudaStream_t st) {
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

}  // namespace

GraphGrids graph_grids(const RenderParams& p, int top_nodes, int block_chunks) {
  const int tn = staged_nodes(p.sc.n_sub, top_nodes);
  const size_t smem = (size_t)tn * p.sc.n_sub * sizeof(Node);
  const size_t shade_smem = bundle_shade_smem(p.bundle);
  allow_dynamic_smem(shade_fn(p), shade_smem);
  return GraphGrids{grid_of(traverse_fn(p), kChunk, smem), grid_of(shade_fn(p), kBlock, shade_smem),
                    grid_of(shadow_fn(p), kChunk), tn, block_chunks};
}

cudaError_t launch_traverse_g(const RenderParams& p, const GraphGrids& g, const int* counts_in, int* work,
                              QueuePair qp, RayBuf rb, float2* hits, Control* ctl, cudaStream_t st) {
  int tn = g.top_nodes, bc = g.block_chunks & 1;
  void* args[] = {(void*)&p, (void*)&counts_in, (void*)&work, (void*)&tn, (void*)&bc, (void*)&qp, (void*)&rb,
                  (void*)&hits, (void*)&ctl};
  const size_t smem = (size_t)tn * p.sc.n_sub * sizeof(Node);
  return cudaLaunchKernel(traverse_fn(p), dim3(g.traverse), dim3(kChunk), args, smem, st);
}

cudaError_t launch_shade_g(const RenderParams& p, const GraphGrids& g, const WaveDesc& w, const int* n_in,
                           RayBuf cur, const float2* hits, RayBuf next, int* next_count, uint32_t* q, int* q_count,
                           int qcap, ShadowBuf sb, uint32_t* sq, int* sq_count, float* path_L, Control* ctl,
                           cudaStream_t st) {
  void* args[] = {(void*)&p,  (void*)&w,       (void*)&n_in, (void*)&cur, (void*)&hits,     (void*)&next,
                  (void*)&next_count, (void*)&q, (void*)&q_count, (void*)&qcap, (void*)&sb, (void*)&sq,
                  (void*)&sq_count, (void*)&path_L, (void*)&ctl};
  return cudaLaunchKernel(shade_fn(p), dim3(g.shade), dim3(kBlock), args, bundle_shade_smem(p.bundle), st);
}

cudaError_t launch_shadow_g(const RenderParams& p, const GraphGrids& g, const WaveDesc& w, const int* counts_in,
                            int* work, QueuePair qp, ShadowBuf sb, float* path_L, Control* ctl, cudaStream_t st) {
  int bc = (g.block_chunks >> 1) & 1;
  void* args[] = {(void*)&p,  (void*)&w,  (void*)&counts_in, (void*)&work, (void*)&bc,
                  (void*)&qp, (void*)&sb, (void*)&path_L,    (void*)&ctl};
  return launch_fn(shadow_fn(p), g.shadow, kChunk, args, st);
}

void launch_set_int(int* dst, int v, cudaStream_t st) { k_set_int<<<1, 1, 0, st>>>(dst, v); }

void launch_loop_cond(cudaGraphConditionalHandle h, const int* counts, int n_sub, int max_iter, int kind,
                      Control* ctl, cudaStream_t st) {
  k_loop_cond<<<1, 1, 0, st>>>(h, counts, n_sub, max_iter, kind, ctl);
}

void launch_check_drained(const int* counts, int n_sub, Control* ctl, cudaStream_t st) {
  k_check_drained<<<1, kMaxSubdomains, 0, st>>>(counts, n_sub, ctl);
}

}  // namespace sdd
