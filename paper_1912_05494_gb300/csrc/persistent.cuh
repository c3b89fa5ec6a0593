// persistent.cuh -- the persistent drain kernel of one wave (persistent.cu).
#pragma once

#include "sdd_internal.h"

namespace sdd {

struct PersistBuffers {
  RayBuf rb[2];       // ray generations
  float2* hits;
  uint32_t* q[2];     // closest-hit queue entries [n_sub][qcap], alternating per pass
  ShadowBuf sb;
  uint32_t* sq[2];    // shadow queue entries
  float* path_L;
  int qcap;
};

// Queue-rotation state of a wave between segment launches (see SEG_* below).
struct PersistState {
  int cq, qe;   // closest queues: counts buffer and entries buffer of the next input
  int sq, se;   // shadow queues
  int cur;      // ray generation buffer being shaded
  int n_rays;   // rays of the current generation; 0 when the wave is drained
  int gen;
  int pad;
};

// What one launch of the persistent kernel covers.  SEG_WAVE drains the whole wave.  For
// scenes whose tile hits go to the network the wave is split: SEG_RAYGEN, then per
// generation SEG_CLOSEST_SHADE (closest passes and shading) and SEG_SHADOW (shadow passes),
// with the fused tile-shading launch between the two; launches after the wave is drained
// return at once, so a fixed sequence of max_depth + 2 generations covers every wave.
enum PersistSegment : int { SEG_WAVE = 0, SEG_RAYGEN = 1, SEG_CLOSEST_SHADE = 2, SEG_SHADOW = 3 };

// Device-side bookkeeping of one persistent wave; the host clears it before each wave.
struct PersistCtl {
  int qc[3][kMaxSubdomains];   // closest queue counts, three rotating buffers
  int sqc[3][kMaxSubdomains];  // shadow queue counts
  int wq[3], wsq[3];           // work counters of the traversal passes
  int next_rays[2], next_shadow[2];
  unsigned bar_count, bar_gen;
  int abort;
  int pad;
  PersistState st;
};

// Blocks of the cooperative launch (SMs x resident blocks) for a scene's tile mode (0 none,
// 1 brute force, 2 network), with or without spectral bundles.
int persistent_grid(bool stats, int tile_mode, int bundle);
// The spectral-bundle kernels (persistent_bundle.cu) per tile mode; nullptr otherwise.
const void* persistent_bundle_kernel(bool stats, int tile_mode);
// Runs k_barrier_selftest (four blocks, the last never arrives) on the legacy stream.
cudaError_t barrier_selftest(PersistCtl* pc, Control* ctl, int timeout_ms);
cudaError_t launch_persistent_wave(const RenderParams& p, const WaveDesc& w, const PersistBuffers& b, PersistCtl* pc,
                                   Control* ctl, int grid, cudaStream_t st, int seg = SEG_WAVE);

}  // namespace sdd
