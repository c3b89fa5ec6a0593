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

// Device-side bookkeeping of one persistent wave; the host clears it before each launch.
struct PersistCtl {
  int qc[3][kMaxSubdomains];   // closest queue counts, three rotating buffers
  int sqc[3][kMaxSubdomains];  // shadow queue counts
  int wq[3], wsq[3];           // work counters of the traversal passes
  int next_rays[2], next_shadow[2];
  unsigned bar_count, bar_gen;
  int abort;
  int pad;
};

int persistent_grid(bool stats, int tile_mode);
cudaError_t launch_persistent_wave(const RenderParams& p, const WaveDesc& w, const PersistBuffers& b, PersistCtl* pc,
                                   Control* ctl, int grid, cudaStream_t st);

}  // namespace sdd
