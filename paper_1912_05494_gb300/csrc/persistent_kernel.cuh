// persistent_kernel.cuh -- the persistent drain kernel of one wave (the batched form),
// included by persistent.cu (one wavelength per path) and persistent_bundle.cu (spectral
// bundles); both translation units are compiled with global loads cached at L2 only.
//
// Sec. 5 of the paper lets a processor keep several sub-domains loaded, work on whichever
// still has many rays, and gather results while other rays are processed; Sec. 4 asks for
// dynamic job balancing so that faster workers take more work.  On one GB300 this becomes a
// persistent kernel: every block loops over
//   raygen -> per generation: [closest-hit passes over all subdomain queues, blocks taking
//   128-ray chunks from a shared work counter] -> shade -> [shadow passes] -> film
// with grid-wide barriers between the steps instead of host round trips.  The per-ray work
// is the same device code as the host-driven kernels (render_device.cuh), so both forms
// produce bit-identical images.
//
// Queue bookkeeping without races: queue counts rotate through three buffers.  The step
// that consumes buffer c appends hand-offs into c+1 and clears c+2 (consumed two steps ago,
// copied by every block before the barrier that ended that step), so a buffer is always
// cleared one barrier before anyone appends to it.  Work counters rotate the same way.  A
// pass that finds its input empty ends without a barrier, so nothing may write its input
// buffer until the next barrier: the following step writes the next buffer instead.
//
// Every grid barrier waits at most kBarrierTimeoutNs; on expiry the block sets the abort
// flag and the frame's error word, all blocks leave at their next barrier and the host
// reports SDD_ERR_TIMEOUT.
#pragma once

#include <cooperative_groups.h>

#include "bundle_device.cuh"
#include "chunk_sched.cuh"
#include "persistent.cuh"

namespace sdd {

namespace {

constexpr int kPB = 128;  // threads per block
static_assert(kPB == kShadeThreads, "bundle shading rows are sized for kShadeThreads threads");
constexpr int kBundleBlocks = 4;  // resident blocks per SM of the spectral-bundle kernels (measured best of 4, 6, 8)
constexpr unsigned long long kBarrierTimeoutNs = 5ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a time limit.  Returns false when the wave must be abandoned.
__device__ bool grid_barrier(PersistCtl* pc, Control* ctl, unsigned long long timeout_ns = kBarrierTimeoutNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &pc->bar_gen;
    volatile int* vabort = &pc->abort;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(&pc->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      pc->bar_count = 0;
      __threadfence();
      atomicAdd(&pc->bar_gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (*vabort) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(&pc->abort, 1);
          atomicOr(&ctl->error, ERR_TIMEOUT);  // survives the next wave's reset of pc
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *vabort == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Clear the count buffer and work counter that the step after next will write.
__device__ __forceinline__ void clear_ahead(int (*counts)[kMaxSubdomains], int* work, int idx) {
  if (blockIdx.x == 0) {
    for (int s = threadIdx.x; s < kMaxSubdomains; s += blockDim.x) counts[idx][s] = 0;
    if (threadIdx.x == 0) work[idx] = 0;
  }
}

}  // namespace

// Eight resident blocks per SM (registers bounded at 64; ~150 B of spills) for scenes
// without brute-force tiles: measured faster than 6 (80 registers, no spills), 10 or 12 (more
// spills); the brute-force tile tracer needs 128 registers (four blocks).
// kBund: spectral bundles (bundle_device.cuh) in place of one wavelength per path.
template <bool kStats, int kTM, bool kBund>
__global__ void __launch_bounds__(kPB, kTM == 1 ? 4 : (kBund ? kBundleBlocks : 8)) k_persistent_wave(RenderParams p, WaveDesc w, PersistBuffers b,
                                                         PersistCtl* pc, Control* ctl, int seg) {
  __shared__ int s_prefix[kMaxSubdomains + 1];
  __shared__ int s_count[kMaxSubdomains];
  __shared__ int s_chunk;
  const int n_sub = p.sc.n_sub;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;

  PersistState S;
  if (seg == SEG_WAVE || seg == SEG_RAYGEN) {
    // raygen: primary rays into generation 0 and the closest queues (counts buffer 0)
    for (uint32_t base = blockIdx.x * blockDim.x; base < w.n_paths; base += nthreads) {
      uint32_t i = base + threadIdx.x;
      if constexpr (kBund) {
        dev_raygen_bundle(p, w, i, i < w.n_paths, b.rb[0], b.q[0], pc->qc[0], b.qcap, ctl);
      } else {
        dev_raygen(p, w, i, i < w.n_paths, b.rb[0], b.q[0], pc->qc[0], b.qcap, ctl);
      }
    }
    if (!grid_barrier(pc, ctl)) return;
    S = PersistState{0, 0, 0, 0, 0, (int)w.n_paths, 0, 0};
    if (seg == SEG_RAYGEN) {
      if (leader) pc->st = S;
      return;
    }
  } else {
    const volatile PersistState* vs = &pc->st;
    S = PersistState{vs->cq, vs->qe, vs->sq, vs->se, vs->cur, vs->n_rays, vs->gen, 0};
    if (S.n_rays <= 0 || *(volatile int*)&pc->abort) return;  // drained or abandoned
  }

  while (S.n_rays > 0) {
    if (S.gen > p.max_depth + 1) {
      if (leader) atomicOr(&ctl->error, ERR_TIMEOUT);
      S.n_rays = 0;
      break;
    }
    const int par = S.gen & 1;
    if (seg != SEG_SHADOW) {
      if (leader) {
        pc->next_rays[par] = 0;
        pc->next_shadow[par] = 0;
      }
      bool ran_pass = false;
      for (int pass = 0; pass <= 2 * kMaxSubdomains + 2; ++pass) {
        int total = load_prefix(pc->qc[S.cq], n_sub, b.qcap, s_prefix, s_count);
        clear_ahead(pc->qc, pc->wq, (S.cq + 2) % 3);
        if (total == 0) break;
        QueuePair qp{b.q[S.qe], b.q[1 - S.qe], pc->qc[(S.cq + 1) % 3], b.qcap};
        for (;;) {
          if (threadIdx.x == 0) s_chunk = atomicAdd(&pc->wq[S.cq], (int)blockDim.x);
          __syncthreads();
          const int c0 = s_chunk;
          __syncthreads();
          if (c0 >= total) break;
          const int s = find_subdomain(s_prefix, n_sub, c0);  // the whole chunk's subdomain
          const int i = c0 - s_prefix[s] + (int)threadIdx.x;
          dev_traverse_warp<kStats>(p, s, i, i < s_count[s], nullptr, 0, qp, b.rb[S.cur], b.hits, ctl);
        }
        ran_pass = true;
        if (!grid_barrier(pc, ctl)) return;
        S.cq = (S.cq + 1) % 3;
        S.qe = 1 - S.qe;
      }
      if (!ran_pass && !grid_barrier(pc, ctl)) return;

      // Shade every ray of this generation.  The last closest pass found its input buffer
      // cq empty and left without a barrier, so slower blocks may still be reading cq:
      // children go to the next buffer in the rotation instead (cleared two steps ago, read
      // by nobody), and the rotation moves past the empty pass.  Shadow rays go to the
      // shadow queues; tile hits for the network go to the tile queue.
      for (uint32_t base = blockIdx.x * blockDim.x; base < (uint32_t)S.n_rays; base += nthreads) {
        int r = (int)(base + threadIdx.x);
        if constexpr (kBund) {
          dev_shade_bundle<kTM>(p, w, r, r < S.n_rays, b.rb[S.cur], b.hits, b.rb[1 - S.cur], &pc->next_rays[par],
                                b.q[1 - S.qe], pc->qc[(S.cq + 1) % 3], b.qcap, b.sb, &pc->next_shadow[par],
                                b.sq[S.se], pc->sqc[S.sq], b.path_L, ctl);
        } else {
          dev_shade<kTM>(p, w, r, r < S.n_rays, b.rb[S.cur], b.hits, b.rb[1 - S.cur], &pc->next_rays[par],
                         b.q[1 - S.qe], pc->qc[(S.cq + 1) % 3], b.qcap, b.sb, &pc->next_shadow[par], b.sq[S.se],
                         pc->sqc[S.sq], b.path_L, ctl);
        }
      }
      S.cq = (S.cq + 1) % 3;
      S.qe = 1 - S.qe;
      if (!grid_barrier(pc, ctl)) return;
      if (seg == SEG_CLOSEST_SHADE) {
        if (leader) pc->st = S;  // every block holds the same state
        return;
      }
    }

    for (int pass = 0; pass <= 2 * kMaxSubdomains + 2; ++pass) {
      int total = load_prefix(pc->sqc[S.sq], n_sub, b.qcap, s_prefix, s_count);
      clear_ahead(pc->sqc, pc->wsq, (S.sq + 2) % 3);
      if (total == 0) break;
      QueuePair qp{b.sq[S.se], b.sq[1 - S.se], pc->sqc[(S.sq + 1) % 3], b.qcap};
      for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(&pc->wsq[S.sq], (int)blockDim.x);
        __syncthreads();
        const int c0 = s_chunk;
        __syncthreads();
        if (c0 >= total) break;
        const int s = find_subdomain(s_prefix, n_sub, c0);
        const int i = c0 - s_prefix[s] + (int)threadIdx.x;
        if constexpr (kBund) {
          dev_shadow_bundle<kStats, kTM, kTM == 1>(p, w, s, i, i < s_count[s], nullptr, 0, qp, b.sb, b.path_L, ctl);
        } else if constexpr (kTM == 1) {  // the same walk choice as the host-driven shadow kernel
          dev_shadow_warp<kStats, kTM>(p, w, s, i, i < s_count[s], nullptr, 0, qp, b.sb, b.path_L, ctl);
        } else {
          dev_shadow<kStats, kTM>(p, w, s, i, i < s_count[s], nullptr, 0, qp, b.sb, b.path_L, ctl);
        }
      }
      if (!grid_barrier(pc, ctl)) return;
      S.sq = (S.sq + 1) % 3;
      S.se = 1 - S.se;
    }
    S.n_rays = min(*(volatile int*)&pc->next_rays[par], b.qcap);
    if (*(volatile int*)&pc->next_rays[par] > b.qcap && leader) atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
    S.cur = 1 - S.cur;
    S.gen++;
    if (seg == SEG_SHADOW) break;
  }
  if (seg != SEG_WAVE && leader) pc->st = S;
}

}  // namespace sdd
