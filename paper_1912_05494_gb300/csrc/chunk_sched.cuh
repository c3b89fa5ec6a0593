// chunk_sched.cuh -- subdomain-aligned chunks of the traversal queues for kernels whose
// grid is fixed and whose queue counts are read on the device (the persistent kernel and the
// graph form's traversal kernels).
#pragma once

#include "sdd_internal.h"

namespace sdd {

namespace {

constexpr int kChunk = 128;  // rays per chunk: one 128-thread block's worth

// Per-subdomain queue counts (clamped to cap) into s_count and the exclusive prefix sums of
// the counts rounded up to whole chunks of kChunk rays into s_prefix; returns the padded total.
// A chunk then never straddles two subdomains, so every block works on one subdomain's
// queue at a time and its warps enter the traversal converged.
// The leading barrier keeps thread 0 from overwriting the shared arrays while another
// thread still reads the previous call's values: a pass that finds its queues empty leaves
// without a grid barrier, so two calls can follow each other with no barrier in between.
__device__ int load_prefix(const int* counts, int n_sub, int cap, int* s_prefix, int* s_count) {
  __shared__ int s_total;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int s = 0; s < n_sub; ++s) {
      const int c = min(max(((volatile const int*)counts)[s], 0), cap);
      s_count[s] = c;
      s_prefix[s] = acc;
      acc += (c + kChunk - 1) / kChunk * kChunk;
    }
    s_prefix[n_sub] = acc;
    s_total = acc;
  }
  __syncthreads();
  return s_total;
}

__device__ __forceinline__ int find_subdomain(const int* s_prefix, int n_sub, int j) {
  int lo = 0, hi = n_sub - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (s_prefix[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace

}  // namespace sdd
