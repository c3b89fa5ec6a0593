// persistent.cu -- the batched form of the wavefront: one cooperative launch drains a
// whole wave (the kernel is in persistent_kernel.cuh; its spectral-bundle instantiations are
// compiled in persistent_bundle.cu).
#include "persistent_kernel.cuh"

namespace sdd {

// The kernel for a scene's tile mode (0 none, 1 brute force, 2 network) and path layout.
static const void* persistent_kernel(bool stats, int tile_mode, bool bundle) {
  if (bundle) return persistent_bundle_kernel(stats, tile_mode);
  switch (tile_mode) {
    case 1: return stats ? (const void*)k_persistent_wave<true, 1, false> : (const void*)k_persistent_wave<false, 1, false>;
    case 2: return stats ? (const void*)k_persistent_wave<true, 2, false> : (const void*)k_persistent_wave<false, 2, false>;
    default: return stats ? (const void*)k_persistent_wave<true, 0, false> : (const void*)k_persistent_wave<false, 0, false>;
  }
}

// Watchdog self-test: every block but the last enters a grid barrier that the last block
// never reaches; the waiting blocks give up after timeout_ns.
__global__ void k_barrier_selftest(PersistCtl* pc, Control* ctl, unsigned long long timeout_ns) {
  if (blockIdx.x == gridDim.x - 1) return;
  grid_barrier(pc, ctl, timeout_ns);
}

cudaError_t barrier_selftest(PersistCtl* pc, Control* ctl, int timeout_ms) {
  k_barrier_selftest<<<4, kPB>>>(pc, ctl, (unsigned long long)timeout_ms * 1000000ull);
  return cudaGetLastError();
}

// Blocks of the cooperative launch: every SM times the blocks of the kernel that fit on one
// (with spectral bundles of width `bundle`, their shading rows in dynamic shared memory).
int persistent_grid(bool stats, int tile_mode, int bundle) {
  const void* fn = persistent_kernel(stats, tile_mode, bundle > 1);
  if (!fn) return 0;
  const size_t smem = bundle_shade_smem(bundle);
  if (allow_dynamic_smem(fn, smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPB, smem);
  return sms * per_sm;
}

cudaError_t launch_persistent_wave(const RenderParams& p, const WaveDesc& w, const PersistBuffers& b, PersistCtl* pc,
                                   Control* ctl, int grid, cudaStream_t st, int seg) {
  void* args[] = {(void*)&p, (void*)&w, (void*)&b, (void*)&pc, (void*)&ctl, (void*)&seg};
  const void* fn = persistent_kernel(p.stats >= 2, tile_mode(p), p.bundle > 1);
  if (!fn) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPB), args, bundle_shade_smem(p.bundle), st);
}

}  // namespace sdd
