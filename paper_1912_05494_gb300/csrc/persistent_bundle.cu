// persistent_bundle.cu -- the persistent drain kernel with spectral bundles
// (persistent_kernel.cuh, bundle_device.cuh), compiled apart from the one-wavelength kernels
// so that the two build in parallel.
#include "persistent_kernel.cuh"

namespace sdd {

const void* persistent_bundle_kernel(bool stats, int tile_mode) {
  switch (tile_mode) {
    case 0: return stats ? (const void*)k_persistent_wave<true, 0, true> : (const void*)k_persistent_wave<false, 0, true>;
    case 1: return stats ? (const void*)k_persistent_wave<true, 1, true> : (const void*)k_persistent_wave<false, 1, true>;
    case 2: return stats ? (const void*)k_persistent_wave<true, 2, true> : (const void*)k_persistent_wave<false, 2, true>;
    default: return nullptr;
  }
}

}  // namespace sdd
