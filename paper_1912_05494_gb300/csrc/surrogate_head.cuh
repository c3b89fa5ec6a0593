// surrogate_head.cuh -- the output head of the tile-BTDF network, shared by its training
// loss (mlp.cu) and by the renderer that samples it (surrogate_render.cu).
//
// Of the network's 16 outputs z, eight are used:
//   T = sigmoid(z0), R = sigmoid(z1)
//   transmitted side: w = sigmoid(z2), log kappa_1 = z3 + 6, log kappa_2 = z4 + 1
//   reflected side:   w = sigmoid(z5), log kappa_1 = z6 + 6, log kappa_2 = z7 + 1
// (log kappa clamped to [-3, 14]).  A side's exit direction follows the mixture
// w vMF(kappa_1) + (1 - w) vMF(kappa_2) about its reference direction (straight through, or
// the mirror direction).  The vMF mass within angle alpha of its axis is
// F(a) = expm1(-kappa a) / expm1(-2 kappa), a = 1 - cos(alpha).
#pragma once

#include <cuda_runtime.h>

namespace sdd {

constexpr int kHeadPred = 8;      // predictions per row
constexpr int kHeadBins = 8;      // deflection-angle bins per side
constexpr int kHeadTargets = 2 + 2 * kHeadBins;
constexpr float kLkOffset1 = 6.f, kLkOffset2 = 1.f, kLkMin = -3.f, kLkMax = 14.f;
constexpr float kLobeWeight = 0.05f, kKlDelta = 1e-4f;

// a = 1 - cos(edge) of the bin edges 0, 1, 2, 4, 8, 16, 32, 64, 180 degrees.
__device__ __forceinline__ float head_bin_a(int e) {
  switch (e) {
    case 0: return 0.f;
    case 1: return 1.5230484360873042e-4f;
    case 2: return 6.0917298090423577e-4f;
    case 3: return 2.4359497401758023e-3f;
    case 4: return 9.7319312584296482e-3f;
    case 5: return 3.8738304061681084e-2f;
    case 6: return 0.15195190384357404f;
    case 7: return 0.56162885321092254f;
    default: return 2.f;
  }
}

// vMF mass within a = 1 - cos(angle) of the axis, and its derivative in kappa.
__device__ __forceinline__ void vmf_cdf(float a, float kappa, float* F, float* dF) {
  const float N = expm1f(-kappa * a), D = expm1f(-2.f * kappa);
  const float e2 = expf(-2.f * kappa);
  *F = N / D;
  *dF = (-a * expf(-kappa * a) * D + 2.f * N * e2) / (D * D);
}

__device__ __forceinline__ float head_sigmoid(float z) { return 1.f / (1.f + expf(-z)); }
__device__ __forceinline__ float head_log_kappa(float z, float off) { return fminf(kLkMax, fmaxf(kLkMin, z + off)); }

// Mass of the mixture (w, kappa_1, kappa_2) within a = 1 - cos(angle).
__device__ __forceinline__ float lobe_mass_within(float w, float k1, float k2, float a) {
  float F1, F2, d;
  vmf_cdf(a, k1, &F1, &d);
  vmf_cdf(a, k2, &F2, &d);
  return w * F1 + (1.f - w) * F2;
}

}  // namespace sdd
