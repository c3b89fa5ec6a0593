// surrogate_head.cuh -- the output head of the tile-BTDF network and its training loss,
// shared by training (train_tc.cuh) and by the renderer that samples it (surrogate_render.cu).
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

// Training loss of one row and its gradient in the network outputs z (targets y: T, R, then
// the tracer's deflection-bin fractions of each side): (T - y_T)^2 + (R - y_R)^2
// + kLobeWeight [y_T KL(h_T | m_T) + y_R KL(h_R | m_R)], m a side's mixture mass per bin,
// KL with kKlDelta added to both sides.  Returns the row's loss; g gets d loss / d z.
__device__ __forceinline__ float head_loss_row(const float* z, const float* y, float* g) {
  float l = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) g[j] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // T, R
    const float p = head_sigmoid(z[j]);
    const float d = p - y[j];
    l += d * d;
    g[j] = 2.f * d * p * (1.f - p);
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int jw = 2 + 3 * side;
    const float wt = kLobeWeight * y[side];
    const float w = head_sigmoid(z[jw]);
    const float u1 = z[jw + 1] + kLkOffset1, u2 = z[jw + 2] + kLkOffset2;
    const float k1 = expf(fminf(kLkMax, fmaxf(kLkMin, u1))), k2 = expf(fminf(kLkMax, fmaxf(kLkMin, u2)));
    const float* h = y + 2 + side * kHeadBins;
    float F1p = 0.f, F2p = 0.f, dF1p = 0.f, dF2p = 0.f;  // CDFs at the bin's lower edge
    float gw = 0.f, gk1 = 0.f, gk2 = 0.f;
    for (int b = 0; b < kHeadBins; ++b) {
      float F1, F2, dF1, dF2;
      if (b == kHeadBins - 1) {
        F1 = F2 = 1.f;
        dF1 = dF2 = 0.f;
      } else {
        const float a = head_bin_a(b + 1);
        vmf_cdf(a, k1, &F1, &dF1);
        vmf_cdf(a, k2, &F2, &dF2);
      }
      const float P1 = F1 - F1p, P2 = F2 - F2p;
      const float m = w * P1 + (1.f - w) * P2;
      const float hb = h[b];
      l += wt * hb * (logf(hb + kKlDelta) - logf(m + kKlDelta));
      const float gm = -wt * hb / (m + kKlDelta);
      gw += gm * (P1 - P2);
      gk1 += gm * w * (dF1 - dF1p);
      gk2 += gm * (1.f - w) * (dF2 - dF2p);
      F1p = F1; F2p = F2; dF1p = dF1; dF2p = dF2;
    }
    g[jw] = gw * w * (1.f - w);
    g[jw + 1] = (u1 > kLkMin && u1 < kLkMax) ? gk1 * k1 : 0.f;
    g[jw + 2] = (u2 > kLkMin && u2 < kLkMax) ? gk2 * k2 : 0.f;
  }
  return l;
}

}  // namespace sdd
