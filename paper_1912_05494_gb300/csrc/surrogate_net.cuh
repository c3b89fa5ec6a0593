// surrogate_net.cuh -- the tile-BTDF network's shape, its activation and feature map, and the
// policy interface of the fused inference kernel (surrogate_tc.cuh); the training kernels
// are in train_tc.cuh.
//
// Network: Fourier features of the 7 normalised inputs (48 wide) -> 4 x 128 GELU -> 16, the
// first 8 outputs mapped by the head of surrogate_head.cuh.  Parameters are one FP32 array,
// per layer W [in][out] row-major then b [out]; the BF16 copy Wt used here holds each layer
// transposed, [out][in].

#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "surrogate_head.cuh"

struct sdd_surrogate;

namespace sdd {
namespace net {

constexpr int kIn = 7, kFourier = 16, kFeat = 48, kHid = 128, kOut = 16, kLayers = 5;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kFeat : kHid; }
__host__ __device__ constexpr int layer_out(int l) { return l == kLayers - 1 ? kOut : kHid; }
__host__ __device__ constexpr int layer_offset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += layer_in(i) * layer_out(i) + layer_out(i);
  return o;
}
constexpr int kParams = layer_offset(kLayers);

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// The raw inputs q of one row normalised to [0, 1].
__device__ __forceinline__ void normalise_row(const float q[kIn], float x[kIn]) {
  x[0] = 0.5f * (q[0] + 1.f);
  x[1] = q[1] * 0.15915494309189535f;
  x[2] = (q[2] - 380.f) / 400.f;
  x[3] = (q[3] - 2e-3f) / 3e-3f;
  x[4] = q[4] / 2e10f;
  x[5] = (q[5] - 1.45f) / 0.2f;
  x[6] = (log10f(fmaxf(q[6], 1e-30f)) + 8.f) / 4.f;
}
// Fourier pair i of the normalised inputs x: sin and cos of 2 pi (B x)_i.  A row's 48 features
// are [sin(2 pi B x) (16), cos(2 pi B x) (16), x (7), zero padding (9)].
__device__ __forceinline__ void fourier_pair(const float x[kIn], const float* __restrict__ Bm, int i, float* s,
                                             float* c) {
  float p = 0.f;
  for (int j = 0; j < kIn; ++j) p += __ldg(Bm + i * kIn + j) * x[j];
  sincospif(2.f * p, s, c);
}

}  // namespace net

// Device view of a network's current weights.
struct SurrogateView {
  const __nv_bfloat16* Wt;  // BF16 weights, layer l transposed [out][in] at net::layer_offset(l)
  const float* params;      // FP32 parameters (biases read from here)
  const float* Bm;          // Fourier matrix [16][7]
};
SurrogateView surrogate_view(const sdd_surrogate* s);
unsigned surrogate_version(const sdd_surrogate* s);

// ------------------------------------------------------------------ fused inference
constexpr int kInferRows = 128;          // rows per chunk (one M = 128 tensor-core tile)
constexpr int kInferZLd = net::kOut;     // output staging row stride (floats)

// Policy interface of the fused inference kernel (k_infer_tc, surrogate_tc.cuh); the
// policy stays in kernel parameter space:
//   Ctx resolve() const                       buffers the launch works on (small)
//   int count(const Ctx&) const               rows to process
//   void load(const Ctx&, int row, float q[7]) const
//   void consume(const Ctx&, int row0, int valid, const float* pred) const
//     pred = [kInferRows][kInferZLd] staging, called by every thread of the block
//   uint32_t* err(const Ctx&) const           error word for the timeout bit

// Rows of raw inputs [n][7] to predictions [n][8]; n read from n_dev when given (capped at n).
struct RawPolicy {
  const float* raw;
  float* out;
  int n;
  const int* n_dev;
  uint32_t* errw;
  struct Ctx {};
  __device__ Ctx resolve() const { return Ctx{}; }
  __device__ int count(const Ctx&) const { return n_dev ? min(*(volatile const int*)n_dev, n) : n; }
  __device__ void load(const Ctx&, int row, float q[net::kIn]) const {
#pragma unroll
    for (int j = 0; j < net::kIn; ++j) q[j] = raw[(size_t)row * net::kIn + j];
  }
  __device__ void consume(const Ctx&, int row0, int valid, const float* pred) const {
    for (int i = threadIdx.x; i < valid * kHeadPred; i += blockDim.x)
      out[(size_t)row0 * kHeadPred + i] = pred[(i / kHeadPred) * kInferZLd + i % kHeadPred];
  }
  __device__ uint32_t* err(const Ctx&) const { return errw; }
};

// Blocks for a fused launch over at most n_max rows: one per SM, fewer for small n.
int infer_grid(int n_max);

}  // namespace sdd
