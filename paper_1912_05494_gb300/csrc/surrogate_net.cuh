// surrogate_net.cuh -- the tile-BTDF network's shape, its BF16 warp-MMA building blocks (the
// training kernels of mlp.cu), the feature map, and the policy interface of the fused
// inference kernel (surrogate_tc.cuh).
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

// ------------------------------------------------------------------ warp MMA helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t r[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// acc[j] (j = n-tile of 8 columns) += A[16 rows of the warp][0..Kd) * Bt[cols][0..Kd)^T, with
// A at sa (row stride lda elements) and Bt at sb (row stride ldb elements), both shared memory.
// Accumulator layout (m16n8 fragment): acc[j][2h + e] is row (lane / 4) + 8 h, column
// 8 j + 2 (lane % 4) + e.
template <int Kd, int NT>
__device__ __forceinline__ void warp_gemm(float (*acc)[4], const __nv_bfloat16* sa, int lda, const __nv_bfloat16* sb,
                                          int ldb) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 0; kk < Kd; kk += 16) {
    uint32_t a[4];
    ldmatrix_x4(a, sa + (lane & 15) * lda + kk + (lane >> 4) * 8);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      uint32_t b[2];
      ldmatrix_x2(b, sb + (j * 8 + (lane & 7)) * ldb + kk + ((lane >> 3) & 1) * 8);
      mma16816(acc[j], a, b);
    }
  }
}

// Copy a [rows][cols] BF16 tile (row-major, `cols` contiguous, cols % 8 == 0) into shared
// memory with row stride ld; rows beyond `valid` are zero.
__device__ __forceinline__ void load_tile(__nv_bfloat16* dst, int ld, const __nv_bfloat16* src, int src_ld, int rows,
                                          int cols, int valid) {
  const int vec = cols / 8;
  for (int i = threadIdx.x; i < rows * vec; i += blockDim.x) {
    int r = i / vec, c = (i - r * vec) * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < valid) v = *reinterpret_cast<const uint4*>(src + (size_t)r * src_ld + c);
    *reinterpret_cast<uint4*>(dst + r * ld + c) = v;
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// The 48 BF16 features of one row of raw inputs q: [sin(2 pi B x), cos(2 pi B x), x, 0 pad]
// with x the inputs normalised to [0, 1].
__device__ __forceinline__ void features_row(const float q[kIn], const float* __restrict__ Bm, __nv_bfloat16* f) {
  const float x[kIn] = {0.5f * (q[0] + 1.f), q[1] * 0.15915494309189535f, (q[2] - 380.f) / 400.f,
                        (q[3] - 2e-3f) / 3e-3f, q[4] / 2e10f, (q[5] - 1.45f) / 0.2f,
                        (log10f(fmaxf(q[6], 1e-30f)) + 8.f) / 4.f};
  for (int i = 0; i < kFourier; ++i) {
    float p = 0.f;
    for (int j = 0; j < kIn; ++j) p += __ldg(Bm + i * kIn + j) * x[j];
    float s, c;
    sincospif(2.f * p, &s, &c);
    f[i] = __float2bfloat16(s);
    f[kFourier + i] = __float2bfloat16(c);
  }
  for (int j = 0; j < kIn; ++j) f[2 * kFourier + j] = __float2bfloat16(x[j]);
  for (int j = 2 * kFourier + kIn; j < kFeat; ++j) f[j] = __float2bfloat16(0.f);
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
