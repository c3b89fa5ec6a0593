// surrogate_net.cuh -- the tile-BTDF network's shape, its BF16 warp-MMA building blocks, and
// the fused inference kernel used by the renderer and by sdd_surrogate_infer.
//
// Network: Fourier features of the 7 normalised inputs (48 wide) -> 4 x 128 GELU -> 16, the
// first 8 outputs mapped by the head of surrogate_head.cuh.  Parameters are one FP32 array,
// per layer W [in][out] row-major then b [out]; the BF16 copy Wt used here holds each layer
// transposed, [out][in].
//
// Fused inference: one block per SM keeps every layer's weights resident in shared memory
// (about 120 KB) and loops over chunks of 128 rows.  Each of its 8 warps owns 16 rows: it
// builds their features, runs the five layers on the tensor cores (mma.sync m16n8k16, BF16
// operands from shared memory by ldmatrix, FP32 accumulation), writes each layer's
// activations back over its own rows, and leaves the head's predictions in shared memory
// for the policy's consumer.  A policy supplies the row count (possibly read from device
// memory), each row's raw inputs and what happens to the predictions, so the renderer can
// gather its inputs from the ray state and sample the exit in the same launch.
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
constexpr int kInferWarps = 8;
constexpr int kInferRows = 16 * kInferWarps;
constexpr int kInferThreads = 32 * kInferWarps;
constexpr int kInferXLd = net::kHid + 8;  // activation tile row stride (elements)
constexpr int kInferZLd = net::kOut;      // output staging row stride (floats)

__host__ __device__ constexpr int infer_w_ld(int l) { return net::layer_in(l) + 8; }
__host__ __device__ constexpr int infer_w_offset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += net::layer_out(i) * infer_w_ld(i);
  return o;
}
constexpr size_t kInferSmem = sizeof(__nv_bfloat16) * ((size_t)infer_w_offset(net::kLayers) + kInferRows * kInferXLd) +
                              sizeof(float) * (size_t)kInferRows * kInferZLd;

namespace net {
// One hidden layer over the warp's 16 rows in place: x <- GELU(x W + b).
template <int K>
__device__ __forceinline__ void hidden_layer(__nv_bfloat16* xw, const __nv_bfloat16* w, const float* __restrict__ bias) {
  const int lane = threadIdx.x & 31;
  float acc[kHid / 8][4];
#pragma unroll
  for (int j = 0; j < kHid / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  warp_gemm<K, kHid / 8>(acc, xw, kInferXLd, w, K + 8);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < kHid / 8; ++j) {
    const int col = j * 8 + (lane & 3) * 2;
    const float b0 = __ldg(bias + col), b1 = __ldg(bias + col + 1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = (lane >> 2) + h * 8;
      *reinterpret_cast<__nv_bfloat162*>(xw + r * kInferXLd + col) =
          __floats2bfloat162_rn(gelu(acc[j][2 * h] + b0), gelu(acc[j][2 * h + 1] + b1));
    }
  }
  __syncwarp();
}
}  // namespace net

// Policy interface (device members, the policy itself stays in kernel parameter space):
//   Ctx resolve() const                       buffers the launch works on (small)
//   int count(const Ctx&) const               rows to process
//   void load(const Ctx&, int row, float q[7]) const
//   void consume(const Ctx&, int row0, int valid, const float* pred) const
//     pred = [kInferRows][kInferZLd] staging, called by every thread of the block.
template <class Policy>
__global__ void __launch_bounds__(kInferThreads, 1) k_infer_fused(SurrogateView v, const Policy pol) {
  using namespace net;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* sx = sw + infer_w_offset(kLayers);
  float* sz = reinterpret_cast<float*>(sx + kInferRows * kInferXLd);
  const typename Policy::Ctx ctx = pol.resolve();
  const int n = pol.count(ctx);
  if ((int)blockIdx.x * kInferRows >= n) return;  // whole block
#pragma unroll
  for (int l = 0; l < kLayers; ++l)
    load_tile(sw + infer_w_offset(l), infer_w_ld(l), v.Wt + layer_offset(l), layer_in(l), layer_out(l), layer_in(l),
              layer_out(l));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* xw = sx + warp * 16 * kInferXLd;
  for (int row0 = blockIdx.x * kInferRows; row0 < n; row0 += gridDim.x * kInferRows) {
    const int valid = min(kInferRows, n - row0);
    __syncthreads();  // weights staged; the previous chunk's consumer is done with sx and sz
    for (int r = threadIdx.x; r < kInferRows; r += blockDim.x) {
      float q[kIn] = {0.f, 0.f, 380.f, 2e-3f, 0.f, 1.45f, 1e-8f};
      if (r < valid) pol.load(ctx, row0 + r, q);
      features_row(q, v.Bm, sx + r * kInferXLd);
    }
    __syncthreads();
    hidden_layer<kFeat>(xw, sw + infer_w_offset(0), v.params + layer_offset(0) + kFeat * kHid);
#pragma unroll 1
    for (int l = 1; l < kLayers - 1; ++l)
      hidden_layer<kHid>(xw, sw + infer_w_offset(l), v.params + layer_offset(l) + kHid * kHid);
    {
      float acc[kOut / 8][4];
#pragma unroll
      for (int j = 0; j < kOut / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
      warp_gemm<kHid, kOut / 8>(acc, xw, kInferXLd, sw + infer_w_offset(kLayers - 1), kHid + 8);
      const float* bias = v.params + layer_offset(kLayers - 1) + kHid * kOut;
#pragma unroll
      for (int j = 0; j < kOut / 8; ++j) {
        const int col = j * 8 + (lane & 3) * 2;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = warp * 16 + (lane >> 2) + h * 8;
          sz[r * kInferZLd + col] = acc[j][2 * h] + __ldg(bias + col);
          sz[r * kInferZLd + col + 1] = acc[j][2 * h + 1] + __ldg(bias + col + 1);
        }
      }
      __syncwarp();
      if (lane < 16) {  // the head, in place over the first 8 outputs of the row
        float* z = sz + (warp * 16 + lane) * kInferZLd;
        float p[kHeadPred];
        p[0] = head_sigmoid(z[0]);
        p[1] = head_sigmoid(z[1]);
        p[2] = head_sigmoid(z[2]);
        p[3] = head_log_kappa(z[3], kLkOffset1);
        p[4] = head_log_kappa(z[4], kLkOffset2);
        p[5] = head_sigmoid(z[5]);
        p[6] = head_log_kappa(z[6], kLkOffset1);
        p[7] = head_log_kappa(z[7], kLkOffset2);
#pragma unroll
        for (int j = 0; j < kHeadPred; ++j) z[j] = p[j];
      }
    }
    __syncthreads();
    pol.consume(ctx, row0, valid, sz);
  }
}

// Rows of raw inputs [n][7] to predictions [n][8]; n read from n_dev when given (capped at n).
struct RawPolicy {
  const float* raw;
  float* out;
  int n;
  const int* n_dev;
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
};

// Blocks for a fused launch over at most n_max rows: one per SM, fewer for small n.
int infer_grid(int n_max);
// Sets the fused kernel's shared-memory limit (once per instantiation).
template <class Policy>
cudaError_t infer_prepare() {
  return cudaFuncSetAttribute(k_infer_fused<Policy>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
}

}  // namespace sdd
