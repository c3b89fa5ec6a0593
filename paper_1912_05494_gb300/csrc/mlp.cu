// mlp.cu -- the tile-BTDF surrogate network on BF16 tensor cores: training (forward,
// backward, Adam) and inference.
//
// The paper models glass as refractive only and names scattering in heterogeneous tiles as
// future work (Sec. 6).  The brute-force tile tracer (tile.cu) resolves it exactly but is
// costly at every tile hit; this network learns the tile's BTDF statistics from the
// tracer's samples:
//   inputs   signed cos(theta_in) (> 0 through the flat front face, < 0 through the rough back),
//            phi_in, lambda, mean thickness, bubble density, n, k, normalised to [0, 1]:
//            (cos + 1) / 2, phi / 2 pi, (lambda - 380) / 400, (d - 2 mm) / 3 mm,
//            rho / 2e10 m^-3, (n - 1.45) / 0.2, (log10 k + 8) / 4
//   features [sin(2 pi B x), cos(2 pi B x), x, 0 pad] (B: 16 x 7), 48 wide
//   layers   48 -> 128 -> 128 -> 128 -> 128 -> 16, exact GELU after the hidden layers
//   head     T, R and a two-lobe vMF mixture per side (surrogate_head.cuh)
//   loss     mean over the batch of (T - y_T)^2 + (R - y_R)^2
//            + 0.05 [y_T KL(h_T | m_T) + y_R KL(h_R | m_R)], h the tracer's deflection-bin
//            fractions, m the mixture's mass per bin; Adam on FP32 master weights
// Training: weights and activations are BF16, products accumulate in FP32 (mma.sync
// m16n8k16, fragments loaded with ldmatrix from padded shared-memory tiles).  Inference
// (sdd_surrogate_infer and the renderer) runs the fused tcgen05 kernel of surrogate_tc.cuh.
// Parameters are one flat FP32 array: for each layer W [in][out] row-major, then b [out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "surrogate_head.cuh"
#include "surrogate_net.cuh"
#include "surrogate_tc.cuh"

namespace sdd {
sdd_status set_last_error(sdd_status st, const char* msg);
}
using namespace sdd;

namespace {

using namespace sdd::net;
constexpr int kTargets = kHeadTargets;
constexpr int kRows = 128;    // batch rows per block
constexpr int kThreads = 256;  // 8 warps, 16 rows each

// ------------------------------------------------------------------ kernels
__global__ void k_features(int n, const float* __restrict__ raw, const float* __restrict__ Bm,
                           __nv_bfloat16* __restrict__ feat) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float q[kIn];
  for (int j = 0; j < kIn; ++j) q[j] = raw[(size_t)r * kIn + j];
  features_row(q, Bm, feat + (size_t)r * kFeat);
}

// Z = X W + b (X [n][K] bf16, Wt = W^T [N][K] bf16); hidden layers store Z (bf16) and GELU(Z)
// (bf16), the output layer stores Z in FP32.
template <int K, int N, bool kHidden>
__global__ void __launch_bounds__(kThreads) k_layer_fwd(int n, const __nv_bfloat16* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ Wt,
                                                         const float* __restrict__ bias, __nv_bfloat16* Zb, float* Zf,
                                                         __nv_bfloat16* A) {
  constexpr int LD = K + 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* sw = sx + kRows * LD;
  const int row0 = blockIdx.x * kRows;
  load_tile(sx, LD, X + (size_t)row0 * K, K, kRows, K, min(kRows, n - row0));
  load_tile(sw, LD, Wt, K, N, K, N);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[N / 8][4];
#pragma unroll
  for (int j = 0; j < N / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  warp_gemm<K, N / 8>(acc, sx + warp * 16 * LD, LD, sw, LD);
#pragma unroll
  for (int j = 0; j < N / 8; ++j) {
    const int col = j * 8 + (lane & 3) * 2;
    const float b0 = bias[col], b1 = bias[col + 1];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = row0 + warp * 16 + (lane >> 2) + h * 8;
      if (r >= n) continue;
      float z0 = acc[j][2 * h] + b0, z1 = acc[j][2 * h + 1] + b1;
      size_t o = (size_t)r * N + col;
      if (kHidden) {
        *reinterpret_cast<__nv_bfloat162*>(Zb + o) = __floats2bfloat162_rn(z0, z1);
        *reinterpret_cast<__nv_bfloat162*>(A + o) = __floats2bfloat162_rn(gelu(z0), gelu(z1));
      } else {
        Zf[o] = z0;
        Zf[o + 1] = z1;
      }
    }
  }
}

// Loss of one row (head and loss in surrogate_head.cuh) and dZ = d(mean loss)/dZ for the
// output layer.
__global__ void k_loss(int n, float inv_batch, const float* __restrict__ Z, const float* __restrict__ Y,
                       __nv_bfloat16* __restrict__ dZ, float* loss_sum) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (r < n) {
    const float* z = Z + (size_t)r * kOut;
    const float* y = Y + (size_t)r * kTargets;
    float g[kOut];
#pragma unroll
    for (int j = 0; j < kOut; ++j) g[j] = 0.f;
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
#pragma unroll
    for (int j = 0; j < kOut; ++j) dZ[(size_t)r * kOut + j] = __float2bfloat16(g[j] * inv_batch);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, l);
}

// dZ_prev = (dZ W^T) * GELU'(Z_prev): dZ [n][N], W [K][N] (as the B operand, K output
// columns, N reduction), Z_prev [n][K].
template <int N, int K>
__global__ void __launch_bounds__(kThreads) k_layer_bwd_data(int n, const __nv_bfloat16* __restrict__ dZ,
                                                              const __nv_bfloat16* __restrict__ W,
                                                              const __nv_bfloat16* __restrict__ Zprev,
                                                              __nv_bfloat16* __restrict__ dZprev) {
  constexpr int LD = N + 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sd = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* sw = sd + kRows * LD;
  const int row0 = blockIdx.x * kRows;
  load_tile(sd, LD, dZ + (size_t)row0 * N, N, kRows, N, min(kRows, n - row0));
  load_tile(sw, LD, W, N, K, N, K);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[K / 8][4];
#pragma unroll
  for (int j = 0; j < K / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  warp_gemm<N, K / 8>(acc, sd + warp * 16 * LD, LD, sw, LD);
#pragma unroll
  for (int j = 0; j < K / 8; ++j) {
    const int col = j * 8 + (lane & 3) * 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = row0 + warp * 16 + (lane >> 2) + h * 8;
      if (r >= n) continue;
      size_t o = (size_t)r * K + col;
      __nv_bfloat162 zp = *reinterpret_cast<const __nv_bfloat162*>(Zprev + o);
      float g0 = acc[j][2 * h] * gelu_grad(__bfloat162float(zp.x));
      float g1 = acc[j][2 * h + 1] * gelu_grad(__bfloat162float(zp.y));
      *reinterpret_cast<__nv_bfloat162*>(dZprev + o) = __floats2bfloat162_rn(g0, g1);
    }
  }
}

// This block's share of dW = X^T dZ and db = column sums of dZ over its row chunks (X [n][K],
// dZ [n][N]), written to part + blockIdx.x (K N + N) as [K][N] then [N]; k_reduce_partials
// sums the blocks' shares in block order, so the gradients do not depend on scheduling.
template <int K, int N>
__global__ void __launch_bounds__(kThreads) k_layer_bwd_weight(int n, const __nv_bfloat16* __restrict__ X,
                                                                const __nv_bfloat16* __restrict__ dZ, float* part) {
  float* dW = part + (size_t)blockIdx.x * (K * N + N);
  float* db = dW + K * N;
  constexpr int LD = kRows + 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sxt = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [K][LD]: X^T of the chunk
  __nv_bfloat16* sdt = sxt + K * LD;                                // [N][LD]: dZ^T of the chunk
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[N / 8][4];
#pragma unroll
  for (int j = 0; j < N / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  float bsum = 0.f;  // thread t < N sums column t
  const int chunks = (n + kRows - 1) / kRows;
  for (int c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int row0 = c * kRows, valid = min(kRows, n - row0);
    __syncthreads();
    for (int i = threadIdx.x; i < kRows * K; i += blockDim.x) {
      int r = i / K, k = i - r * K;
      sxt[k * LD + r] = r < valid ? X[(size_t)(row0 + r) * K + k] : __float2bfloat16(0.f);
    }
    for (int i = threadIdx.x; i < kRows * N; i += blockDim.x) {
      int r = i / N, k = i - r * N;
      sdt[k * LD + r] = r < valid ? dZ[(size_t)(row0 + r) * N + k] : __float2bfloat16(0.f);
    }
    __syncthreads();
    if (warp < K / 16) warp_gemm<kRows, N / 8>(acc, sxt + warp * 16 * LD, LD, sdt, LD);
    if (threadIdx.x < N)
      for (int r = 0; r < valid; ++r) bsum += __bfloat162float(sdt[threadIdx.x * LD + r]);
  }
  if (warp < K / 16) {
#pragma unroll
    for (int j = 0; j < N / 8; ++j) {
      const int col = j * 8 + (lane & 3) * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = warp * 16 + (lane >> 2) + h * 8;
        dW[(size_t)k * N + col] = acc[j][2 * h];
        dW[(size_t)k * N + col + 1] = acc[j][2 * h + 1];
      }
    }
  }
  if (threadIdx.x < N) db[threadIdx.x] = bsum;
}

// out[i] = sum over the blocks b = 0 .. nblk - 1, in order, of part[b len + i].
__global__ void k_reduce_partials(int nblk, int len, const float* __restrict__ part, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float acc = 0.f;
  for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * len + i];
  out[i] = acc;
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of the weights in both layouts: W [K][N] and Wt [N][K].
__global__ void k_weights_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ Wb,
                               __nv_bfloat16* __restrict__ Wtb) {
  int l = blockIdx.y;
  const int K = layer_in(l), N = layer_out(l);
  const float* W = p + layer_offset(l);
  __nv_bfloat16* wb = Wb + layer_offset(l);
  __nv_bfloat16* wt = Wtb + layer_offset(l);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * N; i += gridDim.x * blockDim.x) {
    int k = i / N, c = i - k * N;
    __nv_bfloat16 v = __float2bfloat16(W[i]);
    wb[i] = v;
    wt[c * K + k] = v;
  }
}

// Rows of one minibatch: row j of the batch is row (a (off + j) + c) mod n of the samples,
// a bijection of [0, n) when gcd(a, n) = 1.
__global__ void k_gather_batch(int n, int batch, long long off, long long a, long long c, const float* __restrict__ raw,
                               const float* __restrict__ y, float* __restrict__ braw, float* __restrict__ by) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  const long long src = (a * ((off + j) % n) + c) % n;
  for (int k = 0; k < 7; ++k) braw[(size_t)j * 7 + k] = raw[(size_t)src * 7 + k];
  for (int k = 0; k < kTargets; ++k) by[(size_t)j * kTargets + k] = y[(size_t)src * kTargets + k];
}

__global__ void k_record_loss(const float* loss_sum, float inv_batch, float* out) { *out = *loss_sum * inv_batch; }

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(p, sizeof(T) * (n > 0 ? n : 1));
}

}  // namespace

struct sdd_surrogate {
  int max_batch = 0;
  float* params = nullptr;  // FP32 master weights
  float* grads = nullptr;
  float* partial = nullptr;  // per-block shares of one layer's gradient [partial_blocks][K N + N]
  int partial_blocks = 0;
  float* m = nullptr;
  float* v = nullptr;
  float* Bm = nullptr;      // Fourier matrix [16][7]
  __nv_bfloat16* Wb = nullptr;
  __nv_bfloat16* Wtb = nullptr;
  __nv_bfloat16* feat = nullptr;            // [batch][48]
  __nv_bfloat16* Z[kLayers - 1] = {};        // hidden pre-activations [batch][128]
  __nv_bfloat16* A[kLayers - 1] = {};        // hidden activations
  float* Zout = nullptr;                     // [batch][16]
  __nv_bfloat16* dZ[2] = {};                 // [batch][128]
  float* loss = nullptr;
  uint32_t* err = nullptr;  // timeout bit of the inference kernel's bounded waits
  float* batch_raw = nullptr;  // minibatch scratch of sdd_surrogate_train [max_batch][7]
  float* batch_y = nullptr;    // [max_batch][18]
  int step = 0;
  unsigned version = 0;  // bumped whenever the weights change
  ~sdd_surrogate() {
    cudaFree(params); cudaFree(grads); cudaFree(partial); cudaFree(m); cudaFree(v); cudaFree(Bm); cudaFree(Wb); cudaFree(Wtb);
    cudaFree(feat); cudaFree(Zout); cudaFree(loss); cudaFree(err); cudaFree(batch_raw); cudaFree(batch_y);
    for (auto* p : Z) cudaFree(p);
    for (auto* p : A) cudaFree(p);
    for (auto* p : dZ) cudaFree(p);
  }
};

namespace {

size_t fwd_smem(int K, int N) { return sizeof(__nv_bfloat16) * (size_t)(kRows + N) * (K + 8); }
size_t bwdd_smem(int N, int K) { return sizeof(__nv_bfloat16) * (size_t)(kRows + K) * (N + 8); }
size_t bwdw_smem(int K, int N) { return sizeof(__nv_bfloat16) * (size_t)(K + N) * (kRows + 8); }

template <int K, int N, bool H>
void set_fwd_attr() {
  cudaFuncSetAttribute(k_layer_fwd<K, N, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(K, N));
}

sdd_status check(cudaError_t e) {
  return e == cudaSuccess ? SDD_OK : set_last_error(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,
                                                    cudaGetErrorString(e));
}

// Forward pass of n rows of raw inputs; leaves Zout (FP32) and the hidden Z/A buffers.
cudaError_t forward(sdd_surrogate* s, int n, const float* raw, cudaStream_t st) {
  k_features<<<(n + 127) / 128, 128, 0, st>>>(n, raw, s->Bm, s->feat);
  const int blocks = (n + kRows - 1) / kRows;
  k_layer_fwd<kFeat, kHid, true><<<blocks, kThreads, fwd_smem(kFeat, kHid), st>>>(
      n, s->feat, s->Wtb + layer_offset(0), s->params + layer_offset(0) + kFeat * kHid, s->Z[0], nullptr, s->A[0]);
  for (int l = 1; l < kLayers - 1; ++l)
    k_layer_fwd<kHid, kHid, true><<<blocks, kThreads, fwd_smem(kHid, kHid), st>>>(
        n, s->A[l - 1], s->Wtb + layer_offset(l), s->params + layer_offset(l) + kHid * kHid, s->Z[l], nullptr,
        s->A[l]);
  k_layer_fwd<kHid, kOut, false><<<blocks, kThreads, fwd_smem(kHid, kOut), st>>>(
      n, s->A[kLayers - 2], s->Wtb + layer_offset(4), s->params + layer_offset(4) + kHid * kOut, nullptr, s->Zout,
      nullptr);
  return cudaGetLastError();
}

// Loss and gradients of n rows into s->grads (zeroed first); loss sum in s->loss.
cudaError_t backward(sdd_surrogate* s, int n, const float* raw, const float* y, cudaStream_t st) {
  cudaError_t e = forward(s, n, raw, st);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(s->loss, 0, sizeof(float), st);
  k_loss<<<(n + 127) / 128, 128, 0, st>>>(n, 1.f / n, s->Zout, y, s->dZ[0], s->loss);
  const int blocks = (n + kRows - 1) / kRows;
  const int wblocks = std::min(blocks, s->partial_blocks);
  auto reduce = [&](int l) {
    const int len = layer_in(l) * layer_out(l) + layer_out(l);
    k_reduce_partials<<<(len + 255) / 256, 256, 0, st>>>(wblocks, len, s->partial, s->grads + layer_offset(l));
  };
  // output layer
  k_layer_bwd_weight<kHid, kOut><<<wblocks, kThreads, bwdw_smem(kHid, kOut), st>>>(n, s->A[3], s->dZ[0], s->partial);
  reduce(4);
  k_layer_bwd_data<kOut, kHid><<<blocks, kThreads, bwdd_smem(kOut, kHid), st>>>(n, s->dZ[0], s->Wb + layer_offset(4),
                                                                               s->Z[3], s->dZ[1]);
  int cur = 1;
  for (int l = kLayers - 2; l >= 1; --l) {
    k_layer_bwd_weight<kHid, kHid><<<wblocks, kThreads, bwdw_smem(kHid, kHid), st>>>(n, s->A[l - 1], s->dZ[cur],
                                                                                    s->partial);
    reduce(l);
    k_layer_bwd_data<kHid, kHid><<<blocks, kThreads, bwdd_smem(kHid, kHid), st>>>(
        n, s->dZ[cur], s->Wb + layer_offset(l), s->Z[l - 1], s->dZ[1 - cur]);
    cur = 1 - cur;
  }
  k_layer_bwd_weight<kFeat, kHid><<<wblocks, kThreads, bwdw_smem(kFeat, kHid), st>>>(n, s->feat, s->dZ[cur],
                                                                                    s->partial);
  reduce(0);
  return cudaGetLastError();
}

// One Adam step on n rows (enqueued on st): gradients, moments, parameters, BF16 copies.
cudaError_t adam_step(sdd_surrogate* s, int n, const float* raw, const float* y, float lr, cudaStream_t st) {
  cudaError_t e = backward(s, n, raw, y, st);
  if (e != cudaSuccess) return e;
  s->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
  k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(kParams, s->params, s->grads, s->m, s->v, lr, b1, b2, 1e-8f, c1, c2);
  s->version++;
  k_weights_bf16<<<dim3(16, kLayers), 256, 0, st>>>(s->params, s->Wb, s->Wtb);
  return cudaGetLastError();
}

long long gcd_ll(long long a, long long b) {
  while (b) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

namespace sdd {
SurrogateView surrogate_view(const sdd_surrogate* s) { return SurrogateView{s->Wtb, s->params, s->Bm}; }
unsigned surrogate_version(const sdd_surrogate* s) { return s->version; }

int infer_grid(int n_max) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return std::max(1, std::min(sms, (n_max + kInferRows - 1) / kInferRows));
}

// Predictions [n][8] for raw inputs [n][7] (fused tcgen05 inference), enqueued on st; with
// n_dev the row count is read on the device (at most n).  A timeout of the kernel's bounded
// waits sets the surrogate's error word (checked by sdd_surrogate_infer).
cudaError_t surrogate_predict(sdd_surrogate* s, int n, const float* raw, float* out, cudaStream_t st,
                              const int* n_dev) {
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e = infer_tc_prepare<RawPolicy>();
    if (e != cudaSuccess) return e;
    prepared = true;
  }
  if (n <= 0) return cudaSuccess;
  k_infer_tc<RawPolicy><<<infer_grid(n), tc::kThreads, tc::kSmem, st>>>(surrogate_view(s),
                                                                       RawPolicy{raw, out, n, n_dev, s->err});
  return cudaGetLastError();
}
}  // namespace sdd

extern "C" {

sdd_status sdd_surrogate_create(const float* fourier_B, const float* init_params, int n_params, int max_batch,
                                sdd_surrogate** out) {
  if (!fourier_B || !init_params || !out || max_batch < 1) return set_last_error(SDD_ERR_ARG, "bad arguments");
  if (n_params != kParams)
    return set_last_error(SDD_ERR_ARG, ("n_params must be " + std::to_string(kParams)).c_str());
  *out = nullptr;
  static bool attrs = false;
  if (!attrs) {
    set_fwd_attr<kFeat, kHid, true>();
    set_fwd_attr<kHid, kHid, true>();
    set_fwd_attr<kHid, kOut, false>();
    cudaFuncSetAttribute(k_layer_bwd_data<kHid, kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdd_smem(kHid, kHid));
    cudaFuncSetAttribute(k_layer_bwd_data<kOut, kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdd_smem(kOut, kHid));
    cudaFuncSetAttribute(k_layer_bwd_weight<kHid, kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdw_smem(kHid, kHid));
    cudaFuncSetAttribute(k_layer_bwd_weight<kHid, kOut>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdw_smem(kHid, kOut));
    cudaFuncSetAttribute(k_layer_bwd_weight<kFeat, kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdw_smem(kFeat, kHid));
    attrs = true;
  }
  sdd_surrogate* s = new sdd_surrogate;
  s->max_batch = max_batch;
  const size_t mb = (size_t)max_batch;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  A(dalloc(&s->params, kParams));
  A(dalloc(&s->grads, kParams));
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->partial_blocks = std::max(1, 2 * sms);
    A(dalloc(&s->partial, (size_t)s->partial_blocks * (kHid * kHid + kHid)));
  }
  A(dalloc(&s->m, kParams));
  A(dalloc(&s->v, kParams));
  A(dalloc(&s->Bm, 16 * 7));
  A(dalloc(&s->Wb, kParams));
  A(dalloc(&s->Wtb, kParams));
  A(dalloc(&s->feat, mb * kFeat));
  for (int l = 0; l < kLayers - 1; ++l) {
    A(dalloc(&s->Z[l], mb * kHid));
    A(dalloc(&s->A[l], mb * kHid));
  }
  A(dalloc(&s->Zout, mb * kOut));
  A(dalloc(&s->dZ[0], mb * kHid));
  A(dalloc(&s->dZ[1], mb * kHid));
  A(dalloc(&s->loss, 1));
  A(dalloc(&s->err, 1));
  if (e == cudaSuccess) e = cudaMemcpy(s->params, init_params, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->Bm, fourier_B, sizeof(float) * 16 * 7, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(s->v, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) {
    k_weights_bf16<<<dim3(16, kLayers), 256>>>(s->params, s->Wb, s->Wtb);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    delete s;
    return check(e);
  }
  *out = s;
  return SDD_OK;
}

void sdd_surrogate_destroy(sdd_surrogate* s) { delete s; }

int sdd_surrogate_param_count(void) { return kParams; }

sdd_status sdd_surrogate_get_params(const sdd_surrogate* s, float* host_out, int n) {
  if (!s || !host_out || n != kParams) return set_last_error(SDD_ERR_ARG, "bad arguments");
  return check(cudaMemcpy(host_out, s->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
}

sdd_status sdd_surrogate_set_params(sdd_surrogate* s, const float* host_in, int n) {
  if (!s || !host_in || n != kParams) return set_last_error(SDD_ERR_ARG, "bad arguments");
  cudaError_t e = cudaMemcpy(s->params, host_in, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  s->version++;
  if (e == cudaSuccess) {
    k_weights_bf16<<<dim3(16, kLayers), 256>>>(s->params, s->Wb, s->Wtb);
    e = cudaDeviceSynchronize();
  }
  return check(e);
}

sdd_status sdd_surrogate_gradients(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev, float* grad_host,
                                   float* loss_host, void* stream) {
  if (!s || n < 1 || n > s->max_batch || !raw_dev || !y_dev) return set_last_error(SDD_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = backward(s, n, raw_dev, y_dev, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpy(grad_host, s->grads, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_host) {
    e = cudaMemcpy(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost);
    *loss_host /= n;
  }
  return check(e);
}

sdd_status sdd_surrogate_train_step(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev, float lr,
                                    float* loss_host, void* stream) {
  if (!s || n < 1 || n > s->max_batch || !raw_dev || !y_dev || !(lr > 0.f))
    return set_last_error(SDD_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = adam_step(s, n, raw_dev, y_dev, lr, st);
  if (e == cudaSuccess && loss_host) {
    e = cudaMemcpyAsync(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *loss_host /= n;
  }
  return check(e);
}

sdd_status sdd_surrogate_train(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev,
                               const sdd_train_opts* opts, float* loss_host, void* stream) {
  if (!s || n < 1 || !raw_dev || !y_dev || !opts) return set_last_error(SDD_ERR_ARG, "NULL argument or n < 1");
  if (opts->steps < 1) return set_last_error(SDD_ERR_ARG, "steps must be >= 1");
  if (opts->batch < 1 || opts->batch > s->max_batch || opts->batch > n)
    return set_last_error(SDD_ERR_ARG, "batch must be in [1, min(n, max_batch)]");
  if (!(opts->lr > 0.f)) return set_last_error(SDD_ERR_ARG, "lr must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!s->batch_raw) e = dalloc(&s->batch_raw, (size_t)s->max_batch * 7);
  if (e == cudaSuccess && !s->batch_y) e = dalloc(&s->batch_y, (size_t)s->max_batch * kTargets);
  float* losses = nullptr;
  if (e == cudaSuccess) e = dalloc(&losses, (size_t)opts->steps);
  if (e != cudaSuccess) {
    cudaFree(losses);
    return check(e);
  }
  // each epoch visits the rows in the order (a i + c) mod n, a and c drawn from the seed
  uint64_t rng = opts->seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto next = [&rng]() {
    rng ^= rng >> 12;
    rng ^= rng << 25;
    rng ^= rng >> 27;
    return rng * 0x2545F4914F6CDD1Dull;
  };
  long long a = 1, c = 0, pos = (long long)n;  // pos >= n forces a new epoch
  for (int step = 0; step < opts->steps && e == cudaSuccess; ++step) {
    if (pos + opts->batch > n) {
      do {
        a = (long long)(next() % (uint64_t)n) | 1;
      } while (n > 1 && gcd_ll(a, n) != 1);
      c = (long long)(next() % (uint64_t)n);
      pos = 0;
    }
    k_gather_batch<<<(opts->batch + 255) / 256, 256, 0, st>>>(n, opts->batch, pos, a, c, raw_dev, y_dev,
                                                              s->batch_raw, s->batch_y);
    pos += opts->batch;
    e = adam_step(s, opts->batch, s->batch_raw, s->batch_y, opts->lr, st);
    if (e == cudaSuccess) k_record_loss<<<1, 1, 0, st>>>(s->loss, 1.f / opts->batch, losses + step);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && loss_host)
    e = cudaMemcpyAsync(loss_host, losses, sizeof(float) * opts->steps, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(losses);
  return check(e);
}

sdd_status sdd_surrogate_get_weights(const sdd_surrogate* s, void* host_out, size_t bytes) {
  if (!s || !host_out || bytes != sizeof(float) * (size_t)kParams)
    return set_last_error(SDD_ERR_ARG, "bytes must be 4 x sdd_surrogate_param_count()");
  return sdd_surrogate_get_params(s, static_cast<float*>(host_out), kParams);
}

sdd_status sdd_surrogate_set_weights(sdd_surrogate* s, const void* host_in, size_t bytes) {
  if (!s || !host_in || bytes != sizeof(float) * (size_t)kParams)
    return set_last_error(SDD_ERR_ARG, "bytes must be 4 x sdd_surrogate_param_count()");
  return sdd_surrogate_set_params(s, static_cast<const float*>(host_in), kParams);
}

sdd_status sdd_surrogate_infer(sdd_surrogate* s, int n, const float* raw_dev, float* out_dev, void* stream) {
  if (!s || n < 0 || !raw_dev || !out_dev) return set_last_error(SDD_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = surrogate_predict(s, n, raw_dev, out_dev, st, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  uint32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, s->err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return check(e);
  if (err) {
    cudaMemset(s->err, 0, sizeof(uint32_t));
    return set_last_error(SDD_ERR_TIMEOUT, "tensor-core wait gave up after its time limit");
  }
  return SDD_OK;
}

}  // extern "C"
