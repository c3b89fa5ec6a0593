// train_tc.cuh -- training of the tile-BTDF network on the 5th-generation tensor cores
// (tcgen05 with TMEM accumulators): a fused forward + loss kernel and a fused backward kernel
// whose weight gradients accumulate in TMEM over all of a CTA's row chunks.
//
// Names: layer l (0..4) maps its input in_l (in_0 = the 48 features, in_l = GELU(z_{l-1}))
// to z_l = in_l W_l + b_l (W_l [K_l][N_l]); gz_l = d loss / d z_l.  The products:
//   forward   z_l = in_l W_l           A = in_l    [rows][K_l]   B = W_l^T  [N_l][K_l] (Wt copy)
//   backward  d in_l = gz_l W_l^T      A = gz_l    [rows][N_l]   B = W_l    [K_l][N_l] (Wb copy)
//             gz_{l-1} = d in_l * GELU'(z_{l-1})
//             dW_l^T = gz_l^T in_l     A = gz_l^T  [N_l][rows]   B = in_l^T [K_l][rows]   (l < 4)
//             dW_4 = in_4^T gz_4       A = in_4^T  [128][rows]   B = gz_4^T [16][rows]
// Every shared-memory operand uses the K-major layout without swizzle (8-row x 16-byte core
// matrices).  Operands with features along K (in_l, gz_l) are canonical: element (r, k) of an
// operand with K columns at canon(r, k, K), core matrices 128 bytes apart along K, 8-row
// groups (K / 8) x 128 apart.  Operands with the 128 rows of a chunk along K (the transposed
// in_l^T, gz_l^T) space their core matrices 144 bytes apart along K (tcanon): a warp writes
// one feature of its 32 rows at a time, and with 128-byte spacing those 2-byte stores would
// fall into four banks; with 144 they spread over sixteen.  An MMA's K step of 16 is two core
// matrices further.
//
// The forward writes, per chunk of 128 rows, exactly what the backward needs in these
// operand layouts (a chunk record), so the backward copies contiguous blocks:
//   in_l^T  (l = 0..4)  element (feature f, row r) at tcanon(f, r)
//   z_l     (l = 0..3)  BF16, row-tiled for the epilogue threads: column c of row r at
//                       ((c / 16) 128 + r) 16 + c % 16 elements
//   gz_4                BF16 (scaled by 1 / batch) in the normal layout canon(r, o, 16) and
//                       transposed, tcanon(o, r)
// Rows past the batch get gz_4 = 0, so they add nothing to any gradient.
//
// The backward keeps every layer's weight gradient in TMEM (512 columns: dW_1^T, dW_2^T,
// dW_3^T 128 each, a 64-column working accumulator for d in_l, taken in two halves, dW_0^T
// 48, dW_4 16) and writes one partial gradient per CTA at the end; the partials are summed
// in CTA order, so a step's gradient does not depend on scheduling.  Bias gradients are the
// column sums of the BF16 gz_l, read from the transposed operand.  Every mbarrier wait is
// bounded; on expiry the kernel sets the timeout bit, waits (bounded) for its MMAs in
// flight, frees its TMEM and returns.
#pragma once

#include "surrogate_head.cuh"
#include "surrogate_tc.cuh"

namespace sdd {
namespace trn {

using namespace net;
constexpr int kRows = 128;
constexpr int kThreads = 512;  // 16 warps: 4 lane quadrants x 4 column groups in the epilogues

// Byte offset of element (r, k) of an operand with K columns (canonical K-major, no swizzle).
__host__ __device__ constexpr uint32_t canon(int r, int k, int K) {
  return (uint32_t)(r >> 3) * (uint32_t)(K / 8) * 128u + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}
__host__ __device__ constexpr uint32_t sbo(int K) { return (uint32_t)(K / 8) * 128u; }
// The transposed operands (K = the 128 rows of a chunk): element (feature f, row r).
constexpr uint32_t kTLbo = 144, kTSbo = (kRows / 8) * kTLbo;  // 2,304 bytes per 8 features
__host__ __device__ constexpr uint32_t tcanon(int f, int r) {
  return (uint32_t)(f >> 3) * kTSbo + (uint32_t)(r >> 3) * kTLbo + (uint32_t)(f & 7) * 16u + (uint32_t)(r & 7) * 2u;
}

// ---------------------------------------------------------------- chunk record (bytes)
constexpr uint32_t kInT0Bytes = (kFeat / 8) * kTSbo;  // 13,824
constexpr uint32_t kTileBytes = (kHid / 8) * kTSbo;   // 36,864 (>= the 32,768 of a canonical 128 x 128 tile)
__host__ __device__ constexpr uint32_t rec_in_t(int l) { return l == 0 ? 0u : kInT0Bytes + (uint32_t)(l - 1) * kTileBytes; }
__host__ __device__ constexpr uint32_t rec_z(int l) { return rec_in_t(kLayers) + (uint32_t)l * kTileBytes; }
constexpr uint32_t kGzBytes = kOut * kRows * 2;      // 4,096: gz_4, normal layout
constexpr uint32_t kGzTBytes = (kOut / 8) * kTSbo;   // 4,608: gz_4^T
constexpr uint32_t kRecGz = rec_z(kLayers - 1);
constexpr uint32_t kRecGzT = kRecGz + kGzBytes;
constexpr uint32_t kRecBytes = kRecGzT + kGzTBytes;

// ---------------------------------------------------------------- forward shared memory
// weights W_l^T of layers 0..4 (as the inference kernel), the A operand, a transposed
// staging tile, the mbarrier and the TMEM address
constexpr uint32_t kFwdAOff = tc::w_off(kLayers);            // 114,688
constexpr uint32_t kFwdTOff = kFwdAOff + kHid * kRows * 2;   // 147,456
constexpr uint32_t kFwdBarOff = kFwdTOff + kTileBytes;       // 184,320
constexpr size_t kFwdSmem = kFwdBarOff + 16;

// ---------------------------------------------------------------- backward shared memory
// W_l of layers 4, 3, 2, 1 as the B operand of d in_l ([K_l = 128][N_l], canonical with N_l
// columns), three rotating 36 KB operand buffers, the mbarrier and the TMEM address
__host__ __device__ constexpr uint32_t bwd_w_off(int l) {  // l = 1..4
  return l == 4 ? 0u : (uint32_t)(kHid * kOut * 2) + (uint32_t)(3 - l) * (kHid * kHid * 2);
}
constexpr uint32_t kBwdBufOff = (uint32_t)(kHid * kOut * 2) + 3u * (kHid * kHid * 2);  // 102,400
constexpr uint32_t kBwdBarOff = kBwdBufOff + 3u * kTileBytes;                           // 212,992
constexpr size_t kBwdSmem = kBwdBarOff + 16;

// TMEM columns of the backward (one allocation of 512)
constexpr uint32_t kTmemAll = 512;
__host__ __device__ constexpr uint32_t col_dw(int l) {  // dW_l^T (l = 0..3) or dW_4
  return l == 0 ? 448u : (l == 4 ? 496u : (uint32_t)(l - 1) * 128u);
}
constexpr uint32_t kColWork = 384;  // 64 columns: one half of d in_l

__device__ __forceinline__ void copy16(unsigned char* dst, const unsigned char* src, uint32_t bytes) {
  for (uint32_t i = threadIdx.x * 16u; i < bytes; i += blockDim.x * 16u)
    *reinterpret_cast<uint4*>(dst + i) = *reinterpret_cast<const uint4*>(src + i);
}

// Asynchronous 16-byte global -> shared copies (cp.async, completed by copy_async_wait).
__device__ __forceinline__ void copy16_async(unsigned char* dst, const unsigned char* src, uint32_t bytes) {
  for (uint32_t i = threadIdx.x * 16u; i < bytes; i += blockDim.x * 16u)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::sa(dst + i)), "l"(src + i) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void store_bf16(unsigned char* base, uint32_t off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16(x);
}

// ================================================================ forward + loss
// One CTA per SM over chunks c = blockIdx.x, + gridDim.x, ...: features, the five layers
// (z_l and in_{l+1} into the chunk record), the head's loss and gz_4 (scaled by inv_batch).
// loss_sum collects the batch's summed loss.
__global__ void __launch_bounds__(kThreads, 1)
    k_train_fwd(SurrogateView v, int n, const float* __restrict__ raw, const float* __restrict__ y, float inv_batch,
                unsigned char* __restrict__ rec, float* loss_sum, uint32_t* errw) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem + kFwdAOff;
  unsigned char* sT = smem + kFwdTOff;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kFwdBarOff);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kFwdBarOff + 8);
  __shared__ int s_fail;

  const int chunks = (n + kRows - 1) / kRows;
  if ((int)blockIdx.x >= chunks) return;  // whole block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_a = tc::sa(bar);

#pragma unroll 1
  for (int l = 0; l < kLayers; ++l) {  // W_l^T [N][K] into the canonical layout
    const int N = layer_out(l), K = layer_in(l), kc = K / 8;
    const uint4* src = reinterpret_cast<const uint4*>(v.Wt + layer_offset(l));
    unsigned char* dst = smem + tc::w_off(l);
    for (int i = tid; i < N * kc; i += blockDim.x) {
      const int r = i / kc, c = i - r * kc;
      *reinterpret_cast<uint4*>(dst + tc::chunk_off(r, c, tc::sbo_of(K))) = src[i];
    }
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::sa(s_tmem)),
                 "r"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *s_tmem;
  const int quad = warp & 3, cg = warp >> 2;  // lane quadrant (rows), column group
  const int row = quad * 32 + lane;
  const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;
  float loss = 0.f;

  for (int c = blockIdx.x; c < chunks && !failed; c += gridDim.x) {
    const int row0 = c * kRows, valid = min(kRows, n - row0);
    unsigned char* rc = rec + (size_t)c * kRecBytes;
    __syncthreads();  // the previous chunk's staging copy is done
    {  // features (the inference kernel's map): four threads per row, four Fourier pairs each;
       // layer 0's A operand and in_0^T
      const int r = tid & (kRows - 1), part = tid >> 7;
      float q[kIn] = {0.f, 0.f, 380.f, 2e-3f, 0.f, 1.45f, 1e-8f};
      if (r < valid)
        for (int j = 0; j < kIn; ++j) q[j] = raw[(size_t)(row0 + r) * kIn + j];
      float x[kIn];
      normalise_row(q, x);
      __align__(8) __nv_bfloat16 fs[4], fc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float sn, cs;
        fourier_pair(x, v.Bm, 4 * part + i, &sn, &cs);
        fs[i] = __float2bfloat16(sn);
        fc[i] = __float2bfloat16(cs);
      }
      const uint32_t s48 = tc::sbo_of(kFeat);
      *reinterpret_cast<uint2*>(sA + tc::chunk_off(r, part / 2, s48) + (part & 1) * 8) =
          *reinterpret_cast<const uint2*>(fs);
      *reinterpret_cast<uint2*>(sA + tc::chunk_off(r, 2 + part / 2, s48) + (part & 1) * 8) =
          *reinterpret_cast<const uint2*>(fc);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        *reinterpret_cast<__nv_bfloat16*>(sT + tcanon(4 * part + i, r)) = fs[i];
        *reinterpret_cast<__nv_bfloat16*>(sT + tcanon(kFourier + 4 * part + i, r)) = fc[i];
      }
      if (part == 0) {  // the normalised inputs and the zero padding: features 32..47
        __align__(16) __nv_bfloat16 f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) f[j] = __float2bfloat16(j < kIn ? x[j] : 0.f);
        *reinterpret_cast<uint4*>(sA + tc::chunk_off(r, 4, s48)) = reinterpret_cast<const uint4*>(f)[0];
        *reinterpret_cast<uint4*>(sA + tc::chunk_off(r, 5, s48)) = reinterpret_cast<const uint4*>(f)[1];
#pragma unroll
        for (int j = 0; j < 16; ++j) *reinterpret_cast<__nv_bfloat16*>(sT + tcanon(2 * kFourier + j, r)) = f[j];
      }
    }
    tc::fence_async_smem();
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < kLayers; ++l) {
      const int N = layer_out(l), K = layer_in(l);
      if (tid == 0) {
        tc::fence_after();
        const uint32_t a0 = tc::sa(sA), b0 = tc::sa(smem + tc::w_off(l));
        const uint32_t id = tc::idesc(kRows, N);
        for (int kk = 0; kk < K / 16; ++kk)
          tc::mma(tmem, tc::sdesc(a0 + kk * 256u, 128u, tc::sbo_of(K)), tc::sdesc(b0 + kk * 256u, 128u, tc::sbo_of(K)),
                  id, kk > 0 ? 1u : 0u);
        tc::commit(bar_a);
      }
      // while the MMAs run: the staged in_l^T goes to the chunk record
      copy16(rc + rec_in_t(l), sT, l == 0 ? kInT0Bytes : kTileBytes);
      if (!tc::bar_wait(bar_a, phase)) s_fail = 1;
      phase ^= 1u;
      __syncthreads();
      if (s_fail) {
        failed = true;
        break;
      }
      tc::fence_after();
      const float* bias = v.params + layer_offset(l) + K * N;
      if (l < kLayers - 1) {  // hidden: z_l to the record, in_{l+1} = GELU(z_l) as A and transposed
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
          const int col = cg * 32 + g * 16;
          float z[16], bb[16];
          tc::ld16(t_row + (uint32_t)col, z);
#pragma unroll
          for (int j = 0; j < 4; ++j) *reinterpret_cast<float4*>(bb + 4 * j) = __ldg(reinterpret_cast<const float4*>(bias + col) + j);
          uint32_t zb[8], a8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float z0 = z[2 * j] + bb[2 * j], z1 = z[2 * j + 1] + bb[2 * j + 1];
            zb[j] = tc::pack2(z0, z1);
            const float g0 = gelu(z0), g1 = gelu(z1);
            a8[j] = tc::pack2(g0, g1);
            store_bf16(sT, tcanon(col + 2 * j, row), g0);
            store_bf16(sT, tcanon(col + 2 * j + 1, row), g1);
          }
          uint4* zd = reinterpret_cast<uint4*>(rc + rec_z(l) + (((uint32_t)(col / 16) * kRows + row) * 16u) * 2u);
          zd[0] = make_uint4(zb[0], zb[1], zb[2], zb[3]);
          zd[1] = make_uint4(zb[4], zb[5], zb[6], zb[7]);
          *reinterpret_cast<uint4*>(sA + tc::chunk_off(row, col / 8, tc::sbo_of(kHid))) =
              make_uint4(a8[0], a8[1], a8[2], a8[3]);
          *reinterpret_cast<uint4*>(sA + tc::chunk_off(row, col / 8 + 1, tc::sbo_of(kHid))) =
              make_uint4(a8[4], a8[5], a8[6], a8[7]);
        }
        tc::fence_before();
        tc::fence_async_smem();
        __syncthreads();
      } else {  // output layer: loss and gz_4 of this thread's row
        if (cg == 0) {
          float z[16], gz[16];
          tc::ld16(t_row, z);
#pragma unroll
          for (int j = 0; j < 16; ++j) z[j] += __ldg(bias + j);
          if (row < valid) {
            loss += head_loss_row(z, y + (size_t)(row0 + row) * kHeadTargets, gz);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) gz[j] = 0.f;
          }
          uint32_t g8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float a = gz[2 * j] * inv_batch, b = gz[2 * j + 1] * inv_batch;
            g8[j] = tc::pack2(a, b);
            store_bf16(sT, tcanon(2 * j, row), a);
            store_bf16(sT, tcanon(2 * j + 1, row), b);
          }
          *reinterpret_cast<uint4*>(rc + kRecGz + canon(row, 0, kOut)) = make_uint4(g8[0], g8[1], g8[2], g8[3]);
          *reinterpret_cast<uint4*>(rc + kRecGz + canon(row, 8, kOut)) = make_uint4(g8[4], g8[5], g8[6], g8[7]);
        }
        tc::fence_before();
        __syncthreads();
        copy16(rc + kRecGzT, sT, kGzTBytes);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
  if (lane == 0 && loss != 0.f) atomicAdd(loss_sum, loss);
  if (failed) {
    if (tid == 0) atomicOr(errw, tc::kErrTimeout);
    tc::bar_wait(bar_a, phase ^ 1u);  // the phase that gave up: the MMAs still in flight
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::kTmemCols));
  }
}

// ================================================================ backward
// One CTA per SM over chunks c = blockIdx.x, + gridDim.x, ... (gridDim.x <= chunks): every
// layer's dW and db accumulate over the CTA's chunks; at the end the CTA writes its partial
// gradient, in the parameter layout (per layer W [K][N] then b [N]), to part + blockIdx.x kParams.
__global__ void __launch_bounds__(kThreads, 1)
    k_train_bwd(const __nv_bfloat16* __restrict__ Wb, int n, const unsigned char* __restrict__ rec,
                float* __restrict__ part, uint32_t* errw) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* buf[3] = {smem + kBwdBufOff, smem + kBwdBufOff + kTileBytes, smem + kBwdBufOff + 2 * kTileBytes};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBwdBarOff);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kBwdBarOff + 8);
  __shared__ int s_fail;

  const int chunks = (n + kRows - 1) / kRows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_a = tc::sa(bar);

#pragma unroll 1
  for (int l = 1; l < kLayers; ++l) {  // W_l [K = 128][N_l] as the B operand with N_l columns
    const int N = layer_out(l), nc = N / 8;
    const uint4* src = reinterpret_cast<const uint4*>(Wb + layer_offset(l));
    unsigned char* dst = smem + bwd_w_off(l);
    for (int i = tid; i < kHid * nc; i += blockDim.x) {
      const int f = i / nc, j = i - f * nc;
      *reinterpret_cast<uint4*>(dst + canon(f, 8 * j, N)) = src[i];
    }
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::sa(s_tmem)),
                 "r"(kTmemAll));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *s_tmem;
  const int quad = warp & 3, cg = warp >> 2;  // lane quadrant (rows), column group
  const int row = quad * 32 + lane;
  const uint32_t t_lane = (uint32_t)(quad * 32) << 16;
  uint32_t phase = 0;
  bool failed = false;
  float db[kLayers] = {0.f, 0.f, 0.f, 0.f, 0.f};  // thread t: column t of each layer's bias gradient

  // Bounded wait for the MMAs committed last; false (with s_fail set) when it gave up.
  auto wait_mma = [&]() -> bool {
    if (!tc::bar_wait(bar_a, phase)) s_fail = 1;
    phase ^= 1u;
    __syncthreads();
    return !s_fail;
  };
  // Column sums of a transposed gz operand (feature t's 128 rows) into db[l].
  auto add_bias_grad = [&](int l, const unsigned char* gzt) {
    if (tid < layer_out(l)) {
      float acc = 0.f;
#pragma unroll 4
      for (int rg = 0; rg < kRows / 8; ++rg) {
        const uint4 u = *reinterpret_cast<const uint4*>(gzt + tcanon(tid, 8 * rg));
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc += __bfloat162float(h[e].x) + __bfloat162float(h[e].y);
      }
      db[l] += acc;
    }
  };

  for (int c = blockIdx.x, first = 1; c < chunks && !failed; c += gridDim.x, first = 0) {
    const unsigned char* rc = rec + (size_t)c * kRecBytes;
    int bx = 0, by = 1, bz = 2;  // gz_l (normal), gz_l^T, in_l^T
    __syncthreads();
    copy16(buf[bx], rc + kRecGz, kGzBytes);
    copy16(buf[by], rc + kRecGzT, kGzTBytes);
    copy16(buf[bz], rc + rec_in_t(kLayers - 1), kTileBytes);
    tc::fence_async_smem();
    __syncthreads();
    add_bias_grad(kLayers - 1, buf[by]);
#pragma unroll 1
    for (int l = kLayers - 1; l >= 0 && !failed; --l) {
      const int N = layer_out(l), K = layer_in(l);
      if (tid == 0) {
        tc::fence_after();
        const uint32_t X = tc::sa(buf[bx]), Y = tc::sa(buf[by]), Z = tc::sa(buf[bz]);
        if (l == kLayers - 1) {  // dW_4 [128][16] += in_4^T gz_4
          const uint32_t id = tc::idesc(kRows, kOut);
          for (int kk = 0; kk < kRows / 16; ++kk)
            tc::mma(tmem + col_dw(l), tc::sdesc(Z + kk * 2u * kTLbo, kTLbo, kTSbo),
                    tc::sdesc(Y + kk * 2u * kTLbo, kTLbo, kTSbo), id, (first && kk == 0) ? 0u : 1u);
        } else {  // dW_l^T [N_l][K_l] += gz_l^T in_l
          const uint32_t id = tc::idesc(N, K);
          for (int kk = 0; kk < kRows / 16; ++kk)
            tc::mma(tmem + col_dw(l), tc::sdesc(Y + kk * 2u * kTLbo, kTLbo, kTSbo),
                    tc::sdesc(Z + kk * 2u * kTLbo, kTLbo, kTSbo), id, (first && kk == 0) ? 0u : 1u);
        }
        if (l > 0) {  // first half of d in_l = gz_l W_l^T: columns 0..63
          const uint32_t id = tc::idesc(kRows, 64);
          const uint32_t W = tc::sa(smem + bwd_w_off(l));
          for (int kk = 0; kk < N / 16; ++kk)
            tc::mma(tmem + kColWork, tc::sdesc(X + kk * 256u, 128u, sbo(N)), tc::sdesc(W + kk * 256u, 128u, sbo(N)), id,
                    kk > 0 ? 1u : 0u);
        }
        tc::commit(bar_a);
      }
      // z_{l-1} of this thread's columns of the first half, loaded while the MMAs run
      const unsigned char* zr = rc + rec_z(l > 0 ? l - 1 : 0);
      auto z_of = [&](int h2) {
        const int col = h2 * 64 + cg * 16;
        return reinterpret_cast<const uint4*>(zr + (((uint32_t)(col / 16) * kRows + row) * 16u) * 2u);
      };
      uint4 zz[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      if (l > 0) {
        zz[0] = z_of(0)[0];
        zz[1] = z_of(0)[1];
      }
      if (!wait_mma()) {
        failed = true;
        break;
      }
      if (l == 0) break;
      // gz_{l-1} = d in_l * GELU'(z_{l-1}), two halves of 64 columns; written over gz_l^T
      // (into the normal layout) and in_l^T (transposed), both consumed by dW_l
#pragma unroll 1
      for (int h2 = 0; h2 < 2; ++h2) {
        if (h2 == 1) {
          if (tid == 0) {
            tc::fence_after();
            const uint32_t id = tc::idesc(kRows, 64);
            const uint32_t W = tc::sa(smem + bwd_w_off(l)) + 8u * sbo(N);  // B rows 64..127
            const uint32_t X = tc::sa(buf[bx]);
            for (int kk = 0; kk < N / 16; ++kk)
              tc::mma(tmem + kColWork, tc::sdesc(X + kk * 256u, 128u, sbo(N)), tc::sdesc(W + kk * 256u, 128u, sbo(N)),
                      id, kk > 0 ? 1u : 0u);
            tc::commit(bar_a);
          }
          zz[0] = z_of(1)[0];
          zz[1] = z_of(1)[1];
          if (!wait_mma()) {
            failed = true;
            break;
          }
          // both halves of d in_l are computed: in_{l-1}^T goes into the buffer gz_l used,
          // asynchronously, while this half's epilogue runs
          copy16_async(buf[bx], rc + rec_in_t(l - 1), l - 1 == 0 ? kInT0Bytes : kTileBytes);
        }
        tc::fence_after();
        // this warp: rows of its quadrant, columns cg * 16 .. + 15 of the 64-column half
        {
          const int wc = cg * 16;             // column within the working half
          const int col = h2 * 64 + wc;       // column of d in_l
          float d[16];
          tc::ld16(tmem + t_lane + kColWork + (uint32_t)wc, d);
          const __nv_bfloat162* zh = reinterpret_cast<const __nv_bfloat162*>(zz);
          uint32_t g8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float a = d[2 * j] * gelu_grad(__bfloat162float(zh[j].x));
            const float b = d[2 * j + 1] * gelu_grad(__bfloat162float(zh[j].y));
            g8[j] = tc::pack2(a, b);
            store_bf16(buf[bz], tcanon(col + 2 * j, row), a);
            store_bf16(buf[bz], tcanon(col + 2 * j + 1, row), b);
          }
          *reinterpret_cast<uint4*>(buf[by] + canon(row, col, kHid)) = make_uint4(g8[0], g8[1], g8[2], g8[3]);
          *reinterpret_cast<uint4*>(buf[by] + canon(row, col + 8, kHid)) = make_uint4(g8[4], g8[5], g8[6], g8[7]);
        }
        tc::fence_before();
        __syncthreads();  // every thread's reads of the working columns are done
      }
      copy_async_wait();  // in_{l-1}^T has landed (also on the way out of a failed wait)
      if (failed) break;
      tc::fence_async_smem();
      __syncthreads();
      add_bias_grad(l - 1, buf[bz]);
      const int t = bx;  // rotate: gz_{l-1} normal, gz_{l-1}^T, in_{l-1}^T
      bx = by;
      by = bz;
      bz = t;
    }
  }
  if (!failed) {
    tc::fence_after();
    // partial gradient of this CTA
    float* out = part + (size_t)blockIdx.x * kParams;
    if (cg == 0) {  // dW_4 [in f = row][out o]: 16 columns
      float d[16];
      tc::ld16(tmem + t_lane + col_dw(kLayers - 1), d);
      float* w = out + layer_offset(kLayers - 1) + (size_t)row * kOut;
#pragma unroll
      for (int j = 0; j < 16; ++j) w[j] = d[j];
    }
#pragma unroll 1
    for (int l = 0; l < kLayers - 1; ++l) {  // dW_l^T [out o = row][in f]
      const int K = layer_in(l), N = layer_out(l);
      float* w = out + layer_offset(l);
#pragma unroll 1
      for (int g = cg; g < K / 16; g += 4) {
        float d[16];
        tc::ld16(tmem + t_lane + col_dw(l) + (uint32_t)(16 * g), d);
#pragma unroll
        for (int j = 0; j < 16; ++j) w[(size_t)(16 * g + j) * N + row] = d[j];
      }
    }
#pragma unroll 1
    for (int l = 0; l < kLayers; ++l)
      if (tid < layer_out(l)) out[layer_offset(l) + layer_in(l) * layer_out(l) + tid] = db[l];
  } else {
    if (tid == 0) atomicOr(errw, tc::kErrTimeout);
    tc::bar_wait(bar_a, phase ^ 1u);  // the phase that gave up: the MMAs still in flight
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemAll));
  }
}

}  // namespace trn
}  // namespace sdd
