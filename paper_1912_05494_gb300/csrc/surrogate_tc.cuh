// surrogate_tc.cuh -- fused inference of the tile-BTDF network on the 5th-generation tensor
// cores (tcgen05 with a TMEM accumulator), used by the renderer and by sdd_surrogate_infer.
//
// One CTA of 512 threads per SM keeps every layer's BF16 weights in shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices; element (r, k) of
// an [R][K] operand at (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes,
// SBO = K / 8 * 128) and loops over chunks of 128 rows.  Per chunk:
//   1. threads 0..127 gather one row's raw inputs (policy) and stage them normalised; then
//      all 512 threads write the 48 features as the A operand (four threads per row, four
//      Fourier pairs each);
//   2. per layer, one thread issues K / 16 tcgen05.mma (M = 128, N = 128 or 16, BF16 in,
//      FP32 accumulate) into 128 TMEM columns and commits them to an mbarrier;
//   3. every warp reads its quadrant of rows (warp % 4) and a quarter of the columns
//      (warp / 4) back with tcgen05.ld, adds the bias, applies GELU and writes the BF16
//      activations as the next layer's A operand (the output layer's 16 columns go through
//      the head into a staging array for the policy's consumer).  Sixteen warps per SM
//      rather than eight: the epilogues (exact-erf GELU, packing) bound the kernel, not the
//      tensor cores.
// Every mbarrier wait is bounded by the global timer; on expiry the kernel raises the
// policy's timeout error bit, waits (bounded) for the MMAs in flight, frees its TMEM and
// returns.
#pragma once

#include "surrogate_net.cuh"

namespace sdd {
namespace tc {

constexpr int kThreads = 512;
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kErrTimeout = 4u;  // the renderer's timeout error bit
constexpr unsigned long long kWaitNs = 1000ull * 1000 * 1000;

__host__ __device__ constexpr uint32_t sbo_of(int K) { return (uint32_t)(K / 8) * 128u; }
// Shared-memory map (bytes): weights of layers 0..4, the A operand, the output staging,
// the mbarrier and the TMEM address.  Every region starts on a 1024-byte boundary.
__host__ __device__ constexpr uint32_t w_bytes(int l) { return (uint32_t)net::layer_out(l) * net::layer_in(l) * 2u; }
__host__ __device__ constexpr uint32_t w_off(int l) {
  uint32_t o = 0;
  for (int i = 0; i < l; ++i) o += w_bytes(i);
  return o;
}
constexpr uint32_t kAOff = w_off(net::kLayers);                    // 114,688
constexpr uint32_t kZOff = kAOff + kRows * net::kHid * 2u;         // 147,456
constexpr uint32_t kXOff = kZOff + kRows * kInferZLd * 4u;         // 155,648: normalised inputs [128][8]
constexpr uint32_t kBarOff = kXOff + kRows * 8 * 4u;               // 159,744
constexpr size_t kSmem = kBarOff + 16;

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, leading (K-direction) byte offset >> 4,
// stride (row-group) byte offset >> 4, the fixed version bits 0b001 at 46, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait for the mbarrier phase; false when the time limit passed.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t phase) {
  const unsigned long long t0 = now_ns();
  while (!bar_try(bar, phase))
    if (now_ns() - t0 > kWaitNs) return false;
  return true;
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Byte offset of the 16-byte chunk (row r, columns 8c .. 8c + 7) in the canonical layout.
__device__ __forceinline__ uint32_t chunk_off(int r, int c, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)c * 128u + (uint32_t)(r & 7) * 16u;
}

}  // namespace tc

template <class Policy>
__global__ void __launch_bounds__(tc::kThreads, 1) k_infer_tc(SurrogateView v, const Policy pol) {
  using namespace net;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem + tc::kAOff;
  float* sz = reinterpret_cast<float*>(smem + tc::kZOff);
  float* sx = reinterpret_cast<float*>(smem + tc::kXOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + tc::kBarOff);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + tc::kBarOff + 8);
  __shared__ int s_fail;

  const typename Policy::Ctx ctx = pol.resolve();
  const int n = pol.count(ctx);
  if ((int)blockIdx.x * tc::kRows >= n) return;  // whole block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_a = tc::sa(bar);

  // weights into the canonical layout (16-byte chunks), barrier, TMEM
#pragma unroll 1
  for (int l = 0; l < kLayers; ++l) {
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
  const int quad = warp & 3, quarter = warp >> 2;
  const int row = quad * 32 + lane;  // this thread's row of the chunk in the epilogues
  const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;

  for (int row0 = blockIdx.x * tc::kRows; row0 < n && !failed; row0 += gridDim.x * tc::kRows) {
    const int valid = min(tc::kRows, n - row0);
    __syncthreads();  // the previous chunk's consumer is done with sz
    const uint32_t s48 = tc::sbo_of(kFeat);
    if (tid < tc::kRows) {  // row tid's inputs, normalised; features 32..47 (x, zero padding)
      float q[kIn] = {0.f, 0.f, 380.f, 2e-3f, 0.f, 1.45f, 1e-8f};
      if (tid < valid) pol.load(ctx, row0 + tid, q);
      float x[kIn];
      normalise_row(q, x);
      __align__(16) __nv_bfloat16 f[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) f[j] = __float2bfloat16(j < kIn ? x[j] : 0.f);
      *reinterpret_cast<uint4*>(sA + tc::chunk_off(tid, 4, s48)) = reinterpret_cast<const uint4*>(f)[0];
      *reinterpret_cast<uint4*>(sA + tc::chunk_off(tid, 5, s48)) = reinterpret_cast<const uint4*>(f)[1];
#pragma unroll
      for (int j = 0; j < kIn; ++j) sx[tid * 8 + j] = x[j];
    }
    __syncthreads();
    {  // Fourier pairs 4 part .. 4 part + 3 of row r: sines at features 0..15, cosines 16..31
      const int r = tid & (tc::kRows - 1), part = tid >> 7;
      float x[kIn];
#pragma unroll
      for (int j = 0; j < kIn; ++j) x[j] = sx[r * 8 + j];
      __align__(8) __nv_bfloat16 fs[4], fc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float sn, cs;
        fourier_pair(x, v.Bm, 4 * part + i, &sn, &cs);
        fs[i] = __float2bfloat16(sn);
        fc[i] = __float2bfloat16(cs);
      }
      *reinterpret_cast<uint2*>(sA + tc::chunk_off(r, part / 2, s48) + (part & 1) * 8) =
          *reinterpret_cast<const uint2*>(fs);
      *reinterpret_cast<uint2*>(sA + tc::chunk_off(r, 2 + part / 2, s48) + (part & 1) * 8) =
          *reinterpret_cast<const uint2*>(fc);
    }
    tc::fence_async_smem();
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < kLayers; ++l) {
      const int N = layer_out(l), K = layer_in(l);
      if (tid == 0) {
        tc::fence_after();
        const uint32_t a0 = tc::sa(sA), b0 = tc::sa(smem + tc::w_off(l));
        const uint32_t id = tc::idesc(tc::kRows, N);
        for (int kk = 0; kk < K / 16; ++kk)
          tc::mma(tmem, tc::sdesc(a0 + kk * 256u, 128u, tc::sbo_of(K)), tc::sdesc(b0 + kk * 256u, 128u, tc::sbo_of(K)), id,
                  kk > 0 ? 1u : 0u);
        tc::commit(bar_a);
      }
      if (!tc::bar_wait(bar_a, phase)) s_fail = 1;
      phase ^= 1u;
      __syncthreads();
      if (s_fail) {
        failed = true;
        break;
      }
      tc::fence_after();
      if (l < kLayers - 1) {  // hidden layer: bias + GELU -> next A (K = 128)
        const float* bias = v.params + layer_offset(l) + K * N;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
          const int col = quarter * 32 + g * 16;
          float z[16];
          tc::ld16(t_row + (uint32_t)col, z);
          uint32_t w8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            w8[j] = tc::pack2(gelu(z[2 * j] + __ldg(bias + col + 2 * j)), gelu(z[2 * j + 1] + __ldg(bias + col + 2 * j + 1)));
          *reinterpret_cast<uint4*>(sA + tc::chunk_off(row, col / 8, tc::sbo_of(kHid))) =
              make_uint4(w8[0], w8[1], w8[2], w8[3]);
          *reinterpret_cast<uint4*>(sA + tc::chunk_off(row, col / 8 + 1, tc::sbo_of(kHid))) =
              make_uint4(w8[4], w8[5], w8[6], w8[7]);
        }
        tc::fence_before();
        tc::fence_async_smem();
        __syncthreads();
      } else {  // output layer: the head of the first 8 outputs
        if (quarter == 0) {
          const float* bias = v.params + layer_offset(l) + K * N;
          float z[16];
          tc::ld16(t_row, z);
          float* o = sz + row * kInferZLd;
          o[0] = head_sigmoid(z[0] + __ldg(bias + 0));
          o[1] = head_sigmoid(z[1] + __ldg(bias + 1));
          o[2] = head_sigmoid(z[2] + __ldg(bias + 2));
          o[3] = head_log_kappa(z[3] + __ldg(bias + 3), kLkOffset1);
          o[4] = head_log_kappa(z[4] + __ldg(bias + 4), kLkOffset2);
          o[5] = head_sigmoid(z[5] + __ldg(bias + 5));
          o[6] = head_log_kappa(z[6] + __ldg(bias + 6), kLkOffset1);
          o[7] = head_log_kappa(z[7] + __ldg(bias + 7), kLkOffset2);
        }
        tc::fence_before();
        __syncthreads();
      }
    }
    if (failed) break;
    pol.consume(ctx, row0, valid, sz);
  }
  if (failed) {
    if (tid == 0) atomicOr(pol.err(ctx), tc::kErrTimeout);
    // The phase bit was flipped after the wait that gave up, so the phase still owed by the
    // MMAs in flight is phase ^ 1 (try_wait.parity(p) succeeds at once for a parity p that
    // is not the barrier's current phase).  Wait for it, bounded again, before the TMEM
    // columns are freed; the results of this launch are already flagged invalid.
    tc::bar_wait(bar_a, phase ^ 1u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::kTmemCols));
  }
}

template <class Policy>
cudaError_t infer_tc_prepare() {
  return cudaFuncSetAttribute(k_infer_tc<Policy>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem);
}

}  // namespace sdd
