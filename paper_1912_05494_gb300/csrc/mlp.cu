// mlp.cu -- the tile-BTDF surrogate network on the BF16 tensor cores: training (forward,
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
// Weights and activations are BF16, products accumulate in FP32 on the tcgen05 tensor cores
// with TMEM accumulators.  A training step is three launches: the fused forward + loss
// kernel and the fused backward kernel of train_tc.cuh (per-CTA partial gradients), then
// one kernel that sums the partials in CTA order, applies Adam and refreshes the BF16 weight
// copies.  Inference (sdd_surrogate_infer and the renderer) runs the fused tcgen05 kernel of
// surrogate_tc.cuh.  Parameters are one flat FP32 array: for each layer W [in][out]
// row-major, then b [out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "surrogate_head.cuh"
#include "surrogate_net.cuh"
#include "surrogate_tc.cuh"
#include "train_tc.cuh"

namespace sdd {
sdd_status set_last_error(sdd_status st, const char* msg);
}
using namespace sdd;

namespace {

using namespace sdd::net;
constexpr int kTargets = kHeadTargets;

// The per-CTA partial gradients of a step summed in CTA order (grads, when given); with
// lr > 0 also the Adam step of the FP32 parameters (Kingma & Ba: moments m, v, bias
// corrections c1, c2) and their BF16 copies Wb (W [K][N]) and Wtb (W^T [N][K]).
__global__ void k_reduce_adam(int nblk, const float* __restrict__ part, float* __restrict__ grads,
                              float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                              float b2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ Wb,
                              __nv_bfloat16* __restrict__ Wtb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += part[(size_t)b * kParams + i];
  if (grads) grads[i] = g;
  if (!(lr > 0.f)) return;
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  int l = 0;
  while (l < kLayers - 1 && i >= layer_offset(l + 1)) ++l;
  const int j = i - layer_offset(l), K = layer_in(l), N = layer_out(l);
  if (j < K * N) {
    const __nv_bfloat16 h = __float2bfloat16(pi);
    Wb[i] = h;
    Wtb[layer_offset(l) + (j % N) * K + j / N] = h;
  }
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
  float* partial = nullptr;  // per-CTA partial gradients of a step [partial_blocks][kParams]
  int partial_blocks = 0;
  float* m = nullptr;
  float* v = nullptr;
  float* Bm = nullptr;      // Fourier matrix [16][7]
  __nv_bfloat16* Wb = nullptr;
  __nv_bfloat16* Wtb = nullptr;
  unsigned char* rec = nullptr;  // forward -> backward chunk records [max_batch / 128][trn::kRecBytes]
  float* loss = nullptr;
  uint32_t* err = nullptr;  // timeout bit of the tensor-core kernels' bounded waits
  float* batch_raw = nullptr;  // minibatch scratch of sdd_surrogate_train [max_batch][7]
  float* batch_y = nullptr;    // [max_batch][18]
  int step = 0;
  unsigned version = 0;  // bumped whenever the weights change
  ~sdd_surrogate() {
    cudaFree(params); cudaFree(grads); cudaFree(partial); cudaFree(m); cudaFree(v); cudaFree(Bm); cudaFree(Wb); cudaFree(Wtb);
    cudaFree(rec); cudaFree(loss); cudaFree(err); cudaFree(batch_raw); cudaFree(batch_y);
  }
};

namespace {

sdd_status check(cudaError_t e) {
  return e == cudaSuccess ? SDD_OK : set_last_error(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,
                                                    cudaGetErrorString(e));
}

// CTAs of the training kernels for n rows: one per SM, at most one per 128-row chunk.
int train_grid(const sdd_surrogate* s, int n) {
  return std::max(1, std::min(s->partial_blocks, (n + trn::kRows - 1) / trn::kRows));
}

// Forward, loss (summed into s->loss) and backward of n rows: per-CTA partial gradients in
// s->partial; returns the number of partials.
cudaError_t gradients(sdd_surrogate* s, int n, const float* raw, const float* y, cudaStream_t st, int* nblk) {
  const int g = train_grid(s, n);
  cudaError_t e = cudaMemsetAsync(s->loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  trn::k_train_fwd<<<g, trn::kThreads, trn::kFwdSmem, st>>>(surrogate_view(s), n, raw, y, 1.f / n, s->rec, s->loss,
                                                            s->err);
  trn::k_train_bwd<<<g, trn::kThreads, trn::kBwdSmem, st>>>(s->Wb, n, s->rec, s->partial, s->err);
  *nblk = g;
  return cudaGetLastError();
}

// Loss and gradients of n rows into s->grads; loss sum in s->loss.
cudaError_t backward(sdd_surrogate* s, int n, const float* raw, const float* y, cudaStream_t st) {
  int nblk = 0;
  cudaError_t e = gradients(s, n, raw, y, st, &nblk);
  if (e != cudaSuccess) return e;
  k_reduce_adam<<<(kParams + 255) / 256, 256, 0, st>>>(nblk, s->partial, s->grads, nullptr, nullptr, nullptr, 0.f, 0.f,
                                                         0.f, 0.f, 1.f, 1.f, nullptr, nullptr);
  return cudaGetLastError();
}

// One Adam step on n rows (enqueued on st): gradients, moments, parameters, BF16 copies.
cudaError_t adam_step(sdd_surrogate* s, int n, const float* raw, const float* y, float lr, cudaStream_t st) {
  int nblk = 0;
  cudaError_t e = gradients(s, n, raw, y, st, &nblk);
  if (e != cudaSuccess) return e;
  s->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
  k_reduce_adam<<<(kParams + 255) / 256, 256, 0, st>>>(nblk, s->partial, s->grads, s->params, s->m, s->v, lr, b1, b2,
                                                         1e-8f, c1, c2, s->Wb, s->Wtb);
  s->version++;
  return cudaGetLastError();
}

// The tensor-core kernels' timeout bit, read after the stream was synchronised (and cleared).
sdd_status check_timeout(sdd_surrogate* s) {
  uint32_t err = 0;
  cudaError_t e = cudaMemcpy(&err, s->err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return check(e);
  if (err) {
    cudaMemset(s->err, 0, sizeof(uint32_t));
    return set_last_error(SDD_ERR_TIMEOUT, "tensor-core wait gave up after its time limit");
  }
  return SDD_OK;
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
    cudaFuncSetAttribute(trn::k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trn::kFwdSmem);
    cudaFuncSetAttribute(trn::k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trn::kBwdSmem);
    attrs = true;
  }
  sdd_surrogate* s = new sdd_surrogate;
  s->max_batch = max_batch;
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
    s->partial_blocks = std::max(1, sms);
    A(dalloc(&s->partial, (size_t)s->partial_blocks * kParams));
  }
  A(dalloc(&s->m, kParams));
  A(dalloc(&s->v, kParams));
  A(dalloc(&s->Bm, 16 * 7));
  A(dalloc(&s->Wb, kParams));
  A(dalloc(&s->Wtb, kParams));
  A(dalloc(&s->rec, (size_t)((max_batch + trn::kRows - 1) / trn::kRows) * trn::kRecBytes));
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
  if (e != cudaSuccess) return check(e);
  if (sdd_status t = check_timeout(s)) return t;
  if (grad_host)
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
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check(e);
  if (loss_host) *loss_host /= n;
  return check_timeout(s);
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
  if (e != cudaSuccess) return check(e);
  return check_timeout(s);
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
