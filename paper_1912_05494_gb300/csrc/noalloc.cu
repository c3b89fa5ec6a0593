// noalloc.cu -- sdd_trace_closest_noalloc: the batched closest-hit query of
// sdd_trace_closest, run out of a fixed static device array instead of the scene's
// growable workspace, so that the call itself allocates no memory.
//
// Who needs it: callers that work under a device-memory budget fixed when they start
// (a long-running service that reserves its GPU memory up front, or an application whose
// own allocator owns the device heap) and may not let a library call cudaMalloc when a
// batch arrives.  sdd_trace_closest grows the scene's workspace on demand; this variant
// never does.  The scene itself is still created beforehand with sdd_scene_create.
//
// The scratch array below is part of the library image: every GPU on which the library is
// used holds its kNoAllocScratchBytes from the first call until the process exits.  All
// calls share it and it keeps whatever the last call left there, so the counters that must
// start at zero are cleared on every call, and calls whose work overlaps on the GPU (two
// host threads, or two streams) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/sdd.h"
#include "render_kernels.cuh"
#include "sdd_internal.h"

namespace sdd {
// Defined in api.cu: the device-side description of a scene and the thread-local error text.
const DevScene* scene_device_view(const sdd_scene* s);
bool scene_streaming(const sdd_scene* s);
sdd_status set_last_error(sdd_status st, const char* msg);
}  // namespace sdd

using namespace sdd;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kBlock = 128;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of scratch for n rays across n_sub subdomain queues: ray origin and direction
// (2 x 16 B), ray info (8 B), hit record (8 B), two queue generations (2 x 4 B per
// subdomain), plus the control block.
size_t scratch_bytes(size_t n, int n_sub) {
  return align256(sizeof(Control)) + 2 * align256(16 * n) + align256(8 * n) + align256(8 * n) +
         2 * align256(4 * n * (size_t)n_sub);
}

// Device address of the static scratch on the current device.  The array is a host-side
// stand-in in host code, so its device address is looked up, with the device current, on
// every call: the first lookup on a device loads the library's module there (under CUDA's
// default lazy loading this is when the 16 MiB are placed in device memory); later lookups
// are cheap, and a lookup per call follows a context that was destroyed and created again
// (cudaDeviceReset), where a cached address would go stale.
sdd_status scratch_on_current_device(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    return set_last_error(SDD_ERR_CUDA, (std::string("cudaGetSymbolAddress(scratch): ") +
                                         cudaGetErrorString(e)).c_str());
  }
  *out = static_cast<unsigned char*>(p);
  return SDD_OK;
}

// Status for the error bits the traversal kernels raise in the control block.
sdd_status status_of_error_bits(uint32_t bits) {
  if (bits & ERR_STACK_OVERFLOW)
    return set_last_error(SDD_ERR_STACK, "BVH traversal stack overflow or walk step bound reached");
  if (bits & (ERR_QUEUE_OVERFLOW | ERR_SHADOW_OVERFLOW))
    return set_last_error(SDD_ERR_QUEUE_OVERFLOW, "ray queue capacity exceeded");
  return set_last_error(SDD_ERR_TIMEOUT, "device loop hit its iteration cap");
}

}  // namespace

extern "C" sdd_status sdd_trace_closest_noalloc(sdd_scene* scene, int n, const float* org_dev,
                                                const float* dir_dev, float* t_out_dev, int32_t* prim_out_dev,
                                                void* cuda_stream) {
  if (!scene || n < 0 || (n > 0 && (!org_dev || !dir_dev || !t_out_dev || !prim_out_dev)))
    return set_last_error(SDD_ERR_ARG, "bad arguments");
  if (n == 0) {  // set-up only: place the scratch on this device now
    unsigned char* base = nullptr;
    return scratch_on_current_device(&base);
  }
  if (scene_streaming(scene))
    return set_last_error(SDD_ERR_STATE, "out-of-core subdomains are on (resident_subdomains > 0): the BVH is not resident");
  const DevScene* ds = scene_device_view(scene);
  const size_t need = scratch_bytes((size_t)n, ds->n_sub);
  if (need > kNoAllocScratchBytes) {
    std::string msg = "sdd_trace_closest_noalloc: " + std::to_string(n) + " rays over " + std::to_string(ds->n_sub) +
                      " subdomains need " + std::to_string(need) + " bytes of scratch; the static limit is " +
                      std::to_string(kNoAllocScratchBytes) + " bytes (at most n * (48 + 8 * n_subdomains) bytes of rays)";
    return set_last_error(SDD_ERR_ARG, msg.c_str());
  }
  unsigned char* base = nullptr;
  sdd_status st = scratch_on_current_device(&base);
  if (st) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // carve the scratch
  unsigned char* p = base;
  Control* ctl = reinterpret_cast<Control*>(p);
  p += align256(sizeof(Control));
  RayBuf rb;
  rb.o = reinterpret_cast<float4*>(p);
  p += align256(16 * (size_t)n);
  rb.d = reinterpret_cast<float4*>(p);
  p += align256(16 * (size_t)n);
  rb.info = reinterpret_cast<uint2*>(p);
  p += align256(8 * (size_t)n);
  rb.cap = n;
  float2* hits = reinterpret_cast<float2*>(p);
  p += align256(8 * (size_t)n);
  uint32_t* q[2];
  q[0] = reinterpret_cast<uint32_t*>(p);
  p += align256(4 * (size_t)n * ds->n_sub);
  q[1] = reinterpret_cast<uint32_t*>(p);

  // the shared array keeps the previous call's contents: clear the counters
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Control), stream);
  if (e != cudaSuccess) return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
  launch_rays_from_arrays(n, org_dev, dir_dev, *ds, rb, q[0], ctl->q_count[0], n, stream);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));

  RenderParams prm{};
  prm.sc = *ds;
  Control h;  // host copy of the counters (ordinary host memory)
  int a = 0;
  bool drained = false;
  for (int pass = 0; pass <= 2 * kMaxSubdomains + 2; ++pass) {
    if ((e = cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
      return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
    if (h.error) return status_of_error_bits(h.error);
    Sched sch;
    sch.n_sub = ds->n_sub;
    int blocks = 0;
    long long total = 0;
    for (int s = 0; s < ds->n_sub; ++s) {
      sch.blk_start[s] = blocks;
      sch.count[s] = std::min(std::max(h.q_count[a][s], 0), n);
      blocks += (sch.count[s] + kBlock - 1) / kBlock;
      total += sch.count[s];
    }
    sch.blk_start[ds->n_sub] = blocks;
    if (total == 0) {
      drained = true;
      break;
    }
    if ((e = cudaMemsetAsync(ctl->q_count[1 - a], 0, sizeof(int) * kMaxSubdomains, stream)) != cudaSuccess)
      return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
    QueuePair qp{q[a], q[1 - a], ctl->q_count[1 - a], n};
    launch_traverse(prm, sch, blocks, kBlock, 0, qp, rb, hits, ctl, stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
    a = 1 - a;
  }
  if (!drained) return set_last_error(SDD_ERR_TIMEOUT, "closest-hit passes did not drain the subdomain queues");
  launch_hits_to_arrays(n, hits, t_out_dev, prim_out_dev, stream);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return set_last_error(SDD_ERR_CUDA, cudaGetErrorString(e));
  return SDD_OK;
}
