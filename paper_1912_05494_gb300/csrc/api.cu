// api.cu -- C ABI of libsdd (include/sdd.h): scene creation, the host-driven wavefront
// render loop, and the small query entry points.
//
// Render loop of one wave (a block of spectral paths, Sec. 4: every wavelength is an
// independent path):
//   raygen -> [ closest-hit passes over the subdomain queues until no ray is handed on
//               (Sec. 5) -> shade (children + shadow rays binned by subdomain) ->
//               shadow passes ]  repeated while rays remain -> film accumulation.
// The host reads the queue counters after each launch to size the next grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "graph_form.h"
#include "persistent.cuh"
#include "photon.cuh"
#include "render_kernels.cuh"
#include "scene_build.h"
#include "surrogate_render.cuh"
#include "surrogate_head.cuh"
#include "sdd_internal.h"

using namespace sdd;

namespace {

thread_local std::string g_err;

sdd_status fail(sdd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

template <typename T>
struct DevArr {
  T* p = nullptr;
  size_t n = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t want) {
    if (want <= n && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 1) * sizeof(T));
    if (e == cudaSuccess) n = want;
    else p = nullptr;
    return e;
  }
};

struct HostMaterial {
  int kind;
  std::vector<float> lam, n, k, albedo;
  float thick;
  int tile_id;
};

double interp_table(const std::vector<float>& grid, const std::vector<float>& val, double lam) {
  if (val.empty()) return 0.0;
  size_t n = grid.size();
  if (n == 1 || lam <= grid[0]) return val[0];
  if (lam >= grid[n - 1]) return val[n - 1];
  size_t i = 0;
  while (grid[i + 1] < lam) ++i;
  double f = (lam - grid[i]) / ((double)grid[i + 1] - grid[i]);
  return (1.0 - f) * val[i] + f * val[i + 1];
}

enum TimedKind { TK_RAYGEN = 0, TK_TRAVERSE, TK_SHADE, TK_SHADOW, TK_FILM, TK_TILE, TK_COUNT };

}  // namespace

struct sdd_scene {
  // host copies
  int n_tris = 0;
  std::vector<HostMaterial> mats;
  std::vector<float> il_lam, il_sky, il_sun;
  int sky_mode = 0;
  float sun_dir[3] = {0, 0, 1};
  float sun_half = 0.f;
  float eps = 1e-5f;
  int slab_pol = 0;
  // heterogeneous tiles
  const sdd_tileset* tiles = nullptr;
  std::vector<int> mat_tile;           // tile index per material, -1 otherwise
  std::vector<int> tile_mats;          // the HETERO_TILE materials
  std::vector<float3> tile_mat_normal; // their first triangle's normal
  DevArr<int> t_mat_tile, t_tile_mats;
  DevArr<float3> t_tile_normal;
  DevArr<uint32_t> tile_queue;
  DevArr<float> sun_T;
  unsigned sun_T_version = ~0u;
  const sdd_surrogate* sun_T_net = nullptr;
  // device scene
  DevArr<Node> nodes;
  DevArr<TriRec> tris;
  DevArr<float4> prim;
  DevScene dev{};
  // out-of-core subdomains (sdd_tuning.resident_subdomains > 0): the BVH lives in pinned host
  // memory and at most `cap` subdomains' nodes and triangle records occupy device slots
  struct Streaming {
    int cap = 0;
    Node* h_nodes = nullptr;   // pinned host copy of every subdomain's nodes (absolute links)
    TriRec* h_tris = nullptr;
    int64_t n_nodes = 0, n_tris = 0;
    std::vector<int> node0, nnodes, tri0, ntris;  // per subdomain ranges in the host arrays
    int slot_nodes = 0, slot_tris = 0;            // capacity of one slot
    DevArr<Node> d_nodes;      // cap slots
    DevArr<TriRec> d_tris;
    std::vector<int> slot_of, sub_in_slot;  // subdomain -> slot, slot -> subdomain (-1: none)
  } strm;
  int n_sub = 1, axis = 0, bvh_max_depth = 0;
  int64_t n_refs = 0, n_nodes = 0, n_tri_recs = 0;
  // per-render spectral tables (cached for the last wavelength set)
  std::vector<float> cached_lambda;
  DevArr<float> t_lambda, t_thick, t_n, t_k, t_alb, t_sky, t_sun;
  DevArr<int> t_kind;
  DevArr<double> cmf_w;
  // workspace
  DevArr<float4> rb_o[2], rb_d[2], sb_o, sb_d;
  DevArr<float> rb_w[2], sb_c;  // spectral bundles: per-member throughput / shadow contribution
  DevArr<unsigned long long> rb_m[2], sb_m;  // spectral bundles: member masks of rays / shadow rays
  DevArr<uint2> rb_info[2], sb_info;
  DevArr<float2> hits;
  DevArr<uint32_t> q[2], sq[2];
  DevArr<float> path_L;
  DevArr<uint32_t> path_hash;
  DevArr<double> film;
  DevArr<int32_t> pixel_list;
  DevArr<float> out_spec, out_xyz;
  Control* d_ctl = nullptr;
  Control* h_ctl = nullptr;
  sdd_tuning tuning{128, 0, 0, 0, 0, 0, 0};
  // batched form: persistent-wave bookkeeping, internal stream and the captured frame graph
  PersistCtl* d_pc = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gevent = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t bstream = nullptr;  // graph form: captures the bodies of the pass loops
  std::vector<unsigned char> graph_key;
  std::vector<std::pair<int, int>> graph_ev;  // graph form: (kind, event pair) recorded in the graph
  int64_t graph_launches[TK_COUNT] = {};       // graph form: launches per frame by kind
  cudaEvent_t pev[2] = {nullptr, nullptr};
  // profiling
  int profiling = 0;
  sdd_stats stats{};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;  // (kind, index of the start event)
  size_t ev_next = 0;

  ~sdd_scene() {
    DevArr<Node>* a[] = {&nodes};
    for (auto* x : a) x->release();
    strm.d_nodes.release();
    strm.d_tris.release();
    cudaFreeHost(strm.h_nodes);
    cudaFreeHost(strm.h_tris);
    tris.release();
    prim.release();
    t_lambda.release(); t_thick.release(); t_n.release(); t_k.release(); t_alb.release();
    t_sky.release(); t_sun.release(); t_kind.release(); cmf_w.release();
    t_mat_tile.release(); t_tile_mats.release(); t_tile_normal.release(); tile_queue.release(); sun_T.release();
    for (int i = 0; i < 2; ++i) {
      rb_o[i].release(); rb_d[i].release(); rb_info[i].release(); q[i].release(); sq[i].release();
      rb_w[i].release();
      rb_m[i].release();
    }
    sb_c.release();
    sb_m.release();
    sb_o.release(); sb_d.release(); sb_info.release(); hits.release(); path_L.release();
    path_hash.release(); film.release(); pixel_list.release(); out_spec.release(); out_xyz.release();
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (d_pc) cudaFree(d_pc);
    if (gevent) cudaEventDestroy(gevent);
    for (auto e : pev)
      if (e) cudaEventDestroy(e);
    if (gstream) cudaStreamDestroy(gstream);
    if (bstream) cudaStreamDestroy(bstream);
    if (d_ctl) cudaFree(d_ctl);
    if (h_ctl) cudaFreeHost(h_ctl);
    for (auto e : ev_pool) cudaEventDestroy(e);
  }

  // ---- timing helpers: a pair of events around every launch when profiling >= 1
  int ev_begin(int kind, cudaStream_t st) {
    if (profiling < 1) return -1;
    if (ev_next + 2 > ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ev_pool.push_back(e);
      }
    }
    int idx = (int)ev_next;
    ev_next += 2;
    record(ev_pool[idx], st);
    ev_used.push_back({kind, idx});
    return idx;
  }
  void ev_end(int idx, cudaStream_t st) {
    if (idx >= 0) record(ev_pool[idx + 1], st);
  }
  // In a stream capture a plain event record only orders captured work; an external record
  // becomes an event node of the graph that records at every replay.
  static void record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  // Called after a stream sync: fold every recorded pair into the stats.
  void ev_collect() {
    for (auto& u : ev_used) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev_pool[u.second], ev_pool[u.second + 1]);
      double* dst[TK_COUNT] = {&stats.ms_raygen, &stats.ms_traverse, &stats.ms_shade, &stats.ms_shadow,
                               &stats.ms_film, &stats.ms_tile};
      *dst[u.first] += ms;
    }
    ev_used.clear();
    ev_next = 0;
  }
};

// Photon maps (Sec. 3.2): per map (0 caustic, 1 global) the stored photons as appended
// (kept for sdd_photon_maps_get) and sorted into the buckets of the hashed grid.
struct sdd_photon_maps {
  std::vector<float> lambda;  // wavelengths the maps were built for
  float radius = 0.f, inv_cell = 0.f;
  uint32_t mask = 0;
  int64_t count[2] = {0, 0};
  DevArr<float4> raw_pos[2], raw_nrm[2], pos[2], nrm[2];
  DevArr<uint2> raw_id[2];
  DevArr<uint32_t> start[2];
  ~sdd_photon_maps() {
    for (int m = 0; m < 2; ++m) {
      raw_pos[m].release(); raw_nrm[m].release(); pos[m].release(); nrm[m].release();
      raw_id[m].release(); start[m].release();
    }
  }
  PhotonMapDev view() const {
    PhotonMapDev v{};
    for (int m = 0; m < 2; ++m) {
      v.pos_pw[m] = pos[m].p;
      v.nrm_lam[m] = nrm[m].p;
      v.start[m] = start[m].p;
    }
    v.mask = mask;
    v.inv_cell = inv_cell;
    v.radius = radius;
    return v;
  }
};

namespace sdd {
// Used by the allocation-free entry point (noalloc.cu).
const DevScene* scene_device_view(const sdd_scene* s) { return &s->dev; }
bool scene_streaming(const sdd_scene* s) { return s->strm.cap > 0; }
sdd_status set_last_error(sdd_status st, const char* msg) {
  g_err = msg;
  return st;
}
}  // namespace sdd

namespace {

void count_launch(sdd_scene* s, int kind) {
  int64_t* dst[TK_COUNT] = {&s->stats.launches_raygen, &s->stats.launches_traverse, &s->stats.launches_shade,
                            &s->stats.launches_shadow, &s->stats.launches_film, &s->stats.launches_tile};
  ++*dst[kind];
  ++s->stats.launches_total;
}

sdd_status validate_table(const char* what, int n, const float* lam, const float* v, bool required) {
  if (!v) {
    if (required) return fail(SDD_ERR_ARG, std::string(what) + " table is NULL");
    return SDD_OK;
  }
  if (n < 1 || !lam) return fail(SDD_ERR_ARG, std::string(what) + ": n_lambda < 1 or lambda_nm NULL");
  for (int i = 1; i < n; ++i)
    if (!(lam[i] > lam[i - 1])) return fail(SDD_ERR_ARG, std::string(what) + ": lambda_nm not ascending");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return fail(SDD_ERR_ARG, std::string(what) + ": non-finite value");
  return SDD_OK;
}

sdd_status read_ctl(sdd_scene* s, cudaStream_t st) {
  CK(cudaMemcpyAsync(s->h_ctl, s->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

sdd_status device_error(uint32_t e) {
  if (e & ERR_STACK_OVERFLOW) return fail(SDD_ERR_STACK, "BVH traversal stack overflow");
  if (e & (ERR_QUEUE_OVERFLOW | ERR_SHADOW_OVERFLOW))
    return fail(SDD_ERR_QUEUE_OVERFLOW, "ray queue capacity exceeded (lower wave_paths or max_depth)");
  if (e & ERR_TIMEOUT) return fail(SDD_ERR_TIMEOUT, "device loop hit its iteration cap");
  return SDD_OK;
}

// ------------------------------------------------------------------ out-of-core subdomains
// Sec. 5: sub-domains are loaded according to the memory available and unloaded when few
// rays remain for them.  With streaming on (host-driven form), before every traversal pass a
// resident subdomain stays in its device slot while its queue holds rays; slots whose
// subdomain has none left (or that are empty) go to the waiting subdomains with the most
// queued rays, whose nodes and triangle records are copied in from pinned host memory (one
// asynchronous copy each) and whose links a small kernel then rebases to the slot.  Rays
// queued for subdomains that are not resident wait, unchanged, for a later pass; rays cross
// each slab at most once, so resident queues drain and every waiting queue is reached.  The
// traversal code is the same; only where the nodes lie changes, so every hit, path and image
// is the all-resident one bit for bit.

// Links of a subdomain's nodes copied into slot j: inner children from the subdomain's first
// node n0 to the slot's nbase, leaf triangle ranges from its first record t0 to tbase.
__device__ __forceinline__ int rebase_link(int link, int cnt, int n0, int nbase, int t0, int tbase) {
  if (cnt > 0) return link - t0 + tbase;
  return link >= 0 ? link - n0 + nbase : link;
}
__global__ void k_rebase_nodes(Node* nodes, int nn, int n0, int nbase, int t0, int tbase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int4 l = nodes[i].link;
  const int4 c = nodes[i].cnt;
  l.x = rebase_link(l.x, c.x, n0, nbase, t0, tbase);
  l.y = rebase_link(l.y, c.y, n0, nbase, t0, tbase);
  l.z = rebase_link(l.z, c.z, n0, nbase, t0, tbase);
  l.w = rebase_link(l.w, c.w, n0, nbase, t0, tbase);
  nodes[i].link = l;
}

// Copy subdomain `sub` from pinned host memory into device slot j and rebase its links there.
cudaError_t load_subdomain(sdd_scene* s, int sub, int j, cudaStream_t st) {
  auto& m = s->strm;
  const int n0 = m.node0[sub], nn = m.nnodes[sub], t0 = m.tri0[sub], nt = m.ntris[sub];
  const int nbase = j * m.slot_nodes, tbase = j * m.slot_tris;
  cudaError_t e = cudaMemcpyAsync(m.d_nodes.p + nbase, m.h_nodes + n0, sizeof(Node) * (size_t)nn,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nt > 0)
    e = cudaMemcpyAsync(m.d_tris.p + tbase, m.h_tris + t0, sizeof(TriRec) * (size_t)nt, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nn > 0) {
    k_rebase_nodes<<<(nn + 255) / 256, 256, 0, st>>>(m.d_nodes.p + nbase, nn, n0, nbase, t0, tbase);
    e = cudaGetLastError();
  }
  s->stats.bytes_streamed += (int64_t)(sizeof(Node) * (size_t)nn + sizeof(TriRec) * (size_t)nt);
  s->stats.subdomain_loads++;
  return e;
}

// Keep the resident subdomains that still have queued rays and give the other slots to the
// waiting subdomains with the most queued rays; runs[i] = the queued count of a resident
// subdomain this pass traverses, 0 for the others.  sc gets the slots.
sdd_status stream_in(sdd_scene* s, const int* counts, DevScene* sc, int* runs, cudaStream_t st) {
  auto& m = s->strm;
  std::vector<char> keep(s->n_sub, 0);
  std::vector<int> waiting;
  for (int i = 0; i < s->n_sub; ++i) {
    if (counts[i] <= 0) continue;
    if (m.slot_of[i] >= 0) keep[i] = 1;
    else waiting.push_back(i);
  }
  std::sort(waiting.begin(), waiting.end(), [&](int a, int b) {
    return counts[a] != counts[b] ? counts[a] > counts[b] : a < b;
  });
  size_t next = 0;
  for (int j = 0; j < m.cap && next < waiting.size(); ++j) {
    const int o = m.sub_in_slot[j];
    if (o >= 0 && keep[o]) continue;  // still has rays: stays
    const int i = waiting[next++];
    if (o >= 0) m.slot_of[o] = -1;    // nothing left for it: unloaded
    CK(load_subdomain(s, i, j, st));
    m.slot_of[i] = j;
    m.sub_in_slot[j] = i;
    keep[i] = 1;
  }
  sc->nodes = m.d_nodes.p;
  sc->tris = m.d_tris.p;
  for (int i = 0; i < s->n_sub; ++i) {
    runs[i] = keep[i] ? counts[i] : 0;
    if (m.slot_of[i] >= 0) sc->root[i] = m.slot_of[i] * m.slot_nodes;
  }
  return SDD_OK;
}

// Rays of subdomains this pass leaves out move, unchanged, to the pass's output queues
// (whose counts were just cleared); the traversal then appends behind them.
sdd_status carry_queues(sdd_scene* s, const int* counts, const int* runs, uint32_t* qin, uint32_t* qout,
                        int* out_count, int qcap, cudaStream_t st) {
  for (int i = 0; i < s->n_sub; ++i) {
    const int c = std::min(std::max(counts[i], 0), qcap);
    if (c == 0 || runs[i] > 0) continue;
    CK(cudaMemcpyAsync(qout + (size_t)i * qcap, qin + (size_t)i * qcap, sizeof(uint32_t) * (size_t)c,
                       cudaMemcpyDeviceToDevice, st));
    launch_set_int(out_count + i, c, st);
  }
  return SDD_OK;
}

// Pass bound of one generation's passes (beyond it: SDD_ERR_TIMEOUT): without streaming a ray
// crosses each slab at most once; with it waiting queues add passes, generously bounded.
int pass_bound(const sdd_scene* s) {
  const int n = s->n_sub;
  return s->strm.cap > 0 ? (2 * n + 2) * (n + 1) : 2 * kMaxSubdomains + 2;
}

Sched make_sched(int n_sub, const int* counts, int cap, int block, int* total_blocks, long long* total) {
  Sched sc;
  sc.n_sub = n_sub;
  int b = 0;
  long long t = 0;
  for (int s = 0; s < n_sub; ++s) {
    sc.blk_start[s] = b;
    sc.count[s] = std::min(std::max(counts[s], 0), cap);  // overflow is reported, never read past cap
    b += (counts[s] + block - 1) / block;
    t += counts[s];
  }
  sc.blk_start[n_sub] = b;
  *total_blocks = b;
  *total = t;
  return sc;
}

// Closest-hit passes: the queues in q[a] (counts in ctl->q_count[a]) are traversed and
// rays crossing an interface move to q[1-a], until every ray has a hit record.
sdd_status run_closest_passes(sdd_scene* s, const RenderParams& p0, RayBuf rb, int qcap, cudaStream_t st) {
  RenderParams p = p0;
  int a = 0;
  const int bound = pass_bound(s);
  for (int pass = 0; pass <= bound; ++pass) {
    sdd_status r = read_ctl(s, st);
    if (r) return r;
    if (s->h_ctl->error) return device_error(s->h_ctl->error);
    int nb;
    long long total;
    const int blk = s->tuning.traverse_block;
    const int* counts = s->h_ctl->q_count[a];
    int runs[kMaxSubdomains];
    long long queued = 0;
    for (int i = 0; i < s->n_sub; ++i) queued += std::max(counts[i], 0);
    if (queued == 0) return SDD_OK;
    if (s->strm.cap > 0 && (r = stream_in(s, counts, &p.sc, runs, st))) return r;
    Sched sch = make_sched(s->n_sub, s->strm.cap > 0 ? runs : counts, qcap, blk, &nb, &total);
    CK(cudaMemsetAsync(s->d_ctl->q_count[1 - a], 0, sizeof(int) * kMaxSubdomains, st));
    if (s->strm.cap > 0 &&
        (r = carry_queues(s, counts, runs, s->q[a].p, s->q[1 - a].p, s->d_ctl->q_count[1 - a], qcap, st)))
      return r;
    QueuePair qp{s->q[a].p, s->q[1 - a].p, s->d_ctl->q_count[1 - a], qcap};
    int ev = s->ev_begin(TK_TRAVERSE, st);
    launch_traverse(p, sch, nb, blk, s->tuning.top_nodes, qp, rb, s->hits.p, s->d_ctl, st);
    s->ev_end(ev, st);
    CK(cudaGetLastError());
    count_launch(s, TK_TRAVERSE);
    a = 1 - a;
  }
  return fail(SDD_ERR_TIMEOUT, "closest-hit passes did not drain the subdomain queues");
}

sdd_status run_shadow_passes(sdd_scene* s, const RenderParams& p0, const WaveDesc& w, int qcap, cudaStream_t st) {
  RenderParams p = p0;
  int a = 0;
  ShadowBuf sb{s->sb_o.p, s->sb_d.p, s->sb_info.p, qcap, s->sb_c.p, s->sb_m.p};
  const int bound = pass_bound(s);
  for (int pass = 0; pass <= bound; ++pass) {
    sdd_status r = read_ctl(s, st);
    if (r) return r;
    if (s->h_ctl->error) return device_error(s->h_ctl->error);
    int nb;
    long long total;
    const int blk = s->tuning.traverse_block;
    const int* counts = s->h_ctl->sq_count[a];
    int runs[kMaxSubdomains];
    long long queued = 0;
    for (int i = 0; i < s->n_sub; ++i) queued += std::max(counts[i], 0);
    if (queued == 0) return SDD_OK;
    if (s->strm.cap > 0 && (r = stream_in(s, counts, &p.sc, runs, st))) return r;
    Sched sch = make_sched(s->n_sub, s->strm.cap > 0 ? runs : counts, qcap, blk, &nb, &total);
    CK(cudaMemsetAsync(s->d_ctl->sq_count[1 - a], 0, sizeof(int) * kMaxSubdomains, st));
    if (s->strm.cap > 0 &&
        (r = carry_queues(s, counts, runs, s->sq[a].p, s->sq[1 - a].p, s->d_ctl->sq_count[1 - a], qcap, st)))
      return r;
    QueuePair qp{s->sq[a].p, s->sq[1 - a].p, s->d_ctl->sq_count[1 - a], qcap};
    int ev = s->ev_begin(TK_SHADOW, st);
    launch_shadow(p, w, sch, nb, blk, s->tuning.top_nodes, qp, sb, s->path_L.p, s->d_ctl, st);
    s->ev_end(ev, st);
    CK(cudaGetLastError());
    count_launch(s, TK_SHADOW);
    a = 1 - a;
  }
  return fail(SDD_ERR_TIMEOUT, "shadow passes did not drain the subdomain queues");
}

// Resample every material / illuminant table to the render wavelengths and upload.
sdd_status prepare_spectral(sdd_scene* s, int L, const float* lam, cudaStream_t st) {
  std::vector<float> want(lam, lam + L);
  if (want == s->cached_lambda && s->t_lambda.p) return SDD_OK;
  size_t M = s->mats.size();
  std::vector<int> kind(M);
  std::vector<float> thick(M), tn(M * L), tk(M * L), ta(M * L), sky(L), sun(L);
  for (size_t m = 0; m < M; ++m) {
    const HostMaterial& hm = s->mats[m];
    kind[m] = hm.kind;
    thick[m] = hm.thick;
    for (int l = 0; l < L; ++l) {
      tn[m * L + l] = (float)interp_table(hm.lam, hm.n, lam[l]);
      tk[m * L + l] = (float)interp_table(hm.lam, hm.k, lam[l]);
      ta[m * L + l] = (float)interp_table(hm.lam, hm.albedo, lam[l]);
    }
  }
  for (int l = 0; l < L; ++l) {
    sky[l] = (float)interp_table(s->il_lam, s->il_sky, lam[l]);
    sun[l] = s->il_sun.empty() ? 0.f : (float)interp_table(s->il_lam, s->il_sun, lam[l]);
  }
  CK(s->t_lambda.ensure(L));
  CK(s->t_kind.ensure(M));
  CK(s->t_thick.ensure(M));
  CK(s->t_n.ensure(M * L));
  CK(s->t_k.ensure(M * L));
  CK(s->t_alb.ensure(M * L));
  CK(s->t_sky.ensure(L));
  CK(s->t_sun.ensure(L));
  CK(s->cmf_w.ensure(3 * (size_t)L));
  CK(cudaMemcpyAsync(s->t_lambda.p, lam, sizeof(float) * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_kind.p, kind.data(), sizeof(int) * M, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_thick.p, thick.data(), sizeof(float) * M, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_n.p, tn.data(), sizeof(float) * M * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_k.p, tk.data(), sizeof(float) * M * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_alb.p, ta.data(), sizeof(float) * M * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_sky.p, sky.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_sun.p, sun.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st));
  if (!s->tile_mats.empty()) {
    CK(s->t_mat_tile.ensure(M));
    CK(cudaMemcpyAsync(s->t_mat_tile.p, s->mat_tile.data(), sizeof(int) * M, cudaMemcpyHostToDevice, st));
    CK(s->t_tile_mats.ensure(s->tile_mats.size()));
    CK(cudaMemcpyAsync(s->t_tile_mats.p, s->tile_mats.data(), sizeof(int) * s->tile_mats.size(),
                       cudaMemcpyHostToDevice, st));
    CK(s->t_tile_normal.ensure(s->tile_mats.size()));
    CK(cudaMemcpyAsync(s->t_tile_normal.p, s->tile_mat_normal.data(), sizeof(float3) * s->tile_mats.size(),
                       cudaMemcpyHostToDevice, st));
  }
  s->sun_T_version = ~0u;  // the network's sun table depends on the wavelengths
  launch_cmf_table(L, s->t_lambda.p, s->cmf_w.p, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));  // host vectors above go out of scope
  s->cached_lambda = want;
  return SDD_OK;
}

DevCamera make_camera(const sdd_camera* c) {
  double pos[3] = {c->pos[0], c->pos[1], c->pos[2]};
  double f[3] = {c->look_at[0] - pos[0], c->look_at[1] - pos[1], c->look_at[2] - pos[2]};
  double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (double& x : f) x /= fl;
  double up[3] = {c->up[0], c->up[1], c->up[2]};
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (double& x : r) x /= rl;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  DevCamera dc;
  dc.pos = make_float3((float)pos[0], (float)pos[1], (float)pos[2]);
  dc.fwd = make_float3((float)f[0], (float)f[1], (float)f[2]);
  dc.right = make_float3((float)r[0], (float)r[1], (float)r[2]);
  dc.up = make_float3((float)u[0], (float)u[1], (float)u[2]);
  dc.tan_half = (float)std::tan(0.5 * c->vfov_deg * M_PI / 180.0);
  dc.aspect = (float)c->width / (float)c->height;
  dc.ortho_half = 0.5f * c->ortho_height_m;
  dc.width = c->width;
  dc.height = c->height;
  dc.ortho = c->orthographic;
  return dc;
}

sdd_status ensure_ctl(sdd_scene* s) {
  if (!s->d_ctl) {
    CK(cudaMalloc(&s->d_ctl, sizeof(Control)));
    CK(cudaMallocHost(&s->h_ctl, sizeof(Control)));
  }
  return SDD_OK;
}

// Workspace for `cap` rays per generation and `paths` paths per wave.
sdd_status ensure_workspace(sdd_scene* s, size_t cap, size_t paths, int n_slots, bool hash, int bundle) {
  for (int i = 0; i < 2; ++i) {
    if (bundle > 1) CK(s->rb_w[i].ensure(cap * (size_t)bundle));
    if (bundle > 1) CK(s->rb_m[i].ensure(cap));
    CK(s->rb_o[i].ensure(cap));
    CK(s->rb_d[i].ensure(cap));
    CK(s->rb_info[i].ensure(cap));
    CK(s->q[i].ensure(cap * (size_t)s->n_sub));
    CK(s->sq[i].ensure(cap * (size_t)s->n_sub));
  }
  if (bundle > 1) CK(s->sb_c.ensure(cap * (size_t)bundle));
  if (bundle > 1) CK(s->sb_m.ensure(cap));
  CK(s->sb_o.ensure(cap));
  CK(s->sb_d.ensure(cap));
  CK(s->sb_info.ensure(cap));
  CK(s->hits.ensure(cap));
  CK(s->path_L.ensure(paths * (size_t)n_slots));
  if (hash) CK(s->path_hash.ensure(paths * (size_t)std::max(bundle, 1)));
  return ensure_ctl(s);
}

// Enqueue the whole frame of the batched form on stream `gs`: per wave, clear the wave's
// bookkeeping and path radiance, one persistent cooperative launch, film accumulation; then
// the final film resolve.
// The closest-hit (shadow = false) or shadow passes of one generation of the graph form,
// until its queues drain.  In a graph capture: a conditional 'while' node whose body runs two
// passes (queue buffer 0 to 1, then 1 to 0) and the loop condition, which reads the counts on
// the device (at most n_sub / 2 + 2 iterations; a ray crosses each slab at most once).
// Enqueued directly: n_sub + 1 passes and a drain check.  Timed as a whole.
sdd_status graph_passes(sdd_scene* s, const RenderParams& p, const GraphGrids& gg, const WaveDesc& w,
                        const PersistBuffers& b, int cur, bool shadow, cudaStream_t gs, int64_t* cnt) {
  Control* c = s->d_ctl;
  const int nsub = p.sc.n_sub, qcap = b.qcap;
  int(*counts)[kMaxSubdomains] = shadow ? c->sq_count : c->q_count;
  uint32_t* const* qs = shadow ? b.sq : b.q;
  auto pass = [&](int a, cudaStream_t st) -> sdd_status {
    CK(cudaMemsetAsync(counts[1 - a], 0, sizeof(int) * kMaxSubdomains, st));
    CK(cudaMemsetAsync(&c->work[a], 0, sizeof(int), st));
    QueuePair qp{qs[a], qs[1 - a], counts[1 - a], qcap};
    if (shadow) CK(launch_shadow_g(p, gg, w, counts[a], &c->work[a], qp, b.sb, b.path_L, c, st));
    else CK(launch_traverse_g(p, gg, counts[a], &c->work[a], qp, b.rb[cur], b.hits, c, st));
    return SDD_OK;
  };
  const int kind = shadow ? TK_SHADOW : TK_TRAVERSE;
  int ev = s->ev_begin(kind, gs);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(gs, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    CK(cudaMemsetAsync(&c->loop_iter, 0, sizeof(int), gs));
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(gs, &cs, nullptr, &g, &deps, &edges, &nd));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(gs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(s->bstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    sdd_status r = pass(0, s->bstream);
    if (r == SDD_OK) r = pass(1, s->bstream);
    if (r == SDD_OK) launch_loop_cond(h, counts[0], nsub, nsub / 2 + 2, shadow ? 1 : 0, c, s->bstream);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s->bstream, &out);
    if (r != SDD_OK) return r;
    CK(e);
  } else {
    for (int i = 0, a = 0; i <= nsub; ++i, a = 1 - a) {
      sdd_status r = pass(a, gs);
      if (r != SDD_OK) return r;
      cnt[kind]++;
    }
    launch_check_drained(counts[(nsub + 1) & 1], nsub, c, gs);
  }
  s->ev_end(ev, gs);
  CK(cudaGetLastError());
  return SDD_OK;
}

// One wave of the graph form (graph_kernels.cu): raygen, then per generation the closest-hit
// passes, shading (and the fused tile shading) and the shadow passes, every launch with a
// fixed grid that reads its counts on the device.  Counts host-known launches into cnt.
sdd_status enqueue_graph_wave(sdd_scene* s, const RenderParams& p, const WaveDesc& w, const PersistBuffers& b,
                              const GraphGrids& gg, const sdd_render_opts* o, cudaStream_t gs, int64_t* cnt) {
  Control* c = s->d_ctl;
  const int qcap = b.qcap;
  int ev = s->ev_begin(TK_RAYGEN, gs);
  launch_raygen(p, w, b.rb[0], b.q[0], c->q_count[0], qcap, c, gs);
  launch_set_int(&c->gen_rays[0], (int)w.n_paths, gs);
  s->ev_end(ev, gs);
  CK(cudaGetLastError());
  cnt[TK_RAYGEN] += 2;
  int cur = 0;
  for (int g = 0; g <= p.max_depth + 1; ++g) {
    sdd_status r = graph_passes(s, p, gg, w, b, cur, false, gs, cnt);
    if (r != SDD_OK) return r;
    // shading refills q[0] and sq[0] from cleared counts
    CK(cudaMemsetAsync(c, 0, offsetof(Control, error), gs));
    CK(cudaMemsetAsync(&c->gen_rays[(g + 1) & 1], 0, sizeof(int), gs));
    if (p.use_surrogate) CK(cudaMemsetAsync(&c->tile_hits, 0, sizeof(int), gs));
    ev = s->ev_begin(TK_SHADE, gs);
    CK(launch_shade_g(p, gg, w, &c->gen_rays[g & 1], b.rb[cur], b.hits, b.rb[1 - cur], &c->gen_rays[(g + 1) & 1],
                      b.q[0], c->q_count[0], qcap, b.sb, b.sq[0], c->sq_count[0], b.path_L, c, gs));
    s->ev_end(ev, gs);
    cnt[TK_SHADE]++;
    if (p.use_surrogate) {
      ev = s->ev_begin(TK_TILE, gs);
      CK(launch_tile_shade(p, w, b.rb[cur], b.hits, b.rb[1 - cur], &c->gen_rays[(g + 1) & 1], b.q[0],
                           c->q_count[0], qcap, c, o->surrogate, gs));
      s->ev_end(ev, gs);
      cnt[TK_TILE]++;
    }
    r = graph_passes(s, p, gg, w, b, cur, true, gs, cnt);
    if (r != SDD_OK) return r;
    cur = 1 - cur;
  }
  return SDD_OK;
}

sdd_status enqueue_batched_frame(sdd_scene* s, const RenderParams& p, const std::vector<WaveDesc>& waves,
                                 const PersistBuffers& b, int n_slots, int grid, const GraphGrids& gg,
                                 const sdd_render_opts* o, float* spectral_out, float* xyz_out, cudaStream_t gs,
                                 int64_t* cnt) {
  CK(cudaMemsetAsync(s->d_ctl, 0, sizeof(Control), gs));
  CK(cudaMemsetAsync(s->film.p, 0, sizeof(double) * (size_t)p.n_px * p.sp.n_lambda, gs));
  for (const WaveDesc& w : waves) {
    CK(cudaMemsetAsync(s->path_L.p, 0, sizeof(float) * (size_t)w.n_paths * n_slots, gs));
    if (o->batched == 2) {
      // queue counts of the wave; the error word keeps what earlier waves raised
      CK(cudaMemsetAsync(s->d_ctl, 0, offsetof(Control, error), gs));
      sdd_status r = enqueue_graph_wave(s, p, w, b, gg, o, gs, cnt);
      if (r) return r;
    } else if (!p.use_surrogate) {
      CK(cudaMemsetAsync(s->d_pc, 0, sizeof(PersistCtl), gs));
      CK(launch_persistent_wave(p, w, b, s->d_pc, s->d_ctl, grid, gs, SEG_WAVE));
    } else {
      // the network runs between shading and the shadow rays of every generation
      CK(cudaMemsetAsync(s->d_pc, 0, sizeof(PersistCtl), gs));
      CK(launch_persistent_wave(p, w, b, s->d_pc, s->d_ctl, grid, gs, SEG_RAYGEN));
      for (int g = 0; g <= p.max_depth + 1; ++g) {
        CK(cudaMemsetAsync(&s->d_ctl->tile_hits, 0, sizeof(int), gs));
        CK(launch_persistent_wave(p, w, b, s->d_pc, s->d_ctl, grid, gs, SEG_CLOSEST_SHADE));
        CK(launch_tile_shade_persistent(p, w, b, s->d_pc, s->d_ctl, o->surrogate, gs));
        CK(launch_persistent_wave(p, w, b, s->d_pc, s->d_ctl, grid, gs, SEG_SHADOW));
      }
    }
    int ev = o->batched == 2 ? s->ev_begin(TK_FILM, gs) : -1;
    launch_film_accum(p, w, s->path_L.p, s->film.p, o->path_radiance_out, o->path_hash_out, gs);
    s->ev_end(ev, gs);
    CK(cudaGetLastError());
    cnt[TK_FILM]++;
  }
  launch_film_finalize(p, s->film.p, s->cmf_w.p, spectral_out, xyz_out, gs);
  CK(cudaGetLastError());
  cnt[TK_FILM]++;
  return SDD_OK;
}

// The batched form: the frame runs on the scene's internal stream (ordered after the
// caller's stream), captured once as a CUDA graph and replayed while the key -- every kernel
// parameter and buffer address of the frame -- is unchanged.
sdd_status render_batched(sdd_scene* s, const RenderParams& p, const std::vector<WaveDesc>& waves, int n_slots,
                          int qcap, const sdd_render_opts* o, float* spectral_out, float* xyz_out, cudaStream_t st) {
  if (!s->gstream) {
    CK(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&s->gevent, cudaEventDisableTiming));
    CK(cudaEventCreate(&s->pev[0]));
    CK(cudaEventCreate(&s->pev[1]));
  }
  if (!s->d_pc) CK(cudaMalloc(&s->d_pc, sizeof(PersistCtl)));
  const int form = o->batched;  // 1 persistent kernel, 2 graph form
  int grid = 0;
  GraphGrids gg{};
  if (form == 2) {
    gg = graph_grids(p, s->tuning.top_nodes, s->tuning.block_chunks);  // occupancy queries stay outside the capture
  } else {
    grid = persistent_grid(p.stats >= 2, tile_mode(p), p.bundle);
    if (grid <= 0) return fail(SDD_ERR_CUDA, "persistent kernel does not fit on this device");
  }
  PersistBuffers b;
  for (int i = 0; i < 2; ++i) {
    b.rb[i] = RayBuf{s->rb_o[i].p, s->rb_d[i].p, s->rb_info[i].p, qcap, s->rb_w[i].p, s->rb_m[i].p};
    b.q[i] = s->q[i].p;
    b.sq[i] = s->sq[i].p;
  }
  b.hits = s->hits.p;
  b.sb = ShadowBuf{s->sb_o.p, s->sb_d.p, s->sb_info.p, qcap, s->sb_c.p, s->sb_m.p};
  b.path_L = s->path_L.p;
  b.qcap = qcap;
  // graph key: everything the captured frame depends on
  std::vector<unsigned char> key;
  auto put = [&key](const void* d, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(d);
    key.insert(key.end(), c, c + n);
  };
  put(&p, sizeof(p));
  put(&b, sizeof(b));
  put(&grid, sizeof(grid));
  put(&gg, sizeof(gg));
  put(&form, sizeof(form));
  put(&n_slots, sizeof(n_slots));
  for (const WaveDesc& w : waves) put(&w, sizeof(w));
  const void* ptrs[] = {spectral_out, xyz_out, o->path_radiance_out, o->path_hash_out, s->film.p, s->cmf_w.p,
                        s->d_pc, s->d_ctl, o->surrogate};
  put(ptrs, sizeof(ptrs));

  CK(cudaEventRecord(s->gevent, st));
  CK(cudaStreamWaitEvent(s->gstream, s->gevent, 0));
  if (s->profiling >= 1) CK(cudaEventRecord(s->pev[0], s->gstream));
  bool replay = !s->tuning.no_graph && s->graph_exec && key == s->graph_key;
  if (!replay) {
    if (s->graph_exec) {
      cudaGraphExecDestroy(s->graph_exec);
      s->graph_exec = nullptr;
      s->graph_key.clear();
    }
    cudaGraph_t graph = nullptr;
    bool captured = false;
    int64_t cnt[TK_COUNT] = {};
    s->ev_used.clear();
    s->ev_next = 0;
    if (!s->tuning.no_graph && cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      sdd_status r = enqueue_batched_frame(s, p, waves, b, n_slots, grid, gg, o, spectral_out, xyz_out, s->gstream,
                                           cnt);
      cudaError_t ec = cudaStreamEndCapture(s->gstream, &graph);
      if (r == SDD_OK && ec == cudaSuccess && graph &&
          cudaGraphInstantiate(&s->graph_exec, graph, 0) == cudaSuccess) {
        captured = true;
        s->graph_key = key;
        s->graph_ev = s->ev_used;  // event nodes of the graph, re-recorded at every replay
        for (int k = 0; k < TK_COUNT; ++k) s->graph_launches[k] = cnt[k];
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();  // a failed capture leaves a sticky-free error; clear it
    }
    if (!captured) {
      // capture not available: enqueue the same frame directly
      s->graph_exec = nullptr;
      s->ev_used.clear();
      s->ev_next = 0;
      for (int k = 0; k < TK_COUNT; ++k) cnt[k] = 0;
      sdd_status r = enqueue_batched_frame(s, p, waves, b, n_slots, grid, gg, o, spectral_out, xyz_out, s->gstream,
                                           cnt);
      if (r) return r;
      s->graph_ev.clear();
      for (int k = 0; k < TK_COUNT; ++k) s->graph_launches[k] = cnt[k];
    }
  }
  if (s->graph_exec) {
    CK(cudaGraphLaunch(s->graph_exec, s->gstream));
    if (replay) s->stats.graph_replays++;
  }
  if (s->profiling >= 1) CK(cudaEventRecord(s->pev[1], s->gstream));
  CK(cudaStreamSynchronize(s->gstream));
  if (form == 2) {
    if (s->graph_exec) s->ev_used = s->graph_ev;
    s->ev_collect();
    int64_t* dst[TK_COUNT] = {&s->stats.launches_raygen, &s->stats.launches_traverse, &s->stats.launches_shade,
                              &s->stats.launches_shadow, &s->stats.launches_film, &s->stats.launches_tile};
    for (int k = 0; k < TK_COUNT; ++k) {
      *dst[k] += s->graph_launches[k];
      s->stats.launches_total += s->graph_launches[k];
    }
    if (s->profiling >= 1) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, s->pev[0], s->pev[1]);
      s->stats.ms_persistent = ms;
    }
    return SDD_OK;
  }
  const int64_t per_wave = p.use_surrogate ? 1 + 2 * (int64_t)(p.max_depth + 2) : 1;
  s->stats.launches_persistent += per_wave * (int64_t)waves.size();
  if (p.use_surrogate) s->stats.launches_tile += (int64_t)(p.max_depth + 2) * (int64_t)waves.size();
  s->stats.launches_film += (int64_t)waves.size() + 1;
  s->stats.launches_total += (per_wave + (p.use_surrogate ? p.max_depth + 2 : 0) + 1) * (int64_t)waves.size() + 1;
  if (s->profiling >= 1) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->pev[0], s->pev[1]);
    s->stats.ms_persistent = ms;
  }
  PersistCtl hpc;
  CK(cudaMemcpy(&hpc, s->d_pc, sizeof(PersistCtl), cudaMemcpyDeviceToHost));
  if (hpc.abort) return fail(SDD_ERR_TIMEOUT, "persistent wave abandoned: a grid barrier hit its time limit");
  return SDD_OK;
}

// Each wave as two halves, in order: by samples when it has several (each cell still
// accumulates its samples in order), else by cells.  A wave of one path stays whole.
std::vector<WaveDesc> halve_waves(const std::vector<WaveDesc>& in) {
  std::vector<WaveDesc> out;
  for (const WaveDesc& w : in) {
    if (w.ns <= 1 && w.nc <= 1) {
      out.push_back(w);
      continue;
    }
    WaveDesc a = w, b = w;
    if (w.ns > 1) {
      a.ns = w.ns / 2;
      b.s0 = w.s0 + a.ns;
      b.ns = w.ns - a.ns;
    } else {
      a.nc = w.nc / 2;
      b.c0 = w.c0 + a.nc;
      b.nc = w.nc - a.nc;
    }
    a.n_paths = a.ns * a.nc;
    b.n_paths = b.ns * b.nc;
    out.push_back(a);
    out.push_back(b);
  }
  return out;
}

// (pixel, sample, wavelength) chains of a wave: its cells times the samples, with bundles the
// members of each cell's bundle (the last bundle of a pixel may be partial).
// Parameters every launch over the scene shares: geometry, the spectral tables of the
// current wavelength set (prepare_spectral) and illuminant, and the tile set.
RenderParams scene_params(const sdd_scene* s, int L) {
  RenderParams p{};
  p.sc = s->dev;
  p.sp.n_lambda = L;
  p.sp.lambda_nm = s->t_lambda.p;
  p.sp.mat_kind = s->t_kind.p;
  p.sp.mat_thick = s->t_thick.p;
  p.sp.mat_n = s->t_n.p;
  p.sp.mat_k = s->t_k.p;
  p.sp.mat_albedo = s->t_alb.p;
  p.sp.sky = s->t_sky.p;
  p.sp.sun = s->t_sun.p;
  p.sp.sky_mode = s->sky_mode;
  p.sp.slab_pol = s->slab_pol;
  double sd[3] = {s->sun_dir[0], s->sun_dir[1], s->sun_dir[2]};
  double l = std::sqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
  p.sp.sun_dir = make_float3((float)(sd[0] / l), (float)(sd[1] / l), (float)(sd[2] / l));
  bool has_sun = !s->il_sun.empty() && s->sun_half > 0.f;
  double h = has_sun ? 2.0 * std::sin(0.5 * s->sun_half) * std::sin(0.5 * s->sun_half) : 0.0;
  p.sp.sun_h = (float)h;
  p.sp.sun_omega = (float)(2.0 * M_PI * h);
  if (!s->tile_mats.empty()) {
    p.tiles = *tileset_device_view(s->tiles);
    p.mat_tile = s->t_mat_tile.p;
  }
  return p;
}

int64_t spectral_paths(const RenderParams& p, const WaveDesc& w) {
  if (p.bundle <= 1) return (int64_t)w.n_paths;
  const int64_t nb = p.n_bundles, c0 = w.c0, c1 = (int64_t)w.c0 + w.nc;
  const int64_t last = c1 / nb - c0 / nb;  // cells in [c0, c1) holding a pixel's last bundle
  const int64_t members = (int64_t)w.nc * p.bundle - last * (nb * p.bundle - p.sp.n_lambda);
  return members * (int64_t)w.ns;
}

sdd_status render_impl(sdd_scene* s, const sdd_camera* cam, const sdd_render_opts* o, float* spectral_out,
                       float* xyz_out, cudaStream_t st) {
  if (!s || !cam || !o) return fail(SDD_ERR_ARG, "NULL scene, camera or options");
  if (cam->width <= 0 || cam->height <= 0) return fail(SDD_ERR_ARG, "camera width/height must be positive");
  if ((long long)cam->width * cam->height > (1LL << 30)) return fail(SDD_ERR_ARG, "image too large");
  if (!cam->orthographic && !(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f))
    return fail(SDD_ERR_ARG, "vfov_deg must be in (0, 180)");
  if (cam->orthographic && !(cam->ortho_height_m > 0.f)) return fail(SDD_ERR_ARG, "ortho_height_m must be > 0");
  if (o->n_lambda < 1 || !o->lambda_nm) return fail(SDD_ERR_ARG, "n_lambda < 1 or lambda_nm NULL");
  if (o->n_lambda > 4096) return fail(SDD_ERR_ARG, "n_lambda > 4096");
  for (int i = 0; i < o->n_lambda; ++i)
    if (!(o->lambda_nm[i] > 0.f)) return fail(SDD_ERR_ARG, "lambda_nm must be positive");
  if (o->spp < 1) return fail(SDD_ERR_ARG, "spp must be >= 1");
  if (o->mode != SDD_MODE_DETERMINISTIC && o->mode != SDD_MODE_MONTE_CARLO) return fail(SDD_ERR_ARG, "unknown mode");
  if (o->mode == SDD_MODE_DETERMINISTIC && o->spp != 1) return fail(SDD_ERR_ARG, "deterministic mode needs spp == 1");
  if (o->max_depth < 0 || o->max_depth > 255) return fail(SDD_ERR_ARG, "max_depth must be in [0, 255]");
  if (o->mode == SDD_MODE_DETERMINISTIC && o->max_depth > 10)
    return fail(SDD_ERR_ARG, "deterministic mode supports max_depth <= 10");
  if (o->use_surrogate && !o->surrogate) return fail(SDD_ERR_ARG, "use_surrogate needs opts->surrogate");
  if (!s->tile_mats.empty() && o->mode == SDD_MODE_DETERMINISTIC)
    return fail(SDD_ERR_ARG, "heterogeneous tiles need Monte Carlo mode");
  if (o->n_pixels < 0) return fail(SDD_ERR_ARG, "n_pixels < 0");
  if (o->n_pixels > 0 && !o->pixels) return fail(SDD_ERR_ARG, "pixels is NULL");
  const long long img = (long long)cam->width * cam->height;
  for (int i = 0; i < o->n_pixels; ++i)
    if (o->pixels[i] < 0 || o->pixels[i] >= img) return fail(SDD_ERR_ARG, "pixel index out of range");
  if (o->batched < 0 || o->batched > 2) return fail(SDD_ERR_ARG, "batched must be 0, 1 or 2");
  if (o->batched != 0 && s->strm.cap > 0)
    return fail(SDD_ERR_STATE, "out-of-core subdomains (resident_subdomains > 0) need the host-driven form (batched = 0)");
  if (o->bundle < 0 || o->bundle > kMaxBundle) return fail(SDD_ERR_ARG, "bundle must be in [0, 64]");
  if (const sdd_photon_maps* pm = o->photon_maps) {
    if (o->mode != SDD_MODE_MONTE_CARLO) return fail(SDD_ERR_ARG, "photon maps need Monte Carlo mode");
    if (o->batched == 1) return fail(SDD_ERR_ARG, "photon maps need the host-driven or the graph form (batched = 0 or 2)");
    if (o->use_surrogate) return fail(SDD_ERR_ARG, "photon maps need use_surrogate = 0");
    if (pm->lambda != std::vector<float>(o->lambda_nm, o->lambda_nm + o->n_lambda))
      return fail(SDD_ERR_ARG, "photon maps were built for another wavelength list");
  }
  const int B = o->bundle > 1 ? o->bundle : 1;
  if (B > 1 && o->mode != SDD_MODE_MONTE_CARLO) return fail(SDD_ERR_ARG, "spectral bundles need Monte Carlo mode");
  const int L = o->n_lambda;
  const int n_bundles = (L + B - 1) / B;
  const long long n_px = o->n_pixels > 0 ? o->n_pixels : img;
  if (n_px * L > 0x7FFFFFFFLL) return fail(SDD_ERR_ARG, "pixels x wavelengths exceeds 2^31");
  // cells of the wave partition: (pixel, wavelength), or (pixel, bundle) with bundles
  const long long n_cells = n_px * n_bundles;

  sdd_status r = prepare_spectral(s, L, o->lambda_nm, st);
  if (r) return r;
  r = ensure_ctl(s);
  if (r) return r;

  // waves
  const bool det = o->mode == SDD_MODE_DETERMINISTIC;
  // default: 2^26 paths per wave, 2^25 with bundles (each carrying up to B wavelengths)
  long long wmax = o->wave_paths > 0 ? o->wave_paths
                                     : (s->tuning.wave_paths > 0 ? s->tuning.wave_paths : (B > 1 ? 1LL << 25 : 1LL << 26));
  wmax = std::min<long long>(wmax, 1LL << 28);
  // the network form queues one entry per member of every tile hit: 2 x wave x B of them
  if (o->use_surrogate && B > 1 && o->wave_paths <= 0 && s->tuning.wave_paths <= 0)
    wmax = std::min<long long>(wmax, 0x7FFFFFFFLL / (2LL * B));
  std::vector<WaveDesc> waves;
  if (n_cells <= wmax) {
    uint32_t ns_per = (uint32_t)std::max<long long>(1, wmax / n_cells);
    for (uint32_t s0 = 0; s0 < (uint32_t)o->spp; s0 += ns_per) {
      WaveDesc w;
      w.s0 = s0;
      w.ns = std::min<uint32_t>(ns_per, (uint32_t)o->spp - s0);
      w.c0 = 0;
      w.nc = (uint32_t)n_cells;
      w.n_paths = w.ns * w.nc;
      waves.push_back(w);
    }
  } else {
    for (uint32_t s0 = 0; s0 < (uint32_t)o->spp; ++s0)
      for (long long c0 = 0; c0 < n_cells; c0 += wmax) {
        WaveDesc w;
        w.s0 = s0;
        w.ns = 1;
        w.c0 = (uint32_t)c0;
        w.nc = (uint32_t)std::min<long long>(wmax, n_cells - c0);
        w.n_paths = w.nc;
        waves.push_back(w);
      }
  }
  size_t wave_paths = 0;
  for (auto& w : waves) wave_paths = std::max<size_t>(wave_paths, w.n_paths);
  // contribution slots per path: the deterministic tree's leaves, or one per bundle member
  const int n_slots = det ? (1 << (o->max_depth + 1)) : B;
  // rays of one generation: a Monte Carlo path has one ray; a bundle has one per group of
  // members that agree, queued for twice the paths (a wave that needs more is split, below)
  const size_t cap = det ? wave_paths * 4 : wave_paths * (size_t)(B > 1 ? 2 : 1);
  const bool want_hash = o->path_hash_out != nullptr;
  r = ensure_workspace(s, cap, wave_paths, n_slots, want_hash, B);
  if (r) return r;
  CK(s->film.ensure((size_t)(n_px * L)));
  CK(cudaMemsetAsync(s->film.p, 0, sizeof(double) * n_px * L, st));
  if (o->n_pixels > 0) {
    CK(s->pixel_list.ensure(o->n_pixels));
    CK(cudaMemcpyAsync(s->pixel_list.p, o->pixels, sizeof(int32_t) * o->n_pixels, cudaMemcpyHostToDevice, st));
  }

  RenderParams p = scene_params(s, L);
  p.cam = make_camera(cam);
  p.pixel_list = o->n_pixels > 0 ? s->pixel_list.p : nullptr;
  p.n_px = (int)n_px;
  p.spp = o->spp;
  p.seed = o->seed;
  p.max_depth = o->max_depth;
  p.mode = o->mode;
  p.rr_start = o->rr_start_depth;
  p.n_slots = n_slots;
  p.stats = s->profiling;
  p.path_hash = want_hash ? s->path_hash.p : nullptr;
  p.bundle = B;
  p.n_bundles = n_bundles;
  if (!s->tile_mats.empty()) p.use_surrogate = o->use_surrogate ? 1 : 0;
  if (o->photon_maps) {
    p.use_photons = 1;
    p.pm = o->photon_maps->view();
  }
  if (p.use_surrogate) {
    // one entry per tile hit, with bundles one per member (entries ray << 6 | member)
    const size_t tcap = cap * (size_t)B;
    if (B > 1 && cap > (1u << 26)) return fail(SDD_ERR_ARG, "wave too large for spectral bundles with the network");
    if (tcap > 0x7FFFFFFFu) return fail(SDD_ERR_ARG, "wave too large for the tile queue");
    CK(s->tile_queue.ensure(tcap));
    p.tile_queue = s->tile_queue.p;
    p.tile_count = &s->d_ctl->tile_hits;
    p.tile_cap = (int)tcap;
    // network transmittance toward the sun per tile material and wavelength
    sdd_surrogate* net = const_cast<sdd_surrogate*>(o->surrogate);
    const int nm = (int)s->tile_mats.size();
    if (s->sun_T_net != net || s->sun_T_version != surrogate_version(net)) {
      CK(s->sun_T.ensure(s->mats.size() * (size_t)L));
      CK(cudaMemsetAsync(s->sun_T.p, 0, sizeof(float) * s->mats.size() * L, st));
      DevArr<float> raw, pred;
      CK(raw.ensure((size_t)nm * L * 7));
      CK(pred.ensure((size_t)nm * L * kHeadPred));
      launch_sun_queries(p, s->t_tile_mats.p, s->t_tile_normal.p, nm, raw.p, st);
      CK(surrogate_predict(net, nm * L, raw.p, pred.p, st));
      launch_sun_table(s->t_tile_mats.p, nm, L, pred.p, s->sun_T.p, st);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(st));
      raw.release();
      pred.release();
      s->sun_T_net = net;
      s->sun_T_version = surrogate_version(net);
    }
    p.tile_sun_T = s->sun_T.p;
  }

  s->stats = sdd_stats{};
  // queue capacity seen by the kernels (every append is checked against it); the buffers
  // above keep the automatic size
  const int qcap = (int)(s->tuning.queue_capacity > 0 ? std::min<size_t>(cap, (size_t)s->tuning.queue_capacity) : cap);
  if (o->batched) {
    // A frame whose rays outgrew the queues is rendered again with every wave halved (see the
    // host-driven form below); the frame's film is cleared at its start.
    std::vector<WaveDesc> bw = waves;
    for (int attempt = 0;; ++attempt) {
      r = render_batched(s, p, bw, n_slots, qcap, o, spectral_out, xyz_out, st);
      if (r) return r;
      r = read_ctl(s, s->gstream);
      if (r) return r;
      const uint32_t e = s->h_ctl->error;
      const bool overflow = (e & (ERR_QUEUE_OVERFLOW | ERR_SHADOW_OVERFLOW)) != 0u && !(e & ~(ERR_QUEUE_OVERFLOW | ERR_SHADOW_OVERFLOW));
      bool splittable = false;
      for (const WaveDesc& w : bw) splittable = splittable || w.ns > 1 || w.nc > 1;
      if (overflow && s->tuning.queue_capacity == 0 && attempt < 12 && splittable) {
        bw = halve_waves(bw);
        s->stats.wave_splits++;
        continue;
      }
      if (e) return device_error(e);
      break;
    }
    for (const WaveDesc& w : bw) {
      s->stats.waves++;
      s->stats.paths += spectral_paths(p, w);
    }
    // graph form: passes run by the conditional loops, and their condition launches
    const int64_t gp0 = (int64_t)s->h_ctl->graph_passes[0], gp1 = (int64_t)s->h_ctl->graph_passes[1];
    s->stats.launches_traverse += gp0;
    s->stats.launches_shadow += gp1;
    s->stats.launches_total += gp0 + gp1 + (gp0 + gp1) / 2;
    s->stats.node_visits = (int64_t)s->h_ctl->node_visits;
    s->stats.tri_tests = (int64_t)s->h_ctl->tri_tests;
    s->stats.shadow_node_visits = (int64_t)s->h_ctl->shadow_node_visits;
    s->stats.shadow_tri_tests = (int64_t)s->h_ctl->shadow_tri_tests;
    s->stats.rays_closest = (int64_t)s->h_ctl->rays_closest;
    s->stats.rays_shadow = (int64_t)s->h_ctl->rays_shadow;
    s->stats.crossings = (int64_t)s->h_ctl->crossings;
    s->stats.tile_shaded = (int64_t)s->h_ctl->tile_shaded;
    s->stats.bytes_ray_state = s->stats.rays_closest * 44 + s->stats.rays_shadow * 44;
    s->stats.ms_total = s->stats.ms_persistent;
    return SDD_OK;
  }
  CK(cudaMemsetAsync(s->d_ctl, 0, sizeof(Control), st));
  auto run_wave = [&](const WaveDesc& w) -> sdd_status {
    CK(cudaMemsetAsync(s->d_ctl, 0, offsetof(Control, node_visits), st));
    CK(cudaMemsetAsync(s->path_L.p, 0, sizeof(float) * (size_t)w.n_paths * n_slots, st));
    int cur = 0;
    RayBuf rb0{s->rb_o[0].p, s->rb_d[0].p, s->rb_info[0].p, qcap, s->rb_w[0].p, s->rb_m[0].p};
    int ev = s->ev_begin(TK_RAYGEN, st);
    launch_raygen(p, w, rb0, s->q[0].p, s->d_ctl->q_count[0], qcap, s->d_ctl, st);
    s->ev_end(ev, st);
    CK(cudaGetLastError());
    count_launch(s, TK_RAYGEN);
    int n_rays = (int)w.n_paths;
    for (int gen = 0; n_rays > 0; ++gen) {
      if (gen > o->max_depth + 1) return fail(SDD_ERR_TIMEOUT, "generation count exceeded max_depth + 1");
      RayBuf rc{s->rb_o[cur].p, s->rb_d[cur].p, s->rb_info[cur].p, qcap, s->rb_w[cur].p, s->rb_m[cur].p};
      RayBuf rn{s->rb_o[1 - cur].p, s->rb_d[1 - cur].p, s->rb_info[1 - cur].p, qcap, s->rb_w[1 - cur].p,
                s->rb_m[1 - cur].p};
      r = run_closest_passes(s, p, rc, qcap, st);
      if (r) return r;
      // the closest passes left every count at zero; shade refills q[0] and sq[0]
      CK(cudaMemsetAsync(s->d_ctl, 0, offsetof(Control, error), st));
      CK(cudaMemsetAsync(&s->d_ctl->tile_hits, 0, sizeof(int), st));
      ShadowBuf sb{s->sb_o.p, s->sb_d.p, s->sb_info.p, qcap, s->sb_c.p, s->sb_m.p};
      ev = s->ev_begin(TK_SHADE, st);
      launch_shade(p, w, n_rays, rc, s->hits.p, rn, s->q[0].p, s->d_ctl->q_count[0], qcap, sb, s->sq[0].p,
                   s->d_ctl->sq_count[0], s->path_L.p, s->d_ctl, st);
      s->ev_end(ev, st);
      CK(cudaGetLastError());
      count_launch(s, TK_SHADE);
      if (p.use_surrogate) {
        // the generation's tile hits: inputs, network and exit sampling in one launch
        ev = s->ev_begin(TK_TILE, st);
        CK(launch_tile_shade(p, w, rc, s->hits.p, rn, &s->d_ctl->next_rays, s->q[0].p, s->d_ctl->q_count[0], qcap,
                             s->d_ctl, o->surrogate, st));
        s->ev_end(ev, st);
        count_launch(s, TK_TILE);
      }
      r = run_shadow_passes(s, p, w, qcap, st);
      if (r) return r;
      n_rays = s->h_ctl->next_rays;
      if (n_rays > qcap) return fail(SDD_ERR_QUEUE_OVERFLOW, "ray queue capacity exceeded");
      cur = 1 - cur;
    }
    float* prad = o->path_radiance_out;
    ev = s->ev_begin(TK_FILM, st);
    launch_film_accum(p, w, s->path_L.p, s->film.p, prad, o->path_hash_out, st);
    s->ev_end(ev, st);
    CK(cudaGetLastError());
    count_launch(s, TK_FILM);
    s->stats.waves++;
    s->stats.paths += spectral_paths(p, w);
    return SDD_OK;
  };
  // A wave whose rays outgrow the queues (spectral bundles split into more rays than they
  // have paths only where their members' branches differ, so their queues are sized for twice
  // the paths) is abandoned before its film accumulation and rendered again as two halves:
  // per cell the samples are still accumulated in order, so the image is the same.
  std::vector<std::pair<WaveDesc, int>> work;
  for (auto it = waves.rbegin(); it != waves.rend(); ++it) work.push_back({*it, 0});
  while (!work.empty()) {
    const WaveDesc w = work.back().first;
    const int depth = work.back().second;
    work.pop_back();
    r = run_wave(w);
    if (r == SDD_OK) continue;
    const bool can_split = r == SDD_ERR_QUEUE_OVERFLOW && s->tuning.queue_capacity == 0 && depth < 24 &&
                           (w.ns > 1 || w.nc > 1);
    if (!can_split) return r;
    s->stats.wave_splits++;
    const std::vector<WaveDesc> halves = halve_waves({w});
    for (auto it = halves.rbegin(); it != halves.rend(); ++it) work.push_back({*it, depth + 1});
  }
  int ev = s->ev_begin(TK_FILM, st);
  launch_film_finalize(p, s->film.p, s->cmf_w.p, spectral_out, xyz_out, st);
  s->ev_end(ev, st);
  CK(cudaGetLastError());
  count_launch(s, TK_FILM);
  r = read_ctl(s, st);
  if (r) return r;
  if (s->h_ctl->error) return device_error(s->h_ctl->error);
  s->stats.node_visits = (int64_t)s->h_ctl->node_visits;
  s->stats.tri_tests = (int64_t)s->h_ctl->tri_tests;
  s->stats.shadow_node_visits = (int64_t)s->h_ctl->shadow_node_visits;
  s->stats.shadow_tri_tests = (int64_t)s->h_ctl->shadow_tri_tests;
  s->stats.rays_closest = (int64_t)s->h_ctl->rays_closest;
  s->stats.rays_shadow = (int64_t)s->h_ctl->rays_shadow;
  s->stats.crossings = (int64_t)s->h_ctl->crossings;
  s->stats.tile_shaded = (int64_t)s->h_ctl->tile_shaded;
  // traversal ray-state traffic: per closest visit read queue index 4 B + origin/direction
  // 32 B, write hit 8 B or hand-off 4 B; per shadow visit read 4 + 32 + 8 B.
  s->stats.bytes_ray_state = s->stats.rays_closest * 44 + s->stats.rays_shadow * 44;
  s->ev_collect();
  s->stats.ms_total = s->stats.ms_raygen + s->stats.ms_traverse + s->stats.ms_shade + s->stats.ms_shadow +
                      s->stats.ms_film + s->stats.ms_tile;
  return SDD_OK;
}

// ------------------------------------------------------------------ photon maps (Sec. 3.2)
constexpr int64_t kMaxMapPhotons = 1LL << 30;

// Trace every photon and append the stored ones to the maps' buffers (capacity cap per map);
// *need receives each map's count, or an estimate of it when the tracing stopped early
// because a buffer was full.
sdd_status photon_trace(sdd_scene* s, const RenderParams& p, PhotonEmit pe, int64_t total, int max_depth,
                        sdd_photon_maps* m, int* d_count, int64_t cap, int64_t need[2], cudaStream_t st) {
  // one ray per photon; waves small enough that a wave's stores cannot overflow the counters
  const int W = (int)std::min<int64_t>({total, 1LL << 24, (1LL << 29) / std::max(max_depth, 1)});
  sdd_status r = ensure_workspace(s, (size_t)W, 1, 1, false, 1);
  if (r) return r;
  PhotonStore ps{};
  for (int k = 0; k < 2; ++k) {
    ps.pos_pw[k] = m->raw_pos[k].p;
    ps.nrm_lam[k] = m->raw_nrm[k].p;
    ps.id_seq[k] = m->raw_id[k].p;
  }
  ps.count = d_count;
  ps.cap = (int)cap;
  CK(cudaMemsetAsync(d_count, 0, 2 * sizeof(int), st));
  for (int64_t j0 = 0; j0 < total; j0 += W) {
    const int n = (int)std::min<int64_t>(W, total - j0);
    pe.j0 = (uint32_t)j0;
    CK(cudaMemsetAsync(s->d_ctl, 0, sizeof(Control), st));
    RayBuf rb0{s->rb_o[0].p, s->rb_d[0].p, s->rb_info[0].p, W, nullptr};
    launch_photon_emit(p, pe, n, rb0, s->q[0].p, s->d_ctl->q_count[0], W, s->d_ctl, st);
    CK(cudaGetLastError());
    int cur = 0, n_rays = n;
    for (int gen = 0; n_rays > 0; ++gen) {
      if (gen > max_depth + 1) return fail(SDD_ERR_TIMEOUT, "photon generations exceeded max_depth + 1");
      RayBuf rc{s->rb_o[cur].p, s->rb_d[cur].p, s->rb_info[cur].p, W, nullptr};
      RayBuf rn{s->rb_o[1 - cur].p, s->rb_d[1 - cur].p, s->rb_info[1 - cur].p, W, nullptr};
      r = run_closest_passes(s, p, rc, W, st);
      if (r) return r;
      CK(cudaMemsetAsync(s->d_ctl, 0, offsetof(Control, error), st));
      launch_photon_shade(p, pe, n_rays, rc, s->hits.p, rn, &s->d_ctl->next_rays, s->q[0].p, s->d_ctl->q_count[0], W,
                          ps, s->d_ctl, st);
      CK(cudaGetLastError());
      r = read_ctl(s, st);
      if (r) return r;
      if (s->h_ctl->error) return device_error(s->h_ctl->error);
      n_rays = s->h_ctl->next_rays;
      if (n_rays > W) return fail(SDD_ERR_QUEUE_OVERFLOW, "photon ray buffer exceeded");
      cur = 1 - cur;
    }
    int c[2];
    CK(cudaMemcpyAsync(c, d_count, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t done = j0 + n;
    for (int k = 0; k < 2; ++k) need[k] = c[k];
    if (c[0] > cap || c[1] > cap) {  // stop: project the counts over all photons
      for (int k = 0; k < 2; ++k)
        need[k] = std::min<int64_t>(kMaxMapPhotons + 1, (int64_t)((double)c[k] * (double)total / (double)done * 1.1) + 1024);
      return SDD_OK;
    }
  }
  return SDD_OK;
}

sdd_status photon_build(sdd_scene* s, const sdd_photon_opts* o, sdd_photon_maps* m, cudaStream_t st) {
  const int L = o->n_lambda;
  sdd_status r = prepare_spectral(s, L, o->lambda_nm, st);
  if (r) return r;
  r = ensure_ctl(s);
  if (r) return r;
  RenderParams p = scene_params(s, L);
  p.seed = o->seed;
  p.max_depth = o->max_depth;
  p.mode = SDD_MODE_MONTE_CARLO;
  PhotonEmit pe{};
  {
    double sd[3] = {s->sun_dir[0], s->sun_dir[1], s->sun_dir[2]};
    const double l = std::sqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
    pe.origin = make_float3((float)(o->center[0] + o->distance_m * sd[0] / l),
                            (float)(o->center[1] + o->distance_m * sd[1] / l),
                            (float)(o->center[2] + o->distance_m * sd[2] / l));
    const double h = 2.0 * std::sin(0.5 * s->sun_half) * std::sin(0.5 * s->sun_half);
    const double R = o->radius_m;
    pe.radius = o->radius_m;
    pe.power_scale = (float)(2.0 * M_PI * h * M_PI * R * R / o->n_per_lambda);
    pe.n_per_lambda = o->n_per_lambda;
  }
  const int64_t total = (int64_t)L * o->n_per_lambda;
  DevArr<int> d_count;
  CK(d_count.ensure(2));
  int64_t cap = std::min<int64_t>(std::max<int64_t>(total, 1024), kMaxMapPhotons);
  int64_t need[2] = {0, 0};
  for (int attempt = 0;; ++attempt) {
    for (int k = 0; k < 2; ++k) {
      CK(m->raw_pos[k].ensure((size_t)cap));
      CK(m->raw_nrm[k].ensure((size_t)cap));
      CK(m->raw_id[k].ensure((size_t)cap));
    }
    r = photon_trace(s, p, pe, total, o->max_depth, m, d_count.p, cap, need, st);
    if (r) return r;
    if (need[0] <= cap && need[1] <= cap) break;
    if (need[0] > kMaxMapPhotons || need[1] > kMaxMapPhotons || attempt >= 4)
      return fail(SDD_ERR_QUEUE_OVERFLOW, "a photon map would hold more than 2^30 photons");
    cap = std::min<int64_t>(std::max(need[0], need[1]), kMaxMapPhotons);
  }
  // hashed grids of cell edge 2 r, one table size for both maps
  m->count[0] = need[0];
  m->count[1] = need[1];
  m->radius = o->gather_radius_m;
  m->inv_cell = 1.f / (2.f * o->gather_radius_m);
  int64_t T = 1024;
  while (T < 2 * std::max(need[0], need[1]) && T < (1LL << 27)) T <<= 1;
  m->mask = (uint32_t)(T - 1);
  DevArr<uint32_t> scratch;
  CK(scratch.ensure((size_t)(T + T / 1024)));
  for (int k = 0; k < 2; ++k) {
    CK(m->start[k].ensure((size_t)T + 1));
    CK(m->pos[k].ensure((size_t)need[k]));
    CK(m->nrm[k].ensure((size_t)need[k]));
    CK(build_photon_grid((int)need[k], m->raw_pos[k].p, m->raw_nrm[k].p, m->inv_cell, m->mask, m->start[k].p,
                         scratch.p, m->pos[k].p, m->nrm[k].p, st));
  }
  CK(cudaStreamSynchronize(st));
  scratch.release();
  d_count.release();
  m->lambda.assign(o->lambda_nm, o->lambda_nm + L);
  return SDD_OK;
}

// The geometry checks of a scene description (vertices, indices, subdomain count, axis).
sdd_status validate_geometry(const sdd_scene_desc* d) {
  if (d->n_vertices < 3 || !d->vertices) return fail(SDD_ERR_ARG, "need >= 3 vertices");
  if (d->n_triangles < 1 || !d->indices) return fail(SDD_ERR_ARG, "need >= 1 triangle");
  if (d->n_triangles > (1 << 28)) return fail(SDD_ERR_ARG, "too many triangles");
  if (d->n_subdomains < 1 || d->n_subdomains > kMaxSubdomains) return fail(SDD_ERR_ARG, "n_subdomains must be 1..64");
  if (d->split_axis < -1 || d->split_axis > 2) return fail(SDD_ERR_ARG, "split_axis must be -1, 0, 1 or 2");
  for (long long i = 0; i < 3LL * d->n_vertices; ++i)
    if (!std::isfinite(d->vertices[i])) return fail(SDD_ERR_ARG, "non-finite vertex coordinate");
  for (long long i = 0; i < 3LL * d->n_triangles; ++i)
    if (d->indices[i] >= (uint32_t)d->n_vertices) return fail(SDD_ERR_ARG, "triangle index out of range");
  return SDD_OK;
}

// The split of a validated description (Sec. 5): the scene box, the split axis (the longest
// unless given), S slabs of equal length along it (the outer two open), the ray epsilon
// (*eps) and the slop by which a triangle's slab overlap is widened.
BuildInput split_input(const sdd_scene_desc* d, float* eps) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, amax = 0.0;
  for (int i = 0; i < d->n_vertices; ++i)
    for (int a = 0; a < 3; ++a) {
      double x = d->vertices[3 * i + a];
      lo[a] = std::min(lo[a], x);
      hi[a] = std::max(hi[a], x);
      amax = std::max(amax, std::fabs(x));
    }
  int axis = d->split_axis;
  if (axis < 0) axis = (hi[0] - lo[0] >= hi[1] - lo[1] && hi[0] - lo[0] >= hi[2] - lo[2]) ? 0
                       : (hi[1] - lo[1] >= hi[2] - lo[2] ? 1 : 2);
  *eps = d->ray_epsilon_m > 0.f ? d->ray_epsilon_m : (float)std::max(1e-5, 2e-6 * amax);
  BuildInput in;
  in.verts = d->vertices;
  in.idx = d->indices;
  in.n_tris = d->n_triangles;
  in.n_sub = d->n_subdomains;
  in.axis = axis;
  in.slop = (float)std::max<double>(*eps, 1e-6 * amax);
  for (int i = 0; i <= in.n_sub; ++i) {
    if (i == 0) in.planes[i] = -INFINITY;
    else if (i == in.n_sub) in.planes[i] = INFINITY;
    else in.planes[i] = (float)(lo[axis] + (hi[axis] - lo[axis]) * i / in.n_sub);
  }
  return in;
}

}  // namespace

extern "C" {

const char* sdd_last_error(void) { return g_err.c_str(); }
const char* sdd_version(void) { return "sdd 0.1 (sm_103a)"; }

sdd_status sdd_scene_create(const sdd_scene_desc* d, sdd_scene** out) {
  g_err.clear();
  if (!d || !out) return fail(SDD_ERR_ARG, "NULL desc or out");
  *out = nullptr;
  if (sdd_status r = validate_geometry(d)) return r;
  if (!d->material_of_triangle) return fail(SDD_ERR_ARG, "need >= 1 triangle");
  if (d->n_materials < 1 || !d->materials) return fail(SDD_ERR_ARG, "need >= 1 material");
  for (int t = 0; t < d->n_triangles; ++t)
    if (d->material_of_triangle[t] >= d->n_materials) return fail(SDD_ERR_ARG, "material index out of range");
  sdd_scene* s = new (std::nothrow) sdd_scene;
  if (!s) return fail(SDD_ERR_OOM, "host allocation failed");
  for (int m = 0; m < d->n_materials; ++m) {
    const sdd_material& sm = d->materials[m];
    if (sm.kind < 0 || sm.kind > 4) {
      delete s;
      return fail(SDD_ERR_ARG, "material " + std::to_string(m) + ": unknown kind");
    }
    if (sm.kind == SDD_MAT_HETERO_TILE &&
        (!d->tiles || sm.tile_param_id < 0 || sm.tile_param_id >= tileset_device_view(d->tiles)->n_tiles)) {
      delete s;
      return fail(SDD_ERR_ARG, "material " + std::to_string(m) + ": HETERO_TILE needs desc->tiles and a tile_param_id in range");
    }
    bool glass = sm.kind == SDD_MAT_DIELECTRIC_SOLID || sm.kind == SDD_MAT_THIN_SLAB || sm.kind == SDD_MAT_HETERO_TILE;
    sdd_status v = validate_table("material n", sm.n_lambda, sm.lambda_nm, sm.n, glass);
    if (!v) v = validate_table("material k", sm.n_lambda, sm.lambda_nm, sm.k, glass);
    if (!v) v = validate_table("material albedo", sm.n_lambda, sm.lambda_nm, sm.albedo, sm.kind == SDD_MAT_DIFFUSE);
    if (v) {
      delete s;
      return fail(v, "material " + std::to_string(m) + ": " + g_err);
    }
    HostMaterial hm;
    hm.kind = sm.kind;
    hm.lam.assign(sm.lambda_nm, sm.lambda_nm + sm.n_lambda);
    if (sm.n) hm.n.assign(sm.n, sm.n + sm.n_lambda);
    if (sm.k) hm.k.assign(sm.k, sm.k + sm.n_lambda);
    if (sm.albedo) hm.albedo.assign(sm.albedo, sm.albedo + sm.n_lambda);
    if (glass) {
      for (float x : hm.n)
        if (!(x >= 1.0f)) {
          delete s;
          return fail(SDD_ERR_ARG, "material " + std::to_string(m) + ": glass index n must be >= 1");
        }
      for (float x : hm.k)
        if (!(x >= 0.f)) {
          delete s;
          return fail(SDD_ERR_ARG, "material " + std::to_string(m) + ": k must be >= 0");
        }
    }
    if (sm.kind == SDD_MAT_THIN_SLAB && !(sm.thickness_m > 0.f)) {
      delete s;
      return fail(SDD_ERR_ARG, "material " + std::to_string(m) + ": thin slab needs thickness_m > 0");
    }
    hm.thick = sm.thickness_m;
    hm.tile_id = sm.tile_param_id;
    s->mats.push_back(hm);
    s->mat_tile.push_back(sm.kind == SDD_MAT_HETERO_TILE ? sm.tile_param_id : -1);
    if (sm.kind == SDD_MAT_HETERO_TILE) s->tile_mats.push_back(m);
  }
  const sdd_illuminant& il = d->illum;
  sdd_status v = validate_table("sky_radiance", il.n_lambda, il.lambda_nm, il.sky_radiance, true);
  if (!v && il.sun_radiance) v = validate_table("sun_radiance", il.n_lambda, il.lambda_nm, il.sun_radiance, true);
  if (v) {
    delete s;
    return v;
  }
  s->il_lam.assign(il.lambda_nm, il.lambda_nm + il.n_lambda);
  s->il_sky.assign(il.sky_radiance, il.sky_radiance + il.n_lambda);
  if (il.sun_radiance && il.sun_half_angle_rad > 0.f) s->il_sun.assign(il.sun_radiance, il.sun_radiance + il.n_lambda);
  s->sky_mode = il.sky_mode;
  double sl = std::sqrt((double)il.sun_dir[0] * il.sun_dir[0] + (double)il.sun_dir[1] * il.sun_dir[1] +
                        (double)il.sun_dir[2] * il.sun_dir[2]);
  if (!s->il_sun.empty() && !(sl > 0.0)) {
    delete s;
    return fail(SDD_ERR_ARG, "sun_dir must be non-zero");
  }
  for (int i = 0; i < 3; ++i) s->sun_dir[i] = il.sun_dir[i];
  s->sun_half = il.sun_half_angle_rad;

  if (d->slab_polarisation != 0 && d->slab_polarisation != 1) {
    delete s;
    return fail(SDD_ERR_ARG, "slab_polarisation must be 0 or 1");
  }
  s->slab_pol = d->slab_polarisation;
  const BuildInput in = split_input(d, &s->eps);
  const int axis = in.axis;
  HostBVH bvh;
  try {
    build_scene_bvh(in, bvh);
  } catch (const std::bad_alloc&) {
    delete s;
    return fail(SDD_ERR_OOM, "host allocation failed during BVH build");
  }
  if (bvh.stack_need > kStackSize) {
    delete s;
    return fail(SDD_ERR_ARG, "BVH too deep for the traversal stack");
  }
  // per-primitive normal + material
  std::vector<float4> prim(d->n_triangles);
  for (int t = 0; t < d->n_triangles; ++t) {
    const float* a = d->vertices + 3 * d->indices[3 * t];
    const float* b = d->vertices + 3 * d->indices[3 * t + 1];
    const float* c = d->vertices + 3 * d->indices[3 * t + 2];
    double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
    double e2[3] = {(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(l > 0.0)) l = 1.0;  // degenerate triangle: never hit by the watertight test
    float mf;
    int mi = d->material_of_triangle[t];
    std::memcpy(&mf, &mi, 4);
    prim[t] = make_float4((float)(n[0] / l), (float)(n[1] / l), (float)(n[2] / l), mf);
  }
  s->tiles = d->tiles;
  s->tile_mat_normal.assign(s->tile_mats.size(), make_float3(0.f, 0.f, 1.f));
  {
    std::vector<int> first(d->n_materials, -1);
    for (int t = d->n_triangles - 1; t >= 0; --t) first[d->material_of_triangle[t]] = t;
    for (size_t j = 0; j < s->tile_mats.size(); ++j) {
      int t = first[s->tile_mats[j]];
      if (t >= 0) s->tile_mat_normal[j] = make_float3(prim[t].x, prim[t].y, prim[t].z);
    }
  }
  s->n_tris = d->n_triangles;
  s->n_sub = d->n_subdomains;
  s->axis = axis;
  s->bvh_max_depth = bvh.max_depth;
  s->n_refs = bvh.n_refs;
  s->n_nodes = (int64_t)bvh.nodes.size();
  s->n_tri_recs = (int64_t)bvh.tris.size();
  cudaError_t e;
  if ((e = s->nodes.ensure(bvh.nodes.size())) != cudaSuccess ||
      (e = s->tris.ensure(std::max<size_t>(1, bvh.tris.size()))) != cudaSuccess ||
      (e = s->prim.ensure(prim.size())) != cudaSuccess) {
    delete s;
    return fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(s->nodes.p, bvh.nodes.data(), sizeof(Node) * bvh.nodes.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(s->tris.p, bvh.tris.data(), sizeof(TriRec) * bvh.tris.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(s->prim.p, prim.data(), sizeof(float4) * prim.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete s;
    return fail(SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  DevScene& ds = s->dev;
  ds.nodes = s->nodes.p;
  ds.tris = s->tris.p;
  ds.prim_nrm_mat = s->prim.p;
  ds.n_prims = d->n_triangles;
  ds.n_sub = in.n_sub;
  ds.axis = axis;
  for (int i = 0; i <= in.n_sub; ++i) ds.planes[i] = in.planes[i];
  for (int i = in.n_sub + 1; i <= kMaxSubdomains; ++i) ds.planes[i] = INFINITY;
  for (int i = 0; i < in.n_sub; ++i) {
    ds.root[i] = bvh.root[i];
    ds.n_nodes_sub[i] = bvh.n_nodes[i];
  }
  ds.eps = s->eps;
  *out = s;
  return SDD_OK;
}

void sdd_scene_destroy(sdd_scene* s) { delete s; }

sdd_status sdd_scene_get_info(const sdd_scene* s, sdd_scene_info* out) {
  if (!s || !out) return fail(SDD_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->n_triangles = s->n_tris;
  out->n_subdomains = s->n_sub;
  out->split_axis = s->axis;
  out->bvh_max_depth = s->bvh_max_depth;
  out->n_tri_refs = s->n_refs;
  out->n_nodes = s->n_nodes;
  out->device_bytes = (int64_t)(s->nodes.n * sizeof(Node) + s->tris.n * sizeof(TriRec) + s->prim.n * sizeof(float4));
  for (int i = 0; i <= s->n_sub; ++i) out->planes[i] = s->dev.planes[i];
  return SDD_OK;
}

sdd_status sdd_bvh_build_host(const sdd_scene_desc* d, sdd_bvh_info* info, void* nodes, int64_t nodes_cap,
                              void* tris, int64_t tris_cap, int32_t* root, int32_t* n_nodes_sub, float* planes) {
  g_err.clear();
  if (!d || !info) return fail(SDD_ERR_ARG, "NULL desc or info");
  if (sdd_status r = validate_geometry(d)) return r;
  float eps = 0.f;
  const BuildInput in = split_input(d, &eps);
  HostBVH bvh;
  try {
    build_scene_bvh(in, bvh);
  } catch (const std::bad_alloc&) {
    return fail(SDD_ERR_OOM, "host allocation failed during BVH build");
  }
  info->n_subdomains = in.n_sub;
  info->split_axis = in.axis;
  info->bvh_max_depth = bvh.max_depth;
  info->stack_need = bvh.stack_need;
  info->n_nodes = (int64_t)bvh.nodes.size();
  info->n_tri_records = (int64_t)bvh.tris.size();
  info->slop = in.slop;
  if (nodes) {
    if (nodes_cap < info->n_nodes) return fail(SDD_ERR_ARG, "nodes buffer too small");
    std::memcpy(nodes, bvh.nodes.data(), sizeof(Node) * bvh.nodes.size());
  }
  if (tris) {
    if (tris_cap < info->n_tri_records) return fail(SDD_ERR_ARG, "tris buffer too small");
    std::memcpy(tris, bvh.tris.data(), sizeof(TriRec) * bvh.tris.size());
  }
  for (int k = 0; k < in.n_sub; ++k) {
    if (root) root[k] = bvh.root[k];
    if (n_nodes_sub) n_nodes_sub[k] = bvh.n_nodes[k];
  }
  if (planes)
    for (int k = 0; k <= in.n_sub; ++k) planes[k] = in.planes[k];
  return SDD_OK;
}

sdd_status sdd_render(sdd_scene* scene, const sdd_camera* cam, const sdd_render_opts* opts, float* spectral_out,
                      float* xyz_out, void* stream) {
  g_err.clear();
  if (!spectral_out && !xyz_out) return fail(SDD_ERR_ARG, "spectral_out and xyz_out are both NULL");
  return render_impl(scene, cam, opts, spectral_out, xyz_out, (cudaStream_t)stream);
}

sdd_status sdd_render_to_host(sdd_scene* s, const sdd_camera* cam, const sdd_render_opts* o, float* spec_host,
                              float* xyz_host, void* stream) {
  g_err.clear();
  if (!s || !cam || !o) return fail(SDD_ERR_ARG, "NULL scene, camera or options");
  if (!spec_host && !xyz_host) return fail(SDD_ERR_ARG, "spectral_out and xyz_out are both NULL");
  cudaStream_t st = (cudaStream_t)stream;
  long long n_px = o->n_pixels > 0 ? o->n_pixels : (long long)cam->width * cam->height;
  size_t ns = (size_t)n_px * std::max(o->n_lambda, 1), nx = (size_t)n_px * 3;
  CK(s->out_spec.ensure(ns));
  CK(s->out_xyz.ensure(nx));
  sdd_status r = render_impl(s, cam, o, spec_host ? s->out_spec.p : nullptr, xyz_host ? s->out_xyz.p : nullptr, st);
  if (r) return r;
  if (spec_host) CK(cudaMemcpyAsync(spec_host, s->out_spec.p, ns * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (xyz_host) CK(cudaMemcpyAsync(xyz_host, s->out_xyz.p, nx * sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

sdd_status sdd_watchdog_selftest(int timeout_ms) {
  if (timeout_ms < 1 || timeout_ms > 10000) return fail(SDD_ERR_ARG, "timeout_ms must be in [1, 10000]");
  PersistCtl* pc = nullptr;
  Control* ctl = nullptr;
  cudaError_t e = cudaMalloc(&pc, sizeof(PersistCtl));
  if (e == cudaSuccess) e = cudaMalloc(&ctl, sizeof(Control));
  if (e == cudaSuccess) e = cudaMemset(pc, 0, sizeof(PersistCtl));
  if (e == cudaSuccess) e = cudaMemset(ctl, 0, sizeof(Control));
  if (e == cudaSuccess) e = barrier_selftest(pc, ctl, timeout_ms);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  Control h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost);
  cudaFree(pc);
  cudaFree(ctl);
  if (e != cudaSuccess) return fail(SDD_ERR_CUDA, cudaGetErrorString(e));
  if (h.error & ERR_TIMEOUT) return fail(SDD_ERR_TIMEOUT, "grid barrier gave up after its time limit");
  return SDD_OK;
}

namespace {
void free_streaming(sdd_scene* s) {
  auto& m = s->strm;
  m.d_nodes.release();
  m.d_tris.release();
  cudaFreeHost(m.h_nodes);
  cudaFreeHost(m.h_tris);
  m.h_nodes = nullptr;
  m.h_tris = nullptr;
  m.cap = 0;
}

// Switch to at most `cap` resident subdomains (0 or >= n_sub: all resident).  Entering keeps
// the BVH in pinned host memory, allocates cap slots and frees the all-resident device copy;
// leaving uploads it again.
sdd_status set_streaming(sdd_scene* s, int cap) {
  auto& m = s->strm;
  if (cap >= s->n_sub) cap = 0;
  if (cap == m.cap) return SDD_OK;
  CK(cudaDeviceSynchronize());  // no render in flight reads the BVH
  if (m.cap > 0) {  // restore the all-resident device copy
    CK(s->nodes.ensure((size_t)m.n_nodes));
    CK(s->tris.ensure((size_t)std::max<int64_t>(1, m.n_tris)));
    CK(cudaMemcpy(s->nodes.p, m.h_nodes, sizeof(Node) * (size_t)m.n_nodes, cudaMemcpyHostToDevice));
    if (m.n_tris > 0) CK(cudaMemcpy(s->tris.p, m.h_tris, sizeof(TriRec) * (size_t)m.n_tris, cudaMemcpyHostToDevice));
    s->dev.nodes = s->nodes.p;
    s->dev.tris = s->tris.p;
    for (int i = 0; i < s->n_sub; ++i) s->dev.root[i] = m.node0[i];
    free_streaming(s);
    s->graph_key.clear();
  }
  if (cap == 0) return SDD_OK;
  m.n_nodes = s->n_nodes;
  m.n_tris = (int64_t)s->n_tri_recs;
  m.node0.assign(s->n_sub, 0);
  m.nnodes.assign(s->n_sub, 0);
  m.tri0.assign(s->n_sub, 0);
  m.ntris.assign(s->n_sub, 0);
  cudaError_t e = cudaMallocHost(&m.h_nodes, sizeof(Node) * (size_t)std::max<int64_t>(1, m.n_nodes));
  if (e == cudaSuccess) e = cudaMallocHost(&m.h_tris, sizeof(TriRec) * (size_t)std::max<int64_t>(1, m.n_tris));
  if (e == cudaSuccess) e = cudaMemcpy(m.h_nodes, s->nodes.p, sizeof(Node) * (size_t)m.n_nodes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && m.n_tris > 0)
    e = cudaMemcpy(m.h_tris, s->tris.p, sizeof(TriRec) * (size_t)m.n_tris, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free_streaming(s);
    return fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  // per subdomain: its nodes (one breadth-first block from its root) and the triangle
  // records its leaves reference
  int max_nodes = 1, max_tris = 1;
  for (int i = 0; i < s->n_sub; ++i) {
    const int n0 = s->dev.root[i], nn = s->dev.n_nodes_sub[i];
    int t0 = INT32_MAX, t1 = 0;
    for (int k = n0; k < n0 + nn; ++k) {
      const int* l = &m.h_nodes[k].link.x;
      const int* c = &m.h_nodes[k].cnt.x;
      for (int w = 0; w < kBvhWidth; ++w)
        if (c[w] > 0) {
          t0 = std::min(t0, l[w]);
          t1 = std::max(t1, l[w] + c[w]);
        }
    }
    if (t0 > t1) t0 = t1 = 0;
    m.node0[i] = n0;
    m.nnodes[i] = nn;
    m.tri0[i] = t0;
    m.ntris[i] = t1 - t0;
    max_nodes = std::max(max_nodes, nn);
    max_tris = std::max(max_tris, t1 - t0);
  }
  m.slot_nodes = max_nodes;
  m.slot_tris = max_tris;
  e = m.d_nodes.ensure((size_t)cap * max_nodes);
  if (e == cudaSuccess) e = m.d_tris.ensure((size_t)cap * max_tris);
  if (e != cudaSuccess) {
    free_streaming(s);
    return fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, cudaGetErrorString(e));
  }
  m.slot_of.assign(s->n_sub, -1);
  m.sub_in_slot.assign(cap, -1);
  m.cap = cap;
  s->nodes.release();  // the device now holds only the slots
  s->tris.release();
  s->dev.nodes = nullptr;
  s->dev.tris = nullptr;
  s->graph_key.clear();
  return SDD_OK;
}
}  // namespace

sdd_status sdd_set_tuning(sdd_scene* s, const sdd_tuning* t) {
  if (!s || !t) return fail(SDD_ERR_ARG, "NULL argument");
  if (t->traverse_block != 64 && t->traverse_block != 128 && t->traverse_block != 256)
    return fail(SDD_ERR_ARG, "traverse_block must be 64, 128 or 256");
  // staged nodes take the 48 KB of shared memory a block may use without opting in
  constexpr int kMaxStaged = (int)((48 * 1024) / sizeof(Node));
  static_assert(kMaxStaged == 384, "the message below names the bound");
  if (t->top_nodes < 0 || t->top_nodes > kMaxStaged) return fail(SDD_ERR_ARG, "top_nodes must be in [0, 384]");
  if (t->wave_paths < 0) return fail(SDD_ERR_ARG, "wave_paths must be >= 0");
  if (t->no_graph != 0 && t->no_graph != 1) return fail(SDD_ERR_ARG, "no_graph must be 0 or 1");
  if (t->queue_capacity < 0) return fail(SDD_ERR_ARG, "queue_capacity must be >= 0");
  if (t->block_chunks < 0 || t->block_chunks > 3) return fail(SDD_ERR_ARG, "block_chunks must be in [0, 3]");
  if (t->resident_subdomains < 0) return fail(SDD_ERR_ARG, "resident_subdomains must be >= 0");
  if (sdd_status r = set_streaming(s, t->resident_subdomains)) return r;
  s->tuning = *t;
  s->tuning.resident_subdomains = s->strm.cap;
  return SDD_OK;
}

sdd_status sdd_get_tuning(const sdd_scene* s, sdd_tuning* t) {
  if (!s || !t) return fail(SDD_ERR_ARG, "NULL argument");
  *t = s->tuning;
  return SDD_OK;
}

sdd_status sdd_set_profiling(sdd_scene* s, int level) {
  if (!s || level < 0 || level > 2) return fail(SDD_ERR_ARG, "bad scene or profiling level");
  s->profiling = level;
  return SDD_OK;
}

sdd_status sdd_get_stats(const sdd_scene* s, sdd_stats* out) {
  if (!s || !out) return fail(SDD_ERR_ARG, "NULL argument");
  *out = s->stats;
  return SDD_OK;
}

sdd_status sdd_trace_closest(sdd_scene* s, int n, const float* org, const float* dir, float* t_out, int32_t* prim_out,
                             void* stream) {
  g_err.clear();
  if (!s || n < 0 || (n > 0 && (!org || !dir || !t_out || !prim_out))) return fail(SDD_ERR_ARG, "bad arguments");
  if (n == 0) return SDD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  sdd_status r = ensure_workspace(s, (size_t)n, (size_t)n, 1, false, 1);
  if (r) return r;
  CK(cudaMemsetAsync(s->d_ctl, 0, sizeof(Control), st));
  RayBuf rb{s->rb_o[0].p, s->rb_d[0].p, s->rb_info[0].p, n};
  launch_rays_from_arrays(n, org, dir, s->dev, rb, s->q[0].p, s->d_ctl->q_count[0], n, st);
  CK(cudaGetLastError());
  RenderParams p{};
  p.sc = s->dev;
  p.stats = 0;
  r = run_closest_passes(s, p, rb, n, st);
  if (r) return r;
  launch_hits_to_arrays(n, s->hits.p, t_out, prim_out, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

sdd_status sdd_eval_optics(int n, const float* cos_i, const float* n_re, const float* k, const float* d,
                           const float* lam, int slab_polarisation, float* R, float* Rs, float* Ts, void* stream) {
  g_err.clear();
  if (n < 0 || (n > 0 && (!cos_i || !n_re || !k || !d || !lam || !R || !Rs || !Ts))) return fail(SDD_ERR_ARG, "bad arguments");
  if (slab_polarisation != 0 && slab_polarisation != 1) return fail(SDD_ERR_ARG, "slab_polarisation must be 0 or 1");
  if (n == 0) return SDD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  launch_eval_optics(n, cos_i, n_re, k, d, lam, slab_polarisation, R, Rs, Ts, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

sdd_status sdd_photon_maps_build(sdd_scene* s, const sdd_photon_opts* o, sdd_photon_maps** out, void* stream) {
  g_err.clear();
  if (!s || !o || !out) return fail(SDD_ERR_ARG, "NULL scene, options or output");
  *out = nullptr;
  if (o->n_lambda < 1 || o->n_lambda > 4096 || !o->lambda_nm) return fail(SDD_ERR_ARG, "n_lambda must be in [1, 4096]");
  for (int i = 0; i < o->n_lambda; ++i)
    if (!(o->lambda_nm[i] > 0.f) || !std::isfinite(o->lambda_nm[i])) return fail(SDD_ERR_ARG, "lambda_nm must be positive");
  if (o->n_per_lambda < 1) return fail(SDD_ERR_ARG, "n_per_lambda must be >= 1");
  if ((int64_t)o->n_lambda * o->n_per_lambda > 0x7FFFFFFFLL) return fail(SDD_ERR_ARG, "n_lambda x n_per_lambda exceeds 2^31 - 1");
  if (o->max_depth < 1 || o->max_depth > 255) return fail(SDD_ERR_ARG, "max_depth must be in [1, 255]");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(o->center[i])) return fail(SDD_ERR_ARG, "center must be finite");
  if (!(o->radius_m > 0.f) || !std::isfinite(o->radius_m)) return fail(SDD_ERR_ARG, "radius_m must be > 0");
  if (!(o->distance_m >= 0.f) || !std::isfinite(o->distance_m)) return fail(SDD_ERR_ARG, "distance_m must be >= 0");
  if (!(o->gather_radius_m > 0.f) || !std::isfinite(o->gather_radius_m))
    return fail(SDD_ERR_ARG, "gather_radius_m must be > 0");
  if (s->il_sun.empty() || !(s->sun_half > 0.f)) return fail(SDD_ERR_STATE, "photon maps need a sun");
  sdd_photon_maps* m = new (std::nothrow) sdd_photon_maps;
  if (!m) return fail(SDD_ERR_OOM, "host allocation failed");
  sdd_status r = photon_build(s, o, m, (cudaStream_t)stream);
  if (r) {
    delete m;
    return r;
  }
  *out = m;
  return SDD_OK;
}

void sdd_photon_maps_destroy(sdd_photon_maps* m) { delete m; }

sdd_status sdd_photon_maps_count(const sdd_photon_maps* m, int64_t* n_caustic, int64_t* n_global) {
  g_err.clear();
  if (!m || !n_caustic || !n_global) return fail(SDD_ERR_ARG, "NULL argument");
  *n_caustic = m->count[0];
  *n_global = m->count[1];
  return SDD_OK;
}

sdd_status sdd_photon_maps_get(const sdd_photon_maps* m, int map, float* pos, float* nrm, float* power, int32_t* lam,
                               uint32_t* id, uint32_t* seq) {
  g_err.clear();
  if (!m) return fail(SDD_ERR_ARG, "NULL maps");
  if (map != 0 && map != 1) return fail(SDD_ERR_ARG, "map must be 0 (caustic) or 1 (global)");
  const size_t n = (size_t)m->count[map];
  if (n == 0) return SDD_OK;
  std::vector<float4> a(n), b(n);
  std::vector<uint2> c(n);
  CK(cudaMemcpy(a.data(), m->raw_pos[map].p, n * sizeof(float4), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(b.data(), m->raw_nrm[map].p, n * sizeof(float4), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(c.data(), m->raw_id[map].p, n * sizeof(uint2), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < n; ++i) {
    if (pos) { pos[3 * i] = a[i].x; pos[3 * i + 1] = a[i].y; pos[3 * i + 2] = a[i].z; }
    if (nrm) { nrm[3 * i] = b[i].x; nrm[3 * i + 1] = b[i].y; nrm[3 * i + 2] = b[i].z; }
    if (power) power[i] = a[i].w;
    if (lam) { int v; std::memcpy(&v, &b[i].w, sizeof(int)); lam[i] = v; }
    if (id) id[i] = c[i].x;
    if (seq) seq[i] = c[i].y;
  }
  return SDD_OK;
}

sdd_status sdd_photon_gather(const sdd_photon_maps* m, int n, const float* x, const float* nrm, const int32_t* lam,
                             float* ec, float* eg, void* stream) {
  g_err.clear();
  if (!m || n < 0 || (n > 0 && (!x || !nrm || !lam || !ec || !eg))) return fail(SDD_ERR_ARG, "bad arguments");
  if (n == 0) return SDD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  launch_photon_gather(m->view(), n, x, nrm, lam, ec, eg, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

sdd_status sdd_philox(int n, const uint32_t* ctr, uint64_t key, uint32_t* out, void* stream) {
  g_err.clear();
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(SDD_ERR_ARG, "bad arguments");
  if (n == 0) return SDD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  launch_philox(n, ctr, key, out, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return SDD_OK;
}

}  // extern "C"
