// surrogate_render.cu -- heterogeneous tiles in the renderer through the BTDF network.
//
// The shading kernel queues a generation's tile hits.  One fused launch then shades them
// all (k_infer_tc with TileShadePolicy, on the tcgen05 tensor cores): per chunk of 128 hits it gathers the network's
// inputs from the ray state and the tile's material, runs the network, and samples the
// exit from the prediction -- the side with probability R / (R + T) and throughput
// x (R + T), a von Mises-Fisher lobe by its weight (surrogate_head.cuh), then a direction
// from that lobe about the straight-through or mirror direction -- and appends the ray to
// the next generation.  The hit count is read on the device, so the launch needs no host
// round trip and can sit in a captured frame; in the batched form the buffers are taken
// from the persistent kernel's saved queue state.  Shadow rays through a tile use the
// network's transmittance x the transmitted mixture's mass within 1 degree of straight
// through toward the sun (sun table), the same ballistic convention as the brute-force form.
#include "bundle_device.cuh"
#include "persistent.cuh"
#include "surrogate_head.cuh"
#include "surrogate_net.cuh"
#include "surrogate_tc.cuh"
#include "surrogate_render.cuh"

namespace sdd {

namespace {

__device__ __forceinline__ float clamp01(float x) { return fminf(1.f, fmaxf(0.f, x)); }

// Direction from the vMF lobe about unit axis a with concentration kappa: the cosine by
// inverting the lobe's mass F(1 - cos) (surrogate_head.cuh), uniform azimuth.  Returns
// 1 - cos of the angle to the axis in *a_out.
__device__ float3 vmf_sample(float3 a, float kappa, float u1, float u2, float* a_out) {
  float v = -log1pf(u1 * expm1f(-2.f * kappa)) / kappa;  // 1 - cos
  v = fminf(2.f, fmaxf(0.f, v));
  float st = sqrtf(fmaxf(0.f, v * (2.f - v)));
  float3 b1, b2;
  onb(a, &b1, &b2);
  float sp, cp;
  sincospif(2.f * u2, &sp, &cp);
  *a_out = v;
  return (st * cp) * b1 + (st * sp) * b2 + (1.f - v) * a;
}

struct TileHit {
  PathId id;
  float3 pt, ng, dl, t1, t2;
  int mat;
  float thr;
  uint2 info;
  int lam;     // wavelength index
  int member;  // spectral bundles: the member of the ray's bundle (0 otherwise)
};

// The tile hit of tile-queue entry e: a ray slot, or with spectral bundles ray << 6 | member.
__device__ __forceinline__ TileHit tile_hit(const RenderParams& p, const WaveDesc& w, const RayBuf& cur,
                                            const float2* hits, uint32_t e) {
  TileHit h;
  const bool bund = p.bundle > 1;
  const uint32_t r = bund ? e >> 6 : e;
  h.member = bund ? (int)(e & 63u) : 0;
  const float4 O = cur.o[r], D = cur.d[r];
  h.info = cur.info[r];
  const float2 H = hits[r];
  h.id = bund ? path_id_bundle(p, w, h.info.x) : path_id(p, w, h.info.x);
  h.lam = bund ? (int)h.id.lam * p.bundle + h.member : (int)h.id.lam;
  const float4 nm = __ldg(p.sc.prim_nrm_mat + __float_as_uint(H.y));
  h.ng = f3(nm);
  h.mat = __float_as_int(nm.w);
  const float3 d = f3(D);
  h.pt = f3(O) + H.x * d;
  h.thr = bund ? cur.w[(size_t)r * p.bundle + h.member] : D.w;
  float x, y;
  tile_frame(p.tiles.L, h.pt, h.ng, d, &x, &y, &h.dl, &h.t1, &h.t2);
  return h;
}

}  // namespace

// Fused shading of a generation's tile hits (see the file comment).  With pc set, the ray
// and queue buffers are those of the persistent kernel's saved state (batched form).
struct TileShadePolicy {
  RenderParams p;
  WaveDesc w;
  RayBuf cur, next;
  const float2* hits;
  int* next_count;
  uint32_t* q;
  int* q_count;
  int qcap;
  Control* ctl;
  PersistBuffers b;
  PersistCtl* pc;

  struct Ctx {
    RayBuf cur, next;
    int* next_count;
    uint32_t* q;
    int* q_count;
  };
  __device__ Ctx resolve() const {
    if (!pc) return Ctx{cur, next, next_count, q, q_count};
    const volatile PersistState* st = &pc->st;
    const int c = st->cur, gen = st->gen, qe = st->qe, cq = st->cq;
    return Ctx{b.rb[c], b.rb[1 - c], &pc->next_rays[gen & 1], b.q[qe], pc->qc[cq]};
  }
  __device__ int count(const Ctx&) const { return min(*(volatile const int*)p.tile_count, p.tile_cap); }
  __device__ void load(const Ctx& c, int row, float qv[net::kIn]) const {
    const TileHit h = tile_hit(p, w, c.cur, hits, p.tile_queue[row]);
    const int tile = __ldg(p.mat_tile + h.mat);
    const size_t mi = (size_t)h.mat * p.sp.n_lambda + h.lam;
    float phi = atan2f(h.dl.y, h.dl.x);
    if (phi < 0.f) phi += 6.283185307179586f;
    qv[0] = -h.dl.z;  // signed: > 0 arrives at the flat front face (the side the normal points to)
    qv[1] = phi;
    qv[2] = __ldg(p.sp.lambda_nm + h.lam);
    qv[3] = __ldg(p.tiles.d_mean + tile);
    qv[4] = __ldg(p.tiles.rho + tile);
    qv[5] = __ldg(p.sp.mat_n + mi);
    qv[6] = __ldg(p.sp.mat_k + mi);
  }
  // Threads 0..127 (whole warps) take one row each and append its exit ray (with spectral
  // bundles a ray of the one member, drawing on the bundle's counter word).
  __device__ void consume(const Ctx& c, int row0, int valid, const float* pred) const {
    if (p.stats >= 2 && threadIdx.x == 0) atomicAdd(&ctl->tile_shaded, (unsigned long long)valid);
    if (threadIdx.x >= kInferRows) return;
    const int i = threadIdx.x;
    const bool active = i < valid;
    bool e0 = false;
    float3 o0 = make_float3(0.f, 0.f, 0.f), d0 = o0;
    float thr0 = 0.f, s00 = 0.f;
    uint32_t meta0 = 0, path = 0;
    int member = 0;
    const bool bund = p.bundle > 1;
    if (active) {
      const TileHit h = tile_hit(p, w, c.cur, hits, p.tile_queue[row0 + i]);
      path = h.info.x;
      member = h.member;
      const uint32_t depth = h.info.y & 0xFFu, flags = (h.info.y >> 8) & 0xFFu;
      const uint32_t v = depth + 1;
      const float* pr = pred + i * kInferZLd;
      const float T = clamp01(pr[0]), R = clamp01(pr[1]);
      uint32_t* hp = p.path_hash ? p.path_hash + (bund ? (size_t)path * p.bundle + member : (size_t)path) : nullptr;
      uint32_t hsh = hp ? *hp : 0u;
      const float4 u = draw4(h.id.pixel, h.id.sample, v, STREAM_TILE, 0, h.id.lam, p.seed);
      const float4 up = draw4(h.id.pixel, h.id.sample, v, STREAM_PATH, 0, h.id.lam, p.seed);
      const float tot = T + R;
      if (tot > 0.f) {
        const bool refl = u.x * tot < R;
        const float* lobe = pr + (refl ? 5 : 2);
        const float kappa = expf(u.y < lobe[0] ? lobe[1] : lobe[2]);
        const float3 ref = refl ? make_float3(h.dl.x, h.dl.y, -h.dl.z) : h.dl;  // tile frame
        float a;
        float3 dir = vmf_sample(ref, kappa, u.z, u.w, &a);
        if ((dir.z > 0.f) != (ref.z > 0.f)) dir.z = -dir.z;  // keep the lobe on its side of the tile
        const bool ballistic = a < head_bin_a(1);             // within 1 degree
        hsh = fnv_byte(hsh, refl ? EV_REFLECT : EV_TRANSMIT);
        float thr = h.thr * tot;
        const uint32_t fl = (!refl && ballistic) ? flags : (flags & ~FLAG_SUN_COUNTED);
        e0 = true;
        d0 = normalize3(dir.x * h.t1 + dir.y * h.t2 + dir.z * h.ng);
        meta0 = v | (fl << 8);
        if ((int)v >= p.rr_start) {
          const float qs = fminf(0.95f, thr);
          if (up.w >= qs) {
            e0 = false;
            hsh = fnv_byte(hsh, EV_RR_KILL);
          } else {
            thr = thr / qs;
          }
        }
        thr0 = thr;
        if (e0) {
          o0 = offset_point(h.pt, h.ng, d0, p.sc.eps);
          s00 = seg0_of(h.ng, d0, p.sc.eps);
        }
      } else {
        hsh = fnv_byte(hsh, EV_ABSORB);
      }
      if (hp) *hp = hsh;
    }
    if (bund) {
      const int pos = emit_bundle_ray(e0, p.sc, c.next, c.next_count, c.q, c.q_count, qcap, o0, s00, d0, path, meta0,
                                      1ull << member, ctl);
      if (pos >= 0) {
        float* cw = c.next.w + (size_t)pos * p.bundle;
        for (int k = 0; k < p.bundle; ++k) cw[k] = k == member ? thr0 : 0.f;
      }
    } else {
      emit_ray(e0, p.sc, c.next, c.next_count, c.q, c.q_count, qcap, o0, s00, d0, thr0, path, meta0, ctl);
    }
  }
  __device__ uint32_t* err(const Ctx&) const { return &ctl->error; }
};

namespace {
cudaError_t launch_tile_shade_policy(const TileShadePolicy& pol, const sdd_surrogate* net, cudaStream_t st) {
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e = infer_tc_prepare<TileShadePolicy>();
    if (e != cudaSuccess) return e;
    prepared = true;
  }
  k_infer_tc<TileShadePolicy><<<infer_grid(pol.p.tile_cap), tc::kThreads, tc::kSmem, st>>>(surrogate_view(net), pol);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tile_shade(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits, RayBuf next,
                              int* next_count, uint32_t* q, int* q_count, int qcap, Control* ctl,
                              const sdd_surrogate* net, cudaStream_t st) {
  TileShadePolicy pol{};
  pol.p = p;
  pol.w = w;
  pol.cur = cur;
  pol.next = next;
  pol.hits = hits;
  pol.next_count = next_count;
  pol.q = q;
  pol.q_count = q_count;
  pol.qcap = qcap;
  pol.ctl = ctl;
  pol.pc = nullptr;
  return launch_tile_shade_policy(pol, net, st);
}

cudaError_t launch_tile_shade_persistent(const RenderParams& p, const WaveDesc& w, const PersistBuffers& b,
                                         PersistCtl* pc, Control* ctl, const sdd_surrogate* net, cudaStream_t st) {
  TileShadePolicy pol{};
  pol.p = p;
  pol.w = w;
  pol.hits = b.hits;
  pol.qcap = b.qcap;
  pol.ctl = ctl;
  pol.b = b;
  pol.pc = pc;
  return launch_tile_shade_policy(pol, net, st);
}

__global__ void k_sun_queries(RenderParams p, const int* mats, const float3* mat_normal, int n_mats, float* raw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int L = p.sp.n_lambda;
  if (i >= n_mats * L) return;
  int j = i / L, l = i - j * L;
  int mat = mats[j];
  float3 nrm = mat_normal[j];
  float3 t1, t2;
  onb(nrm, &t1, &t2);
  float3 d = p.sp.sun_dir;  // the shadow ray's direction
  float3 dl = make_float3(dot3(d, t1), dot3(d, t2), dot3(d, nrm));
  float phi = atan2f(dl.y, dl.x);
  if (phi < 0.f) phi += 6.283185307179586f;
  int tile = p.mat_tile[mat];
  size_t mi = (size_t)mat * L + l;
  float* q = raw + 7 * (size_t)i;
  q[0] = -dl.z;
  q[1] = phi;
  q[2] = p.sp.lambda_nm[l];
  q[3] = p.tiles.d_mean[tile];
  q[4] = p.tiles.rho[tile];
  q[5] = p.sp.mat_n[mi];
  q[6] = p.sp.mat_k[mi];
}

__global__ void k_sun_table(const int* mats, int n_mats, int L, const float* pred, float* table) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_mats * L) return;
  int j = i / L, l = i - j * L;
  const float* pr = pred + kHeadPred * (size_t)i;
  const float ball = lobe_mass_within(pr[2], expf(pr[3]), expf(pr[4]), head_bin_a(1));
  table[(size_t)mats[j] * L + l] = clamp01(pr[0]) * clamp01(ball);
}

void launch_sun_queries(const RenderParams& p, const int* mats, const float3* mat_normal, int n_mats, float* raw,
                        cudaStream_t st) {
  int n = n_mats * p.sp.n_lambda;
  if (n > 0) k_sun_queries<<<(n + 127) / 128, 128, 0, st>>>(p, mats, mat_normal, n_mats, raw);
}

void launch_sun_table(const int* mats, int n_mats, int L, const float* pred, float* table, cudaStream_t st) {
  int n = n_mats * L;
  if (n > 0) k_sun_table<<<(n + 255) / 256, 256, 0, st>>>(mats, n_mats, L, pred, table);
}

}  // namespace sdd
