// surrogate_render.cu -- heterogeneous tiles in the renderer through the BTDF network.
//
// A generation's tile hits are queued by the shading kernel; this file gathers their network
// inputs, and after the network has predicted T, R and the two von Mises-Fisher lobes of
// each side (surrogate_head.cuh), samples the exit: the side with probability R / (R + T) and
// throughput x (R + T), a lobe by its weight, then a direction from it about the
// straight-through or mirror direction.  Shadow rays through a tile use the network's
// transmittance x the transmitted mixture's mass within 1 degree of straight through
// toward the sun (sun_table), the same ballistic convention as the brute-force form.
#include "render_device.cuh"
#include "surrogate_head.cuh"
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

__device__ __forceinline__ void tile_query(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits,
                                           uint32_t r, PathId* id, float3* pt, float3* ng, float3* dl, float3* t1,
                                           float3* t2, int* mat, float4* O, float4* D, uint2* inf) {
  *O = cur.o[r];
  *D = cur.d[r];
  *inf = cur.info[r];
  float2 H = hits[r];
  *id = path_id(p, w, inf->x);
  uint32_t prim = __float_as_uint(H.y);
  float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
  *ng = f3(nm);
  *mat = __float_as_int(nm.w);
  float3 d = f3(*D);
  *pt = f3(*O) + H.x * d;
  float x, y;
  tile_frame(p.tiles.L, *pt, *ng, d, &x, &y, dl, t1, t2);
}

}  // namespace

__global__ void k_tile_inputs(RenderParams p, WaveDesc w, RayBuf cur, const float2* hits, const uint32_t* queue, int n,
                              float* raw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  PathId id;
  float3 pt, ng, dl, t1, t2;
  int mat;
  float4 O, D;
  uint2 inf;
  tile_query(p, w, cur, hits, queue[i], &id, &pt, &ng, &dl, &t1, &t2, &mat, &O, &D, &inf);
  int tile = __ldg(p.mat_tile + mat);
  size_t mi = (size_t)mat * p.sp.n_lambda + id.lam;
  float phi = atan2f(dl.y, dl.x);
  if (phi < 0.f) phi += 6.283185307179586f;
  float* q = raw + 7 * (size_t)i;
  q[0] = -dl.z;  // signed: > 0 arrives at the flat front face (the side the normal points to)
  q[1] = phi;
  q[2] = __ldg(p.sp.lambda_nm + id.lam);
  q[3] = __ldg(p.tiles.d_mean + tile);
  q[4] = __ldg(p.tiles.rho + tile);
  q[5] = __ldg(p.sp.mat_n + mi);
  q[6] = __ldg(p.sp.mat_k + mi);
}

__global__ void k_tile_apply(RenderParams p, WaveDesc w, RayBuf cur, const float2* hits, const uint32_t* queue, int n,
                             const float* pred, RayBuf next, int* next_count, uint32_t* q, int* q_count, int qcap,
                             Control* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool active = i < n;
  bool e0 = false;
  float3 o0 = make_float3(0.f, 0.f, 0.f), d0 = o0;
  float thr0 = 0.f, s00 = 0.f;
  uint32_t meta0 = 0, path = 0;
  if (active) {
    PathId id;
    float3 pt, ng, dl, t1, t2;
    int mat;
    float4 O, D;
    uint2 inf;
    tile_query(p, w, cur, hits, queue[i], &id, &pt, &ng, &dl, &t1, &t2, &mat, &O, &D, &inf);
    path = inf.x;
    uint32_t depth = inf.y & 0xFFu, flags = (inf.y >> 8) & 0xFFu;
    uint32_t v = depth + 1;
    const float* pr = pred + kHeadPred * (size_t)i;
    float T = clamp01(pr[0]), R = clamp01(pr[1]);
    uint32_t hsh = p.path_hash ? p.path_hash[path] : 0u;
    float4 u = draw4(id.pixel, id.sample, v, STREAM_TILE, 0, id.lam, p.seed);
    float4 up = draw4(id.pixel, id.sample, v, STREAM_PATH, 0, id.lam, p.seed);
    float tot = T + R;
    if (tot > 0.f) {
      bool refl = u.x * tot < R;
      const float* lobe = pr + (refl ? 5 : 2);
      float kappa = expf(u.y < lobe[0] ? lobe[1] : lobe[2]);
      float3 ref = refl ? make_float3(dl.x, dl.y, -dl.z) : dl;  // mirror or straight through (tile frame)
      float a;
      float3 dir = vmf_sample(ref, kappa, u.z, u.w, &a);
      if ((dir.z > 0.f) != (ref.z > 0.f)) dir.z = -dir.z;  // keep the lobe on its side of the tile
      bool ballistic = a < head_bin_a(1);                    // within 1 degree
      hsh = fnv_byte(hsh, refl ? EV_REFLECT : EV_TRANSMIT);
      float thr = D.w * tot;
      bool keep = !refl && ballistic;
      uint32_t fl = keep ? flags : (flags & ~FLAG_SUN_COUNTED);
      e0 = true;
      d0 = normalize3(dir.x * t1 + dir.y * t2 + dir.z * ng);
      meta0 = v | (fl << 8);
      if ((int)v >= p.rr_start) {
        float qs = fminf(0.95f, thr);
        if (up.w >= qs) {
          e0 = false;
          hsh = fnv_byte(hsh, EV_RR_KILL);
        } else {
          thr = thr / qs;
        }
      }
      thr0 = thr;
      if (e0) {
        o0 = offset_point(pt, ng, d0, p.sc.eps);
        s00 = seg0_of(ng, d0, p.sc.eps);
      }
    } else {
      hsh = fnv_byte(hsh, EV_ABSORB);
    }
    if (p.path_hash) p.path_hash[path] = hsh;
  }
  emit_ray(e0, p.sc, next, next_count, q, q_count, qcap, o0, s00, d0, thr0, path, meta0, ctl);
}

// Network queries toward the sun for every tile material and wavelength.
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

void launch_tile_inputs(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits,
                        const uint32_t* queue, int n, float* raw, cudaStream_t st) {
  if (n > 0) k_tile_inputs<<<(n + 127) / 128, 128, 0, st>>>(p, w, cur, hits, queue, n, raw);
}

void launch_tile_apply(const RenderParams& p, const WaveDesc& w, RayBuf cur, const float2* hits,
                       const uint32_t* queue, int n, const float* pred, RayBuf next, int* next_count, uint32_t* q,
                       int* q_count, int qcap, Control* ctl, cudaStream_t st) {
  if (n > 0)
    k_tile_apply<<<(n + 127) / 128, 128, 0, st>>>(p, w, cur, hits, queue, n, pred, next, next_count, q, q_count, qcap,
                                                  ctl);
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
