// photon.cu -- photon maps (Sec. 3.2: Jensen's photon mapping, the paper's global-illumination
// algorithm): photon tracing from the sun on the renderer's wavefront (the same subdomain
// queues and closest-hit passes as the camera paths), the maps' hashed uniform grids, and
// density estimation.
//
// Photon i of wavelength index l leaves a disc of radius R centred on C + D s (s toward the
// sun), perpendicular to s, at a point uniform over the disc, travelling along -w with w
// uniform in the sun's cone; it carries Phi = L_sun(l) Omega (s . w) pi R^2 / N.  Its draws are
// Philox(photon i, 0, bounce | photon stream, wavelength l).  At glass it follows the camera
// paths' Monte Carlo rules; at a diffuse surface it is stored, then survives with probability
// albedo (power unchanged) into a cosine-distributed direction.  Stored in the caustic map when
// a specular event changed its direction before any diffuse bounce, in the global map after
// a diffuse bounce; light that reached its first diffuse surface only through straight slab
// transmission (or ballistic tile exits) is direct light, counted by the renderer's sun NEE,
// and is not stored.
#include "photon.cuh"
#include "photon_device.cuh"
#include "render_device.cuh"

namespace sdd {

namespace {

constexpr int kPB = 128;

__global__ void __launch_bounds__(kPB) k_photon_emit(RenderParams p, PhotonEmit pe, int n, RayBuf rb, uint32_t* q,
                                                     int* q_count, int qcap, Control* ctl) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = r < n;
  float3 o = make_float3(0.f, 0.f, 0.f);
  if (active) {
    const uint32_t j = pe.j0 + (uint32_t)r;
    const uint32_t l = j / (uint32_t)pe.n_per_lambda, i = j - l * (uint32_t)pe.n_per_lambda;
    const float4 u = draw4(i, 0, 0, STREAM_PHOTON, 0, l, p.seed);
    const float3 s = p.sp.sun_dir;
    float3 t1, t2;
    onb(s, &t1, &t2);
    const float rr = pe.radius * sqrtf(u.x), phi = 2.f * kPhotonPi * u.y;
    o = pe.origin + (rr * cosf(phi)) * t1 + (rr * sinf(phi)) * t2;
    const float3 w = cone_dir(s, p.sp.sun_h, u.z, u.w);
    const float power = __ldg(p.sp.sun + l) * pe.power_scale * dot3(s, w);
    rb.o[r] = make_float4(o.x, o.y, o.z, 0.f);
    rb.d[r] = make_float4(-w.x, -w.y, -w.z, power);
    rb.info[r] = make_uint2(j, 0u);  // depth 0, no flags, no diffuse surface met
  }
  const int sd = active ? subdomain_of(p.sc, o) : 0;
  const int pos = warp_append(q_count, sd, active);
  if (active) {
    if (pos < qcap) q[(size_t)sd * qcap + pos] = (uint32_t)r;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
}

enum : uint32_t { PF_SPEC = 1u, PF_DIFF = 2u };

// One generation of photons: interaction at the hit, storage, continuation.
template <int kTM>
__global__ void __launch_bounds__(kPB) k_photon_shade(RenderParams p, PhotonEmit pe, int n_rays, RayBuf cur,
                                                      const float2* __restrict__ hits, RayBuf next, int* next_count,
                                                      uint32_t* q, int* q_count, int qcap, PhotonStore st,
                                                      Control* ctl) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  bool emit = false, store = false;
  int map = 0;
  float3 o0 = make_float3(0.f, 0.f, 0.f), d0 = o0, pt = o0, nf = o0;
  float pw0 = 0.f, s00 = 0.f, stored_pw = 0.f;
  uint32_t path = 0, meta0 = 0, seq = 0, lam = 0, id = 0, stored_seq = 0;
  if (r < n_rays) {
    const float4 O = cur.o[r], D = cur.d[r];
    const uint2 inf = cur.info[r];
    const float2 H = hits[r];
    path = inf.x;
    const uint32_t depth = inf.y & 0xFFu;
    uint32_t flags = (inf.y >> 8) & 0xFFu;
    seq = inf.y >> 16;
    const int l = (int)(path / (uint32_t)pe.n_per_lambda);
    const uint32_t i = path - (uint32_t)l * (uint32_t)pe.n_per_lambda;
    lam = (uint32_t)l;
    id = i;
    const uint32_t prim = __float_as_uint(H.y);
    const uint32_t v = depth + 1;
    if (prim != kMissPrim && prim < (uint32_t)p.sc.n_prims && (int)v <= p.max_depth) {
      float power = D.w;
      const float seg0 = O.w;
      const float3 o = f3(O), d = f3(D);
      const float lambda = __ldg(p.sp.lambda_nm + l);
      const float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
      const float3 ng = f3(nm);
      const int mat = __float_as_int(nm.w);
      const int kind = __ldg(p.sp.mat_kind + mat);
      const size_t mi = (size_t)mat * p.sp.n_lambda + l;
      pt = o + H.x * d;
      const float cos_n = dot3(d, ng);
      nf = cos_n < 0.f ? ng : -1.f * ng;
      const float cos_i = fabsf(cos_n);
      const float4 u = draw4(i, 0, v, STREAM_PHOTON, 0, (uint32_t)l, p.seed);
      if (kind == MAT_SOLID) {
        const bool inside = cos_n > 0.f;
        const float nre = __ldg(p.sp.mat_n + mi), kk = __ldg(p.sp.mat_k + mi);
        if (inside) power *= beer_lambert(kk, H.x + seg0, lambda);
        const float n1 = inside ? nre : 1.f;
        const float n2re = inside ? 1.f : nre, n2im = inside ? 0.f : kk;
        const float R = fresnel_R(cos_i, n1, n2re, n2im);
        const float eta = n1 / n2re;
        const float c2 = 1.f - eta * eta * (1.f - cos_i * cos_i);
        d0 = (u.x < R || c2 <= 0.f) ? reflect3(d, nf) : normalize3(eta * d + (eta * cos_i - sqrtf(c2)) * nf);
        flags |= PF_SPEC;
        emit = true;
      } else if (kind == MAT_SLAB) {
        float Rs, Ts;
        slab_RT(cos_i, __ldg(p.sp.mat_n + mi), __ldg(p.sp.mat_k + mi), __ldg(p.sp.mat_thick + mat), lambda, &Rs, &Ts,
                p.sp.slab_pol);
        power *= Rs + Ts;
        if (u.x < Rs / (Rs + Ts)) {
          d0 = reflect3(d, nf);
          flags |= PF_SPEC;
        } else {
          d0 = d;
        }
        emit = true;
      } else if (kTM == 1 && kind == MAT_TILE) {
        float x, y;
        float3 dl, t1v, t2v;
        tile_frame(p.tiles.L, pt, ng, d, &x, &y, &dl, &t1v, &t2v);
        const TileOut to = tile_trace(tile_of(p.tiles, __ldg(p.mat_tile + mat)), x, y, dl, __ldg(p.sp.mat_n + mi),
                                      __ldg(p.sp.mat_k + mi), lambda, i, 0, v, (uint32_t)l, p.seed, kTileEvents,
                                      STREAM_PHOTON_TILE);
        if (to.side != 2) {
          power *= to.w;
          d0 = normalize3(to.dir.x * t1v + to.dir.y * t2v + to.dir.z * ng);
          if (!(to.side == 1 && dot3(to.dir, dl) > kCos1Deg)) flags |= PF_SPEC;
          emit = true;
        }
      } else if (kind == MAT_DIFFUSE) {
        if (flags & (PF_SPEC | PF_DIFF)) {
          store = true;
          map = (flags & PF_DIFF) ? 1 : 0;
          stored_pw = power;
          stored_seq = seq;
        }
        if (u.w < __ldg(p.sp.mat_albedo + mi)) {  // survives with probability albedo
          d0 = cosine_dir(nf, u.y, u.z);
          flags |= PF_DIFF;
          ++seq;
          emit = true;
        }
      }
      if (emit) {
        o0 = offset_point(pt, ng, d0, p.sc.eps);
        s00 = seg0_of(ng, d0, p.sc.eps);
        pw0 = power;
        meta0 = v | (flags << 8) | (seq << 16);
      }
    }
  }
  // store into the map's append buffer (the count runs on past cap: the host grows and repeats)
  const int k = warp_append(st.count, map, store);
  if (store && k >= 0 && k < st.cap) {
    st.pos_pw[map][k] = make_float4(pt.x, pt.y, pt.z, stored_pw);
    st.nrm_lam[map][k] = make_float4(nf.x, nf.y, nf.z, __int_as_float((int)lam));
    st.id_seq[map][k] = make_uint2(id, stored_seq);
  }
  emit_ray(emit, p.sc, next, next_count, q, q_count, qcap, o0, s00, d0, pw0, path, meta0, ctl);
}

// ---------------------------------------------------------------- hashed grid
__device__ __forceinline__ uint32_t bucket_of(float3 x, float inv_cell, uint32_t mask) {
  return photon_bucket(photon_cell(x.x, inv_cell), photon_cell(x.y, inv_cell), photon_cell(x.z, inv_cell), mask);
}

__global__ void k_bucket_count(int n, const float4* __restrict__ pos, float inv_cell, uint32_t mask, uint32_t* count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) atomicAdd(count + bucket_of(f3(pos[k]), inv_cell, mask), 1u);
}

// Exclusive prefix sums of 1024-entry blocks (Hillis-Steele in shared memory); block totals out.
__global__ void __launch_bounds__(1024) k_scan_blocks(int n, const uint32_t* __restrict__ in, uint32_t* out,
                                                      uint32_t* totals) {
  __shared__ uint32_t s[1024];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t v = i < n ? in[i] : 0u;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t a = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
    __syncthreads();
    s[threadIdx.x] += a;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) totals[blockIdx.x] = s[1023];
}

// Exclusive prefix sums of the block totals in place (one block, sequential over chunks).
__global__ void __launch_bounds__(1024) k_scan_totals(int nb, uint32_t* totals, uint32_t* grand) {
  __shared__ uint32_t s[1024];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nb ? totals[i] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const uint32_t a = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
      __syncthreads();
      s[threadIdx.x] += a;
      __syncthreads();
    }
    if (i < nb) totals[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int n, uint32_t* out, const uint32_t* __restrict__ totals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += totals[i / 1024];
}

__global__ void k_bucket_scatter(int n, const float4* __restrict__ pos, const float4* __restrict__ nrm, float inv_cell,
                                 uint32_t mask, uint32_t* cursor, float4* out_pos, float4* out_nrm) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float4 p = pos[k];
  const uint32_t dst = atomicAdd(cursor + bucket_of(f3(p), inv_cell, mask), 1u);
  out_pos[dst] = p;
  out_nrm[dst] = nrm[k];
}

__global__ void k_photon_gather(PhotonMapDev pm, int n, const float* __restrict__ x, const float* __restrict__ nrm,
                                const int32_t* __restrict__ lam, float* ec, float* eg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float3 p = make_float3(x[3 * i], x[3 * i + 1], x[3 * i + 2]);
  const float3 nn = make_float3(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]);
  const float2 e = photon_irradiance(pm, p, nn, lam[i]);
  ec[i] = e.x;
  eg[i] = e.y;
}

int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_photon_emit(const RenderParams& p, const PhotonEmit& pe, int n, RayBuf rb, uint32_t* q, int* q_count,
                        int qcap, Control* ctl, cudaStream_t st) {
  if (n > 0) k_photon_emit<<<blocks(n, kPB), kPB, 0, st>>>(p, pe, n, rb, q, q_count, qcap, ctl);
}

void launch_photon_shade(const RenderParams& p, const PhotonEmit& pe, int n_rays, RayBuf cur, const float2* hits,
                         RayBuf next, int* next_count, uint32_t* q, int* q_count, int qcap, const PhotonStore& s,
                         Control* ctl, cudaStream_t st) {
  if (n_rays <= 0) return;
  if (p.tiles.n_tiles > 0)  // photons trace through heterogeneous tiles by brute force
    k_photon_shade<1><<<blocks(n_rays, kPB), kPB, 0, st>>>(p, pe, n_rays, cur, hits, next, next_count, q, q_count, qcap,
                                                           s, ctl);
  else
    k_photon_shade<0><<<blocks(n_rays, kPB), kPB, 0, st>>>(p, pe, n_rays, cur, hits, next, next_count, q, q_count, qcap,
                                                           s, ctl);
}

// Sort n photons into the buckets of a table of mask + 1 entries (a power of two, >= 1024),
// cells of edge 1 / inv: start [mask + 2] (its last entry the total), scratch
// [mask + 1 + (mask + 1) / 1024] words.
cudaError_t build_photon_grid(int n, const float4* pos, const float4* nrm, float inv, uint32_t mask, uint32_t* start,
                              uint32_t* scratch, float4* out_pos, float4* out_nrm, cudaStream_t st) {
  const int T = (int)mask + 1;
  uint32_t* count = scratch;
  uint32_t* totals = scratch + T;
  const int nb = blocks(T, 1024);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * T, st);
  if (e != cudaSuccess) return e;
  if (n > 0) k_bucket_count<<<blocks(n, 256), 256, 0, st>>>(n, pos, inv, mask, count);
  k_scan_blocks<<<nb, 1024, 0, st>>>(T, count, start, totals);
  k_scan_totals<<<1, 1024, 0, st>>>(nb, totals, start + T);
  k_scan_add<<<blocks(T, 256), 256, 0, st>>>(T, start, totals);
  e = cudaMemcpyAsync(count, start, sizeof(uint32_t) * T, cudaMemcpyDeviceToDevice, st);  // scatter cursors
  if (e != cudaSuccess) return e;
  if (n > 0) k_bucket_scatter<<<blocks(n, 256), 256, 0, st>>>(n, pos, nrm, inv, mask, count, out_pos, out_nrm);
  return cudaGetLastError();
}

void launch_photon_gather(const PhotonMapDev& pm, int n, const float* x, const float* nrm, const int32_t* lam, float* ec,
                          float* eg, cudaStream_t st) {
  if (n > 0) k_photon_gather<<<blocks(n, 128), 128, 0, st>>>(pm, n, x, nrm, lam, ec, eg);
}

}  // namespace sdd
