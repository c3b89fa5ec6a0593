// bundle_device.cuh -- spectral bundles: the wavefront path with several wavelengths per ray.
//
// Sec. 4 of the paper cuts the 81-value spectral array into groups of n wavelengths as units
// of work.  Here a bundle is B consecutive wavelengths (B = RenderParams::bundle, 2..64) of one (pixel,
// sample).  Every random number of the bundle's chains is drawn on the bundle index j in
// place of the wavelength index (the rule the oracle follows), so as long as their decisions
// agree the B chains share every vertex and one traversal serves them all.  A ray carries the
// 64-bit mask of the members that still follow it (RayBuf::m) and one throughput per member
// (RayBuf::w, [cap][B]).  At a vertex the members are split:
//   thin-slab glass    reflected members and transmitted members (at most two rays);
//   diffuse            one ray (the cosine direction does not depend on the wavelength) and
//                      one shadow ray whose per-member contributions (ShadowBuf::c) the
//                      shadow walk multiplies by each member's slab transmittance;
//   solid dielectric   the reflected members in one ray, each transmitted member on its own
//                      ray (Snell's direction depends on n(lambda));
//   brute-force tiles  each member on its own ray (its own trace through the tile).
// Russian roulette is decided per member with the shared uniform.  Path radiance goes to
// path_L[path][B] and, with event hashes enabled, each member keeps its own hash, so every
// member's chain can be compared with the oracle's chain of that wavelength event for event.
// Every function that appends must be called by all 32 lanes of a warp.
#pragma once

#include "render_device.cuh"

namespace sdd {

namespace {

// Path id of a bundle ray: the `lam` field holds the bundle index j (cells are
// pixel_index * n_bundles + j).
__device__ __forceinline__ PathId path_id_bundle(const RenderParams& p, const WaveDesc& w, uint32_t path) {
  PathId r;
  uint32_t ls = path / w.nc;
  uint32_t lc = path - ls * w.nc;
  r.sample = w.s0 + ls;
  r.cell = w.c0 + lc;
  r.px_i = r.cell / (uint32_t)p.n_bundles;
  r.lam = r.cell - r.px_i * (uint32_t)p.n_bundles;
  r.pixel = p.pixel_list ? (uint32_t)p.pixel_list[r.px_i] : r.px_i;
  return r;
}

using Members = unsigned long long;

// Members of bundle j: wavelengths j B .. min(j B + B, L) - 1.
__device__ __forceinline__ Members bundle_members(const RenderParams& p, uint32_t j) {
  int n = min(p.bundle, p.sp.n_lambda - (int)j * p.bundle);
  return n >= 64 ? ~0ull : ((1ull << n) - 1ull);
}

// Index of the lowest member in m (m != 0).
__device__ __forceinline__ int first_member(Members m) { return __ffsll((long long)m) - 1; }

// Hash updates of every member in `mask` (no-op without hashes).
__device__ __forceinline__ void hash_word(uint32_t* hp, Members mask, uint32_t w) {
  if (!hp) return;
  for (Members m = mask; m; m &= m - 1) {
    int b = first_member(m);
    hp[b] = fnv_word(hp[b], w);
  }
}
__device__ __forceinline__ void hash_event(uint32_t* hp, Members mask, uint32_t ev) {
  if (!hp) return;
  for (Members m = mask; m; m &= m - 1) {
    int b = first_member(m);
    hp[b] = fnv_byte(hp[b], ev);
  }
}

// Append a bundle ray to the next generation and bin it by the subdomain of its origin;
// returns its slot (-1 when not appended).  The caller writes its throughputs.
__device__ __forceinline__ int emit_bundle_ray(bool want, const DevScene& sc, RayBuf nb, int* next_count, uint32_t* q,
                                               int* q_count, int qcap, float3 o, float seg0, float3 d, uint32_t path,
                                               uint32_t meta, Members members, Control* ctl) {
  int pos = warp_append(next_count, 0, want);
  bool ok = want && pos < nb.cap;
  if (want && !ok) atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  if (ok) {
    nb.o[pos] = make_float4(o.x, o.y, o.z, seg0);
    nb.d[pos] = make_float4(d.x, d.y, d.z, 0.f);
    nb.info[pos] = make_uint2(path, meta);
    nb.m[pos] = members;
  }
  int s = ok ? subdomain_of(sc, o) : 0;
  int qpos = warp_append(q_count, s, ok);
  if (ok) {
    if (qpos < qcap) q[(size_t)s * qcap + qpos] = (uint32_t)pos;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
  return ok ? pos : -1;
}

// Child throughput of a member after the roulette it survived (q = min(0.95, t)).
__device__ __forceinline__ float after_roulette(float t, bool roulette) { return roulette ? t / fminf(0.95f, t) : t; }

// Writes the B member values val(0..B-1) of the record in slot pos (pos < 0: none) of dst
// ([slots][B]).  Every lane of the warp calls this; the lanes with a slot hold consecutive
// slots in lane order (warp_append), so their values go through the warp's staging area
// (32 x B floats of shared memory) and the warp's block of dst is written with coalesced
// stores instead of B strided partial-sector stores per lane.
template <class F>
__device__ __forceinline__ void store_members(float* dst, int pos, int B, float* stage, F val) {
  const unsigned m = __ballot_sync(0xffffffffu, pos >= 0);
  if (m == 0u) return;
  const int first = __shfl_sync(0xffffffffu, pos, __ffs(m) - 1);
  if (pos >= 0) {
    const int rank = pos - first;
    for (int b = 0; b < B; ++b) stage[rank * B + b] = val(b);
  }
  __syncwarp();
  const int n = __popc(m) * B;
  float* d = dst + (size_t)first * B;
  for (int k = (int)(threadIdx.x & 31); k < n; k += 32) d[k] = stage[k];
  __syncwarp();
}

// The warp's rows when lane l holds row r0 + l and the lanes with a row form a prefix (the
// kernels index rays by a block-strided base plus threadIdx.x): their count, with *r0 the
// first; -1 otherwise, and the caller then accesses its row per lane.  Every lane calls it.
__device__ __forceinline__ int warp_rows(uint32_t r, bool active, uint32_t* r0) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  const uint32_t first = r - (threadIdx.x & 31u);
  *r0 = __shfl_sync(0xffffffffu, first, 0);
  const bool ok = __all_sync(0xffffffffu, first == *r0) && (act & (act + 1u)) == 0u;
  return ok ? __popc(act) : -1;
}

}  // namespace

// ------------------------------------------------------------------------------ raygen
// One primary ray per wave-local bundle path i (every lane of the warp calls this).
__device__ __forceinline__ void dev_raygen_bundle(const RenderParams& p, const WaveDesc& w, uint32_t i, bool active,
                                                  RayBuf rb, uint32_t* q, int* q_count, int qcap, Control* ctl) {
  const int B = p.bundle;
  float3 o = make_float3(0.f, 0.f, 0.f), d = o;
  if (active) {
    PathId id = path_id_bundle(p, w, i);
    float4 u = draw4(id.pixel, id.sample, 0, STREAM_PATH, 0, id.lam, p.seed);
    primary_ray(p, id.pixel, u.x - 0.5f, u.y - 0.5f, &o, &d);
    rb.o[i] = make_float4(o.x, o.y, o.z, 0.f);
    rb.d[i] = make_float4(d.x, d.y, d.z, 0.f);
    rb.info[i] = make_uint2(i, 0u);  // depth 0, no flags
    rb.m[i] = bundle_members(p, id.lam);
  }
  // member throughputs 1 and fresh event hashes: the warp's rows with coalesced stores
  uint32_t i0;
  const int nrow = warp_rows(i, active, &i0);
  if (nrow >= 0) {
    const int lane = (int)(threadIdx.x & 31u);
    float* wd = rb.w + (size_t)i0 * B;
    for (int k = lane; k < nrow * B; k += 32) wd[k] = 1.f;
    if (p.path_hash) {
      uint32_t* hd = p.path_hash + (size_t)i0 * B;
      for (int k = lane; k < nrow * B; k += 32) hd[k] = 0x811C9DC5u;
    }
  } else if (active) {
    for (int b = 0; b < B; ++b) rb.w[(size_t)i * B + b] = 1.f;
    if (p.path_hash)
      for (int b = 0; b < B; ++b) p.path_hash[(size_t)i * B + b] = 0x811C9DC5u;
  }
  int s = active ? subdomain_of(p.sc, o) : 0;
  int pos = warp_append(q_count, s, active);
  if (active) {
    if (pos < qcap) q[(size_t)s * qcap + pos] = i;
    else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
  }
}

// ------------------------------------------------------------------------------ shade
// Shade bundle ray r of the current generation (every lane of the warp calls this).  The
// per-member loop over the vertex's material (Eq. 1 with the complex index, the thin-slab
// series, Beer-Lambert, the Lambertian albedo) decides each member's branch with the shared
// uniforms; the members are then grouped into child rays as the header describes.  Each
// member's throughput after the vertex (before the roulette) is kept in shared memory, one
// row of B floats per thread; the children's member values are written through a per-warp
// staging area of 32 x B floats.  The kernel's dynamic shared memory holds both:
// bundle_shade_smem(B) bytes for blocks of kBlock threads.
// kPM: photon maps (Sec. 3.2), as in dev_shade: the first diffuse vertex adds each member's
// albedo / pi x (E_caustic + E_global) of its wavelength; the continuation carries
// FLAG_PHOTON_DONE (sky light only: no NEE, no sun disc on escape).
template <int kTM, bool kPM = false>
__device__ __forceinline__ void dev_shade_bundle(const RenderParams& p, const WaveDesc& w, int r, bool active,
                                                 RayBuf cur, const float2* __restrict__ hits, RayBuf next,
                                                 int* next_count, uint32_t* q, int* q_count, int qcap, ShadowBuf sb,
                                                 int* shadow_count, uint32_t* sq, int* sq_count, float* path_L,
                                                 Control* ctl) {
  const int B = p.bundle;
  const float eps = p.sc.eps;
  // children: group 0 (members leaving in direction gd0), group 1 (thin-slab transmission:
  // members going straight on) and singles (each member on its own direction).  Origins and
  // the facing normal are recomputed where needed rather than kept live.
  Members gm[2] = {0ull, 0ull}, singles = 0ull, msh = 0ull, tile_m = 0ull;
  uint32_t gf[2] = {0u, 0u};
  float3 gd0 = make_float3(0.f, 0.f, 0.f), dsh = gd0;
  uint32_t path = 0, v = 0, flags = 0, j = 0, lam0 = 0;
  int kind = -1, mat = 0;
  bool roulette = false;
  float uw = 0.f, cl_sh = 0.f, cos_i = 0.f, seg0 = 0.f;
  float3 pt = gd0, ng = gd0, d = gd0;
  extern __shared__ float s_bundle_rows[];
  float* wr = s_bundle_rows + threadIdx.x * B;
  float* stage = s_bundle_rows + (kBlock + (threadIdx.x & ~31u)) * B;
  uint32_t* hp = nullptr;
  PathId id{};
  {
    // the member throughputs into the rows: the warp's block of cur.w with coalesced loads
    uint32_t r0;
    const int nrow = warp_rows((uint32_t)r, active, &r0);
    if (nrow >= 0) {
      // sixteen loads in flight per lane before their shared-memory stores (nave frame: shading
      // 36.0 ms per frame against 36.5 with eight, 38.0 with four, 36.7 with per-lane row loads)
      constexpr int kU = 16;
      float* rows = s_bundle_rows + (threadIdx.x & ~31u) * B;
      const float* src = cur.w + (size_t)r0 * B;
      const int n = nrow * B;
      int k = (int)(threadIdx.x & 31u);
      for (; k + 32 * (kU - 1) < n; k += 32 * kU) {
        float v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) v[u] = src[k + 32 * u];
#pragma unroll
        for (int u = 0; u < kU; ++u) rows[k + 32 * u] = v[u];
      }
      for (; k < n; k += 32) rows[k] = src[k];
      __syncwarp();
    } else if (active) {
      for (int b = 0; b < B; ++b) wr[b] = cur.w[(size_t)r * B + b];
    }
  }
  if (active) {
    float4 O = cur.o[r], D = cur.d[r];
    uint2 inf = cur.info[r];
    float2 H = hits[r];
    path = inf.x;
    const uint32_t depth = inf.y & 0xFFu;
    const Members mask = cur.m[r];
    flags = (inf.y >> 8) & 0xFFu;
    seg0 = O.w;
    const float3 o = f3(O);
    d = f3(D);
    id = path_id_bundle(p, w, path);
    j = id.lam;
    lam0 = j * (uint32_t)B;
    hp = p.path_hash ? p.path_hash + (size_t)path * B : nullptr;
    float* Lp = path_L + (size_t)path * B;
    const uint32_t prim = __float_as_uint(H.y);
    if (prim != kMissPrim && prim >= (uint32_t)p.sc.n_prims) {
      atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);  // stale hit record of a dropped ray
    } else if (prim == kMissPrim) {
      const bool sun_counted = (flags & (FLAG_SUN_COUNTED | FLAG_PHOTON_DONE)) != 0u;
      for (Members m = mask; m; m &= m - 1) {
        int b = first_member(m);
        Lp[b] += wr[b] * escape_radiance(p.sp, d, (int)lam0 + b, sun_counted);
      }
      hash_word(hp, mask, 0xFFFFFFFFu);
      hash_event(hp, mask, EV_ESCAPE);
    } else {
      hash_word(hp, mask, prim);
      v = depth + 1;
      if ((int)v > p.max_depth) {
        hash_event(hp, mask, EV_DEPTH_CAP);
      } else {
        float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
        ng = f3(nm);
        mat = __float_as_int(nm.w);
        kind = __ldg(p.sp.mat_kind + mat);
        pt = o + H.x * d;
        const float cos_n = dot3(d, ng);
        const float3 nf = cos_n < 0.f ? ng : -1.f * ng;
        cos_i = fabsf(cos_n);
        const float4 u = draw4(id.pixel, id.sample, v, STREAM_PATH, 0, j, p.seed);
        uw = u.w;
        const float* mn = p.sp.mat_n + (size_t)mat * p.sp.n_lambda + lam0;
        const float* mk = p.sp.mat_k + (size_t)mat * p.sp.n_lambda + lam0;
        if (kind == MAT_SOLID) {
          const bool inside = cos_n > 0.f;
          for (Members m = mask; m; m &= m - 1) {
            int b = first_member(m);
            float nre = __ldg(mn + b), kk = __ldg(mk + b);
            float thr = wr[b];
            if (inside) thr *= beer_lambert(kk, H.x + seg0, __ldg(p.sp.lambda_nm + lam0 + b));
            float n1 = inside ? nre : 1.f;
            float n2re = inside ? 1.f : nre, n2im = inside ? 0.f : kk;
            float R = fresnel_R(cos_i, n1, n2re, n2im);
            float eta = n1 / n2re;
            float c2 = 1.f - eta * eta * (1.f - cos_i * cos_i);
            wr[b] = thr;
            if (u.x < R || c2 <= 0.f) gm[0] |= 1ull << b;
            else singles |= 1ull << b;
          }
          hash_event(hp, gm[0], EV_REFLECT);
          hash_event(hp, singles, EV_TRANSMIT);
          gd0 = reflect3(d, nf);
          gf[0] = flags & ~FLAG_SUN_COUNTED;
        } else if (kind == MAT_SLAB) {
          const float thick = __ldg(p.sp.mat_thick + mat);
          for (Members m = mask; m; m &= m - 1) {
            int b = first_member(m);
            float Rs, Ts;
            slab_RT(cos_i, __ldg(mn + b), __ldg(mk + b), thick, __ldg(p.sp.lambda_nm + lam0 + b), &Rs, &Ts, p.sp.slab_pol);
            float P = Rs / (Rs + Ts);
            wr[b] = wr[b] * (Rs + Ts);
            if (u.x < P) gm[0] |= 1ull << b;  // (a computed index would put gm in local memory)
            else gm[1] |= 1ull << b;
          }
          hash_event(hp, gm[0], EV_REFLECT);
          hash_event(hp, gm[1], EV_TRANSMIT);
          gd0 = reflect3(d, nf);
          gf[0] = flags & ~FLAG_SUN_COUNTED;
          gf[1] = flags;
        } else if (kind == MAT_DIFFUSE) {
          const float* ma = p.sp.mat_albedo + (size_t)mat * p.sp.n_lambda + lam0;
          hash_event(hp, mask, EV_DIFFUSE);
          for (Members m = mask; m; m &= m - 1) {
            int b = first_member(m);
            wr[b] = wr[b] * __ldg(ma + b);
          }
          const bool photon_done = kPM && (flags & FLAG_PHOTON_DONE) != 0u;
          if (kPM && !photon_done) {
            for (Members m = mask; m; m &= m - 1) {
              int b = first_member(m);
              const float2 E = photon_irradiance(p.pm, pt, nf, (int)lam0 + b);
              Lp[b] += wr[b] * kInvPi * (E.x + E.y);
            }
          }
          if (p.sp.sun_h > 0.f && !photon_done) {
            float4 un = draw4(id.pixel, id.sample, v, STREAM_NEE, 0, j, p.seed);
            float3 wl = cone_dir(p.sp.sun_dir, p.sp.sun_h, un.x, un.y);
            float cl = dot3(nf, wl);
            if (cl > 0.f) {
              msh = mask;
              dsh = wl;
              cl_sh = cl;
            }
          }
          gm[0] = mask;
          gd0 = cosine_dir(nf, u.y, u.z);
          gf[0] = flags | FLAG_SUN_COUNTED | (kPM ? FLAG_PHOTON_DONE : 0u);
        } else if (kTM == 1 && kind == MAT_TILE) {
          singles = mask;  // each member traces its own ray through the tile
        } else if (kTM == 2 && kind == MAT_TILE) {
          tile_m = mask;  // each member is shaded from the network's prediction for its wavelength
        } else {
          hash_event(hp, mask, EV_ABSORB);
        }
        if ((int)v >= p.rr_start) {
          roulette = true;
          // tile members meet their roulette after their own trace (singles loop)
          const Members cand = gm[0] | gm[1] | (kind == MAT_SOLID ? singles : 0ull);
          for (Members m = cand; m; m &= m - 1) {
            int b = first_member(m);
            if (uw >= fminf(0.95f, wr[b])) {
              const Members bit = 1ull << b;
              gm[0] &= ~bit;
              gm[1] &= ~bit;
              if (kind == MAT_SOLID) singles &= ~bit;
              hash_event(hp, bit, EV_RR_KILL);
            }
          }
        }
      }
    }
  }
  // group children
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const float3 dg = g == 0 ? gd0 : d;
    float3 og = dg;
    float sg = 0.f;
    if (gm[g]) {
      og = offset_point(pt, ng, dg, eps);
      sg = seg0_of(ng, dg, eps);
    }
    const int pos = emit_bundle_ray(gm[g] != 0ull, p.sc, next, next_count, q, q_count, qcap, og, sg, dg, path,
                                    v | (gf[g] << 8), gm[g], ctl);
    const Members mg = gm[g];
    store_members(next.w, pos, B, stage, [&](int b) { return ((mg >> b) & 1ull) ? after_roulette(wr[b], roulette) : 0.f; });
  }
  // singles: each member on its own direction (transmission into or out of solid glass,
  // brute-force tiles)
  if (__any_sync(0xffffffffu, singles != 0ull)) {
    const float* mn = p.sp.mat_n + (size_t)mat * p.sp.n_lambda + lam0;
    const float* mk = p.sp.mat_k + (size_t)mat * p.sp.n_lambda + lam0;
    for (int b = 0; b < B; ++b) {
      bool want = (singles >> b) & 1ull;
      float3 ds = d, os = d;
      float ts = 0.f, ss = 0.f;
      uint32_t fs = 0u;
      if (want) {
        const float lambda = __ldg(p.sp.lambda_nm + lam0 + b);
        const float3 nf = dot3(d, ng) < 0.f ? ng : -1.f * ng;
        if (kind == MAT_SOLID) {
          const bool inside = dot3(d, ng) > 0.f;
          const float nre = __ldg(mn + b);
          const float eta = inside ? nre : 1.f / nre;
          const float c2 = 1.f - eta * eta * (1.f - cos_i * cos_i);
          ds = normalize3(eta * d + (eta * cos_i - sqrtf(c2)) * nf);
          ts = after_roulette(wr[b], roulette);
          fs = flags & ~FLAG_SUN_COUNTED;
        } else {
          float x, y;
          float3 dl, t1v, t2v;
          tile_frame(p.tiles.L, pt, ng, d, &x, &y, &dl, &t1v, &t2v);
          TileOut tr = tile_trace(tile_of(p.tiles, __ldg(p.mat_tile + mat)), x, y, dl, __ldg(mn + b), __ldg(mk + b),
                                  lambda, id.pixel, id.sample, v, j, p.seed, kTileEvents, STREAM_TILE);
          const Members bit = 1ull << b;
          if (tr.side == 2) {
            hash_event(hp, bit, EV_ABSORB);
            want = false;
          } else {
            hash_event(hp, bit, tr.side == 0 ? EV_REFLECT : EV_TRANSMIT);
            ds = normalize3(tr.dir.x * t1v + tr.dir.y * t2v + tr.dir.z * ng);
            ts = wr[b] * tr.w;
            const bool keep = tr.side == 1 && dot3(tr.dir, dl) > kCos1Deg;
            fs = keep ? flags : (flags & ~FLAG_SUN_COUNTED);
            if (roulette) {
              const float qs = fminf(0.95f, ts);
              if (uw >= qs) {
                hash_event(hp, bit, EV_RR_KILL);
                want = false;
              } else {
                ts = ts / qs;
              }
            }
          }
        }
        if (want) {
          os = offset_point(pt, ng, ds, eps);
          ss = seg0_of(ng, ds, eps);
        }
      }
      const int pos = emit_bundle_ray(want, p.sc, next, next_count, q, q_count, qcap, os, ss, ds, path, v | (fs << 8),
                                      1ull << b, ctl);
      store_members(next.w, pos, B, stage, [&](int k) { return k == b ? ts : 0.f; });
    }
  }
  // network form: one tile-queue entry (ray << 6 | member) per member at a tile hit
  if (kTM == 2 && __any_sync(0xffffffffu, tile_m != 0ull)) {
    for (int b = 0; b < B; ++b) {
      const bool want = (tile_m >> b) & 1ull;
      const int tpos = warp_append(p.tile_count, 0, want);
      if (want) {
        if (tpos < p.tile_cap) p.tile_queue[tpos] = ((uint32_t)r << 6) | (uint32_t)b;
        else atomicOr(&ctl->error, ERR_QUEUE_OVERFLOW);
      }
    }
  }
  // shadow ray toward the sun, one contribution per member
  const bool esh = msh != 0ull;
  const float3 osh = esh ? offset_point(pt, ng, dsh, eps) : dsh;
  int pos = warp_append(shadow_count, 0, esh);
  bool ok = esh && pos < sb.cap;
  if (esh && !ok) atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  if (ok) {
    sb.o[pos] = make_float4(osh.x, osh.y, osh.z, 0.f);
    sb.d[pos] = make_float4(dsh.x, dsh.y, dsh.z, 0.f);
    sb.info[pos] = make_uint2(path, v << 16);
    sb.m[pos] = msh;
  }
  store_members(sb.c, ok ? pos : -1, B, stage, [&](int b) {
    return ((msh >> b) & 1ull) ? wr[b] * kInvPi * cl_sh * __ldg(p.sp.sun + lam0 + b) * p.sp.sun_omega : 0.f;
  });
  int ss = ok ? subdomain_of(p.sc, osh) : 0;
  int qpos = warp_append(sq_count, ss, ok);
  if (ok) {
    if (qpos < qcap) sq[(size_t)ss * qcap + qpos] = (uint32_t)pos;
    else atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  }
}

// ------------------------------------------------------------------------------ shadow
// Shadow-queue entry i of subdomain s toward the sun for a bundle (every lane of the warp
// calls this): each surface met multiplies every live member's contribution by that
// member's transmittance; a brute-force tile trace that fails for a member drops that
// member only; opaque geometry blocks them all.  Survivors are handed on to the neighbouring
// subdomain or added to their paths.  kWarp selects the warp-uniform walk.
template <bool kStats, int kTM, bool kWarp>
__device__ __forceinline__ void dev_shadow_bundle(const RenderParams& p, const WaveDesc& w, int s, int i, bool active,
                                                  const Node* s_nodes, int n_staged, QueuePair qp, ShadowBuf sb,
                                                  float* path_L, Control* ctl) {
  const int B = p.bundle;
  uint32_t r = active ? qp.in[(size_t)s * qp.cap + i] : 0u;
  bool cross = false;
  int next = -1;
  uint32_t nn = 0, nt = 0;
  float4 O = make_float4(0.f, 0.f, 0.f, 0.f), D = make_float4(0.f, 0.f, 1.f, 0.f);
  uint2 inf = make_uint2(0u, 0u);
  float t0 = 0.f, t1 = 0.f;
  if (active) {
    O = sb.o[r];
    D = sb.d[r];
    inf = sb.info[r];
    slab_interval(p.sc, s, f3(O), f3(D), &t0, &t1, &next);
  }
  const float3 o = f3(O), d = f3(D);
  const PathId id = path_id_bundle(p, w, inf.x);
  const uint32_t lam0 = id.lam * (uint32_t)B;
  const uint32_t bounce = inf.y >> 16;
  const ShadowKey key{id.pixel, id.sample, bounce, p.seed, id.lam};
  Members live = active ? sb.m[r] : 0ull;
  float* c = sb.c + (size_t)r * B;
  uint32_t* hp = (active && p.path_hash && p.mode == 1) ? p.path_hash + (size_t)inf.x * B : nullptr;
  const RayPre rp = ray_pre(o, d);
  auto hit = [&](float t, uint32_t prim) -> bool {
    float4 nm = __ldg(p.sc.prim_nrm_mat + prim);
    int mat = __float_as_int(nm.w);
    int kind = __ldg(p.sp.mat_kind + mat);
    const size_t m0 = (size_t)mat * p.sp.n_lambda + lam0;
    if (kind == MAT_SLAB) {
      const float cos_i = fabsf(dot3(d, f3(nm)));
      const float thick = __ldg(p.sp.mat_thick + mat);
      for (Members m = live; m; m &= m - 1) {
        int b = first_member(m);
        float Rs, Ts;
        slab_RT(cos_i, __ldg(p.sp.mat_n + m0 + b), __ldg(p.sp.mat_k + m0 + b), thick,
                __ldg(p.sp.lambda_nm + lam0 + b), &Rs, &Ts, p.sp.slab_pol);
        c[b] *= Ts;
      }
      return false;
    }
    if (kTM == 2 && kind == MAT_TILE) {
      for (Members m = live; m; m &= m - 1) {
        int b = first_member(m);
        c[b] *= __ldg(p.tile_sun_T + m0 + b);
      }
      return false;
    }
    if (kTM == 1 && kind == MAT_TILE) {
      float x, y;
      float3 dl, t1v, t2v;
      tile_frame(p.tiles.L, rp.o + t * d, f3(nm), d, &x, &y, &dl, &t1v, &t2v);
      const TileDev tile = tile_of(p.tiles, __ldg(p.mat_tile + mat));
      for (Members m = live; m; m &= m - 1) {
        int b = first_member(m);
        TileOut tr = tile_trace(tile, x, y, dl, __ldg(p.sp.mat_n + m0 + b), __ldg(p.sp.mat_k + m0 + b),
                                __ldg(p.sp.lambda_nm + lam0 + b), key.pixel, key.sample, key.bounce, key.word,
                                key.seed, kTileEvents, STREAM_SHADOW_TILE);
        if (tr.side == 1 && dot3(tr.dir, dl) > kCos1Deg) {
          c[b] *= tr.w;
        } else {
          live &= ~(1ull << b);
          hash_event(hp, 1ull << b, EV_SHADOW_BLOCKED);
        }
      }
      return live == 0ull;
    }
    return true;
  };
  const bool walk = active && t1 > t0;
  bool ovf = false, blocked = false;
  if constexpr (kWarp) {
    blocked = any_hit_walk_warp<kStats>(p.sc, s_nodes, n_staged, s, rp, t0, t1, walk, &nn, &nt, &ovf, hit);
  } else {
    if (walk) blocked = any_hit_walk<kStats>(p.sc, s_nodes, n_staged, s, rp, t0, t1, &nn, &nt, &ovf, hit);
  }
  if (active) {
    if (ovf) atomicOr(&ctl->error, ERR_STACK_OVERFLOW);
    cross = !blocked && next >= 0;
    if (cross) {
      sb.m[r] = live;
    } else if (!blocked) {
      float* Lp = path_L + (size_t)inf.x * B;
      for (Members m = live; m; m &= m - 1) {
        int b = first_member(m);
        Lp[b] += c[b];
      }
      hash_event(hp, live, EV_SHADOW_OPEN);
    } else {
      hash_event(hp, live, EV_SHADOW_BLOCKED);
    }
  }
  int pos = warp_append(qp.out_count, cross ? next : 0, cross);
  if (cross) {
    if (pos < qp.cap) qp.out[(size_t)next * qp.cap + pos] = r;
    else atomicOr(&ctl->error, ERR_SHADOW_OVERFLOW);
  }
  if (kStats) {
    unsigned long long a = warp_sum<unsigned long long>(active ? 1ull : 0ull);
    unsigned long long n1 = warp_sum<unsigned long long>(nn);
    unsigned long long n2 = warp_sum<unsigned long long>(nt);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctl->rays_shadow, a);
      atomicAdd(&ctl->shadow_node_visits, n1);
      atomicAdd(&ctl->shadow_tri_tests, n2);
    }
  }
}

}  // namespace sdd
