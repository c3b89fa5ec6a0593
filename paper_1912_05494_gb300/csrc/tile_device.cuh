// tile_device.cuh -- brute-force light transport through one heterogeneous glass tile (FP32).
//
// The paper's medieval tiles have non-uniform thickness and air micro-bubbles that scatter
// light (Sec. 1; Sec. 6 names scattering as the missing piece).  Tile model:
//   * periodic square tile of side L, flat front face z = 0, back face z = -h(x, y) given by a
//     G x G triangulated height field (heights from 2-octave value noise, clamped to 2-5 mm);
//   * air bubbles: a Poisson process of density rho in the glass, radius log-uniform in
//     [10, 100] um; free path ~ Exp(rho * pi * E[r^2]); a met bubble's radius is drawn with
//     weight r^2, the impact point uniformly over its cross-section; the outgoing direction
//     follows the exact sphere optics, the encounter does not displace the ray (bubbles are
//     points at the tile's millimetre scale);
//   * complex-index Fresnel, Snell with the real index and Beer-Lambert along glass segments;
//     each interaction consumes one Philox draw on the tile stream;
//   * the ray leaves through the face on its incident side (reflected) or the other face
//     (transmitted) and does not re-enter; beyond max_events interactions it is absorbed.
#pragma once

#include <math_constants.h>

#include "device_math.cuh"

namespace sdd {

struct TileDev {
  const float* h;     // [(G+1)^2] thickness at the grid vertices, row j, column i
  float hmin, hmax;   // range of h
  float rho;          // bubbles per cubic metre
  int G;
  float L;
};

struct TileOut {
  int side;        // 0 reflected, 1 transmitted, 2 absorbed at the interaction cap
  float w;
  float3 dir;
  int bubbles, events;
};

constexpr float kTileEps = 1e-7f;
constexpr int kTileMaxCells = 4096;

// Lattice value of octave `oct` at integer lattice point (ix, iy).
__device__ __forceinline__ float tile_lattice(uint32_t seed, int ix, int iy, int oct) {
  uint4 o = philox4x32_10(make_uint4((uint32_t)ix, (uint32_t)iy, (uint32_t)oct, seed), 0x5EED7113u, 0u);
  return u01(o.x);
}

__device__ __forceinline__ float tile_value_noise(uint32_t seed, float x, float y, float L, int cells, int oct) {
  float gx = x / L * cells, gy = y / L * cells;
  float fx0 = floorf(gx), fy0 = floorf(gy);
  float fx = gx - fx0, fy = gy - fy0;
  int ix = (((int)fx0 % cells) + cells) % cells, iy = (((int)fy0 % cells) + cells) % cells;
  int jx = (ix + 1) % cells, jy = (iy + 1) % cells;
  float sx = fx * fx * (3.f - 2.f * fx), sy = fy * fy * (3.f - 2.f * fy);
  float a = tile_lattice(seed, ix, iy, oct), b = tile_lattice(seed, jx, iy, oct);
  float c = tile_lattice(seed, ix, jy, oct), d = tile_lattice(seed, jx, jy, oct);
  return (1.f - sy) * ((1.f - sx) * a + sx * b) + sy * ((1.f - sx) * c + sx * d);
}

__device__ __forceinline__ float tile_thickness(uint32_t seed, float d_mean, float amp, float x, float y, float L) {
  float n = (2.f / 3.f) * tile_value_noise(seed, x, y, L, 10, 0) + (1.f / 3.f) * tile_value_noise(seed, x, y, L, 20, 1);
  return fminf(0.005f, fmaxf(0.002f, d_mean + amp * (n - 0.5f)));
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// First back-face hit along o + t d, t in (0, t_max]; n_out: unit normal pointing up (+z,
// into the glass).  Walks the grid cells the ray's xy projection crosses.
__device__ __forceinline__ float tile_back_hit(const TileDev& g, float3 o, float3 d, float t_max, float3* n_out) {
  const float cs = g.L / g.G;
  int ci = (int)floorf(o.x / cs), cj = (int)floorf(o.y / cs);
  const int sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0), sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
  const float tdx = sx ? cs / fabsf(d.x) : CUDART_INF_F, tdy = sy ? cs / fabsf(d.y) : CUDART_INF_F;
  float tx = sx > 0 ? ((ci + 1) * cs - o.x) / d.x : (sx < 0 ? (ci * cs - o.x) / d.x : CUDART_INF_F);
  float ty = sy > 0 ? ((cj + 1) * cs - o.y) / d.y : (sy < 0 ? (cj * cs - o.y) / d.y : CUDART_INF_F);
  float t_in = 0.f;
  RayPre rp = ray_pre(o, d);
  for (int step = 0; step < kTileMaxCells && t_in <= t_max; ++step) {
    float t_out = fminf(fminf(tx, ty), t_max);
    float z0 = o.z + d.z * t_in, z1 = o.z + d.z * t_out;
    if (fminf(z0, z1) <= -g.hmin) {
      int wi = ((ci % g.G) + g.G) % g.G, wj = ((cj % g.G) + g.G) % g.G;
      const float* H = g.h;
      const int W = g.G + 1;
      float x0 = ci * cs, y0 = cj * cs;
      float4 p00 = make_float4(x0, y0, -__ldg(H + wj * W + wi), 0.f);
      float4 p10 = make_float4(x0 + cs, y0, -__ldg(H + wj * W + wi + 1), 0.f);
      float4 p01 = make_float4(x0, y0 + cs, -__ldg(H + (wj + 1) * W + wi), 0.f);
      float4 p11 = make_float4(x0 + cs, y0 + cs, -__ldg(H + (wj + 1) * W + wi + 1), 0.f);
      float ta = tri_hit(rp, p00, p10, p11, 0.f, t_max);
      float tb = tri_hit(rp, p00, p11, p01, 0.f, t_max);
      float best = -1.f;
      float3 bn = make_float3(0.f, 0.f, 1.f);
      if (ta >= 0.f) {
        best = ta;
        bn = cross3(f3(p10) - f3(p00), f3(p11) - f3(p00));
      }
      if (tb >= 0.f && (best < 0.f || tb < best)) {
        best = tb;
        bn = cross3(f3(p11) - f3(p00), f3(p01) - f3(p00));
      }
      if (best >= 0.f) {
        bn = normalize3(bn);
        if (bn.z < 0.f) bn = -1.f * bn;
        *n_out = bn;
        return best;
      }
    }
    if (tx < ty) {
      ci += sx;
      t_in = tx;
      tx += tdx;
    } else {
      cj += sy;
      t_in = ty;
      ty += tdy;
    }
  }
  return -1.f;
}

// One ray through the tile from entry point (x0, y0) with direction d in the tile frame
// (d.z < 0: through the front, d.z > 0: through the back).  Draws keyed (px, sample,
// bounce | tile stream | event, lam).
static __device__ inline TileOut tile_trace(const TileDev& g, float x0, float y0, float3 d, float n, float k, float lambda_nm,
                              uint32_t px, uint32_t sample, uint32_t bounce, uint32_t lam, uint64_t seed,
                              int max_events, uint32_t stream = STREAM_TILE) {
  const float r_lo = 10e-6f, r_hi = 100e-6f;
  const float Er2 = (r_hi * r_hi - r_lo * r_lo) / (2.f * logf(r_hi / r_lo));
  const float sig = g.rho * 3.14159265358979f * Er2;
  const float alpha = kFourPi * k / (lambda_nm * 1e-9f);
  TileOut out{2, 0.f, d, 0, 0};
  const float3 d_in = d;
  float w = 1.f;
  int e = 0;
  float3 p, nrm;
  if (d.z < 0.f) {
    p = make_float3(x0, y0, 0.f);
    nrm = make_float3(0.f, 0.f, 1.f);
  } else {
    float3 nb;
    float3 o2 = make_float3(x0, y0, -g.hmax - 1e-4f);
    float t2 = tile_back_hit(g, o2, d, 1.f, &nb);
    if (t2 < 0.f) {
      out.side = 1;
      out.w = 1.f;
      return out;
    }
    p = o2 + t2 * d;
    nrm = -1.f * nb;
  }
  bool in_glass = false;
  for (;;) {
    if (e >= max_events) break;
    const float cos_i = -dot3(d, nrm);
    float4 u = draw4(px, sample, bounce, stream, (uint32_t)(e++ & 0xFF), lam, seed);
    const float n1 = in_glass ? n : 1.f;
    const float n2re = in_glass ? 1.f : n, n2im = in_glass ? 0.f : k;
    const float R = fresnel_R(cos_i, n1, n2re, n2im);
    const float eta = n1 / n2re;
    const float c2 = 1.f - eta * eta * (1.f - cos_i * cos_i);
    if (u.x < R || c2 <= 0.f) {
      d = d - (2.f * dot3(d, nrm)) * nrm;
    } else {
      d = normalize3(eta * d + (eta * cos_i - sqrtf(c2)) * nrm);
      in_glass = !in_glass;
    }
    if (!in_glass) {
      out.side = ((d.z > 0.f) == (d_in.z < 0.f)) ? 0 : 1;
      out.w = w;
      out.dir = d;
      out.events = e;
      return out;
    }
    p = p + (dot3(d, nrm) >= 0.f ? kTileEps : -kTileEps) * nrm;
    bool surfaced = false;
    while (!surfaced) {
      if (e >= max_events) {
        out.w = w;
        out.events = e;
        return out;
      }
      float4 us = draw4(px, sample, bounce, stream, (uint32_t)(e++ & 0xFF), lam, seed);
      float t_front = d.z > 0.f ? -p.z / d.z : CUDART_INF_F;
      float3 nb = make_float3(0.f, 0.f, 1.f);
      float t_back = tile_back_hit(g, p, d, fminf(t_front, 1.f), &nb);
      float t_surf = t_back >= 0.f ? t_back : t_front;
      float t_bub = sig > 0.f ? -logf(1.f - us.x) / sig : CUDART_INF_F;
      if (!(t_surf < CUDART_INF_F) && !(t_bub < CUDART_INF_F)) {
        out.w = w;
        out.events = e;
        return out;
      }
      if (t_bub < t_surf) {
        p = p + t_bub * d;
        w *= expf(-alpha * t_bub);
        out.bubbles++;
        float r = sqrtf(r_lo * r_lo + us.y * (r_hi * r_hi - r_lo * r_lo));
        float sin_i = sqrtf(us.z);
        float cos_i0 = sqrtf(fmaxf(0.f, 1.f - sin_i * sin_i));
        float3 t1, t2;
        onb(d, &t1, &t2);
        float sp, cp;
        sincospif(2.f * us.w, &sp, &cp);
        float3 rad = cp * t1 + sp * t2;
        float3 q = r * ((-cos_i0) * d + sin_i * rad);
        bool inside = false;
        for (;;) {
          if (e >= max_events) {
            out.w = w;
            out.events = e;
            return out;
          }
          float4 ub = draw4(px, sample, bounce, stream, (uint32_t)(e++ & 0xFF), lam, seed);
          float3 nn = (1.f / r) * q;
          float dn = dot3(d, nn);
          float ci = fabsf(dn);
          float3 nf = dn < 0.f ? nn : -1.f * nn;
          float m1 = inside ? 1.f : n;
          float m2re = inside ? n : 1.f, m2im = inside ? k : 0.f;
          float Rb = fresnel_R(ci, m1, m2re, m2im);
          float et = m1 / m2re;
          float cc = 1.f - et * et * (1.f - ci * ci);
          if (ub.x < Rb || cc <= 0.f) {
            d = d - (2.f * dot3(d, nf)) * nf;
          } else {
            d = normalize3(et * d + (et * ci - sqrtf(cc)) * nf);
            inside = !inside;
          }
          if (!inside) break;
          q = q + (-2.f * dot3(q, d)) * d;
        }
        continue;
      }
      p = p + t_surf * d;
      w *= expf(-alpha * t_surf);
      nrm = t_back >= 0.f ? nb : make_float3(0.f, 0.f, -1.f);
      p.x -= g.L * floorf(p.x / g.L);
      p.y -= g.L * floorf(p.y / g.L);
      surfaced = true;
    }
  }
  out.w = w;
  out.events = e;
  return out;
}

}  // namespace sdd
