// device_math.cuh -- per-ray arithmetic of the GB300 renderer: random numbers, the spectral
// material module, sampling and ray/primitive tests.  FP32 throughout, except the
// near-grazing slab series which is evaluated in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdd {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of the 4x32 Philox S-box.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform in [0,1) from the top 24 bits (exact in FP32).
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

enum Stream : uint32_t {
  STREAM_PATH = 0,
  STREAM_NEE = 1,
  STREAM_TILE = 2,
  STREAM_SHADOW_TILE = 3,
  STREAM_PHOTON = 4,       // photon emission and interactions (Sec. 3.2)
  STREAM_PHOTON_TILE = 5   // a photon's brute-force ray through a heterogeneous tile
};

// Four uniforms keyed by (pixel, sample, bounce | stream | group, lambda index).
__device__ __forceinline__ float4 draw4(uint32_t pixel, uint32_t sample, uint32_t bounce,
                                        uint32_t stream, uint32_t group, uint32_t lam,
                                        uint64_t seed) {
  uint4 o = philox4x32_10(make_uint4(pixel, sample, (bounce << 16) | (stream << 8) | group, lam),
                          (uint32_t)seed, (uint32_t)(seed >> 32));
  return make_float4(u01(o.x), u01(o.y), u01(o.z), u01(o.w));
}

// ------------------------------------------------------------------ small vector helpers
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 normalize3(float3 a) { return rsqrtf(dot3(a, a)) * a; }
__device__ __forceinline__ float comp3(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ------------------------------------------------------------------ double-float sums
// (hi, lo) += v without rounding error: Knuth's TwoSum (TAOCP vol. 2, 4.2.2) adds v to hi and
// keeps the rounding error of that addition in lo (explicitly rounded operations, so the
// compiler cannot reassociate them).  hi + lo then carries about 48 significant bits; a sum
// of a few dozen FP32 values of one sign is exact to well below FP32 rounding.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bv = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// ------------------------------------------------------------------ complex FP32
struct cf { float re, im; };
__device__ __forceinline__ cf cmul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cadd(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf csub(cf a, cf b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ float cnorm(cf a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cf cdiv_real(float x, cf b) {  // x / b
  float inv = x / cnorm(b);
  return {b.re * inv, -b.im * inv};
}
// Principal square root, computed without cancellation in either half-plane.
__device__ __forceinline__ cf csqrt(cf z) {
  float r = hypotf(z.re, z.im);
  if (r == 0.f) return {0.f, 0.f};
  if (z.re >= 0.f) {
    float re = sqrtf(0.5f * (r + z.re));
    return {re, z.im / (2.f * re)};
  }
  float im = copysignf(sqrtf(0.5f * (r - z.re)), z.im);
  return {fabsf(z.im) / (2.f * fabsf(im)), im};
}

// Fresnel reflectances |r_s|^2 and |r_p|^2 from a medium of real index n1 into one of
// complex index n2 = (n2re, n2im) (Eq. 1), cos(theta_t) from the complex Snell law.
__device__ __forceinline__ float2 fresnel_RsRp(float cos_i, float n1, float n2re, float n2im) {
  float sin2 = fmaxf(0.f, 1.f - cos_i * cos_i);
  cf n2 = {n2re, n2im};
  cf eta = cdiv_real(n1, n2);
  cf e2 = cmul(eta, eta);
  cf cos_t = csqrt({1.f - e2.re * sin2, -e2.im * sin2});
  cf n2ct = cmul(n2, cos_t);
  cf n1ci = {n1 * cos_i, 0.f};
  float Rs = cnorm(csub(n1ci, n2ct)) / cnorm(cadd(n1ci, n2ct));
  cf n2ci = {n2re * cos_i, n2im * cos_i};
  cf n1ct = {n1 * cos_t.re, n1 * cos_t.im};
  float Rp = cnorm(csub(n2ci, n1ct)) / cnorm(cadd(n2ci, n1ct));
  return make_float2(Rs, Rp);
}
// Unpolarised reflectance: the mean of the two.
__device__ __forceinline__ float fresnel_R(float cos_i, float n1, float n2re, float n2im) {
  const float2 r = fresnel_RsRp(cos_i, n1, n2re, n2im);
  return 0.5f * (r.x + r.y);
}

// The same in FP64 (near-grazing branch).
__device__ __forceinline__ double2 fresnel_RsRp_f64(double cos_i, double n1, double n2re, double n2im) {
  double sin2 = fmax(0.0, 1.0 - cos_i * cos_i);
  double den = n2re * n2re + n2im * n2im;
  double er = n1 * n2re / den, ei = -n1 * n2im / den;           // eta = n1 / n2
  double e2r = er * er - ei * ei, e2i = 2.0 * er * ei;          // eta^2
  double zr = 1.0 - e2r * sin2, zi = -e2i * sin2;
  double r = hypot(zr, zi), ctr, cti;
  if (r == 0.0) {
    ctr = cti = 0.0;
  } else if (zr >= 0.0) {
    ctr = sqrt(0.5 * (r + zr));
    cti = zi / (2.0 * ctr);
  } else {
    cti = copysign(sqrt(0.5 * (r - zr)), zi);
    ctr = fabs(zi) / (2.0 * fabs(cti));
  }
  double ar = n2re * ctr - n2im * cti, ai = n2re * cti + n2im * ctr;   // n2 cos_t
  double a1 = n1 * cos_i;
  double Rs = ((a1 - ar) * (a1 - ar) + ai * ai) / ((a1 + ar) * (a1 + ar) + ai * ai);
  double br = n2re * cos_i, bi = n2im * cos_i, cr = n1 * ctr, ci = n1 * cti;
  double Rp = ((br - cr) * (br - cr) + (bi - ci) * (bi - ci)) / ((br + cr) * (br + cr) + (bi + ci) * (bi + ci));
  return make_double2(Rs, Rp);
}

constexpr float kFourPi = 12.566370614359172f;
constexpr float kGrazingCos = 0.0625f;  // below this cosine the slab series runs in FP64

// Thin slab (air / glass / air): incoherent sum over internal reflections.
//   R_slab = R + (1-R)^2 R tau^2 / (1 - R^2 tau^2),  T_slab = (1-R)^2 tau / (1 - R^2 tau^2)
// with tau = exp(-4 pi k d / (lambda cos theta_t)).  pol = 0: one series on the unpolarised
// interface reflectance (R_s + R_p) / 2; pol = 1: s and p light do not mix at the parallel
// faces, so the series runs on R_s and on R_p and the two results are averaged.
__device__ __forceinline__ void slab_series_f64(double R, double tau, double* Rs_out, double* Ts_out) {
  double den = (1.0 - R * tau) * (1.0 + R * tau);
  *Rs_out = R + (1.0 - R) * (1.0 - R) * R * tau * tau / den;
  *Ts_out = (1.0 - R) * (1.0 - R) * tau / den;
}
// The FP32 branch, with air outside the slab (n1 = 1): eta = 1 / (n + ik) by one reciprocal of
// n^2 + k^2, the complex square root without the overflow guard of hypotf (|z| is of order
// one here), and its divisions and exponential through __fdividef and __expf (within a few
// ulp for these well-scaled operands; IEEE division took most of the slab's shading cost).
// Every product and sum is an explicitly rounded intrinsic, so the compiler cannot contract
// them differently in the kernels that inline this (the forms' per-path results stay
// bit-identical).
__device__ __forceinline__ void slab_RT_f32(float cos_i, float n, float k, float d, float lambda_nm,
                                            float* Rs_out, float* Ts_out, int pol) {
  const float sin2 = fmaxf(0.f, __fmaf_rn(-cos_i, cos_i, 1.f));
  const float inv_nk = __fdividef(1.f, __fmaf_rn(n, n, __fmul_rn(k, k)));
  const float er = __fmul_rn(n, inv_nk), ei = -__fmul_rn(k, inv_nk);  // eta = 1 / n2
  const float e2r = __fmaf_rn(er, er, -__fmul_rn(ei, ei)), e2i = __fmul_rn(__fmul_rn(2.f, er), ei);
  const float zr = __fmaf_rn(-e2r, sin2, 1.f), zi = -__fmul_rn(e2i, sin2);  // cos_t^2 = 1 - eta^2 sin^2
  const float rz = sqrtf(__fmaf_rn(zr, zr, __fmul_rn(zi, zi)));
  float ctr, cti;
  if (zr >= 0.f) {
    ctr = sqrtf(__fmul_rn(0.5f, __fadd_rn(rz, zr)));
    cti = ctr > 0.f ? __fdividef(zi, __fmul_rn(2.f, ctr)) : 0.f;
  } else {
    cti = copysignf(sqrtf(__fmul_rn(0.5f, __fsub_rn(rz, zr))), zi);
    ctr = __fdividef(fabsf(zi), __fmul_rn(2.f, fabsf(cti)));
  }
  const float ar = __fmaf_rn(n, ctr, -__fmul_rn(k, cti)), ai = __fmaf_rn(n, cti, __fmul_rn(k, ctr));  // n2 cos_t
  auto ratio = [](float xr, float xi, float yr, float yi) {  // |x - y|^2 / |x + y|^2
    const float mr = __fsub_rn(xr, yr), mi = __fsub_rn(xi, yi), pr = __fadd_rn(xr, yr), pi = __fadd_rn(xi, yi);
    return __fdividef(__fmaf_rn(mr, mr, __fmul_rn(mi, mi)), __fmaf_rn(pr, pr, __fmul_rn(pi, pi)));
  };
  const float Rsi = ratio(cos_i, 0.f, ar, ai);
  const float Rpi = ratio(__fmul_rn(n, cos_i), __fmul_rn(k, cos_i), ctr, cti);  // n2 cos_i against cos_t
  const float cos_t = sqrtf(__fsub_rn(1.f, __fdividef(sin2, __fmul_rn(n, n))));
  const float tau = __expf(-__fdividef(__fmul_rn(__fmul_rn(kFourPi, k), d), __fmul_rn(__fmul_rn(lambda_nm, 1e-9f), cos_t)));
  auto series = [tau](float R, float* Rsl, float* Tsl) {
    const float omr = __fsub_rn(1.f, R), rt = __fmul_rn(R, tau);
    const float g = __fdividef(__fmul_rn(__fmul_rn(omr, omr), tau), __fmul_rn(__fsub_rn(1.f, rt), __fadd_rn(1.f, rt)));
    *Rsl = __fmaf_rn(g, rt, R);
    *Tsl = g;
  };
  if (pol == 0) {
    series(__fmul_rn(0.5f, __fadd_rn(Rsi, Rpi)), Rs_out, Ts_out);
    return;
  }
  float R1, T1, R2, T2;
  series(Rsi, &R1, &T1);
  series(Rpi, &R2, &T2);
  *Rs_out = __fmul_rn(0.5f, __fadd_rn(R1, R2));
  *Ts_out = __fmul_rn(0.5f, __fadd_rn(T1, T2));
}

__device__ __forceinline__ void slab_RT(float cos_i, float n, float k, float d, float lambda_nm,
                                        float* Rs_out, float* Ts_out, int pol = 0) {
  if (cos_i < kGrazingCos) {
    double ci = cos_i;
    const double2 rsp = fresnel_RsRp_f64(ci, 1.0, n, k);
    double sin2t = (1.0 - ci * ci) / ((double)n * n);
    double cos_t = sqrt(1.0 - sin2t);
    double tau = exp(-12.566370614359172 * (double)k * (double)d / ((double)lambda_nm * 1e-9 * cos_t));
    double Rsl, Tsl;
    if (pol == 0) {
      slab_series_f64(0.5 * (rsp.x + rsp.y), tau, &Rsl, &Tsl);
    } else {
      double R1, T1, R2, T2;
      slab_series_f64(rsp.x, tau, &R1, &T1);
      slab_series_f64(rsp.y, tau, &R2, &T2);
      Rsl = 0.5 * (R1 + R2);
      Tsl = 0.5 * (T1 + T2);
    }
    *Rs_out = (float)Rsl;
    *Ts_out = (float)Tsl;
    return;
  }
  slab_RT_f32(cos_i, n, k, d, lambda_nm, Rs_out, Ts_out, pol);
}

// Beer-Lambert transmittance over `len` metres.
__device__ __forceinline__ float beer_lambert(float k, float len, float lambda_nm) {
  return expf(-kFourPi * k * len / (lambda_nm * 1e-9f));
}

// ------------------------------------------------------------------ sampling
// Orthonormal basis (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3* b1, float3* b2) {
  float sign = copysignf(1.f, n.z);
  float a = -1.f / (sign + n.z);
  float b = n.x * n.y * a;
  *b1 = make_float3(1.f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *b2 = make_float3(b, sign + n.y * n.y * a, -n.y);
}
// Cosine-weighted hemisphere about n (Malley).
__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2) {
  float3 b1, b2;
  onb(n, &b1, &b2);
  float r = sqrtf(u1), s, c;
  sincospif(2.f * u2, &s, &c);
  float z = sqrtf(fmaxf(0.f, 1.f - u1));
  return (r * c) * b1 + (r * s) * b2 + z * n;
}
// Uniform in the cone about s with 1 - cos(half angle) = h.
__device__ __forceinline__ float3 cone_dir(float3 s, float h, float u0, float u1) {
  float3 b1, b2;
  onb(s, &b1, &b2);
  float omc = u0 * h;
  float cos_t = 1.f - omc;
  float sin_t = sqrtf(fmaxf(0.f, omc * (2.f - omc)));
  float sp, cp;
  sincospif(2.f * u1, &sp, &cp);
  return (sin_t * cp) * b1 + (sin_t * sp) * b2 + cos_t * s;
}

// ------------------------------------------------------------------ ray setup
// Per-ray constants of the watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013)
// and of the slab box test.
struct RayPre {
  float3 o, inv, oinv;   // origin, 1/d, o/d
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  // An exactly zero component would make o/d and l/d infinite and their difference NaN in
  // the FMA form of the slab test; a 1e-12 stand-in keeps every term finite.
  float dx = fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x);
  float dy = fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y);
  float dz_ = fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z);
  r.inv = make_float3(1.f / dx, 1.f / dy, 1.f / dz_);
  r.oinv = make_float3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  float dz = comp3(d, kz);
  if (dz < 0.f) {
    int t = kx;
    kx = ky;
    ky = t;
  }
  r.kx = kx;
  r.ky = ky;
  r.kz = kz;
  r.Sx = comp3(d, kx) / dz;
  r.Sy = comp3(d, ky) / dz;
  r.Sz = 1.f / dz;
  return r;
}

// Watertight ray/triangle test.  Accepts t in (t_lo, t_hi]; returns t or -1 on a miss.
__device__ __forceinline__ float tri_hit(const RayPre& r, float4 v0, float4 v1, float4 v2, float t_lo,
                                         float t_hi) {
  float3 A = make_float3(v0.x - r.o.x, v0.y - r.o.y, v0.z - r.o.z);
  float3 B = make_float3(v1.x - r.o.x, v1.y - r.o.y, v1.z - r.o.z);
  float3 C = make_float3(v2.x - r.o.x, v2.y - r.o.y, v2.z - r.o.z);
  // Explicitly rounded products and differences: a contracted FMA would evaluate the
  // edge function of an edge shared by two triangles differently in each (one product
  // exact, the other rounded), and a ray through that edge could miss both.
  float Az = comp3(A, r.kz), Bz = comp3(B, r.kz), Cz = comp3(C, r.kz);
  float Ax = __fsub_rn(comp3(A, r.kx), __fmul_rn(r.Sx, Az)), Ay = __fsub_rn(comp3(A, r.ky), __fmul_rn(r.Sy, Az));
  float Bx = __fsub_rn(comp3(B, r.kx), __fmul_rn(r.Sx, Bz)), By = __fsub_rn(comp3(B, r.ky), __fmul_rn(r.Sy, Bz));
  float Cx = __fsub_rn(comp3(C, r.kx), __fmul_rn(r.Sx, Cz)), Cy = __fsub_rn(comp3(C, r.ky), __fmul_rn(r.Sy, Cz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
  float det = U + V + W;
  if (det == 0.f) return -1.f;
  float T = U * (r.Sz * Az) + V * (r.Sz * Bz) + W * (r.Sz * Cz);
  float t = T / det;
  return (t > t_lo && t <= t_hi) ? t : -1.f;
}

}  // namespace sdd
