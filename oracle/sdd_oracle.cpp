// sdd_oracle.cpp -- plain, slow, FP64 CPU reference of the spectral glass ray tracer.
//
// TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is checked
// against.  Only the test suite, the smoke check and the bench's CPU-baseline leg load
// it.  It shares no code, header, table or constant generator with the CUDA library;
// the two only see the same seeded input arrays.
//
// What it computes, and where the paper states it (arXiv:1912.05494):
//   * optical constants n~(lambda) = n + i k                            -- Sec. 2, Eq. 1
//   * rendering equation estimated per (pixel, sample, wavelength) path  -- Sec. 3, Eq. 2
//   * light-source sum (sun as a directional source, shadow rays)       -- Sec. 3, Eq. 3
//   * inverse ray tracing: one ray per pixel, closest hit, shadow rays to each light,
//     reflect/refract secondaries, stop at a bounce cap                  -- Sec. 3.1
//   * Monte Carlo path tracing with random rays from the pixels          -- Sec. 3.2
//   * 81-sample (or any) spectral sampling, wavelengths independent      -- Sec. 4
//   * glass refracts only (no scattering); per-tile maps of (n, k, d)    -- Sec. 6
// The paper gives no formula for Fresnel factors, absorption, slabs, sampling, camera or
// film; the readings used here are textbook optics and are listed in the design notes:
//   complex-index Fresnel (unpolarised mean of s and p), Snell with the real index,
//   Beer-Lambert exp(-4 pi k l / lambda), the incoherent infinite slab series,
//   Philox4x32-10 (Salmon et al., SC'11) counters keyed by (pixel, sample, bounce, lambda),
//   the Duff et al. (JCGT 2017) orthonormal basis, Malley cosine sampling, uniform cone
//   sampling of the sun disc, and the Wyman-Sloan-Shirley (JCGT 2013) CMF fit.
// The oracle traces the whole scene with one median-split BVH: it has no subdomains,
// because the domain decomposition (Sec. 5) must not change the image.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

using cd = std::complex<double>;
const double PI = 3.14159265358979323846;
const double INF = std::numeric_limits<double>::infinity();

struct V3 {
  double x, y, z;
};
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
V3 normalize(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }
double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11.
// Ten rounds of the 4x32 Philox S-box with key bumps between rounds.
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;  // golden-ratio Weyl increments
    k1 += 0xBB67AE85u;  // (sqrt(3)-1)
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// 24 high bits of a 32-bit draw, scaled to [0,1): exact in both float and double.
double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// The four uniforms of one draw group.  Counter = (pixel, sample, bounce<<16 | stream<<8 |
// group, lambda index), key = the 64-bit seed.
struct Draw { double u[4]; };
Draw draw(uint32_t pixel, uint32_t sample, uint32_t bounce, uint32_t stream, uint32_t group,
          uint32_t lam, uint64_t seed) {
  uint32_t ctr[4] = {pixel, sample, (bounce << 16) | (stream << 8) | group, lam};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  return Draw{{u01(o[0]), u01(o[1]), u01(o[2]), u01(o[3])}};
}
enum { STREAM_PATH = 0, STREAM_NEE = 1, STREAM_TILE = 2 };

// ---------------------------------------------------------------- optics
// Unpolarised Fresnel reflectance at a plane interface, incident medium with real index
// n1, transmitting medium with complex index n2 = n + i k (Eq. 1).  Textbook s/p
// amplitude coefficients with cos(theta_t) from the complex Snell law (principal
// square root).  Beyond the critical angle cos(theta_t) is imaginary and |r| = 1.
double fresnel_R(double cos_i, double n1, cd n2, double* Rs_out = nullptr,
                 double* Rp_out = nullptr) {
  double sin2_i = std::max(0.0, 1.0 - cos_i * cos_i);
  cd eta = n1 / n2;
  cd cos_t = std::sqrt(1.0 - eta * eta * sin2_i);
  cd rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
  cd rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
  double Rs = std::norm(rs), Rp = std::norm(rp);
  if (Rs_out) *Rs_out = Rs;
  if (Rp_out) *Rp_out = Rp;
  return 0.5 * (Rs + Rp);
}

// Beer-Lambert: intensity left after a path of length len_m in a medium of absorption
// index k; the absorption coefficient is 4 pi k / lambda.
double beer_lambert(double k, double len_m, double lambda_nm) {
  return std::exp(-4.0 * PI * k * len_m / (lambda_nm * 1e-9));
}

// Thin slab of thickness d: incoherent sum over all internal reflections.  R is the
// single-interface reflectance at the incidence angle, tau the one-way internal
// transmittance along the refracted direction (real-index Snell).
void slab_RT(double cos_i, double n, double k, double d_m, double lambda_nm, double* R_slab,
             double* T_slab) {
  double R = fresnel_R(cos_i, 1.0, cd(n, k));
  double sin2_t = (1.0 - cos_i * cos_i) / (n * n);
  double cos_t = std::sqrt(1.0 - sin2_t);
  double tau = beer_lambert(k, d_m / cos_t, lambda_nm);
  double denom = (1.0 - R * tau) * (1.0 + R * tau);  // 1 - R^2 tau^2
  *R_slab = R + (1.0 - R) * (1.0 - R) * R * tau * tau / denom;
  *T_slab = (1.0 - R) * (1.0 - R) * tau / denom;
}

// ---------------------------------------------------------------- CMF fit
// Wyman, Sloan, Shirley, "Simple Analytic Approximations to the CIE XYZ Color Matching
// Functions", JCGT 2(2), 2013: the multi-lobe piecewise-Gaussian fit of CIE 1931.
double pw_gauss(double x, double mu, double s1, double s2) {
  double t = (x - mu) / (x < mu ? s1 : s2);
  return std::exp(-0.5 * t * t);
}
void cmf_xyz(double lam, double out[3]) {
  out[0] = 1.056 * pw_gauss(lam, 599.8, 37.9, 31.0) + 0.362 * pw_gauss(lam, 442.0, 16.0, 26.7) -
           0.065 * pw_gauss(lam, 501.1, 20.4, 26.2);
  out[1] = 0.821 * pw_gauss(lam, 568.8, 46.9, 40.5) + 0.286 * pw_gauss(lam, 530.9, 16.3, 31.1);
  out[2] = 1.217 * pw_gauss(lam, 437.0, 11.8, 36.0) + 0.681 * pw_gauss(lam, 459.0, 26.0, 13.8);
}

// ---------------------------------------------------------------- sampling
// Orthonormal basis around a unit vector: Duff et al., "Building an Orthonormal Basis,
// Revisited", JCGT 6(1), 2017.
void onb(V3 n, V3* b1, V3* b2) {
  double sign = std::copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *b1 = {1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x};
  *b2 = {b, sign + n.y * n.y * a, -n.y};
}
// Cosine-weighted hemisphere direction about n (Malley's method).
V3 cosine_dir(V3 n, double u1, double u2) {
  V3 b1, b2;
  onb(n, &b1, &b2);
  double r = std::sqrt(u1), phi = 2.0 * PI * u2;
  double z = std::sqrt(std::max(0.0, 1.0 - u1));
  return r * std::cos(phi) * b1 + r * std::sin(phi) * b2 + z * n;
}
// Uniform direction inside the cone of half-angle alpha about s; h = 1 - cos(alpha).
V3 cone_dir(V3 s, double h, double u0, double u1) {
  V3 b1, b2;
  onb(s, &b1, &b2);
  double one_minus_cos = u0 * h;
  double cos_t = 1.0 - one_minus_cos;
  double sin_t = std::sqrt(std::max(0.0, one_minus_cos * (2.0 - one_minus_cos)));
  double phi = 2.0 * PI * u1;
  return sin_t * std::cos(phi) * b1 + sin_t * std::sin(phi) * b2 + cos_t * s;
}

// ---------------------------------------------------------------- geometry
// Moller-Trumbore ray/triangle test.  Edges are inclusive and widened by a barycentric
// tolerance far above double rounding (1e-12), so that a ray through an edge shared by two
// triangles always hits the surface (the plain test can reject it in both).
bool ray_triangle(V3 o, V3 d, V3 a, V3 b, V3 c, double* t_out) {
  const double tol = 1e-12;
  V3 e1 = b - a, e2 = c - a;
  V3 p = cross(d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  V3 s = o - a;
  double u = dot(s, p) * inv;
  if (u < -tol || u > 1.0 + tol) return false;
  V3 q = cross(s, e1);
  double v = dot(d, q) * inv;
  if (v < -tol || u + v > 1.0 + tol) return false;
  *t_out = dot(e2, q) * inv;
  return true;
}

struct Box {
  V3 lo{INF, INF, INF}, hi{-INF, -INF, -INF};
  void grow(V3 p) {
    lo = {std::min(lo.x, p.x), std::min(lo.y, p.y), std::min(lo.z, p.z)};
    hi = {std::max(hi.x, p.x), std::max(hi.y, p.y), std::max(hi.z, p.z)};
  }
  void grow(const Box& b) { grow(b.lo); grow(b.hi); }
};
// Slab test of a ray against a box over [t0, t1].
bool ray_box(V3 o, V3 d, const Box& b, double t0, double t1) {
  for (int a = 0; a < 3; ++a) {
    double inv = 1.0 / comp(d, a);
    double ta = (comp(b.lo, a) - comp(o, a)) * inv;
    double tb = (comp(b.hi, a) - comp(o, a)) * inv;
    if (std::isnan(ta) || std::isnan(tb)) {  // ray parallel to and on a slab plane
      if (comp(o, a) < comp(b.lo, a) || comp(o, a) > comp(b.hi, a)) return false;
      continue;
    }
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1) return false;
  }
  return true;
}

// Median-split BVH over all triangles of the scene (the oracle's own, deliberately simple).
struct BNode {
  Box box;
  int left = -1, right = -1, first = 0, count = 0;
};

struct Material {
  int kind;  // 0 solid dielectric, 1 thin slab, 2 heterogeneous tile, 3 diffuse, 4 opaque
  double thickness;
  std::vector<double> n, k, albedo;  // resampled to the render wavelengths
};
enum { MAT_SOLID = 0, MAT_SLAB = 1, MAT_TILE = 2, MAT_DIFFUSE = 3, MAT_OPAQUE = 4 };

struct Scene {
  std::vector<V3> v0, v1, v2, nrm;  // per triangle, and unit geometric normal
  std::vector<int> mat;
  std::vector<Material> mats;
  std::vector<BNode> nodes;
  std::vector<int> order;  // triangle indices referenced by the leaves
  std::vector<double> sky, sun;  // per render wavelength
  int sky_mode = 0;              // 0: every direction, 1: upper hemisphere (z > 0) only
  V3 sun_dir{0, 0, 1};
  double sun_h = 0.0;            // 1 - cos(sun half-angle)
  double eps = 1e-5;             // origin offset along the geometric normal (m)
};

int build_node(Scene& s, std::vector<int>& idx, int first, int count,
               const std::vector<V3>& cen) {
  BNode nd;
  for (int i = first; i < first + count; ++i) {
    int t = idx[i];
    nd.box.grow(s.v0[t]); nd.box.grow(s.v1[t]); nd.box.grow(s.v2[t]);
  }
  int me = (int)s.nodes.size();
  s.nodes.push_back(nd);
  if (count <= 4) {
    s.nodes[me].first = first;
    s.nodes[me].count = count;
    return me;
  }
  Box cb;
  for (int i = first; i < first + count; ++i) cb.grow(cen[idx[i]]);
  V3 ext = cb.hi - cb.lo;
  int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
  int mid = first + count / 2;
  std::nth_element(idx.begin() + first, idx.begin() + mid, idx.begin() + first + count,
                   [&](int a, int b) { return comp(cen[a], axis) < comp(cen[b], axis); });
  int l = build_node(s, idx, first, mid - first, cen);
  int r = build_node(s, idx, mid, first + count - mid, cen);
  s.nodes[me].left = l;
  s.nodes[me].right = r;
  return me;
}

struct Hit {
  double t = INF;
  int prim = -1;
};

// Closest hit over t in (0, t_max); equal distances go to the lower triangle index.
void closest_rec(const Scene& s, int ni, V3 o, V3 d, Hit& h) {
  const BNode& nd = s.nodes[ni];
  if (!ray_box(o, d, nd.box, 0.0, h.t)) return;
  if (nd.left < 0) {
    for (int i = nd.first; i < nd.first + nd.count; ++i) {
      int t = s.order[i];
      double th;
      if (ray_triangle(o, d, s.v0[t], s.v1[t], s.v2[t], &th) && th > 0.0 &&
          (th < h.t || (th == h.t && t < h.prim))) {
        h.t = th;
        h.prim = t;
      }
    }
    return;
  }
  closest_rec(s, nd.left, o, d, h);
  closest_rec(s, nd.right, o, d, h);
}
Hit closest(const Scene& s, V3 o, V3 d) {
  Hit h;
  if (!s.nodes.empty()) closest_rec(s, 0, o, d, h);
  return h;
}

// Transmittance of a shadow ray to infinity: thin-slab tiles multiply their slab
// transmittance, anything else blocks it (returns 0).
void shadow_rec(const Scene& s, int ni, V3 o, V3 d, int lam, double lambda_nm, double& T) {
  if (T == 0.0) return;
  const BNode& nd = s.nodes[ni];
  if (!ray_box(o, d, nd.box, 0.0, INF)) return;
  if (nd.left < 0) {
    for (int i = nd.first; i < nd.first + nd.count; ++i) {
      int t = s.order[i];
      double th;
      if (!(ray_triangle(o, d, s.v0[t], s.v1[t], s.v2[t], &th) && th > 0.0)) continue;
      const Material& m = s.mats[s.mat[t]];
      if (m.kind == MAT_SLAB) {
        double cos_i = std::fabs(dot(d, s.nrm[t]));
        double Rs, Ts;
        slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda_nm, &Rs, &Ts);
        T *= Ts;
      } else {
        T = 0.0;
        return;
      }
    }
    return;
  }
  shadow_rec(s, nd.left, o, d, lam, lambda_nm, T);
  shadow_rec(s, nd.right, o, d, lam, lambda_nm, T);
}
double shadow_T(const Scene& s, V3 o, V3 d, int lam, double lambda_nm) {
  double T = 1.0;
  if (!s.nodes.empty()) shadow_rec(s, 0, o, d, lam, lambda_nm, T);
  return T;
}

// Linear interpolation of a table over an ascending wavelength grid, clamped at the ends.
double interp(const float* grid, const float* val, int n, double lam) {
  if (n == 1 || lam <= grid[0]) return val[0];
  if (lam >= grid[n - 1]) return val[n - 1];
  int i = 0;
  while (grid[i + 1] < lam) ++i;
  double f = (lam - grid[i]) / ((double)grid[i + 1] - grid[i]);
  return (1.0 - f) * val[i] + f * val[i + 1];
}

// ---------------------------------------------------------------- path hash
// FNV-1a over the events of one Monte Carlo path; used only to count branch flips.
struct PathHash {
  uint32_t h = 0x811C9DC5u;
  void byte(uint32_t b) { h = (h ^ (b & 0xFFu)) * 0x01000193u; }
  void word(uint32_t w) { byte(w); byte(w >> 8); byte(w >> 16); byte(w >> 24); }
};
enum {
  EV_REFLECT = 0, EV_TRANSMIT = 1, EV_DIFFUSE = 2, EV_ABSORB = 3, EV_RR_KILL = 4,
  EV_DEPTH_CAP = 5, EV_ESCAPE = 6, EV_SHADOW_BLOCKED = 7, EV_SHADOW_OPEN = 8
};

// ---------------------------------------------------------------- camera
struct Camera {
  V3 pos, fwd, right, up;
  double tan_half, aspect, ortho_half;
  int width, height, ortho;
};
void camera_ray(const Camera& c, int px, double xi_x, double xi_y, V3* o, V3* d) {
  int i = px % c.width, j = px / c.width;
  double sx = ((i + 0.5 + xi_x) / c.width) * 2.0 - 1.0;
  double sy = 1.0 - ((j + 0.5 + xi_y) / c.height) * 2.0;
  if (c.ortho) {
    *o = c.pos + (sx * c.ortho_half * c.aspect) * c.right + (sy * c.ortho_half) * c.up;
    *d = c.fwd;
  } else {
    *o = c.pos;
    *d = normalize(c.fwd + (sx * c.tan_half * c.aspect) * c.right + (sy * c.tan_half) * c.up);
  }
}

// ---------------------------------------------------------------- shading helpers
double escape_radiance(const Scene& s, V3 d, int lam, bool sun_counted) {
  double L = (s.sky_mode == 0 || d.z > 0.0) ? s.sky[lam] : 0.0;
  if (!sun_counted && s.sun_h > 0.0) {
    V3 c = d - s.sun_dir;  // chord test: |d - s|^2 = 2 (1 - cos)
    if (dot(c, c) <= 2.0 * s.sun_h) L += s.sun[lam];
  }
  return L;
}
// Offset a point off the surface to the side the new direction points to.
V3 offset(const Scene& s, V3 p, V3 n, V3 dir) {
  return dot(dir, n) >= 0.0 ? p + s.eps * n : p - s.eps * n;
}
V3 reflect(V3 d, V3 n) { return d - (2.0 * dot(d, n)) * n; }
// A spawned ray starts eps off the surface along the normal; seen from the new ray, the
// surface plane lies eps / |n.d| behind its origin.  Absorption lengths inside glass are
// measured from that plane: l = t_hit + seg0.
double seg0_of(const Scene& s, V3 n, V3 dir) {
  return s.eps / std::max(std::fabs(dot(n, dir)), 1e-6);
}

struct RenderCtx {
  const Scene* s;
  const Camera* cam;
  const double* lambda_nm;
  int n_lambda, spp, max_depth, rr_start;
  uint64_t seed;
};

// Deterministic splitting (Sec. 3.1): the radiance carried back along one ray, spawning
// both the reflected and the transmitted child at every glass interface.  `vertex` is the
// number of surface interactions already made.
double trace_split(const RenderCtx& cx, V3 o, V3 d, double seg0, int vertex, int lam) {
  const Scene& s = *cx.s;
  double lambda = cx.lambda_nm[lam];
  Hit h = closest(s, o, d);
  if (h.prim < 0) return escape_radiance(s, d, lam, false);
  int v = vertex + 1;
  if (v > cx.max_depth) return 0.0;
  const Material& m = s.mats[s.mat[h.prim]];
  V3 p = o + h.t * d;
  V3 ng = s.nrm[h.prim];
  double cos_n = dot(d, ng);
  V3 nf = cos_n < 0.0 ? ng : -1.0 * ng;  // normal facing the incoming ray
  double cos_i = std::fabs(cos_n);
  switch (m.kind) {
    case MAT_SOLID: {
      bool inside = cos_n > 0.0;  // outward normals: leaving the glass body
      double atten = inside ? beer_lambert(m.k[lam], h.t + seg0, lambda) : 1.0;
      double n1 = inside ? m.n[lam] : 1.0;
      cd n2 = inside ? cd(1.0, 0.0) : cd(m.n[lam], m.k[lam]);
      double R = fresnel_R(cos_i, n1, n2);
      V3 dr = reflect(d, nf);
      double L = R * trace_split(cx, offset(s, p, ng, dr), dr, seg0_of(s, ng, dr), v, lam);
      double eta = n1 / std::real(n2);
      double c2 = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
      if (c2 > 0.0 && R < 1.0) {
        V3 dt = normalize(eta * d + (eta * cos_i - std::sqrt(c2)) * nf);
        L += (1.0 - R) * trace_split(cx, offset(s, p, ng, dt), dt, seg0_of(s, ng, dt), v, lam);
      }
      return atten * L;
    }
    case MAT_SLAB: {
      double Rs, Ts;
      slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda, &Rs, &Ts);
      V3 dr = reflect(d, nf);
      return Rs * trace_split(cx, offset(s, p, ng, dr), dr, seg0_of(s, ng, dr), v, lam) +
             Ts * trace_split(cx, offset(s, p, ng, d), d, seg0_of(s, ng, d), v, lam);
    }
    case MAT_DIFFUSE: {
      // Local illumination (Eq. 3): the sun as one directional source toward its centre,
      // irradiance L_sun * solid angle, seen through thin-slab glass.
      if (s.sun_h <= 0.0) return 0.0;
      double cl = dot(nf, s.sun_dir);
      if (cl <= 0.0) return 0.0;
      double T = shadow_T(s, offset(s, p, ng, s.sun_dir), s.sun_dir, lam, lambda);
      double omega = 2.0 * PI * s.sun_h;
      return m.albedo[lam] / PI * cl * s.sun[lam] * omega * T;
    }
    default:
      return 0.0;
  }
}

// Monte Carlo path (Sec. 3.2): one chain per (pixel, sample, wavelength) with the same
// Philox draws the GPU uses.  Returns the path radiance; optionally its event hash.
double trace_mc(const RenderCtx& cx, uint32_t px, uint32_t sample, int lam, uint32_t* hash_out) {
  const Scene& s = *cx.s;
  double lambda = cx.lambda_nm[lam];
  PathHash ph;
  Draw jit = draw(px, sample, 0, STREAM_PATH, 0, lam, cx.seed);  // pixel jitter
  V3 o, d;
  camera_ray(*cx.cam, (int)px, jit.u[0] - 0.5, jit.u[1] - 0.5, &o, &d);
  double thr = 1.0, L = 0.0, seg0 = 0.0;
  bool sun_counted = false;
  for (int v = 1;; ++v) {
    Hit h = closest(s, o, d);
    if (h.prim < 0) {
      L += thr * escape_radiance(s, d, lam, sun_counted);
      ph.word(0xFFFFFFFFu); ph.byte(EV_ESCAPE);
      break;
    }
    ph.word((uint32_t)h.prim);
    if (v > cx.max_depth) { ph.byte(EV_DEPTH_CAP); break; }
    const Material& m = s.mats[s.mat[h.prim]];
    V3 p = o + h.t * d;
    V3 ng = s.nrm[h.prim];
    double cos_n = dot(d, ng);
    V3 nf = cos_n < 0.0 ? ng : -1.0 * ng;
    double cos_i = std::fabs(cos_n);
    Draw u = draw(px, sample, (uint32_t)v, STREAM_PATH, 0, lam, cx.seed);
    V3 nd;
    int nee_event = -1;  // shadow outcome, hashed after the roulette decision of this vertex
    if (m.kind == MAT_SOLID) {
      bool inside = cos_n > 0.0;
      if (inside) thr *= beer_lambert(m.k[lam], h.t + seg0, lambda);
      double n1 = inside ? m.n[lam] : 1.0;
      cd n2 = inside ? cd(1.0, 0.0) : cd(m.n[lam], m.k[lam]);
      double R = fresnel_R(cos_i, n1, n2);
      double eta = n1 / std::real(n2);
      double c2 = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
      if (u.u[0] < R || c2 <= 0.0) {  // c2 <= 0: total internal reflection
        nd = reflect(d, nf);
        ph.byte(EV_REFLECT);
      } else {
        nd = normalize(eta * d + (eta * cos_i - std::sqrt(c2)) * nf);
        ph.byte(EV_TRANSMIT);
      }
      sun_counted = false;
    } else if (m.kind == MAT_SLAB) {
      double Rs, Ts;
      slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda, &Rs, &Ts);
      double P = Rs / (Rs + Ts);
      thr *= (Rs + Ts);
      if (u.u[0] < P) {
        nd = reflect(d, nf);
        sun_counted = false;
        ph.byte(EV_REFLECT);
      } else {
        nd = d;  // straight through; the NEE of an earlier diffuse vertex still covers it
        ph.byte(EV_TRANSMIT);
      }
    } else if (m.kind == MAT_DIFFUSE) {
      ph.byte(EV_DIFFUSE);
      if (s.sun_h > 0.0) {
        Draw un = draw(px, sample, (uint32_t)v, STREAM_NEE, 0, lam, cx.seed);
        V3 wl = cone_dir(s.sun_dir, s.sun_h, un.u[0], un.u[1]);
        double cl = dot(nf, wl);
        if (cl > 0.0) {
          double T = shadow_T(s, offset(s, p, ng, wl), wl, lam, lambda);
          double omega = 2.0 * PI * s.sun_h;
          L += thr * m.albedo[lam] / PI * cl * s.sun[lam] * omega * T;
          nee_event = T > 0.0 ? EV_SHADOW_OPEN : EV_SHADOW_BLOCKED;
        }
      }
      thr *= m.albedo[lam];
      nd = cosine_dir(nf, u.u[1], u.u[2]);
      sun_counted = true;
    } else {
      ph.byte(EV_ABSORB);
      break;
    }
    bool killed = false;
    if (v >= cx.rr_start) {
      double q = std::min(0.95, thr);
      if (u.u[3] >= q) {
        killed = true;
        ph.byte(EV_RR_KILL);
      } else {
        thr /= q;
      }
    }
    if (nee_event >= 0) ph.byte((uint32_t)nee_event);
    if (killed) break;
    o = offset(s, p, ng, nd);
    seg0 = seg0_of(s, ng, nd);
    d = nd;
  }
  if (hash_out) *hash_out = ph.h;
  return L;
}

}  // namespace

// ================================================================ C entry points
// Flat arrays in, doubles out.  All pointers are host memory owned by the caller.
extern "C" {

// Philox4x32-10 on n counters (4 words each) under one key (2 words).
void orc_philox(int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  for (int i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

// Single-interface Fresnel reflectance (unpolarised, and s / p separately).
void orc_fresnel(int n, const double* cos_i, const double* n1, const double* n2_re,
                 const double* n2_im, double* R, double* Rs, double* Rp) {
  for (int i = 0; i < n; ++i) R[i] = fresnel_R(cos_i[i], n1[i], cd(n2_re[i], n2_im[i]), Rs + i, Rp + i);
}

// Thin-slab reflectance and transmittance (air on both sides).
void orc_slab(int n, const double* cos_i, const double* nre, const double* k, const double* d_m,
              const double* lambda_nm, double* R_slab, double* T_slab) {
  for (int i = 0; i < n; ++i) slab_RT(cos_i[i], nre[i], k[i], d_m[i], lambda_nm[i], R_slab + i, T_slab + i);
}

double orc_beer_lambert(double k, double len_m, double lambda_nm) {
  return beer_lambert(k, len_m, lambda_nm);
}

void orc_cmf(int n, const double* lambda_nm, double* xyz) {
  for (int i = 0; i < n; ++i) cmf_xyz(lambda_nm[i], xyz + 3 * i);
}

// Sampling helpers exposed for invariance tests: cosine and cone directions.
void orc_cosine_dir(int n, const double* nrm, const double* u, double* out) {
  for (int i = 0; i < n; ++i) {
    V3 r = cosine_dir({nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]}, u[2 * i], u[2 * i + 1]);
    out[3 * i] = r.x; out[3 * i + 1] = r.y; out[3 * i + 2] = r.z;
  }
}
void orc_cone_dir(int n, const double* axis, double h, const double* u, double* out) {
  for (int i = 0; i < n; ++i) {
    V3 r = cone_dir({axis[3 * i], axis[3 * i + 1], axis[3 * i + 2]}, h, u[2 * i], u[2 * i + 1]);
    out[3 * i] = r.x; out[3 * i + 1] = r.y; out[3 * i + 2] = r.z;
  }
}

struct OrcScene {
  int n_vertices;
  const float* vertices;      // [V][3]
  int n_triangles;
  const uint32_t* indices;    // [T][3]
  const uint16_t* tri_material;  // [T]
  int n_materials;
  const int32_t* mat_kind;    // [M]
  const float* mat_thickness; // [M] metres
  int n_table;                // wavelength table shared by all material / light tables
  const float* table_nm;      // [n_table]
  const float* mat_n;         // [M][n_table]
  const float* mat_k;         // [M][n_table]
  const float* mat_albedo;    // [M][n_table]
  const float* sky;           // [n_table]
  int sky_mode;               // 0 every direction, 1 upper hemisphere only
  float sun_dir[3];           // unit vector toward the sun
  float sun_half_angle;       // radians; <= 0 means no sun
  const float* sun;           // [n_table] or NULL
  float ray_eps;              // offset of spawned origins along the normal (m)
};

struct OrcCamera {
  float pos[3], look_at[3], up[3];
  float vfov_deg;
  int width, height;
  int ortho;           // 1: orthographic
  float ortho_height;  // full image height in metres (orthographic only)
};

struct OrcOpts {
  int n_lambda;
  const float* lambda_nm;
  int spp;
  uint64_t seed;
  int max_depth;
  int mode;            // 0 deterministic splitting, 1 Monte Carlo
  int rr_start_depth;
  int n_pixels;        // number of entries in `pixels`; 0 = every pixel in row-major order
  const int32_t* pixels;
  int n_threads;       // 0 = hardware concurrency
};

struct OrcHandle {
  Scene s;
  int n_table = 0;
  std::vector<float> table_nm;
  std::vector<float> mat_n, mat_k, mat_alb, sky, sun;
  std::vector<int> mat_kind;
  std::vector<float> mat_thick;
};

void* orc_scene_create(const OrcScene* d) {
  OrcHandle* h = new OrcHandle;
  Scene& s = h->s;
  for (int t = 0; t < d->n_triangles; ++t) {
    V3 p[3];
    for (int c = 0; c < 3; ++c) {
      uint32_t vi = d->indices[3 * t + c];
      p[c] = {d->vertices[3 * vi], d->vertices[3 * vi + 1], d->vertices[3 * vi + 2]};
    }
    s.v0.push_back(p[0]); s.v1.push_back(p[1]); s.v2.push_back(p[2]);
    s.nrm.push_back(normalize(cross(p[1] - p[0], p[2] - p[0])));
    s.mat.push_back(d->tri_material[t]);
  }
  h->n_table = d->n_table;
  h->table_nm.assign(d->table_nm, d->table_nm + d->n_table);
  size_t mt = (size_t)d->n_materials * d->n_table;
  h->mat_n.assign(d->mat_n, d->mat_n + mt);
  h->mat_k.assign(d->mat_k, d->mat_k + mt);
  h->mat_alb.assign(d->mat_albedo, d->mat_albedo + mt);
  h->mat_kind.assign(d->mat_kind, d->mat_kind + d->n_materials);
  h->mat_thick.assign(d->mat_thickness, d->mat_thickness + d->n_materials);
  h->sky.assign(d->sky, d->sky + d->n_table);
  if (d->sun) h->sun.assign(d->sun, d->sun + d->n_table);
  s.sky_mode = d->sky_mode;
  s.sun_dir = normalize({d->sun_dir[0], d->sun_dir[1], d->sun_dir[2]});
  double ha = d->sun_half_angle;
  s.sun_h = (d->sun && ha > 0.0) ? 2.0 * std::sin(0.5 * ha) * std::sin(0.5 * ha) : 0.0;
  s.eps = d->ray_eps;
  std::vector<int> idx(d->n_triangles);
  std::vector<V3> cen(d->n_triangles);
  for (int t = 0; t < d->n_triangles; ++t) {
    idx[t] = t;
    cen[t] = (1.0 / 3.0) * (s.v0[t] + s.v1[t] + s.v2[t]);
  }
  if (d->n_triangles > 0) build_node(s, idx, 0, d->n_triangles, cen);
  s.order = idx;
  return h;
}

void orc_scene_destroy(void* h) { delete (OrcHandle*)h; }

// Closest hit of n rays (origin, direction; t in (0, inf)): by brute force over every
// triangle, or through the oracle's BVH.  prim = -1 on a miss.
void orc_closest(void* hp, int n, const double* org, const double* dir, int brute, double* t_out,
                 int32_t* prim_out) {
  const Scene& s = ((OrcHandle*)hp)->s;
  for (int i = 0; i < n; ++i) {
    V3 o{org[3 * i], org[3 * i + 1], org[3 * i + 2]}, d{dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]};
    Hit h;
    if (brute) {
      for (int t = 0; t < (int)s.v0.size(); ++t) {
        double th;
        if (ray_triangle(o, d, s.v0[t], s.v1[t], s.v2[t], &th) && th > 0.0 &&
            (th < h.t || (th == h.t && t < h.prim))) {
          h.t = th;
          h.prim = t;
        }
      }
    } else {
      h = closest(s, o, d);
    }
    t_out[i] = h.prim < 0 ? INF : h.t;
    prim_out[i] = h.prim;
  }
}

// Render the listed pixels.  film[pixel][lambda] is the mean over samples; path_L and
// path_hash ([pixel][sample][lambda], optional) hold every path's radiance and event hash
// (Monte Carlo only).  Returns 0, or -1 on bad arguments.
int orc_render(void* hp, const OrcCamera* cam_in, const OrcOpts* op, double* film,
               double* path_L, uint32_t* path_hash) {
  OrcHandle* h = (OrcHandle*)hp;
  Scene& s = h->s;
  if (op->n_lambda <= 0 || op->spp <= 0 || op->max_depth < 0) return -1;
  if (op->mode == 0 && op->spp != 1) return -1;
  // Resample every table to the render wavelengths.
  s.mats.assign(h->mat_kind.size(), Material{});
  for (size_t m = 0; m < h->mat_kind.size(); ++m) {
    Material& mm = s.mats[m];
    mm.kind = h->mat_kind[m];
    mm.thickness = h->mat_thick[m];
    for (int l = 0; l < op->n_lambda; ++l) {
      double lam = op->lambda_nm[l];
      const size_t o = m * (size_t)h->n_table;
      mm.n.push_back(interp(h->table_nm.data(), h->mat_n.data() + o, h->n_table, lam));
      mm.k.push_back(interp(h->table_nm.data(), h->mat_k.data() + o, h->n_table, lam));
      mm.albedo.push_back(interp(h->table_nm.data(), h->mat_alb.data() + o, h->n_table, lam));
    }
  }
  s.sky.clear(); s.sun.clear();
  for (int l = 0; l < op->n_lambda; ++l) {
    s.sky.push_back(interp(h->table_nm.data(), h->sky.data(), h->n_table, op->lambda_nm[l]));
    s.sun.push_back(h->sun.empty() ? 0.0
                                   : interp(h->table_nm.data(), h->sun.data(), h->n_table, op->lambda_nm[l]));
  }
  Camera cam;
  V3 pos{cam_in->pos[0], cam_in->pos[1], cam_in->pos[2]};
  V3 at{cam_in->look_at[0], cam_in->look_at[1], cam_in->look_at[2]};
  V3 up{cam_in->up[0], cam_in->up[1], cam_in->up[2]};
  cam.pos = pos;
  cam.fwd = normalize(at - pos);
  cam.right = normalize(cross(cam.fwd, up));
  cam.up = cross(cam.right, cam.fwd);
  cam.tan_half = std::tan(0.5 * cam_in->vfov_deg * PI / 180.0);
  cam.aspect = (double)cam_in->width / cam_in->height;
  cam.ortho = cam_in->ortho;
  cam.ortho_half = 0.5 * cam_in->ortho_height;
  cam.width = cam_in->width;
  cam.height = cam_in->height;
  std::vector<double> lam_d(op->lambda_nm, op->lambda_nm + op->n_lambda);
  RenderCtx cx{&s, &cam, lam_d.data(), op->n_lambda, op->spp, op->max_depth, op->rr_start_depth, op->seed};

  int npx = op->n_pixels > 0 ? op->n_pixels : cam.width * cam.height;
  int nth = op->n_threads > 0 ? op->n_threads : (int)std::thread::hardware_concurrency();
  if (nth < 1) nth = 1;
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= npx) break;
      uint32_t px = op->n_pixels > 0 ? (uint32_t)op->pixels[i] : (uint32_t)i;
      V3 o, d;
      for (int l = 0; l < op->n_lambda; ++l) {
        double sum = 0.0;
        for (int sp = 0; sp < op->spp; ++sp) {
          double L;
          uint32_t hh = 0;
          if (op->mode == 0) {
            camera_ray(cam, (int)px, 0.0, 0.0, &o, &d);
            L = trace_split(cx, o, d, 0.0, 0, l);
          } else {
            L = trace_mc(cx, px, (uint32_t)sp, l, &hh);
          }
          size_t slot = ((size_t)i * op->spp + sp) * op->n_lambda + l;
          if (path_L) path_L[slot] = L;
          if (path_hash) path_hash[slot] = hh;
          sum += L;
        }
        film[(size_t)i * op->n_lambda + l] = sum / op->spp;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  return 0;
}

// XYZ of spectral images: X = sum_i L_i xbar(l_i) w_i / sum_i ybar(l_i) w_i, trapezoid
// weights w_i over the wavelength grid.
void orc_xyz(int n_px, int n_lambda, const float* lambda_nm, const double* film, double* xyz) {
  std::vector<double> w(n_lambda, 1.0), cmf(3 * n_lambda);
  if (n_lambda > 1) {
    for (int l = 0; l < n_lambda; ++l) {
      double lo = lambda_nm[l > 0 ? l - 1 : l], hi = lambda_nm[l + 1 < n_lambda ? l + 1 : l];
      w[l] = 0.5 * (hi - lo);
    }
  }
  double ysum = 0.0;
  for (int l = 0; l < n_lambda; ++l) {
    cmf_xyz(lambda_nm[l], &cmf[3 * l]);
    ysum += cmf[3 * l + 1] * w[l];
  }
  for (int p = 0; p < n_px; ++p)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int l = 0; l < n_lambda; ++l) acc += film[(size_t)p * n_lambda + l] * cmf[3 * l + c] * w[l];
      xyz[3 * p + c] = acc / ysum;
    }
}

int orc_hardware_threads(void) { return (int)std::thread::hardware_concurrency(); }

}  // extern "C"
