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
V3 reflect(V3 d, V3 n) { return d - (2.0 * dot(d, n)) * n; }

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
enum { STREAM_PATH = 0, STREAM_NEE = 1, STREAM_TILE = 2, STREAM_SHADOW_TILE = 3, STREAM_PHOTON = 4,
       STREAM_PHOTON_TILE = 5 };

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

// Thin slab of thickness d: incoherent sum over all internal reflections, for an interface
// reflectance R and the one-way internal transmittance tau:
//   R_slab = R + (1 - R)^2 R tau^2 / (1 - R^2 tau^2),  T_slab = (1 - R)^2 tau / (1 - R^2 tau^2).
void slab_series(double R, double tau, double* R_slab, double* T_slab) {
  double denom = (1.0 - R * tau) * (1.0 + R * tau);  // 1 - R^2 tau^2
  *R_slab = R + (1.0 - R) * (1.0 - R) * R * tau * tau / denom;
  *T_slab = (1.0 - R) * (1.0 - R) * tau / denom;
}

// The slab at incidence cos_i (Sec. 2, Eq. 1 optical constants; tau along the refracted
// direction, real-index Snell).  pol = 0: the series runs once on the unpolarised
// interface reflectance (Rs + Rp) / 2; pol = 1: s and p light do not mix at the slab's
// parallel faces, so the series runs for each polarisation on its own reflectance and the
// two results are averaged (unpolarised light is half s, half p).
void slab_RT(double cos_i, double n, double k, double d_m, double lambda_nm, double* R_slab,
             double* T_slab, int pol = 0) {
  double Rs, Rp;
  double R = fresnel_R(cos_i, 1.0, cd(n, k), &Rs, &Rp);
  double sin2_t = (1.0 - cos_i * cos_i) / (n * n);
  double cos_t = std::sqrt(1.0 - sin2_t);
  double tau = beer_lambert(k, d_m / cos_t, lambda_nm);
  if (pol == 0) {
    slab_series(R, tau, R_slab, T_slab);
    return;
  }
  double Rss, Tss, Rsp, Tsp;
  slab_series(Rs, tau, &Rss, &Tss);
  slab_series(Rp, tau, &Rsp, &Tsp);
  *R_slab = 0.5 * (Rss + Rsp);
  *T_slab = 0.5 * (Tss + Tsp);
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

// ---------------------------------------------------------------- heterogeneous tiles
// A medieval glass tile with non-uniform thickness and air micro-bubbles (Sec. 1: "non
// uniform thickness and ... micro particles of air inside the tiles"; Sec. 6: scattering as
// future work).  Model (readings, the paper gives none):
//   * periodic square tile of side L, flat front face z = 0, back face z = -h(x, y);
//   * h = clamp(d_mean + A (n(x, y) - 1/2), 2 mm, 5 mm) with n = 2/3 v(L/10) + 1/3 v(L/20),
//     v = value noise with smoothstep interpolation of lattice values drawn from Philox;
//   * the back face is the G x G triangulated height field through h at the grid vertices;
//   * bubbles form a Poisson process of density rho in the glass, radii log-uniform in
//     [10, 100] um: the free path to the next bubble is exponential with rate rho sigma,
//     sigma = pi E[r^2]; a hit bubble's radius is drawn with weight r^2, the impact point
//     uniformly over its cross-section, and the outgoing direction follows the exact sphere
//     optics (reflections and refractions at its surface); at the tile's scale (mm) the
//     bubble is a point: the encounter does not displace the ray;
//   * complex Fresnel, Snell and Beer-Lambert as for the other glass; every interaction
//     draws its own four uniforms on the tile stream;
//   * a ray leaves through the front face (reflected side) or the back face (transmitted
//     side) and does not re-enter; more than max_events interactions absorb it.
struct TileParams {
  double d_mean, amp, rho;
  uint32_t seed;
};

double tile_lattice(uint32_t seed, int ix, int iy, int oct) {
  uint32_t ctr[4] = {(uint32_t)ix, (uint32_t)iy, (uint32_t)oct, seed};
  uint32_t key[2] = {0x5EED7113u, 0u};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  return u01(o[0]);
}

double tile_value_noise(uint32_t seed, double x, double y, double L, int cells, int oct) {
  double gx = x / L * cells, gy = y / L * cells;
  double fx0 = std::floor(gx), fy0 = std::floor(gy);
  double fx = gx - fx0, fy = gy - fy0;
  int ix = ((int)fx0 % cells + cells) % cells, iy = ((int)fy0 % cells + cells) % cells;
  int jx = (ix + 1) % cells, jy = (iy + 1) % cells;
  double sx = fx * fx * (3.0 - 2.0 * fx), sy = fy * fy * (3.0 - 2.0 * fy);
  double a = tile_lattice(seed, ix, iy, oct), b = tile_lattice(seed, jx, iy, oct);
  double c = tile_lattice(seed, ix, jy, oct), d = tile_lattice(seed, jx, jy, oct);
  return (1 - sy) * ((1 - sx) * a + sx * b) + sy * ((1 - sx) * c + sx * d);
}

double tile_thickness(const TileParams& tp, double x, double y, double L) {
  double n = (2.0 / 3.0) * tile_value_noise(tp.seed, x, y, L, 10, 0) +
             (1.0 / 3.0) * tile_value_noise(tp.seed, x, y, L, 20, 1);
  double h = tp.d_mean + tp.amp * (n - 0.5);
  return std::min(0.005, std::max(0.002, h));
}

struct TileGeom {
  int G;
  double L;
  const double* h;  // [(G+1) * (G+1)] thickness at the grid vertices, row j, column i
  double hmin, hmax;
};

// Back-face triangles of cell (ci, cj) in unwrapped cell coordinates.
void tile_cell_tris(const TileGeom& g, long ci, long cj, V3 tri[2][3]) {
  long wi = ((ci % g.G) + g.G) % g.G, wj = ((cj % g.G) + g.G) % g.G;
  double cs = g.L / g.G;
  double x0 = ci * cs, y0 = cj * cs;
  auto H = [&](long i, long j) { return g.h[(size_t)j * (g.G + 1) + i]; };
  V3 p00{x0, y0, -H(wi, wj)}, p10{x0 + cs, y0, -H(wi + 1, wj)};
  V3 p01{x0, y0 + cs, -H(wi, wj + 1)}, p11{x0 + cs, y0 + cs, -H(wi + 1, wj + 1)};
  tri[0][0] = p00; tri[0][1] = p10; tri[0][2] = p11;
  tri[1][0] = p00; tri[1][1] = p11; tri[1][2] = p01;
}

// First hit of the back face along o + t d, t in (0, t_max], walking the grid cells the
// ray's xy projection crosses (at most max_cells).  Returns t or -1; n_out = unit normal
// of the hit triangle pointing into the glass (+z side).
double tile_back_hit(const TileGeom& g, V3 o, V3 d, double t_max, int max_cells, V3* n_out) {
  double cs = g.L / g.G;
  long ci = (long)std::floor(o.x / cs), cj = (long)std::floor(o.y / cs);
  int sx = d.x > 0 ? 1 : (d.x < 0 ? -1 : 0), sy = d.y > 0 ? 1 : (d.y < 0 ? -1 : 0);
  double tdx = sx ? cs / std::fabs(d.x) : INF, tdy = sy ? cs / std::fabs(d.y) : INF;
  double tx = sx > 0 ? ((ci + 1) * cs - o.x) / d.x : (sx < 0 ? (ci * cs - o.x) / d.x : INF);
  double ty = sy > 0 ? ((cj + 1) * cs - o.y) / d.y : (sy < 0 ? (cj * cs - o.y) / d.y : INF);
  double t_in = 0.0;
  for (int step = 0; step < max_cells && t_in <= t_max; ++step) {
    double t_out = std::min(std::min(tx, ty), t_max);
    double z0 = o.z + d.z * t_in, z1 = o.z + d.z * t_out;
    if (std::min(z0, z1) <= -g.hmin) {  // the ray reaches the band of the back face here
      V3 tri[2][3];
      tile_cell_tris(g, ci, cj, tri);
      double best = -1.0;
      V3 bn{0, 0, 1};
      for (int k = 0; k < 2; ++k) {
        double t;
        if (ray_triangle(o, d, tri[k][0], tri[k][1], tri[k][2], &t) && t > 0.0 && t <= t_max &&
            (best < 0.0 || t < best)) {
          best = t;
          bn = normalize(cross(tri[k][1] - tri[k][0], tri[k][2] - tri[k][0]));
        }
      }
      if (best >= 0.0) {
        if (bn.z < 0) bn = -1.0 * bn;
        *n_out = bn;
        return best;
      }
    }
    if (tx < ty) { ci += sx; t_in = tx; tx += tdx; }
    else { cj += sy; t_in = ty; ty += tdy; }
  }
  return -1.0;
}

// Exact optics of one air bubble in the glass (Sec. 1: air micro-bubbles; Fresnel and Snell
// at each of its surfaces, the glass of index n + ik outside, air inside).  The ray with
// direction *d meets a sphere of radius r at impact parameter b = sin_i * r, displaced from
// the centre line toward the unit vector rad (normal to *d).  At every surface met,
// choice() gives the uniform that picks reflection (u < R) or refraction; inside the air the
// ray crosses the chord to the next surface point.  choice() returns a negative value when
// the event cap is reached: the function then returns false (the ray is lost in the bubble).
// On true, *d holds the direction with which the ray leaves the sphere into the glass.
template <class Choice>
bool bubble_scatter(V3* dp, V3 rad, double sin_i, double r, double n, double k, Choice&& choice) {
  V3 d = *dp;
  double cos_i0 = std::sqrt(std::max(0.0, 1.0 - sin_i * sin_i));
  // the sphere in its own frame: q is the current point relative to the centre
  V3 q = r * ((-cos_i0) * d + sin_i * rad);  // entry point (outward normal q / r)
  bool inside = false;                          // inside the bubble (air)
  for (;;) {
    double u = choice();
    if (u < 0.0) { *dp = d; return false; }
    V3 nn = (1.0 / r) * q;
    double ci = std::fabs(dot(d, nn));
    V3 nf = dot(d, nn) < 0 ? nn : -1.0 * nn;  // facing the incoming ray
    double m1 = inside ? 1.0 : n;
    cd m2 = inside ? cd(n, k) : cd(1.0, 0.0);
    double Rb = fresnel_R(ci, m1, m2);
    double et = m1 / std::real(m2);
    double cc = 1.0 - et * et * (1.0 - ci * ci);
    if (u < Rb || cc <= 0.0) {
      d = reflect(d, nf);
    } else {
      d = normalize(et * d + (et * ci - std::sqrt(cc)) * nf);
      inside = !inside;
    }
    if (!inside) break;           // back in the glass, leaving the sphere
    q = q + (-2.0 * dot(q, d)) * d;  // across the chord to the next point on the sphere
  }
  *dp = d;
  return true;
}

struct TileRay {
  int side;     // 0 reflected (front), 1 transmitted (back), 2 absorbed (event cap)
  double w;     // throughput
  V3 dir;       // exit direction (tile frame)
  int bubbles;  // bubble encounters
  int events;
};

// Trace one ray through the tile.  (x0, y0): entry point; d: direction in the tile frame
// (d.z < 0 enters through the front, d.z > 0 through the back); draws are keyed
// (pixel, sample, bounce<<16 | 2<<8 | event, lam).
TileRay tile_trace(const TileGeom& g, const TileParams& tp, double x0, double y0, V3 d, double n, double k,
                   double lambda_nm, uint32_t px, uint32_t sample, uint32_t bounce, uint32_t lam, uint64_t seed,
                   int max_events, uint32_t stream = STREAM_TILE) {
  const double eps = 1e-7, r_lo = 10e-6, r_hi = 100e-6;
  const double Er2 = (r_hi * r_hi - r_lo * r_lo) / (2.0 * std::log(r_hi / r_lo));
  const double sig = tp.rho * PI * Er2;  // bubble encounters per metre
  const double alpha = 4.0 * PI * k / (lambda_nm * 1e-9);
  TileRay out{2, 0.0, d, 0, 0};
  const V3 d_in = d;
  double w = 1.0;
  int e = 0;
  auto next_u = [&]() { return draw(px, sample, bounce, stream, (uint32_t)(e++ & 0xFF), lam, seed); };
  // entry interface: air -> glass at the front plane or the back face below the entry point
  V3 p, nrm;
  if (d.z < 0) {
    p = {x0, y0, 0.0};
    nrm = {0, 0, 1};
  } else {
    // start below the back face on the vertical through the entry point and walk along d
    V3 nb;
    V3 o2 = {x0, y0, -g.hmax - 1e-4};
    double t2 = tile_back_hit(g, o2, d, 1.0, 4096, &nb);
    if (t2 < 0) { out.side = 1; out.w = 1.0; out.dir = d; return out; }  // passed under the tile
    p = o2 + t2 * d;
    nrm = -1.0 * nb;  // facing the incoming ray (below)
  }
  bool in_glass = false;
  for (;;) {
    if (e >= max_events) { out.side = 2; out.w = w; out.events = e; return out; }
    // interface at p with normal nrm facing the incoming ray
    double cos_i = -dot(d, nrm);
    Draw u = next_u();
    double n1 = in_glass ? n : 1.0;
    cd n2 = in_glass ? cd(1.0, 0.0) : cd(n, k);
    double R = fresnel_R(cos_i, n1, n2);
    double eta = n1 / std::real(n2);
    double c2 = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
    if (u.u[0] < R || c2 <= 0.0) {
      d = reflect(d, nrm);
    } else {
      d = normalize(eta * d + (eta * cos_i - std::sqrt(c2)) * nrm);
      in_glass = !in_glass;
    }
    if (!in_glass) {  // left the glass (or never entered): reflected if back on the incident side
      out.side = ((d.z > 0) == (d_in.z < 0)) ? 0 : 1;
      out.w = w;
      out.dir = d;
      out.events = e;
      return out;
    }
    p = p + (dot(d, nrm) >= 0 ? eps : -eps) * nrm;  // step off the surface into the glass
    // the segment inside the glass: front plane, back face, or a bubble
    for (;;) {
      if (e >= max_events) { out.side = 2; out.w = w; out.events = e; return out; }
      Draw us = next_u();
      double t_front = d.z > 0 ? -p.z / d.z : INF;
      V3 nb{0, 0, 1};
      double t_back = tile_back_hit(g, p, d, std::min(t_front, 1.0), 4096, &nb);
      double t_surf = t_back >= 0 ? t_back : t_front;
      double t_bub = sig > 0 ? -std::log(1.0 - us.u[0]) / sig : INF;
      if (!(t_surf < INF) && !(t_bub < INF)) { out.side = 2; out.w = w; out.events = e; return out; }
      if (t_bub < t_surf) {
        // bubble encounter: exact sphere optics, then continue in the glass (the bubble is
        // not geometry: nothing of it can be hit again)
        p = p + t_bub * d;
        w *= std::exp(-alpha * t_bub);
        out.bubbles++;
        double r = std::sqrt(r_lo * r_lo + us.u[1] * (r_hi * r_hi - r_lo * r_lo));
        double sin_i = std::sqrt(us.u[2]);  // impact parameter / r, uniform over the disc
        V3 t1, t2;
        onb(d, &t1, &t2);
        double phi = 2.0 * PI * us.u[3];
        V3 rad = std::cos(phi) * t1 + std::sin(phi) * t2;
        auto choice = [&]() -> double {
          if (e >= max_events) return -1.0;
          return next_u().u[0];
        };
        if (!bubble_scatter(&d, rad, sin_i, r, n, k, choice)) { out.side = 2; out.w = w; out.events = e; return out; }
        // bubbles (<= 100 um) are point scatterers at the scale of the tile: the ray leaves
        // the encounter where it met it, with the direction the sphere optics gave
        continue;
      }
      // surface hit
      p = p + t_surf * d;
      w *= std::exp(-alpha * t_surf);
      nrm = t_back >= 0 ? nb : V3{0, 0, -1};  // normal facing the ray arriving from the glass
      // re-wrap the position into the base tile
      p.x -= g.L * std::floor(p.x / g.L);
      p.y -= g.L * std::floor(p.y / g.L);
      break;
    }
  }
}

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
  int slab_pol = 0;              // thin-slab series: 0 unpolarised interface R, 1 per polarisation
  // heterogeneous tiles: per material the tile index (-1 for other kinds)
  std::vector<int> mat_tile;
  std::vector<TileParams> tiles;
  std::vector<std::vector<double>> tile_h;  // per tile, (G+1)^2 vertex thicknesses
  std::vector<TileGeom> tile_geom;
  int tile_G = 64;
  double tile_L = 0.1;
};

// Tile-frame coordinates of a hit: the tile's front face is the +n side of the geometric
// normal; (t1, t2) = Duff basis of n; positions wrap with the tile period.
void tile_frame(const Scene& s, V3 p, V3 n, V3 d, double* x, double* y, V3* dl, V3* t1, V3* t2) {
  onb(n, t1, t2);
  double a = dot(p, *t1), b = dot(p, *t2);
  *x = a - s.tile_L * std::floor(a / s.tile_L);
  *y = b - s.tile_L * std::floor(b / s.tile_L);
  *dl = {dot(d, *t1), dot(d, *t2), dot(d, n)};
}
const double kCos1Deg = 0.99984769515639124;

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
// Counter words of the shadow ray's draws; `word` is the wavelength word (the wavelength
// index, or its bundle's index when wavelengths share draws).
struct ShadowKey {
  uint32_t px, sample, bounce;
  uint64_t seed;
  uint32_t word;
};

void shadow_rec(const Scene& s, int ni, V3 o, V3 d, int lam, double lambda_nm, const ShadowKey& key, double& T) {
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
        slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda_nm, &Rs, &Ts, s.slab_pol);
        T *= Ts;
      } else if (m.kind == MAT_TILE) {
        // one brute-force ray through the tile: it counts only if it leaves on the far side
        // within 1 degree of the shadow direction (ballistic), with its throughput
        int ti = s.mat_tile[s.mat[t]];
        double x, y;
        V3 dl, t1, t2;
        tile_frame(s, o + th * d, s.nrm[t], d, &x, &y, &dl, &t1, &t2);
        TileRay r = tile_trace(s.tile_geom[ti], s.tiles[ti], x, y, dl, m.n[lam], m.k[lam], lambda_nm, key.px,
                               key.sample, key.bounce, key.word, key.seed, 64, STREAM_SHADOW_TILE);
        if (r.side == 1 && dot(r.dir, dl) > kCos1Deg) T *= r.w;
        else { T = 0.0; return; }
      } else {
        T = 0.0;
        return;
      }
    }
    return;
  }
  shadow_rec(s, nd.left, o, d, lam, lambda_nm, key, T);
  shadow_rec(s, nd.right, o, d, lam, lambda_nm, key, T);
}
double shadow_T(const Scene& s, V3 o, V3 d, int lam, double lambda_nm, const ShadowKey& key = ShadowKey{0, 0, 0, 0, 0}) {
  double T = 1.0;
  if (!s.nodes.empty()) shadow_rec(s, 0, o, d, lam, lambda_nm, key, T);
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
// A spawned ray starts eps off the surface along the normal; seen from the new ray, the
// surface plane lies eps / |n.d| behind its origin.  Absorption lengths inside glass are
// measured from that plane: l = t_hit + seg0.
double seg0_of(const Scene& s, V3 n, V3 dir) {
  return s.eps / std::max(std::fabs(dot(n, dir)), 1e-6);
}

// ---------------------------------------------------------------- photon maps (Sec. 3.2)
// Jensen's photon mapping as the paper describes it: a pre-rendering step shoots photons
// from the light source and stores those that hit (diffuse) objects in two maps, one for
// caustics and one for global illumination; the rendering step takes the direct and
// specular contributions by ray tracing and the caustic and indirect diffuse ones from the
// maps.  Here the light source is the sun (the sky's light is left to the camera paths).
// Photon i of wavelength index l leaves a disc of radius R centred on C + D s (s the
// direction toward the sun), perpendicular to s, at a point uniform over the disc, travelling
// along -w with w uniform in the sun's cone about s; it carries the power
//   Phi = L_sun(l) Omega (s . w) pi R^2 / N,   Omega = 2 pi (1 - cos half-angle),
// so that the photons' summed power through any surface is, in expectation, the sun's flux.
// Its path follows the Monte Carlo rules of the camera paths (Fresnel choice at solid glass,
// R / (R + T) at thin slabs with the power times R + T, one brute-force ray through a tile)
// and at a diffuse surface it is stored, then survives with probability albedo (power
// unchanged) into a cosine-distributed direction.  Map of a stored photon:
//   caustic  the photon met no diffuse surface yet, and some specular event changed its
//            direction (solid glass, a reflection at a slab, a non-ballistic tile exit);
//   global   the photon was reflected by a diffuse surface before;
// a photon that reached its first diffuse surface only through straight slab transmission
// (or ballistic tile exits) is direct light, which the renderer's sun NEE counts: not stored.
enum { MAP_CAUSTIC = 0, MAP_GLOBAL = 1 };
struct Photon {
  V3 pos, nrm;   // hit point, geometric normal facing the arriving photon
  double power;
  int lam, map;
  uint32_t id, seq;  // photon index, diffuse surfaces met before this one
};
struct PhotonEmitter {
  V3 center;
  double radius, distance;
};

void trace_photon(const Scene& s, const PhotonEmitter& em, uint32_t i, int l, double lambda_nm, uint64_t seed,
                  int n_per_lambda, int max_depth, std::vector<Photon>& out) {
  const V3 sdir = s.sun_dir;
  Draw ue = draw(i, 0, 0, STREAM_PHOTON, 0, (uint32_t)l, seed);
  V3 t1, t2;
  onb(sdir, &t1, &t2);
  const double rr = em.radius * std::sqrt(ue.u[0]), phi = 2.0 * PI * ue.u[1];
  V3 o = em.center + em.distance * sdir + (rr * std::cos(phi)) * t1 + (rr * std::sin(phi)) * t2;
  const V3 w = cone_dir(sdir, s.sun_h, ue.u[2], ue.u[3]);
  V3 d = -1.0 * w;
  const double omega = 2.0 * PI * s.sun_h;
  double power = s.sun[l] * omega * dot(sdir, w) * PI * em.radius * em.radius / n_per_lambda;
  bool spec = false, diff = false;
  uint32_t seq = 0;
  double seg0 = 0.0;
  for (int v = 1; v <= max_depth; ++v) {
    Hit h = closest(s, o, d);
    if (h.prim < 0) return;
    const Material& m = s.mats[s.mat[h.prim]];
    V3 p = o + h.t * d;
    V3 ng = s.nrm[h.prim];
    double cos_n = dot(d, ng);
    V3 nf = cos_n < 0.0 ? ng : -1.0 * ng;
    double cos_i = std::fabs(cos_n);
    Draw u = draw(i, 0, (uint32_t)v, STREAM_PHOTON, 0, (uint32_t)l, seed);
    V3 nd;
    if (m.kind == MAT_SOLID) {
      bool inside = cos_n > 0.0;
      if (inside) power *= beer_lambert(m.k[l], h.t + seg0, lambda_nm);
      double n1 = inside ? m.n[l] : 1.0;
      cd n2 = inside ? cd(1.0, 0.0) : cd(m.n[l], m.k[l]);
      double R = fresnel_R(cos_i, n1, n2);
      double eta = n1 / std::real(n2);
      double c2 = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
      if (u.u[0] < R || c2 <= 0.0) nd = reflect(d, nf);
      else nd = normalize(eta * d + (eta * cos_i - std::sqrt(c2)) * nf);
      spec = true;
    } else if (m.kind == MAT_SLAB) {
      double Rs, Ts;
      slab_RT(cos_i, m.n[l], m.k[l], m.thickness, lambda_nm, &Rs, &Ts, s.slab_pol);
      power *= (Rs + Ts);
      if (u.u[0] < Rs / (Rs + Ts)) {
        nd = reflect(d, nf);
        spec = true;
      } else {
        nd = d;
      }
    } else if (m.kind == MAT_TILE) {
      int ti = s.mat_tile[s.mat[h.prim]];
      double x, y;
      V3 dl, tt1, tt2;
      tile_frame(s, p, ng, d, &x, &y, &dl, &tt1, &tt2);
      TileRay r = tile_trace(s.tile_geom[ti], s.tiles[ti], x, y, dl, m.n[l], m.k[l], lambda_nm, i, 0, (uint32_t)v,
                             (uint32_t)l, seed, 64, STREAM_PHOTON_TILE);
      if (r.side == 2) return;
      power *= r.w;
      nd = normalize(r.dir.x * tt1 + r.dir.y * tt2 + r.dir.z * ng);
      if (!(r.side == 1 && dot(r.dir, dl) > kCos1Deg)) spec = true;
    } else if (m.kind == MAT_DIFFUSE) {
      if (spec || diff) out.push_back(Photon{p, nf, power, l, diff ? MAP_GLOBAL : MAP_CAUSTIC, i, seq});
      if (u.u[3] >= m.albedo[l]) return;  // absorbed: survival with probability albedo
      nd = cosine_dir(nf, u.u[1], u.u[2]);
      diff = true;
      ++seq;
    } else {
      return;
    }
    o = offset(s, p, ng, nd);
    seg0 = seg0_of(s, ng, nd);
    d = nd;
  }
}

// Irradiance estimate of one map at x on a surface with normal n: the power of the map's
// photons of wavelength l within distance r of x that arrived on the same side (n_p . n > 0),
// over the disc area pi r^2.
double photon_gather(const std::vector<Photon>& ph, int map, V3 x, V3 n, int l, double r) {
  double sum = 0.0;
  for (const Photon& p : ph) {
    if (p.map != map || p.lam != l || dot(p.nrm, n) <= 0.0) continue;
    V3 e = p.pos - x;
    if (dot(e, e) < r * r) sum += p.power;
  }
  return sum / (PI * r * r);
}

struct PhotonMapD {
  std::vector<Photon> ph;
  std::vector<double> lambda_nm;
  double radius;
};

struct RenderCtx {
  const Scene* s;
  const Camera* cam;
  const double* lambda_nm;
  int n_lambda, spp, max_depth, rr_start;
  uint64_t seed;
  int bundle;  // wavelengths per draw bundle (1: every wavelength draws on its own)
  const PhotonMapD* pm = nullptr;  // photon maps: the first diffuse vertex takes the sun's caustic
                                   // and indirect light from them
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
      slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda, &Rs, &Ts, s.slab_pol);
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
// Spectral bundling: with cx.bundle = B > 1 the wavelengths l = jB .. jB + B - 1 draw every
// random number on the counter word j instead of l (one draw serves the B wavelengths; Sec. 4
// cuts the spectral array into groups).  Each wavelength still follows its own chain with its
// own decisions; only the uniforms are shared, so each chain has the distribution it has with
// B = 1 and the wavelengths of a bundle are correlated.
double trace_mc(const RenderCtx& cx, uint32_t px, uint32_t sample, int lam, uint32_t* hash_out) {
  const Scene& s = *cx.s;
  double lambda = cx.lambda_nm[lam];
  const uint32_t word = (uint32_t)lam / (uint32_t)cx.bundle;
  PathHash ph;
  Draw jit = draw(px, sample, 0, STREAM_PATH, 0, word, cx.seed);  // pixel jitter
  V3 o, d;
  camera_ray(*cx.cam, (int)px, jit.u[0] - 0.5, jit.u[1] - 0.5, &o, &d);
  double thr = 1.0, L = 0.0, seg0 = 0.0;
  bool sun_counted = false;
  bool photon_done = false;  // with photon maps: the sun's light was taken at a diffuse vertex
  for (int v = 1;; ++v) {
    Hit h = closest(s, o, d);
    if (h.prim < 0) {
      L += thr * escape_radiance(s, d, lam, sun_counted || photon_done);
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
    Draw u = draw(px, sample, (uint32_t)v, STREAM_PATH, 0, word, cx.seed);
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
      slab_RT(cos_i, m.n[lam], m.k[lam], m.thickness, lambda, &Rs, &Ts, s.slab_pol);
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
      if (cx.pm && !photon_done) {  // the sun's caustic and indirect light from the maps
        const double r = cx.pm->radius;
        const double E = photon_gather(cx.pm->ph, MAP_CAUSTIC, p, nf, lam, r) +
                         photon_gather(cx.pm->ph, MAP_GLOBAL, p, nf, lam, r);
        L += thr * m.albedo[lam] / PI * E;
      }
      if (s.sun_h > 0.0 && !photon_done) {
        Draw un = draw(px, sample, (uint32_t)v, STREAM_NEE, 0, word, cx.seed);
        V3 wl = cone_dir(s.sun_dir, s.sun_h, un.u[0], un.u[1]);
        double cl = dot(nf, wl);
        if (cl > 0.0) {
          double T = shadow_T(s, offset(s, p, ng, wl), wl, lam, lambda, ShadowKey{px, sample, (uint32_t)v, cx.seed, word});
          double omega = 2.0 * PI * s.sun_h;
          L += thr * m.albedo[lam] / PI * cl * s.sun[lam] * omega * T;
          nee_event = T > 0.0 ? EV_SHADOW_OPEN : EV_SHADOW_BLOCKED;
        }
      }
      thr *= m.albedo[lam];
      nd = cosine_dir(nf, u.u[1], u.u[2]);
      sun_counted = true;
      if (cx.pm) photon_done = true;  // later vertices: sky light only
    } else if (m.kind == MAT_TILE) {
      // heterogeneous tile: one brute-force ray through the tile on the tile stream
      int ti = s.mat_tile[s.mat[h.prim]];
      double x, y;
      V3 dl, t1, t2;
      tile_frame(s, p, ng, d, &x, &y, &dl, &t1, &t2);
      TileRay r = tile_trace(s.tile_geom[ti], s.tiles[ti], x, y, dl, m.n[lam], m.k[lam], lambda, px, sample,
                             (uint32_t)v, word, cx.seed, 64);
      if (r.side == 2) { ph.byte(EV_ABSORB); break; }
      thr *= r.w;
      nd = normalize(r.dir.x * t1 + r.dir.y * t2 + r.dir.z * ng);
      ph.byte(r.side == 0 ? EV_REFLECT : EV_TRANSMIT);
      if (!(r.side == 1 && dot(r.dir, dl) > kCos1Deg)) sun_counted = false;
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
// Deflection-angle bins of the tile statistics: bin b holds angles in [e_b, e_{b+1}).
constexpr int kTileBins = 8, kTileStatCols = 4 + 2 * kTileBins;
static int deflection_bin(double c) {
  static const double edges_deg[kTileBins + 1] = {0, 1, 2, 4, 8, 16, 32, 64, 180};
  int b = 0;
  while (b < kTileBins - 1 && c < std::cos(edges_deg[b + 1] * PI / 180.0)) ++b;
  return b;
}

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
              const double* lambda_nm, int pol, double* R_slab, double* T_slab) {
  for (int i = 0; i < n; ++i) slab_RT(cos_i[i], nre[i], k[i], d_m[i], lambda_nm[i], R_slab + i, T_slab + i, pol);
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
  int n_tiles;                // heterogeneous tiles (0 = none)
  const void* tiles;          // OrcTile[n_tiles]
  const int32_t* mat_tile;    // [M] tile index of HETERO_TILE materials, -1 otherwise (or NULL)
  int tile_grid;
  double tile_size;
  int slab_polarisation;      // 0: thin-slab series on the unpolarised R; 1: per polarisation
};

struct OrcTile {
  double d_mean, amp, rho;
  uint32_t seed;
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
  int bundle;          // Monte Carlo: wavelengths sharing their draws (0 or 1: none)
  const void* photons; // photon maps of orc_photons_trace for the same wavelengths, or NULL
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
  s.slab_pol = d->slab_polarisation;
  std::vector<int> idx(d->n_triangles);
  std::vector<V3> cen(d->n_triangles);
  for (int t = 0; t < d->n_triangles; ++t) {
    idx[t] = t;
    cen[t] = (1.0 / 3.0) * (s.v0[t] + s.v1[t] + s.v2[t]);
  }
  if (d->n_triangles > 0) build_node(s, idx, 0, d->n_triangles, cen);
  s.order = idx;
  s.mat_tile.assign(d->n_materials, -1);
  if (d->n_tiles > 0 && d->tiles && d->mat_tile) {
    s.mat_tile.assign(d->mat_tile, d->mat_tile + d->n_materials);
    s.tile_G = d->tile_grid;
    s.tile_L = d->tile_size;
    const OrcTile* ot = static_cast<const OrcTile*>(d->tiles);
    for (int t = 0; t < d->n_tiles; ++t) {
      TileParams tp{ot[t].d_mean, ot[t].amp, ot[t].rho, ot[t].seed};
      s.tiles.push_back(tp);
      std::vector<double> hh((size_t)(s.tile_G + 1) * (s.tile_G + 1));
      for (int j = 0; j <= s.tile_G; ++j)
        for (int i = 0; i <= s.tile_G; ++i)
          hh[(size_t)j * (s.tile_G + 1) + i] = tile_thickness(tp, i * s.tile_L / s.tile_G, j * s.tile_L / s.tile_G, s.tile_L);
      s.tile_h.push_back(hh);
    }
    for (int t = 0; t < d->n_tiles; ++t) {
      TileGeom g{s.tile_G, s.tile_L, s.tile_h[t].data(), INF, -INF};
      for (double v : s.tile_h[t]) {
        g.hmin = std::min(g.hmin, v);
        g.hmax = std::max(g.hmax, v);
      }
      s.tile_geom.push_back(g);
    }
  }
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
// Resample every material and light table to a list of wavelengths.
void prepare_tables(OrcHandle* h, int n_lambda, const float* lambda_nm) {
  Scene& s = h->s;
  s.mats.assign(h->mat_kind.size(), Material{});
  for (size_t m = 0; m < h->mat_kind.size(); ++m) {
    Material& mm = s.mats[m];
    mm.kind = h->mat_kind[m];
    mm.thickness = h->mat_thick[m];
    for (int l = 0; l < n_lambda; ++l) {
      double lam = lambda_nm[l];
      const size_t o = m * (size_t)h->n_table;
      mm.n.push_back(interp(h->table_nm.data(), h->mat_n.data() + o, h->n_table, lam));
      mm.k.push_back(interp(h->table_nm.data(), h->mat_k.data() + o, h->n_table, lam));
      mm.albedo.push_back(interp(h->table_nm.data(), h->mat_alb.data() + o, h->n_table, lam));
    }
  }
  s.sky.clear(); s.sun.clear();
  for (int l = 0; l < n_lambda; ++l) {
    s.sky.push_back(interp(h->table_nm.data(), h->sky.data(), h->n_table, lambda_nm[l]));
    s.sun.push_back(h->sun.empty() ? 0.0 : interp(h->table_nm.data(), h->sun.data(), h->n_table, lambda_nm[l]));
  }
}

struct OrcPhotonOpts {
  int n_per_lambda;     // photons shot per wavelength
  uint64_t seed;
  int max_depth;        // surface interactions per photon
  float center[3];      // emitter disc: centre C + distance * (direction to the sun), radius
  float radius, distance;
  float gather_radius;  // density-estimation radius (m)
  int n_threads;        // 0 = hardware concurrency
};

// Photon maps (Sec. 3.2) for a list of wavelengths; returns a handle (orc_photons_destroy).
void* orc_photons_trace(void* hp, const OrcPhotonOpts* po, int n_lambda, const float* lambda_nm) {
  OrcHandle* h = (OrcHandle*)hp;
  if (!po || n_lambda <= 0 || po->n_per_lambda <= 0 || po->radius <= 0.f || !(h->s.sun_h > 0.0)) return nullptr;
  prepare_tables(h, n_lambda, lambda_nm);
  PhotonEmitter em{{po->center[0], po->center[1], po->center[2]}, po->radius, po->distance};
  const int total = po->n_per_lambda * n_lambda;
  int nth = po->n_threads > 0 ? po->n_threads : (int)std::thread::hardware_concurrency();
  if (nth < 1) nth = 1;
  std::vector<std::vector<Photon>> part(nth);
  std::atomic<int> next{0};
  auto worker = [&](int t) {
    for (;;) {
      int j = next.fetch_add(1);
      if (j >= total) break;
      const int l = j / po->n_per_lambda;
      trace_photon(h->s, em, (uint32_t)(j % po->n_per_lambda), l, lambda_nm[l], po->seed, po->n_per_lambda,
                   po->max_depth, part[t]);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) pool.emplace_back(worker, t);
  for (auto& t : pool) t.join();
  PhotonMapD* pm = new PhotonMapD;
  for (auto& v : part) pm->ph.insert(pm->ph.end(), v.begin(), v.end());
  std::sort(pm->ph.begin(), pm->ph.end(), [](const Photon& a, const Photon& b) {
    if (a.lam != b.lam) return a.lam < b.lam;
    if (a.id != b.id) return a.id < b.id;
    return a.seq < b.seq;
  });
  pm->lambda_nm.assign(lambda_nm, lambda_nm + n_lambda);
  pm->radius = po->gather_radius;
  return pm;
}

void orc_photons_destroy(void* pm) { delete (PhotonMapD*)pm; }

int64_t orc_photons_count(const void* pmv, int map) {
  const PhotonMapD* pm = (const PhotonMapD*)pmv;
  int64_t c = 0;
  for (const Photon& p : pm->ph) c += p.map == map;
  return c;
}

// The photons of one map in (wavelength, photon index, order along its path) order.
void orc_photons_get(const void* pmv, int map, double* pos, double* nrm, double* power, int32_t* lam,
                     uint32_t* id) {
  const PhotonMapD* pm = (const PhotonMapD*)pmv;
  size_t k = 0;
  for (const Photon& p : pm->ph) {
    if (p.map != map) continue;
    pos[3 * k] = p.pos.x; pos[3 * k + 1] = p.pos.y; pos[3 * k + 2] = p.pos.z;
    nrm[3 * k] = p.nrm.x; nrm[3 * k + 1] = p.nrm.y; nrm[3 * k + 2] = p.nrm.z;
    power[k] = p.power;
    lam[k] = p.lam;
    id[k] = p.id;
    ++k;
  }
}

// Irradiance estimates of both maps at n query points (position, unit normal, wavelength index).
void orc_photons_gather(const void* pmv, int n, const double* x, const double* nrm, const int32_t* lam,
                        double* E_caustic, double* E_global) {
  const PhotonMapD* pm = (const PhotonMapD*)pmv;
  for (int i = 0; i < n; ++i) {
    V3 p{x[3 * i], x[3 * i + 1], x[3 * i + 2]}, nn{nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
    E_caustic[i] = photon_gather(pm->ph, MAP_CAUSTIC, p, nn, lam[i], pm->radius);
    E_global[i] = photon_gather(pm->ph, MAP_GLOBAL, p, nn, lam[i], pm->radius);
  }
}

int orc_render(void* hp, const OrcCamera* cam_in, const OrcOpts* op, double* film,
               double* path_L, uint32_t* path_hash) {
  OrcHandle* h = (OrcHandle*)hp;
  Scene& s = h->s;
  if (op->n_lambda <= 0 || op->spp <= 0 || op->max_depth < 0) return -1;
  if (op->mode == 0 && op->spp != 1) return -1;
  if (op->bundle < 0 || op->bundle > 64 || (op->bundle > 1 && op->mode == 0)) return -1;
  const PhotonMapD* pm = (const PhotonMapD*)op->photons;
  if (pm) {  // the maps must be for the same wavelengths, and are for Monte Carlo paths
    if (op->mode == 0 || (int)pm->lambda_nm.size() != op->n_lambda) return -1;
    for (int l = 0; l < op->n_lambda; ++l)
      if (pm->lambda_nm[l] != op->lambda_nm[l]) return -1;
  }
  prepare_tables(h, op->n_lambda, op->lambda_nm);
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
  RenderCtx cx{&s, &cam, lam_d.data(), op->n_lambda, op->spp, op->max_depth, op->rr_start_depth, op->seed,
               op->bundle > 1 ? op->bundle : 1, pm};

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

// ---------------------------------------------------------------- tiles

// Thickness at the (G+1) x (G+1) grid vertices of a tile of side L (row j, column i).
void orc_tile_heights(const OrcTile* t, int G, double L, double* h) {
  TileParams tp{t->d_mean, t->amp, t->rho, t->seed};
  for (int j = 0; j <= G; ++j)
    for (int i = 0; i <= G; ++i) h[(size_t)j * (G + 1) + i] = tile_thickness(tp, i * L / G, j * L / G, L);
}

static TileGeom make_geom(int G, double L, const double* h) {
  TileGeom g{G, L, h, INF, -INF};
  for (int i = 0; i < (G + 1) * (G + 1); ++i) {
    g.hmin = std::min(g.hmin, h[i]);
    g.hmax = std::max(g.hmax, h[i]);
  }
  return g;
}

// Trace n rays through one tile: entry points xy [n][2], directions [n][3] (tile frame),
// draws keyed (px[i], sample[i], bounce, tile stream, event, lam).  Outputs side, weight,
// exit direction [n][3], bubble encounters and interactions per ray.
void orc_tile_trace(const OrcTile* t, int G, double L, const double* h, int n, const double* xy, const double* dir,
                    double n_re, double k, double lambda_nm, const uint32_t* px, const uint32_t* sample,
                    uint32_t bounce, uint32_t lam, uint64_t seed, int max_events, int32_t* side, double* w,
                    double* dout, int32_t* bubbles, int32_t* events) {
  TileParams tp{t->d_mean, t->amp, t->rho, t->seed};
  TileGeom g = make_geom(G, L, h);
  for (int i = 0; i < n; ++i) {
    TileRay r = tile_trace(g, tp, xy[2 * i], xy[2 * i + 1], {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]}, n_re, k,
                           lambda_nm, px[i], sample[i], bounce, lam, seed, max_events);
    side[i] = r.side;
    w[i] = r.w;
    dout[3 * i] = r.dir.x; dout[3 * i + 1] = r.dir.y; dout[3 * i + 2] = r.dir.z;
    bubbles[i] = r.bubbles;
    events[i] = r.events;
  }
}

// The bubble optics alone, driven by given uniforms instead of Philox draws: ray i has
// direction d[i], impact direction rad[i] and impact parameter sin_i[i] (b / r); its surface
// interactions take u[i * n_u + j] in turn.  dout gets the exit direction and n_events the
// number of surfaces met, or -1 when the n_u uniforms ran out inside the bubble.
void orc_bubble_scatter(int n, const double* d, const double* rad, const double* sin_i, double r, double n_re,
                        double k, int n_u, const double* u, double* dout, int32_t* n_events) {
  for (int i = 0; i < n; ++i) {
    V3 di{d[3 * i], d[3 * i + 1], d[3 * i + 2]};
    int j = 0;
    auto choice = [&]() -> double { return j < n_u ? u[(size_t)i * n_u + j++] : -1.0; };
    bool ok = bubble_scatter(&di, {rad[3 * i], rad[3 * i + 1], rad[3 * i + 2]}, sin_i[i], r, n_re, k, choice);
    dout[3 * i] = di.x; dout[3 * i + 1] = di.y; dout[3 * i + 2] = di.z;
    n_events[i] = ok ? j : -1;
  }
}

// Per-sample statistics of rays_per_sample rays entering a tile at uniform points with the
// sample's direction (cos_in, phi_in, from the front): out[8] = T, R, absorbed-by-cap,
// ballistic fraction of T (within 1 degree of straight through), mean cosine to straight
// through of T, the same two for R about the mirror direction, bubble encounters per ray.
// Sample s draws its entry points on (s, ray, 0, tile stream, 0) and its interactions on
// bounce 1.
// Per-query tile statistics: T, R, absorbed weight and bubbles per ray, then per side the
// fraction of its weight in each deflection-angle bin (angle to the straight-through or
// mirror direction; edges 0, 1, 2, 4, 8, 16, 32, 64, 180 degrees).
void orc_tile_samples(int n_tiles, const OrcTile* tiles, int G, double L, const double* heights, int n_samples,
                      const double* cos_in, const double* phi_in, const double* lambda_nm, const double* n_re,
                      const double* k, const int32_t* tile, int rays, uint64_t seed, int max_events, int n_threads,
                      double* out) {
  (void)n_tiles;
  int nth = n_threads > 0 ? n_threads : (int)std::thread::hardware_concurrency();
  std::atomic<int> next{0};
  auto work = [&]() {
    for (;;) {
      int s = next.fetch_add(1);
      if (s >= n_samples) break;
      const OrcTile& ot = tiles[tile[s]];
      TileParams tp{ot.d_mean, ot.amp, ot.rho, ot.seed};
      TileGeom g = make_geom(G, L, heights + (size_t)tile[s] * (G + 1) * (G + 1));
      // cos_in < 0: the ray enters through the rough back face (travelling toward +z)
      double st = std::sqrt(std::max(0.0, 1.0 - cos_in[s] * cos_in[s]));
      V3 d{st * std::cos(phi_in[s]), st * std::sin(phi_in[s]), -cos_in[s]};
      V3 dm{d.x, d.y, -d.z};
      double T = 0, R = 0, A = 0, bub = 0, hT[kTileBins] = {}, hR[kTileBins] = {};
      for (int r = 0; r < rays; ++r) {
        Draw ue = draw((uint32_t)s, (uint32_t)r, 0, STREAM_TILE, 0, 0, seed);
        TileRay tr = tile_trace(g, tp, ue.u[0] * L, ue.u[1] * L, d, n_re[s], k[s], lambda_nm[s], (uint32_t)s,
                                (uint32_t)r, 1, 0, seed, max_events);
        bub += tr.bubbles;
        if (tr.side == 1) {
          T += tr.w;
          hT[deflection_bin(dot(tr.dir, d))] += tr.w;
        } else if (tr.side == 0) {
          R += tr.w;
          hR[deflection_bin(dot(tr.dir, dm))] += tr.w;
        } else {
          A += tr.w;
        }
      }
      double* o = out + kTileStatCols * (size_t)s;
      o[0] = T / rays; o[1] = R / rays; o[2] = A / rays; o[3] = bub / rays;
      for (int b = 0; b < kTileBins; ++b) {
        o[4 + b] = T > 0 ? hT[b] / T : 0.0;
        o[4 + kTileBins + b] = R > 0 ? hR[b] / R : 0.0;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int i = 0; i < nth; ++i) pool.emplace_back(work);
  for (auto& th : pool) th.join();
}

int orc_hardware_threads(void) { return (int)std::thread::hardware_concurrency(); }

}  // extern "C"
