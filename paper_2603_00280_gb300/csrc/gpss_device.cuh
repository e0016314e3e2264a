// gpss_device.cuh -- device-side data layout and arithmetic of the GPSS medium.
//
// Everything here is FP32 CUDA for sm_103a.  It implements, from the paper
// "Macrofacet Theory for Gaussian Process Statistical Surfaces":
//   - trilinear field fetch of the mean (a signed distance), variance and albedo
//     grids, with the analytic gradient of the interpolant (Sec. 4: the normal is
//     the normalised gradient of the SDF);
//   - the extinction sigma_t = rho * sigma(d)  (Eq. generalized_sigma_t,
//     Eq. generalized_lambda), rho = phi/Phi of mu/sigma over sigma;
//   - the NDF D(m) = int_0^inf t^3 P(t m) dt (Eq. gdf_to_ndf with Eq. gdf) in closed
//     form through moments M_k(q) = int_0^inf s^k exp(-s^2 + 2 q s) ds;
//   - the conductor phase function (Eq. phase, Eq. microfacet_vndf) and the
//     sampling mixture R * Beckmann-vNDF + (1-R) * uniform hemisphere (end of
//     Sec. 4.2), and exact visible-normal sampling in slope space;
//   - height-field macrofacets with Beckmann or GGX NDFs (Sec. 4.1) and anisotropic,
//     non-stationary kernels (the local-frame roughness of Sec. 4.2 with a tangent
//     field and a correlation-scale grid);
//   - Philox4x32-10 (Salmon et al., SC'11) keyed by (seed) with counter
//     (pixel, sample, bounce | purpose << 16, draw);
//   - Amanatides-Woo traversal of the majorant grid with skip cubes, local majorants
//     for thin shells and the surface-limit analytic pieces.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace gpss {

constexpr int kMaxObjects = 4;

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInv4Pi = 0.07957747154594767280f;
constexpr float kInvSqrtPi = 0.56418958354775628695f;
constexpr float kSqrtPi = 1.77245385090551602730f;
constexpr float kSqrt2 = 1.41421356237309504880f;
constexpr float kInvSqrt2 = 0.70710678118654752440f;
constexpr float kSqrt2OverPi = 0.79788456080286535588f;
constexpr float kInvPi32 = 0.17958712212516656f;  // pi^(-3/2)
constexpr float kSqrtPiOver2 = 1.25331413731550025121f;
constexpr float kInvSqrt2Pi = 0.39894228040143267794f;

// ---------------------------------------------------------------- layouts

// One GPSS object: node-centred grids over [bmin, bmax], x fastest.
struct ObjectDev {
  float bmin[3], bmax[3];
  float inv_h[3];          // (n-1)/(bmax-bmin)
  int n[3];
  int channels;            // albedo channels, 1 or 3
  int ndf;                 // kNdfGpss or a height-field macrofacet NDF (gpss_ndf)
  float alpha_scale;       // sqrt(2)/l_t: alpha = sigma * alpha_scale (Eq. roughness)
  const float2* mv;        // (mean, variance) per node
  const float* albedo;     // channels planes
  // Anisotropic / non-stationary kernel (all neutral for the isotropic stationary one):
  // gradient covariance sigma^2 diag(1/l_t^2, 1/l_b^2, 1/l_n^2) in the frame
  // (tangent, bitangent, n = grad mu/|grad mu|), every l scaled by s(x).
  float kb, kn;            // l_t/l_b, l_t/l_n: alpha_y = kb alpha, alpha_z = kn alpha
  float amax;              // max(1, kb, kn)
  const float* cscale;     // correlation-scale factor s per node, or null (s = 1)
  const float* tangent;    // tangent field, 3 planes of nodes, or null
  int general;             // kb != 1, kn != 1, cscale or tangent
};

// Majorant grid: piecewise-constant upper bound of sigma_t over all directions,
// per cell of `brick` field cells.  For traversal each cell also stores a skip
// entry (M_r, r): the largest radius r in {0, 1, 2, 4, 8, 16} such that the max
// M_r of the majorant over the cube of cells [c-r, c+r]^3 satisfies
// M_r * r * h_min <= kappa (r = 0: the cell's own majorant).  A ray inside cell c
// stays inside that cube for at least r cells, so one load covers up to r cells
// of empty or thin space with a valid (larger) majorant.
struct MajorantDev {
  float gmin[3];
  float cell[3];           // cell size
  float inv_cell[3];
  int dims[3];             // cells per axis
  const float* maj;        // per-cell majorant
  const float2* skip;      // per-cell (M_r, r)
  // Local majorants (single-object scenes; 0 = off): where the cell's majorant
  // times the rest of the ray's segment in the cell exceeds `hot` (expected
  // tentative collisions), the walk bounds sigma_t over shorter pieces from the
  // field at the piece's start (local_piece).
  float hot;
  // Surface-limit analytic flight in those pieces (1 = on, opt-in): the majorant follows
  // a linear lower bound of mu along the ray and is sampled in closed form (lin_depth).
  int lin;
};

enum LightKind : int { kLightDirectional = 0, kLightSky = 1, kLightUniform = 2 };

struct LightDev {
  int kind;
  float dir[3];            // directional: unit vector toward the light
  float radiance[3];
};

struct SceneDev {
  int n_objs;
  ObjectDev obj[kMaxObjects];
  MajorantDev mg;          // over the union of the boxes (majorants of all objects added)
  // Per-object traversal (split = 1, scenes of several objects): og[k] is object k's own
  // majorant grid over its box, at its node spacing, with its local majorants.
  int split;
  MajorantDev og[kMaxObjects];
  LightDev light;
};

struct CameraDev {
  int ortho;
  float eye[3], fwd[3], right[3], up[3];
  float half_w, half_h;    // ortho: half film extent; perspective: tan(fov/2)*aspect, tan(fov/2)
  int width, height;
};

// ---------------------------------------------------------------- small vector helpers
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 normalize(V3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ V3 fma3(float s, V3 a, V3 b) { return {fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)}; }

// ---------------------------------------------------------------- Philox4x32-10
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Out-of-line copy used by the path streams: the ten unrolled rounds then exist
// once in the kernel instead of at every draw site (instruction-cache footprint).
static __device__ __noinline__ U4 philox_block(U4 c, uint32_t k0, uint32_t k1) { return philox4x32_10(c, k0, k1); }

// uniform in (0,1): 24 bits, centred
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }

enum Purpose : uint32_t { kPurposeCamera = 0, kPurposeFlight = 1, kPurposeNee = 2, kPurposePhase = 3 };

// Counter-based stream for one path: (pixel, sample, bounce|purpose<<16, draw).
struct Rng {
  uint32_t k0, k1, pixel, sample, tag, draw;
  uint32_t b0, b1, b2, b3;
  int avail;
  __device__ __forceinline__ void init(uint64_t seed, uint32_t px, uint32_t s) {
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    pixel = px;
    sample = s;
    tag = 0;
    draw = 0;
    avail = 0;
  }
  __device__ __forceinline__ void start(uint32_t bounce, uint32_t purpose) {
    tag = (bounce & 0xFFFFu) | (purpose << 16);
    draw = 0;
    avail = 0;
  }
  __device__ __forceinline__ float next() {
    if (avail == 0) {
      const U4 r = philox_block(U4{pixel, sample, tag, draw}, k0, k1);
      ++draw;
      b0 = r.x; b1 = r.y; b2 = r.z; b3 = r.w;
      avail = 4;
    }
    const uint32_t v = b0;
    b0 = b1; b1 = b2; b2 = b3;
    --avail;
    return u01(v);
  }
};

// ---------------------------------------------------------------- special functions
// lambda(u) = phi(u)/Phi(u) = sqrt(2/pi) / erfcx(-u/sqrt2)   (inverse Mills ratio).  The
// division is the fast one (2 ulp; it returns 0 where erfcx overflows, lambda's limit).
__device__ __forceinline__ float inv_mills(float u) { return __fdividef(kSqrt2OverPi, erfcxf(-u * kInvSqrt2)); }

// e^{-a^2} without the rounding error of a*a: a^2 = hi + lo exactly (lo from an FMA,
// the error-free product of Dekker / Ogita-Rump-Oishi), e^{-a^2} = e^{-hi} (1 - lo) to
// first order in lo <= ulp(hi)/2.  Plain expf(-a*a) is off by ~a^2 ulp for large a.
__device__ __forceinline__ float exp_neg_sq(float a) {
  const float hi = a * a;
  const float lo = fmaf(a, a, -hi);
  return expf(-hi) * (1.0f - lo);
}

// erfc(a) from one erfcx evaluation: erfcx(|a|) e^{-a^2} for a >= 0, 2 minus that for
// a < 0 (ex = e^{-a^2} is passed in because the callers need it too).
__device__ __forceinline__ float erfc_from(float a, float ex, float erfcx_abs) {
  const float t = erfcx_abs * ex;
  return a >= 0.0f ? t : 2.0f - t;
}

// Laplace's continued fraction K(y) = 1/(y + 2/(y + 3/(y + ...))) of the Mills ratio,
// 20 terms, evaluated backward (y >= 2 sqrt2 at the call sites).
__device__ __forceinline__ float mills_cf(float y) {
  float r = 0.0f;
#pragma unroll 1
  for (int k = 20; k >= 1; --k) r = __fdividef((float)k, y + r);
  return r;
}

// psi(a) = exp(-a^2)/(2 sqrt(pi)) - (a/2) erfc(a) = E[max(0, Z/sqrt2 - a)] with Z ~ N(0,1),
// so the projected area is sigma(d) = alpha * psi((d . grad mu)/alpha).  For a > 2 the
// difference cancels; there psi = erfc(a) * K(sqrt2 a) / (2 sqrt2).
__device__ __forceinline__ float psi(float a) {
  const float ex = exp_neg_sq(a);
  const float ec = erfc_from(a, ex, erfcxf(fabsf(a)));
  if (a <= 2.0f) return fmaf(-0.5f * a, ec, 0.5f * kInvSqrtPi * ex);
  return ec * mills_cf(kSqrt2 * a) * (0.5f * kInvSqrt2);
}

// ---------------------------------------------------------------- fields
struct Field {
  float mu, var;
  V3 g;        // gradient of the mean interpolant
  int ndf;     // the object's NDF kind (gpss_ndf)
  float as;    // alpha scale at x: sqrt(2)/(s(x) l_t), alpha = sigma * as
  float cs;    // correlation-scale factor s(x)
  float kb, kn;  // the object's l_t/l_b, l_t/l_n
  V3 t;        // tangent field at x (zero without one)
};

enum NdfKind : int { kNdfGpss = 0, kNdfBeckmann = 1, kNdfGgx = 2 };

// Cell lookup + trilinear weights; returns the node index of the cell's corner 000.
__device__ __forceinline__ int cell_of(const ObjectDev& o, V3 x, float& wx, float& wy, float& wz) {
  const float fx = (x.x - o.bmin[0]) * o.inv_h[0];
  const float fy = (x.y - o.bmin[1]) * o.inv_h[1];
  const float fz = (x.z - o.bmin[2]) * o.inv_h[2];
  const int ix = min(max((int)floorf(fx), 0), o.n[0] - 2);
  const int iy = min(max((int)floorf(fy), 0), o.n[1] - 2);
  const int iz = min(max((int)floorf(fz), 0), o.n[2] - 2);
  wx = fminf(fmaxf(fx - (float)ix, 0.0f), 1.0f);
  wy = fminf(fmaxf(fy - (float)iy, 0.0f), 1.0f);
  wz = fminf(fmaxf(fz - (float)iz, 0.0f), 1.0f);
  return ix + o.n[0] * (iy + o.n[1] * iz);
}

__device__ __forceinline__ bool inside(const ObjectDev& o, V3 x) {
  return x.x >= o.bmin[0] && x.x <= o.bmax[0] && x.y >= o.bmin[1] && x.y <= o.bmax[1] &&
         x.z >= o.bmin[2] && x.z <= o.bmax[2];
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Field of an object with the isotropic stationary kernel (the kernel members neutral).
__device__ __forceinline__ Field fetch_iso(const ObjectDev& o, V3 x) {
  float wx, wy, wz;
  const int b = cell_of(o, x, wx, wy, wz);
  const int sx = 1, sy = o.n[0], sz = o.n[0] * o.n[1];
  const float2 v000 = __ldg(o.mv + b), v100 = __ldg(o.mv + b + sx);
  const float2 v010 = __ldg(o.mv + b + sy), v110 = __ldg(o.mv + b + sy + sx);
  const float2 v001 = __ldg(o.mv + b + sz), v101 = __ldg(o.mv + b + sz + sx);
  const float2 v011 = __ldg(o.mv + b + sz + sy), v111 = __ldg(o.mv + b + sz + sy + sx);
  // mean: interpolate along x, keep the x-differences for the gradient
  const float m00 = lerpf(v000.x, v100.x, wx), m10 = lerpf(v010.x, v110.x, wx);
  const float m01 = lerpf(v001.x, v101.x, wx), m11 = lerpf(v011.x, v111.x, wx);
  const float d00 = v100.x - v000.x, d10 = v110.x - v010.x, d01 = v101.x - v001.x, d11 = v111.x - v011.x;
  const float m0 = lerpf(m00, m10, wy), m1 = lerpf(m01, m11, wy);
  Field f;
  f.ndf = o.ndf;
  f.mu = lerpf(m0, m1, wz);
  f.g.x = lerpf(lerpf(d00, d10, wy), lerpf(d01, d11, wy), wz) * o.inv_h[0];
  f.g.y = lerpf(m10 - m00, m11 - m01, wz) * o.inv_h[1];
  f.g.z = (m1 - m0) * o.inv_h[2];
  const float s00 = lerpf(v000.y, v100.y, wx), s10 = lerpf(v010.y, v110.y, wx);
  const float s01 = lerpf(v001.y, v101.y, wx), s11 = lerpf(v011.y, v111.y, wx);
  f.var = lerpf(lerpf(s00, s10, wy), lerpf(s01, s11, wy), wz);
  f.as = o.alpha_scale;
  f.cs = 1.0f;
  f.kb = 1.0f;
  f.kn = 1.0f;
  f.t = v3(0.0f, 0.0f, 0.0f);
  return f;
}

// Trilinear interpolation of a scalar node grid in the cell with corner node b.
__device__ __forceinline__ float trilerp(const float* __restrict__ p, int b, int sy, int sz, float wx, float wy,
                                         float wz) {
  p += b;
  const float a0 = lerpf(lerpf(__ldg(p), __ldg(p + 1), wx), lerpf(__ldg(p + sy), __ldg(p + sy + 1), wx), wy);
  const float a1 =
      lerpf(lerpf(__ldg(p + sz), __ldg(p + sz + 1), wx), lerpf(__ldg(p + sz + sy), __ldg(p + sz + sy + 1), wx), wy);
  return lerpf(a0, a1, wz);
}

// Field of any object: adds the correlation-scale factor and the tangent field
// (non-stationary and anisotropic kernels) where the object has them.
__device__ __forceinline__ Field fetch(const ObjectDev& o, V3 x) {
  Field f = fetch_iso(o, x);
  if (o.general) {
    f.kb = o.kb;
    f.kn = o.kn;
    if (o.cscale || o.tangent) {
      float wx, wy, wz;
      const int b = cell_of(o, x, wx, wy, wz);
      const int sy = o.n[0], sz = o.n[0] * o.n[1], plane = sz * o.n[2];
      if (o.cscale) {
        f.cs = trilerp(o.cscale, b, sy, sz, wx, wy, wz);
        f.as = o.alpha_scale / f.cs;
      }
      if (o.tangent)
        f.t = v3(trilerp(o.tangent, b, sy, sz, wx, wy, wz), trilerp(o.tangent + plane, b, sy, sz, wx, wy, wz),
                 trilerp(o.tangent + 2 * plane, b, sy, sz, wx, wy, wz));
    }
  }
  return f;
}

// Albedo (F of Eq. phase) at x, per channel.
__device__ __forceinline__ V3 fetch_albedo(const ObjectDev& o, V3 x) {
  float wx, wy, wz;
  const int b = cell_of(o, x, wx, wy, wz);
  const int sy = o.n[0], sz = o.n[0] * o.n[1];
  const int plane = sz * o.n[2];
  float c[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    if (ch >= o.channels) { c[ch] = c[0]; continue; }
    const float* a = o.albedo + ch * plane + b;
    const float a0 = lerpf(lerpf(__ldg(a), __ldg(a + 1), wx), lerpf(__ldg(a + sy), __ldg(a + sy + 1), wx), wy);
    const float a1 = lerpf(lerpf(__ldg(a + sz), __ldg(a + sz + 1), wx), lerpf(__ldg(a + sz + sy), __ldg(a + sz + sy + 1), wx), wy);
    c[ch] = lerpf(a0, a1, wz);
  }
  return {c[0], c[1], c[2]};
}

// ---------------------------------------------------------------- extinction
// Derived quantities of a field sample used by sigma_t and the phase function.
struct Local {
  float sigma;   // sqrt(var)
  float alpha;   // sqrt(2) sigma / l
  float rho;     // lambda(mu/sigma)/sigma
};

// One reciprocal square root serves sigma, mu/sigma and rho (a few ulp each: far below the
// 1e-5 bar, and lambda's sensitivity to u is |u + lambda|, so also at |u| ~ 10).
__device__ __forceinline__ Local local_of(const ObjectDev& o, const Field& f) {
  Local l;
  const float inv_sig = rsqrtf(f.var);
  l.sigma = f.var * inv_sig;
  l.alpha = l.sigma * f.as;
  l.rho = inv_mills(f.mu * inv_sig) * inv_sig;
  return l;
}

// Orthonormal basis around a unit vector (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb_z(V3 n, V3& t1, V3& t2) {
  const float s = copysignf(1.0f, n.z);
  const float a = -1.0f / (s + n.z);
  const float b = n.x * n.y * a;
  t1 = {1.0f + s * n.x * n.x * a, s * b, -s * n.x};
  t2 = {b, s + n.y * n.y * a, -n.y};
}

// sigma(d) = Lambda(d) cos(theta) = alpha psi(d . grad mu / alpha)
// ---------------------------------------------------------------- height-field macrofacets
// Sec. 4.1 (Eq. macro_sigma_t): the density rho times Lambda(w) cos(theta) of a chosen
// microfacet NDF about n = grad mu/|grad mu|, roughness alpha.  For the marching
// direction d (c = d.n, s = sin theta) and the continuation Lambda(-w) = -1 - Lambda(w)
// both signs of c take one form:
//   Beckmann: alpha s psi(c/(alpha s))   (the GPSS projected area with alpha_z = 0)
//   GGX:      (sqrt(c^2 + alpha^2 s^2) - c)/2
__device__ __forceinline__ V3 hf_normal(V3 g) {
  const float G2 = dot(g, g);
  return G2 > 1e-30f ? rsqrtf(G2) * g : v3(0.0f, 0.0f, 1.0f);
}

__device__ __forceinline__ float hf_projected_area(int ndf, V3 d, V3 n, float alpha) {
  const float c = dot(d, n);
  const V3 dxn = cross(d, n);
  const float s2 = dot(dxn, dxn);  // sin^2 theta without the cancellation of 1 - c^2 near the normal
  if (ndf == kNdfGgx) {
    const float r = sqrtf(fmaf(alpha * alpha, s2, c * c));
    return c > 0.0f ? 0.5f * alpha * alpha * s2 / (r + c) : 0.5f * (r - c);  // no cancellation
  }
  const float ae = alpha * sqrtf(s2);
  if (!(ae > 0.0f)) return fmaxf(0.0f, -c);
  return ae * psi(c / ae);
}

// Microfacet NDF about n, normalised by int D(m) (m.n) dm = 1; zero for m.n <= 0.
__device__ __forceinline__ float hf_ndf(int ndf, V3 m, V3 n, float alpha) {
  const float c = dot(m, n);
  if (c <= 0.0f) return 0.0f;
  const float c2 = c * c, a2 = alpha * alpha;
  if (ndf == kNdfGgx) {
    const float q = fmaf(c2, a2 - 1.0f, 1.0f);  // c^4 (a^2 + tan^2)^2 = (1 + c^2 (a^2 - 1))^2
    return a2 / (kPi * q * q);
  }
  return expf(-(1.0f - c2) / (c2 * a2)) / (kPi * a2 * c2 * c2);
}

// ---------------------------------------------------------------- anisotropic kernels
// Gradient covariance (alpha^2/2) diag(1, kb^2, kn^2) in the frame (t, b, n) with n =
// grad mu/|grad mu| (world z where grad mu = 0), t the tangent field's component
// orthogonal to n (any unit vector orthogonal to n where there is none), b = n x t.
// alpha is the tangential roughness sqrt(2) sigma/l_t at x.
struct KFrame {
  V3 t, b, n;
};

__device__ __forceinline__ KFrame kernel_frame(const Field& f) {
  KFrame k;
  k.n = hf_normal(f.g);
  const V3 tp = fma3(-dot(f.t, k.n), k.n, f.t);
  const float l2 = dot(tp, tp);
  if (l2 > 1e-12f * dot(f.t, f.t) && l2 > 0.0f) {
    k.t = rsqrtf(l2) * tp;
    k.b = cross(k.n, k.t);
  } else {
    onb_z(k.n, k.t, k.b);
  }
  return k;
}

// sigma(d) = E[max(0, -d.g)] = alpha_e psi(d.grad mu/alpha_e), alpha_e^2 = 2 d^T Sigma d =
// alpha^2 ((d.t)^2 + kb^2 (d.b)^2 + kn^2 (d.n)^2)  (Eq. generalized_lambda times cos theta
// in the local frame; (d.t)^2 + (d.b)^2 = |d x n|^2 without cancellation).
__device__ __forceinline__ float area_aniso(V3 d, const Field& f, float alpha) {
  const V3 n = hf_normal(f.g);
  const float dn = dot(d, n);
  const V3 dxn = cross(d, n);
  float e2 = fmaf(f.kn * f.kn * dn, dn, dot(dxn, dxn));
  if (f.kb != 1.0f) {
    const KFrame k = kernel_frame(f);
    const float db = dot(d, k.b);
    e2 = fmaf((f.kb * f.kb - 1.0f) * db, db, e2);
  }
  const float ae = alpha * sqrtf(fmaxf(e2, 0.0f));
  if (!(ae > 0.0f)) return fmaxf(0.0f, -dot(d, f.g));
  return ae * psi(dot(d, f.g) / ae);
}

__device__ __forceinline__ float ndf_local(V3 m, float G, float ax, float ay, float az);

// D(m) of the anisotropic GPSS: the local-frame NDF (Eq. macro_ndf) with alpha_x = alpha,
// alpha_y = kb alpha, alpha_z = kn alpha, mean gradient (0, 0, |grad mu|).
__device__ __forceinline__ float ndf_aniso(V3 m, const Field& f, float alpha) {
  const float G = sqrtf(dot(f.g, f.g));
  V3 ml;
  if (f.kb != 1.0f) {
    const KFrame k = kernel_frame(f);
    ml = v3(dot(m, k.t), dot(m, k.b), dot(m, k.n));
  } else {
    const V3 n = hf_normal(f.g);
    const V3 c = cross(m, n);
    ml = v3(sqrtf(dot(c, c)), 0.0f, dot(m, n));
  }
  return ndf_local(ml, G, alpha, alpha * f.kb, alpha * f.kn);
}

__device__ __forceinline__ bool is_aniso(const Field& f) { return f.kb != 1.0f || f.kn != 1.0f; }

__device__ __forceinline__ float projected_area(V3 d, const Field& f, float alpha) {
  if (f.ndf != kNdfGpss) return hf_projected_area(f.ndf, d, hf_normal(f.g), alpha);
  if (is_aniso(f)) return area_aniso(d, f, alpha);
  return alpha * psi(__fdividef(dot(d, f.g), alpha));
}

// sigma_t of one object at x for direction d (0 outside its box); fills f/l.
// GEN = false: the object is known to be an isotropic stationary GPSS.
template <bool GEN = true>
__device__ __forceinline__ float sigma_t_object(const ObjectDev& o, V3 x, V3 d, Field& f, Local& l) {
  if constexpr (GEN) {
    f = fetch(o, x);
  } else {
    f = fetch_iso(o, x);
    f.ndf = kNdfGpss;
  }
  l = local_of(o, f);
  return l.rho * projected_area(d, f, l.alpha);
}

// ---------------------------------------------------------------- NDF
// Moments M3, M4 of exp(-s^2 + 2 q s) on [0, inf), returned scaled:
//   q >= 0:        Mk * exp(-q^2), forward recurrence M_{k+1} = q M_k + (k/2) M_{k-1}
//                  from M0 = sqrt(pi)/2 (1 + erf q), M1 = q M0 + exp(-q^2)/2 (all terms
//                  positive, no cancellation);
//   -3 <= q < 0:   Mk from a degree-10 Chebyshev fit of ln Mk (moment_fit.inc; there the
//                  recurrence cancels in FP32);
//   q < -3:        Mk from M0 = sqrt(pi)/2 erfcx(-q) and the continued fraction
//                  M_k/M_{k-1} = (k/2)/(|q| + M_{k+1}/M_k) (24 terms).
#include "moment_fit.inc"

__device__ __forceinline__ float cheb_eval(const float* c, float x) {
  float b1 = 0.0f, b2 = 0.0f;
  const float x2 = 2.0f * x;
#pragma unroll
  for (int k = kMomentFitDeg; k >= 1; --k) {
    const float t = fmaf(x2, b1, c[k] - b2);
    b2 = b1;
    b1 = t;
  }
  return fmaf(x, b1, c[0] - b2);
}

__device__ __forceinline__ void moments34(float q, float& m3, float& m4) {
  if (q >= 0.0f) {
    const float e = expf(-q * q);
    const float M0 = 0.5f * kSqrtPi * (1.0f + erff(q));
    const float M1 = fmaf(q, M0, 0.5f * e);
    const float M2 = fmaf(q, M1, 0.5f * M0);
    m3 = fmaf(q, M2, M1);
    m4 = fmaf(q, m3, 1.5f * M2);
  } else if (q >= kMomentFitLo) {
    const float x = fmaf(q - kMomentFitLo, 2.0f / (kMomentFitHi - kMomentFitLo), -1.0f);
    m3 = expf(cheb_eval(c_lnM3_cheb, x));
    m4 = expf(cheb_eval(c_lnM4_cheb, x));
  } else {
    const float x = -q;
    float r = 0.0f, r1 = 0.0f, r2 = 0.0f, r3 = 0.0f, r4 = 0.0f;
#pragma unroll 1
    for (int k = 24; k >= 1; --k) {
      r = (0.5f * (float)k) / (x + r);
      if (k == 4) r4 = r;
      if (k == 3) r3 = r;
      if (k == 2) r2 = r;
      if (k == 1) r1 = r;
    }
    const float M0 = 0.5f * kSqrtPi * erfcxf(x);
    m3 = M0 * r1 * r2 * r3;
    m4 = m3 * r4;
  }
}

// Isotropic world-frame NDF: g ~ N(grad mu, alpha^2/2 I).  With a = m . grad mu,
// b^2 = |grad mu x m|^2, q = a/alpha:  D = alpha/pi^(3/2) * E * M3(q), where
// E = exp(-b^2/alpha^2) for q >= 0 (moments scaled by exp(-q^2)) and
// E = exp(-|grad mu|^2/alpha^2) for q < 0.   (Appendix A result, rearranged.)
__device__ __forceinline__ float ndf_iso(V3 m, V3 g, float alpha, float* m4_over_m3 = nullptr) {
  const float inv_a = 1.0f / alpha;
  const float q = dot(m, g) * inv_a;
  float m3, m4;
  moments34(q, m3, m4);
  float E;
  if (q >= 0.0f) {
    const V3 c = cross(g, m);
    E = expf(-dot(c, c) * inv_a * inv_a);
  } else {
    E = expf(-dot(g, g) * inv_a * inv_a);
  }
  if (m4_over_m3) *m4_over_m3 = m4 / m3;
  return alpha * kInvPi32 * E * m3;
}

// Local-frame NDF with mean gradient (0,0,G) and roughness alpha_x, alpha_y, alpha_z
// (Eq. macro_ndf): D = exp(-C) M3(q) / (pi^(3/2) ax ay az A^2),  q = B/sqrt(A).
__device__ __forceinline__ float ndf_local(V3 m, float G, float ax, float ay, float az) {
  m = normalize(m);
  const float A = m.x * m.x / (ax * ax) + m.y * m.y / (ay * ay) + m.z * m.z / (az * az);
  const float B = G * m.z / (az * az);
  const float C = G * G / (az * az);
  const float sA = sqrtf(A);
  const float q = B / sA;
  float m3, m4;
  moments34(q, m3, m4);
  // q >= 0: exp(-C + q^2) = exp(-G^2 S/(az^2 A)) with S = mx^2/ax^2 + my^2/ay^2
  float E;
  if (q >= 0.0f) {
    const float S = m.x * m.x / (ax * ax) + m.y * m.y / (ay * ay);
    E = expf(-C * S / A);
  } else {
    E = expf(-C);
  }
  return E * m3 * kInvPi32 / (ax * ay * az * A * A);
}

// Local-frame projected area (Eq. generalized_lambda times cos theta, mean (0,0,G)).
__device__ __forceinline__ float projected_area_local(V3 w, float G, float ax, float ay, float az) {
  const float ae = sqrtf(ax * ax * w.x * w.x + ay * ay * w.y * w.y + az * az * w.z * w.z);
  return ae * psi(G * w.z / ae);
}

// ---------------------------------------------------------------- sampling mixture
__device__ __forceinline__ void onb(V3 n, V3& t1, V3& t2) { onb_z(n, t1, t2); }

// Beckmann proposal frame and roughness: z = sign(-d.n) n, alpha_B = clamp(alpha/|g|, 1e-3, 16);
// z = -d where |g| < 1e-6.
__device__ __forceinline__ void beckmann_frame(V3 d, V3 g, float alpha, V3& z, float& aB) {
  const float G = sqrtf(dot(g, g));
  if (G < 1e-6f) {
    z = -d;
    aB = 16.0f;
    return;
  }
  const V3 n = (1.0f / G) * g;
  z = (-dot(d, n) >= 0.0f) ? n : -n;
  aB = fminf(fmaxf(alpha / G, 1e-3f), 16.0f);
}

// (1 + Lambda(wi)) cos theta_i of the Beckmann NDF (roughness a, axis z): the normaliser
// of its visible-normal density.
__device__ __forceinline__ float beckmann_vis_den(V3 wi, V3 z, float a) {
  const float ci = fmaxf(dot(wi, z), 0.0f);
  const V3 wxz = cross(wi, z);
  const float si = sqrtf(dot(wxz, wxz));  // no cancellation near the axis
  if (si <= 0.0f) return ci;
  const float ac = ci / (a * si);
  return 0.5f * ci * (1.0f + erff(ac)) + a * si * expf(-ac * ac) * (0.5f * kInvSqrtPi);
}

// Beckmann visible-normal density <wi,m> D_B(m) / den, den = beckmann_vis_den(wi, z, a).
__device__ __forceinline__ float beckmann_vis_pdf_den(V3 m, V3 wi, V3 z, float a, float den) {
  const float wm = dot(wi, m);
  const float c = dot(m, z);
  if (wm <= 0.0f || c <= 0.0f) return 0.0f;
  const float c2 = c * c;
  const float t2 = (1.0f - c2) / c2;
  const float D = expf(-t2 / (a * a)) / (kPi * a * a * c2 * c2);
  return wm * D / den;
}

__device__ __forceinline__ float beckmann_vis_pdf(V3 m, V3 wi, V3 z, float a) {
  return beckmann_vis_pdf_den(m, wi, z, a, beckmann_vis_den(wi, z, a));
}

// Visible-normal sampling of the Beckmann NDF after Heitz & d'Eon (2014): stretch
// the incident direction to unit roughness, draw the x slope by inverting its CDF
// C(x) = cot (1+erf x)/2 + exp(-x^2)/(2 sqrt pi) (Newton, bracketed), the y slope
// from its Gaussian conditional, rotate, unstretch, slope -> normal.
__device__ __forceinline__ V3 beckmann_sample_vis(V3 wi, V3 z, float a, float u1, float u2) {
  V3 t1, t2;
  onb(z, t1, t2);
  V3 ws = normalize(v3(a * dot(wi, t1), a * dot(wi, t2), dot(wi, z)));
  const float ct = ws.z;
  // sin from the tangential components: sqrt(1 - ct^2) cancels near the axis (ct rounded
  // to 1 - 2^-24 gives 3.5e-4 for a true 1e-7), and the slope rotation below would then
  // shrink every slope toward 0 -- a rough proposal about -d (a zero mean gradient) met
  // this on a share of its samples and rendered 30% bright
  const float st = sqrtf(ws.x * ws.x + ws.y * ws.y);
  float cphi = 1.0f, sphi = 0.0f;
  if (st > 1e-7f) {
    cphi = ws.x / st;
    sphi = ws.y / st;
  }
  float sx;
  const float ux = fminf(fmaxf(2.0f * u1 - 1.0f, -0.99999994f), 0.99999994f);
  if (st < 1e-4f) {
    sx = erfinvf(ux);
  } else {
    const float cot = ct / st;
    const float total = 0.5f * cot * (1.0f + erff(cot)) + expf(-cot * cot) * (0.5f * kInvSqrtPi);
    const float target = u1 * total;
    float lo = -6.0f, hi = cot;
    float x = fminf(fmaxf(erfinvf(ux), lo), hi);
    for (int it = 0; it < 24; ++it) {
      const float e = expf(-x * x);
      const float Cx = 0.5f * cot * (1.0f + erff(x)) + e * (0.5f * kInvSqrtPi);
      const float f = Cx - target;
      if (fabsf(f) <= 2e-7f * total) break;
      if (f > 0.0f) hi = x; else lo = x;
      const float df = (cot - x) * e * kInvSqrtPi;
      float xn = df > 0.0f ? x - f / df : 0.5f * (lo + hi);
      if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
      if (hi - lo < 1e-6f * (1.0f + fabsf(x))) { x = xn; break; }
      x = xn;
    }
    sx = x;
  }
  const float uy = fminf(fmaxf(2.0f * u2 - 1.0f, -0.99999994f), 0.99999994f);
  const float sy = erfinvf(uy);
  const float px = (cphi * sx - sphi * sy) * a;
  const float py = (sphi * sx + cphi * sy) * a;
  const V3 ml = normalize(v3(-px, -py, 1.0f));
  return normalize(ml.x * t1 + ml.y * t2 + ml.z * z);
}

__device__ __forceinline__ V3 uniform_hemisphere(V3 wi, float u1, float u2) {
  V3 t1, t2;
  onb(wi, t1, t2);
  const float c = u1, s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  return normalize((s * cp) * t1 + (s * sp) * t2 + c * wi);
}

// ---------------------------------------------------------------- height-field sampling
// Visible-normal sampling of the GGX NDF (Heitz 2018, "Sampling the GGX distribution of
// visible normals"): stretch the incident direction to unit roughness, sample the
// projected hemisphere (a disk warped toward the incident direction), unstretch.
// wi.n > 0 required.
__device__ __forceinline__ V3 ggx_sample_vis(V3 wi, V3 n, float a, float u1, float u2) {
  V3 b1, b2;
  onb(n, b1, b2);
  const V3 vh = normalize(v3(a * dot(wi, b1), a * dot(wi, b2), dot(wi, n)));
  const float lensq = vh.x * vh.x + vh.y * vh.y;
  const V3 T1 = lensq > 0.0f ? rsqrtf(lensq) * v3(-vh.y, vh.x, 0.0f) : v3(1.0f, 0.0f, 0.0f);
  const V3 T2 = cross(vh, T1);
  const float r = sqrtf(u1);
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  const float t1 = r * cp;
  const float sh = 0.5f * (1.0f + vh.z);
  const float t2 = (1.0f - sh) * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1)) + sh * (r * sp);
  const V3 nh = fma3(t1, T1, fma3(t2, T2, sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2)) * vh));
  const V3 ne = normalize(v3(a * nh.x, a * nh.y, fmaxf(nh.z, 1e-7f)));
  return normalize(fma3(ne.x, b1, fma3(ne.y, b2, ne.z * n)));
}

// NDF of a field sample's object (GPSS, anisotropic GPSS or height field).
__device__ __forceinline__ float ndf_field(V3 m, const Field& f, float alpha) {
  if (f.ndf != kNdfGpss) return hf_ndf(f.ndf, m, hf_normal(f.g), alpha);
  if (is_aniso(f)) return ndf_aniso(m, f, alpha);
  return ndf_iso(m, f.g, alpha);
}

// Height-field objects: exact visible normals when the ray arrives from above n (pdf over
// half vectors max(0, wi.m) D(m)/sigma(d)), otherwise m uniform on the hemisphere about wi.
__device__ __forceinline__ float hf_pdf_m(V3 d, V3 m, const Field& f, float alpha, float sd) {
  const V3 wi = -d;
  const V3 n = hf_normal(f.g);
  if (dot(wi, m) <= 0.0f) return 0.0f;
  if (dot(wi, n) > 0.0f) return dot(wi, m) * hf_ndf(f.ndf, m, n, alpha) / sd;
  return 1.0f / kTwoPi;
}

__device__ __forceinline__ V3 hf_sample_m(V3 d, const Field& f, float alpha, float u1, float u2) {
  const V3 wi = -d;
  const V3 n = hf_normal(f.g);
  if (dot(wi, n) > 0.0f)
    return f.ndf == kNdfGgx ? ggx_sample_vis(wi, n, alpha, u1, u2) : beckmann_sample_vis(wi, n, alpha, u1, u2);
  return uniform_hemisphere(wi, u1, u2);
}

// The quantities of the sampling mixture that depend on the incoming d only: the
// Beckmann frame and roughness and its visible-normal normaliser.  A vertex sets
// them up once for its phase sample and its NEE evaluation.
struct Mix {
  V3 z;
  float aB, den, R;
};

__device__ __forceinline__ Mix mix_setup(V3 d, V3 g, float alpha, float R) {
  Mix mx;
  beckmann_frame(d, g, alpha, mx.z, mx.aB);
  mx.den = beckmann_vis_den(-d, mx.z, mx.aB);
  mx.R = R;
  return mx;
}

// mixture pdf over half-vectors m facing -d
__device__ __forceinline__ float mix_pdf_m(const Mix& mx, V3 d, V3 m) {
  const V3 wi = -d;
  if (dot(wi, m) <= 0.0f) return 0.0f;
  return mx.R * beckmann_vis_pdf_den(m, wi, mx.z, mx.aB, mx.den) + (1.0f - mx.R) * (1.0f / kTwoPi);
}

__device__ __forceinline__ float mixture_pdf_m(V3 d, V3 m, V3 g, float alpha, float R) {
  return mix_pdf_m(mix_setup(d, g, alpha, R), d, m);
}

// Phase function p(d,d2)/F = D(m) / (4 sigma(d)) and the mixture pdf over d2, with the
// mixture set up and sd = sigma(d) given.  Returns false where p = 0.
__device__ __forceinline__ bool phase_eval_mix(const Mix& mx, float sd, V3 d, V3 d2, const Field& f, float alpha,
                                               float& p_over_F, float& pdf) {
  V3 m = d2 - d;
  const float len2 = dot(m, m);
  p_over_F = 0.0f;
  pdf = 0.0f;
  if (!(len2 > 0.0f)) return false;
  m = rsqrtf(len2) * m;
  const float dm = dot(d, m);
  if (dm >= 0.0f) return false;
  p_over_F = ndf_field(m, f, alpha) / (4.0f * sd);
  pdf = (f.ndf == kNdfGpss ? mix_pdf_m(mx, d, m) : hf_pdf_m(d, m, f, alpha, sd)) / (4.0f * fabsf(dm));
  return true;
}

// Samples d2 (mixture set up, sd = sigma(d)); returns the weight p/pdf divided by F, and the pdf.
__device__ __forceinline__ bool phase_sample_mix(const Mix& mx, float sd, V3 d, const Field& f, float alpha, float u0,
                                                 float u1, float u2, V3& d2, float& w_over_F, float& pdf) {
  const V3 wi = -d;
  const bool hf = f.ndf != kNdfGpss;
  const V3 m = hf ? hf_sample_m(d, f, alpha, u1, u2)
                  : (u0 < mx.R ? beckmann_sample_vis(wi, mx.z, mx.aB, u1, u2) : uniform_hemisphere(wi, u1, u2));
  const float dm = dot(d, m);
  w_over_F = 0.0f;
  pdf = 0.0f;
  if (!(dm < 0.0f)) return false;
  d2 = normalize(fma3(-2.0f * dm, m, d));
  const float pdf_m = hf ? hf_pdf_m(d, m, f, alpha, sd) : mix_pdf_m(mx, d, m);
  if (!(pdf_m > 0.0f)) return false;
  w_over_F = ndf_field(m, f, alpha) * fabsf(dm) / (sd * pdf_m);
  // The pdf for the MIS weight of this direction is evaluated from d2 as the NEE side
  // evaluates it (half vector normalize(d2 - d)), so that the two weights of every
  // direction add to 1.  For m near grazing, d2 is close to d and the half vector
  // recomputed from d2 is not m (cancellation): the sample's own pdf_m then differs
  // from the NEE side's value, and mixing the two biased the estimate (a zero-gradient
  // fog, whose Beckmann proposal is very rough, rendered 30% bright).  The weight
  // w_over_F keeps the sample's own pdf_m, the density it was drawn from.
  pdf = 0.0f;
  V3 h = d2 - d;
  const float hl2 = dot(h, h);
  if (hl2 > 0.0f) {
    h = rsqrtf(hl2) * h;
    const float dh = dot(d, h);
    if (dh < 0.0f) pdf = (hf ? hf_pdf_m(d, h, f, alpha, sd) : mix_pdf_m(mx, d, h)) / (4.0f * fabsf(dh));
  }
  return isfinite(w_over_F);
}

// The mixture's set-up for a field sample (unused by height-field objects).
__device__ __forceinline__ Mix mix_for(V3 d, const Field& f, float alpha, float R) {
  if (f.ndf != kNdfGpss) {
    Mix mx;
    mx.z = -d;
    mx.aB = 1.0f;
    mx.den = 1.0f;
    mx.R = R;
    return mx;
  }
  return mix_setup(d, f.g, alpha, R);
}

__device__ __forceinline__ bool phase_eval(V3 d, V3 d2, const Field& f, float alpha, float R, float& p_over_F,
                                           float& pdf) {
  return phase_eval_mix(mix_for(d, f, alpha, R), projected_area(d, f, alpha), d, d2, f, alpha, p_over_F, pdf);
}

__device__ __forceinline__ bool phase_sample(V3 d, const Field& f, float alpha, float R, float u0, float u1,
                                             float u2, V3& d2, float& w_over_F, float& pdf) {
  return phase_sample_mix(mix_for(d, f, alpha, R), projected_area(d, f, alpha), d, f, alpha, u0, u1, u2, d2,
                          w_over_F, pdf);
}

// ---------------------------------------------------------------- exact visible-normal sampling
// The GPSS visible-normal distribution max(0, -d.m) D(m)/sigma(d) is the direction
// of a slope g drawn with density proportional to max(0, -d.g) N(g; grad mu, s^2 I),
// s = alpha/sqrt2 (Eq. gdf_to_ndf: D(m) = int t^3 P(t m) dt, and dg = t^2 dt dm).  In
// the frame of d, u = -d.g has density proportional to u N(u; -d.grad mu, s^2) on u > 0
// and the two components orthogonal to d are independent N(grad mu_perp, s^2).  With
// m = g/|g| and d2 = reflect(d, m) the sample's pdf is p(d,d2)/F and its weight p/pdf
// is exactly F.  (The paper leaves this sampling open and uses the mixture above.)

// Mills ratio R(x) = (1 - Phi(x))/phi(x) = sqrt(pi/2) erfcx(x/sqrt2).
__device__ __forceinline__ float mills_ratio(float x) { return kSqrtPiOver2 * erfcxf(x * kInvSqrt2); }

// q(x) = 1 - x R(x) for x >= 0, without cancellation: R(x) K(x) with Laplace's
// continued fraction K (R = 1/(x + K)) for x >= 2.
__device__ __forceinline__ float one_minus_x_mills(float x, float R) {
  return x < 2.0f ? fmaf(-x, R, 1.0f) : R * mills_cf(x);
}

// Unnormalised CDF H(y) = int_0^y t phi(t - beta) dt of the visible slope y = u/s and its
// derivative y phi(y - beta).  beta >= 0: direct form.  beta < 0 (B = -beta): both
// scaled by 1/phi(beta), H = q(B) - E (q(y+B) + y R(y+B)), E = phi(y - beta)/phi(beta).
__device__ __forceinline__ void visible_slope_cdf(float beta, float y, float& H, float& dH) {
  if (beta >= 0.0f) {
    const float t = y - beta;
    const float pt = kInvSqrt2Pi * expf(-0.5f * t * t);
    const float pb = kInvSqrt2Pi * expf(-0.5f * beta * beta);
    const float Pt = 0.5f * erfcf(-t * kInvSqrt2), Pb = 0.5f * erfcf(beta * kInvSqrt2);  // Phi(t), Phi(-beta)
    H = pb - pt + beta * (Pt - Pb);
    dH = y * pt;
  } else {
    const float B = -beta;
    const float E = expf(-y * (B + 0.5f * y));
    const float x = y + B;
    const float Rb = mills_ratio(B), Rx = mills_ratio(x);
    H = one_minus_x_mills(B, Rb) - E * (one_minus_x_mills(x, Rx) + y * Rx);
    dH = y * E;
  }
}

// The visible slope y > 0 with density proportional to y exp(-(y - beta)^2/2) at CDF
// value xi: Newton on H(y) = xi H(inf), safeguarded by bisection (at most 40 steps).
__device__ __forceinline__ float sample_visible_slope(float beta, float xi) {
  float Z;
  if (beta >= 0.0f) {
    Z = beta * 0.5f * erfcf(-beta * kInvSqrt2) + kInvSqrt2Pi * expf(-0.5f * beta * beta);
  } else {
    Z = one_minus_x_mills(-beta, mills_ratio(-beta));
  }
  const float target = xi * Z;
  float lo = 0.0f, hi;
  float y;
  if (beta >= 0.0f) {
    hi = beta + 9.0f;
    y = fmaxf(beta + kSqrt2 * erfinvf(fminf(fmaxf(2.0f * xi - 1.0f, -0.999999f), 0.999999f)), 0.5f * beta);
  } else {
    // about Gamma(2, B) for large B: mean 2/B
    hi = 9.0f + 40.0f / (1.0f - beta);
    y = 2.0f * xi / (0.5f - beta);
  }
  y = fminf(fmaxf(y, 1e-7f), hi);
#pragma unroll 1
  for (int it = 0; it < 40; ++it) {
    float H, dH;
    visible_slope_cdf(beta, y, H, dH);
    const float f = H - target;
    if (f > 0.0f) hi = y; else lo = y;
    if (fabsf(f) <= 1e-6f * Z || hi - lo <= 1e-7f * (1.0f + y)) break;
    float yn = dH > 0.0f ? y - f / dH : 0.5f * (lo + hi);
    if (!(yn > lo && yn < hi)) yn = 0.5f * (lo + hi);
    y = yn;
  }
  return y;
}

// Exact visible-normal sample (uniforms u0: slope along -d, u1, u2: the orthogonal
// slopes).  Returns false for the measure-zero case g = 0.
__device__ __forceinline__ bool vndf_sample_exact(V3 d, V3 g, float alpha, float u0, float u1, float u2, V3& m) {
  const float s = alpha * kInvSqrt2;
  const float beta = -dot(d, g) / s;
  const float y = sample_visible_slope(beta, u0);
  V3 t1, t2;
  onb(d, t1, t2);
  const float n1 = kSqrt2 * erfinvf(fminf(fmaxf(2.0f * u1 - 1.0f, -0.99999994f), 0.99999994f));
  const float n2 = kSqrt2 * erfinvf(fminf(fmaxf(2.0f * u2 - 1.0f, -0.99999994f), 0.99999994f));
  const V3 gs = fma3(-s * y, d, fma3(fmaf(s, n1, dot(g, t1)), t1, fmaf(s, n2, dot(g, t2)) * t2));
  const float len2 = dot(gs, gs);
  if (!(len2 > 0.0f)) return false;
  m = rsqrtf(len2) * gs;
  return true;
}

// Anisotropic kernels: g = grad mu + L xi with xi ~ N(0, I) and L = Sigma^(1/2) =
// (alpha/sqrt2) (I + (kb - 1) b b^T + (kn - 1) n n^T).  With v = L d, s = |v| and e = -v/s,
// -d.g = s (beta + xi.e), beta = -d.grad mu/s: the component xi.e = y - beta with y the
// visible slope above, the two components of xi orthogonal to e plain normals.
__device__ __forceinline__ V3 apply_sqrt_cov(V3 w, const KFrame& k, float kb, float kn, float s0) {
  V3 r = fma3((kb - 1.0f) * dot(w, k.b), k.b, w);
  r = fma3((kn - 1.0f) * dot(w, k.n), k.n, r);
  return s0 * r;
}

__device__ __forceinline__ bool vndf_sample_aniso(V3 d, const Field& f, float alpha, float u0, float u1, float u2,
                                                  V3& m) {
  const KFrame k = kernel_frame(f);
  const float s0 = alpha * kInvSqrt2;
  const V3 v = apply_sqrt_cov(d, k, f.kb, f.kn, s0);
  const float s = sqrtf(dot(v, v));
  if (!(s > 0.0f)) return false;
  const V3 e = (-1.0f / s) * v;
  const float beta = -dot(d, f.g) / s;
  const float y = sample_visible_slope(beta, u0);
  V3 t1, t2;
  onb(e, t1, t2);
  const float n1 = kSqrt2 * erfinvf(fminf(fmaxf(2.0f * u1 - 1.0f, -0.99999994f), 0.99999994f));
  const float n2 = kSqrt2 * erfinvf(fminf(fmaxf(2.0f * u2 - 1.0f, -0.99999994f), 0.99999994f));
  const V3 xi = fma3(y - beta, e, fma3(n1, t1, n2 * t2));
  const V3 g = f.g + apply_sqrt_cov(xi, k, f.kb, f.kn, s0);
  const float len2 = dot(g, g);
  if (!(len2 > 0.0f)) return false;
  m = rsqrtf(len2) * g;
  return true;
}

// Exact-vNDF counterpart of phase_sample_mix: weight p/pdf/F = 1, pdf = p/F.
__device__ __forceinline__ bool phase_sample_vndf(float sd, V3 d, const Field& f, float alpha, float u0, float u1,
                                                  float u2, V3& d2, float& w_over_F, float& pdf) {
  if (f.ndf != kNdfGpss) return phase_sample_mix(mix_for(d, f, alpha, 0.5f), sd, d, f, alpha, u0, u1, u2, d2, w_over_F, pdf);
  V3 m;
  w_over_F = 0.0f;
  pdf = 0.0f;
  if (!(is_aniso(f) ? vndf_sample_aniso(d, f, alpha, u0, u1, u2, m) : vndf_sample_exact(d, f.g, alpha, u0, u1, u2, m)))
    return false;
  const float dm = dot(d, m);
  if (!(dm < 0.0f)) return false;
  d2 = normalize(fma3(-2.0f * dm, m, d));
  pdf = ndf_field(m, f, alpha) / (4.0f * sd);
  w_over_F = 1.0f;
  return pdf > 0.0f && isfinite(pdf);
}

// Out-of-line entry points used at real vertices (rare compared with the
// extinction evaluations of the traversal loop); results are returned by value.
struct PhaseEval {
  float p_over_F, pdf;
  int ok;
};
struct PhaseSample {
  V3 d2;
  float w_over_F, pdf;
  int ok;
};

static __device__ __noinline__ PhaseEval phase_eval_call(V3 d, V3 d2, Field f, float alpha, float R) {
  PhaseEval r;
  r.ok = phase_eval(d, d2, f, alpha, R, r.p_over_F, r.pdf);
  return r;
}

static __device__ __noinline__ PhaseSample phase_sample_call(V3 d, Field f, float alpha, float R, float u0, float u1,
                                                      float u2) {
  PhaseSample r;
  r.d2 = d;
  r.ok = phase_sample(d, f, alpha, R, u0, u1, u2, r.d2, r.w_over_F, r.pdf);
  return r;
}

// Both phase-function uses of a real vertex with incoming d: the NEE evaluation toward
// wl and (if `sample`) the phase sample, sharing sigma(d) and the mixture's set-up.
struct VertexShade {
  PhaseEval nee;
  PhaseSample next;
};

// exact = true: the exact visible-normal sampler (its pdf is p/F, also for the NEE
// direction's MIS weight) instead of the mixture.
__device__ __forceinline__ VertexShade shade_vertex_call(V3 d, V3 wl, Field f, float alpha, float R, int sample,
                                                         bool exact, float u0, float u1, float u2) {
  const float sd = projected_area(d, f, alpha);
  VertexShade r;
  r.next.d2 = d;
  r.next.w_over_F = 0.0f;
  r.next.pdf = 0.0f;
  if (exact && f.ndf == kNdfGpss) {
    V3 m = wl - d;
    const float len2 = dot(m, m);
    r.nee.ok = 0;
    r.nee.p_over_F = 0.0f;
    r.nee.pdf = 0.0f;
    if (len2 > 0.0f) {
      m = rsqrtf(len2) * m;
      if (dot(d, m) < 0.0f) {
        r.nee.p_over_F = ndf_field(m, f, alpha) / (4.0f * sd);
        r.nee.pdf = r.nee.p_over_F;
        r.nee.ok = 1;
      }
    }
    r.next.ok = sample ? phase_sample_vndf(sd, d, f, alpha, u0, u1, u2, r.next.d2, r.next.w_over_F, r.next.pdf) : 0;
    return r;
  }
  const Mix mx = mix_for(d, f, alpha, R);
  r.nee.ok = phase_eval_mix(mx, sd, d, wl, f, alpha, r.nee.p_over_F, r.nee.pdf);
  r.next.ok = sample ? phase_sample_mix(mx, sd, d, f, alpha, u0, u1, u2, r.next.d2, r.next.w_over_F, r.next.pdf) : 0;
  return r;
}

// ---------------------------------------------------------------- lights and camera
__device__ __forceinline__ V3 env_radiance(const LightDev& L, V3 w) {
  if (L.kind == kLightSky) {
    V3 c;
    if (w.z >= 0.0f) {
      const float t = w.z;
      c = {(1.0f - t) + t * 0.35f, (1.0f - t) + t * 0.55f, 1.0f};
    } else {
      c = {0.25f, 0.22f, 0.20f};
    }
    return {c.x * L.radiance[0], c.y * L.radiance[1], c.z * L.radiance[2]};
  }
  return {L.radiance[0], L.radiance[1], L.radiance[2]};
}

__device__ __forceinline__ void camera_ray(const CameraDev& c, int px, int py, float jx, float jy, V3& o, V3& d) {
  const float x = 2.0f * ((float)px + jx) / (float)c.width - 1.0f;
  const float y = 1.0f - 2.0f * ((float)py + jy) / (float)c.height;
  const V3 f = {c.fwd[0], c.fwd[1], c.fwd[2]}, r = {c.right[0], c.right[1], c.right[2]}, u = {c.up[0], c.up[1], c.up[2]};
  const V3 e = {c.eye[0], c.eye[1], c.eye[2]};
  if (c.ortho) {
    o = e + (x * c.half_w) * r + (y * c.half_h) * u;
    d = f;
  } else {
    o = e;
    d = normalize(f + (x * c.half_w) * r + (y * c.half_h) * u);
  }
}

__device__ __forceinline__ float power_heuristic(float a, float b) {
  const float a2 = a * a, b2 = b * b;
  return a2 / (a2 + b2);
}

// ---------------------------------------------------------------- local majorant
// ln Phi(u) of the standard normal, without underflow or cancellation: log1p of the
// upper tail for u >= 0, ln(erfcx(-u/sqrt2)/2) - u^2/2 below.
__device__ __forceinline__ float log_ndtr(float u) {
  if (u >= 0.0f) return log1pf(-0.5f * erfcf(u * kInvSqrt2));
  return logf(0.5f * erfcxf(-u * kInvSqrt2)) - 0.5f * u * u;
}

// The u with ln Phi(u) = L (L <= 0): Phi^-1 through erfcinv where Phi is representable
// (the upper tail 1 - Phi = -expm1(L) above the median), else the asymptote
// u^2 = -2L - ln(-2L) - ln(2 pi) below e^-80 refined by two Newton steps on ln Phi,
// whose derivative is the inverse Mills ratio lambda(u).
__device__ __forceinline__ float inv_log_ndtr(float L) {
  if (L > -0.69314718f) return kSqrt2 * erfcinvf(fmaxf(-2.0f * expm1f(L), 1e-37f));
  if (L > -80.0f) return -kSqrt2 * erfcinvf(2.0f * expf(L));
  const float a = -2.0f * L;
  float u = -sqrtf(a - logf(a) - 1.8378771f);  // ln(2 pi)
#pragma unroll
  for (int it = 0; it < 2; ++it) u -= (log_ndtr(u) - L) / inv_mills(u);
  return u;
}

// A piece of a ray inside one field cell and its majorant: a constant sbar on
// [t0, t_end), or (lin) the linear-exponential majorant of the surface limit,
//   sbar(t) = K lambda(u(t))/s_lo,  u(t) = (mu0 - B (t - t0))/sigma_u,
// with mu0 - B (t - t0) a linear lower bound of the mean along the ray and sigma_u =
// s_hi where that bound is >= 0, s_lo where it is < 0 (lambda decreasing, so either
// choice bounds lambda(mu/sigma) for sigma in [s_lo, s_hi] on its side of 0).  Its
// optical depth is closed form, because d ln Phi(u)/du = lambda(u):
//   int sbar dt = K sigma_u/(s_lo B) [ln Phi(u(t_a)) - ln Phi(u(t_b))]
// (the Smith-height form of the transmittance of a linear mean, Sec. 4.1), for either
// sign of B, and a tentative collision at depth tau inverts it with inv_log_ndtr.
struct LocalPiece {
  float t0, t_end, sbar;       // sbar: the constant majorant, or lin's value at t0
  float mu0, B, s_hi, s_lo, K;
  int lin;
};

// Upper bound of sigma_t along the ray piece that starts at x = o + t d, from the 8
// corners of the field cell of `ob` containing x (the piece ends at that cell's exit at
// the latest).  In the cell the mean is trilinear, so:
//   - each gradient component d_a * dmu/dx_a is a bilinear blend of the cell's
//     4 edge differences along a, hence -d.grad mu <= B = sum_a max over those
//     edges of (-d_a * diff_a / h_a), and along the piece mu >= mu(x) - B (t'-t);
//   - the variance lies between the corner minimum and maximum;
//   - sigma(d) = alpha_e psi(d.grad mu/alpha_e) (Eq. generalized_lambda times cos) grows
//     with alpha_e (its derivative is e^{-a^2}/(2 sqrt pi)) and falls with d.grad mu, so
//     with d.grad mu >= -B (B signed here) and alpha_e <= a_hi, the largest roughness
//     over the cell (anisotropic kernels: the largest axis; non-stationary: the
//     smallest correlation scale at the corners), sigma(d) <= a_hi psi(-B/a_hi): about
//     B for rays approaching the shell, exponentially small for rays leaving it;
// with rho bounded as for the grid majorant (lambda decreasing).
// Rays approaching the shell (B > 0) take constant pieces whose length follows the
// distance to the shell, l = (mu(x) - 2 sigma_hi)/B, at least sigma_lo/B: a few pieces
// with about one tentative collision each instead of (cell size / sigma)^2 null
// collisions.  Rays leaving it (the signed bound B < 0: mu rises at least at rate -B,
// so the density falls along the piece) take one linear-exponential piece to the cell's
// exit (allow_lin, when mu rises by more than sigma_lo over it and the majorant at its
// start is below `cap`, the cell's grid majorant); a constant piece would hold the
// density of the start over the whole cell.
// The bound depends on x only (not on the piece's random numbers), so delta and ratio
// tracking stay unbiased.  Returns t_end <= t when x is not inside the object's box
// (the caller then keeps the cell majorant).  GEN = false: the object is known to have
// the isotropic stationary kernel.
template <bool GEN = true>
__device__ __forceinline__ LocalPiece local_piece(const ObjectDev& ob, V3 o, V3 d, float t, float t_max,
                                                  bool allow_lin, float cap) {
  LocalPiece p;
  p.t0 = t;
  p.t_end = t;
  p.sbar = 0.0f;
  p.lin = 0;
  const V3 x = fma3(t, d, o);
  if (!inside(ob, x)) return p;
  const float xx[3] = {x.x, x.y, x.z}, dd[3] = {d.x, d.y, d.z};
  float f[3];
  int ii[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f[a] = (xx[a] - ob.bmin[a]) * ob.inv_h[a];
    ii[a] = min(max((int)floorf(f[a]), 0), ob.n[a] - 2);
  }
  const int sy = ob.n[0], sz = ob.n[0] * ob.n[1];
  const int b = ii[0] + sy * ii[1] + sz * ii[2];
  float2 c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = __ldg(ob.mv + b + (k & 1) + ((k >> 1) & 1) * sy + (k >> 2) * sz);
  const float wx = fminf(fmaxf(f[0] - (float)ii[0], 0.0f), 1.0f);
  const float wy = fminf(fmaxf(f[1] - (float)ii[1], 0.0f), 1.0f);
  const float wz = fminf(fmaxf(f[2] - (float)ii[2], 0.0f), 1.0f);
  const float mu = lerpf(lerpf(lerpf(c[0].x, c[1].x, wx), lerpf(c[2].x, c[3].x, wx), wy),
                         lerpf(lerpf(c[4].x, c[5].x, wx), lerpf(c[6].x, c[7].x, wx), wy), wz);
  float v_lo = c[0].y, v_hi = c[0].y;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    v_lo = fminf(v_lo, c[k].y);
    v_hi = fmaxf(v_hi, c[k].y);
  }
  // directional decrease-rate bound B (edges along x: corner pairs k, k+1; y: k, k+2; z: k, k+4)
  float ex = -INFINITY, ey = -INFINITY, ez = -INFINITY;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!(k & 1)) ex = fmaxf(ex, -d.x * (c[k + 1].x - c[k].x));
    if (!(k & 2)) ey = fmaxf(ey, -d.y * (c[k + 2].x - c[k].x));
    if (!(k & 4)) ez = fmaxf(ez, -d.z * (c[k + 4].x - c[k].x));
  }
  const float Bs = ex * ob.inv_h[0] + ey * ob.inv_h[1] + ez * ob.inv_h[2];  // signed
  const float B = fmaxf(0.0f, Bs);
  // exit of the field cell
  float l_max = t_max - t;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0f) continue;
    const float frac = dd[a] > 0.0f ? (float)(ii[a] + 1) - f[a] : f[a] - (float)ii[a];
    l_max = fminf(l_max, fmaxf(frac, 0.0f) / (fabsf(dd[a]) * ob.inv_h[a]));
  }
  const float s_lo = sqrtf(v_lo), s_hi = sqrtf(v_hi);
  // largest roughness over the cell: alpha_max = sigma_hi sqrt2/(s_lo l_min), s_lo the
  // smallest correlation-scale factor at the corners (the interpolant stays above it)
  float a_hi = s_hi * ob.alpha_scale;
  if constexpr (GEN) {
    a_hi *= ob.amax;
    if (ob.cscale) {
      float c_lo = __ldg(ob.cscale + b);
#pragma unroll
      for (int k = 1; k < 8; ++k)
        c_lo = fminf(c_lo, __ldg(ob.cscale + b + (k & 1) + ((k >> 1) & 1) * sy + (k >> 2) * sz));
      a_hi /= c_lo;
    }
  }
  // sigma(d) = alpha_e psi(d.grad mu/alpha_e) grows with alpha_e and falls with
  // d.grad mu >= -Bs, so sigma(d) <= a_hi psi(-Bs/a_hi) (<= max(0, Bs) + a_hi/(2 sqrt pi);
  // exponentially small for rays leaving the surface)
  const float area_ub = ob.ndf == kNdfGpss ? a_hi * psi(-Bs / a_hi)
                      : 1.0f + a_hi * (ob.ndf == kNdfGgx ? 0.5f : 0.5f * kInvSqrtPi);
  const float K = area_ub * 1.001f;
  if (allow_lin && -Bs * l_max > s_lo) {
    // rounding of mu and of the positions along the piece
    const float mu0 = mu - (1e-6f * (fabsf(mu) - Bs * l_max) + 1e-7f * s_lo);
    const float s0 = K * inv_mills(mu0 / (mu0 >= 0.0f ? s_hi : s_lo)) / s_lo;
    if (s0 < cap) {
      p.t_end = t + l_max;
      p.sbar = s0;
      p.mu0 = mu0;
      p.B = Bs;
      p.s_hi = s_hi;
      p.s_lo = s_lo;
      p.K = K;
      p.lin = 1;
      return p;
    }
  }
  float l = l_max;
  if (B > 0.0f) l = fminf(fmaxf((mu - 2.0f * s_hi) / B, s_lo / B), l_max);
  float mu_b = mu - B * l;
  mu_b -= 1e-6f * (fabsf(mu) + B * l) + 1e-7f * s_lo;  // rounding of mu and of the piece's end
  const float u = mu_b >= 0.0f ? mu_b / s_hi : mu_b / s_lo;
  p.t_end = t + l;
  p.sbar = inv_mills(u) / s_lo * K;
  return p;
}

// Constant-majorant form (t_end, sbar) of local_piece (parity evaluators).
template <bool GEN = true>
static __device__ __noinline__ float2 local_majorant(const ObjectDev& ob, V3 o, V3 d, float t, float t_max) {
  const LocalPiece p = local_piece<GEN>(ob, o, d, t, t_max, false, INFINITY);
  return make_float2(p.t_end, p.sbar);
}

// Linear-exponential piece: the depth of one side of the crossing tz of the linear
// bound (sigma_u fixed) over [ta, tb].
__device__ __forceinline__ float lin_side_depth(const LocalPiece& p, float su, float ta, float tb) {
  const float ua = (p.mu0 - p.B * (ta - p.t0)) / su, ub = (p.mu0 - p.B * (tb - p.t0)) / su;
  return p.K * su / (p.s_lo * p.B) * (log_ndtr(ua) - log_ndtr(ub));
}

// sigma_u before and after the crossing tz = t0 + mu0/B along the ray: the bound falls
// through 0 for B > 0 (s_hi, then s_lo) and rises through it for B < 0.
__device__ __forceinline__ float lin_s_first(const LocalPiece& p) { return p.B > 0.0f ? p.s_hi : p.s_lo; }
__device__ __forceinline__ float lin_s_second(const LocalPiece& p) { return p.B > 0.0f ? p.s_lo : p.s_hi; }

// Linear-exponential piece: optical depth of the majorant over [ta, tb] (within the piece).
__device__ __forceinline__ float lin_depth(const LocalPiece& p, float ta, float tb) {
  const float tz = p.t0 + p.mu0 / p.B;
  float tau = 0.0f;
  if (ta < tz) tau += lin_side_depth(p, lin_s_first(p), ta, fminf(tb, tz));
  if (tb > tz) tau += lin_side_depth(p, lin_s_second(p), fmaxf(ta, tz), tb);
  return fmaxf(tau, 0.0f);
}

// Linear-exponential piece: the tentative collision at optical depth tau beyond ta
// (tau below the depth to t_max), clamped to [ta, t_max], and the majorant there.
__device__ __forceinline__ float2 lin_collision(const LocalPiece& p, float ta, float t_max, float tau) {
  const float tz = p.t0 + p.mu0 / p.B;
  float su = lin_s_second(p);
  float La;
  bool first = false;
  if (ta < tz) {
    const float s1 = lin_s_first(p);
    La = log_ndtr((p.mu0 - p.B * (ta - p.t0)) / s1);
    const float d1 = p.K * s1 / (p.s_lo * p.B) * (La + 0.69314718f);  // to the crossing: ln Phi(0) = -ln 2
    if (tau < d1) {
      su = s1;
      first = true;
    } else {
      tau -= d1;
      ta = tz;
    }
  }
  if (!first) La = log_ndtr((p.mu0 - p.B * (ta - p.t0)) / su);
  const float u = inv_log_ndtr(La - tau * p.s_lo * p.B / (p.K * su));
  const float t = fminf(fmaxf(p.t0 + (p.mu0 - su * u) / p.B, ta), t_max);
  return make_float2(t, p.K * inv_mills(u) / p.s_lo);
}

// One local piece of the traversal from t (segment end seg_end, cell majorant cap)
// consuming the optical depth tau, kept out of line so the piece's state never lives in
// the traversal loop: returns (t_hit, sbar, 0, 1) for a tentative collision,
// (piece end, sbar, tau left, 2) when the piece is crossed, and w = 0 when no local
// piece beats the cell majorant.
template <bool GEN = true>
static __device__ __noinline__ float4 local_step(const ObjectDev& ob, V3 o, V3 d, float t, float seg_end, float cap,
                                                 int lin, float tau) {
  const LocalPiece p = local_piece<GEN>(ob, o, d, t, seg_end, lin != 0, cap);
  if (!(p.t_end > t && p.sbar < cap)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float pe = fminf(p.t_end, seg_end);
  const float need = p.lin ? lin_depth(p, t, pe) : p.sbar * (pe - t);
  if (tau < need) {
    if (p.lin) {
      const float2 h = lin_collision(p, t, pe, tau);
      return make_float4(h.x, h.y, 0.0f, 1.0f);
    }
    return make_float4(t + tau / p.sbar, p.sbar, 0.0f, 1.0f);
  }
  return make_float4(pe, p.sbar, tau - fmaxf(need, 0.0f), 2.0f);
}

// ---------------------------------------------------------------- majorant traversal
// Majorant traversal consuming an optical-depth budget tau: advances to the next
// tentative collision (returns true, w.t and w.sbar set) or to the end of the ray
// (returns false).  Each step looks up the skip entry of the cell ahead of the
// current point and covers the segment to the exit of that entry's cube at its
// majorant -- a single cell (r = 0, Amanatides-Woo-style face stepping) or a cube
// of (2r+1)^3 cells in thin space.  Every segment is sampled against a valid
// upper bound of sigma_t, so delta and ratio tracking stay unbiased.
struct Walk {
  float t, t_end;
  float sbar;            // majorant at the current tentative collision
  float idx, idy, idz;   // 1/d per axis (0 where d = 0)
  int cx, cy, cz;        // current cell (exact integer stepping, no position nudging)
};

__device__ __forceinline__ int cell_index(float p, float gmin, float inv_cell, int dims) {
  return min(max((int)floorf((p - gmin) * inv_cell), 0), dims - 1);
}

// Starts a walk of grid g along the ray over [tmin, tmax] clipped to the grid's box;
// false when that is empty.
__device__ __forceinline__ bool walk_begin(const MajorantDev& g, V3 o, V3 d, float tmin, float tmax, Walk& w) {
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  float t0 = tmin, t1 = tmax;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float gmax = g.gmin[a] + g.cell[a] * g.dims[a];
    if (dd[a] == 0.0f) {
      if (oo[a] < g.gmin[a] || oo[a] > gmax) return false;
    } else {
      const float inv = 1.0f / dd[a];
      float ta = (g.gmin[a] - oo[a]) * inv, tb = (gmax - oo[a]) * inv;
      if (ta > tb) { const float tmp = ta; ta = tb; tb = tmp; }
      t0 = fmaxf(t0, ta);
      t1 = fminf(t1, tb);
    }
  }
  if (!(t1 > t0)) return false;
  w.t = t0;
  w.t_end = t1;
  w.idx = d.x != 0.0f ? 1.0f / d.x : 0.0f;
  w.idy = d.y != 0.0f ? 1.0f / d.y : 0.0f;
  w.idz = d.z != 0.0f ? 1.0f / d.z : 0.0f;
  w.cx = cell_index(fmaf(t0, d.x, o.x), g.gmin[0], g.inv_cell[0], g.dims[0]);
  w.cy = cell_index(fmaf(t0, d.y, o.y), g.gmin[1], g.inv_cell[1], g.dims[1]);
  w.cz = cell_index(fmaf(t0, d.z, o.z), g.gmin[2], g.inv_cell[2], g.dims[2]);
  return true;
}

// parameter at which the ray leaves the slab [lo, hi] of one axis (INFINITY if parallel)
__device__ __forceinline__ float slab_exit(float lo, float hi, float o, float inv, float dcomp) {
  if (dcomp == 0.0f) return INFINITY;
  return ((dcomp > 0.0f ? hi : lo) - o) * inv;
}

// LOCAL = false compiles the local-majorant branch out (scenes without thin
// objects: no register cost for it in the render kernels); GEN as for local_majorant.
// Returns kWalkHit (w.t and w.sbar at the tentative collision) or kWalkExit (the ray
// left the grid); tau is consumed.
enum WalkResult : int { kWalkExit = 0, kWalkHit = 1 };

template <bool LOCAL = true, bool GEN = true>
__device__ __forceinline__ int walk_advance(const MajorantDev& g, const ObjectDev& lob, V3 o, V3 d, Walk& w, float& tau,
                                            uint32_t& steps) {
  // Each step moves the cell index strictly past the face the ray left by (or, in
  // a local piece, t strictly forward); the cap only guards against non-finite
  // input (the ray then counts as leaving).
  for (int guard = 0; guard < (1 << 22); ++guard) {
    const float2 sk = __ldg(g.skip + w.cx + g.dims[0] * (w.cy + g.dims[1] * w.cz));
    const int r = (int)sk.y;
    const int lx = max(w.cx - r, 0), hx = min(w.cx + r, g.dims[0] - 1);
    const int ly = max(w.cy - r, 0), hy = min(w.cy + r, g.dims[1] - 1);
    const int lz = max(w.cz - r, 0), hz = min(w.cz + r, g.dims[2] - 1);
    const float ex = slab_exit(g.gmin[0] + (float)lx * g.cell[0], g.gmin[0] + (float)(hx + 1) * g.cell[0], o.x, w.idx, d.x);
    const float ey = slab_exit(g.gmin[1] + (float)ly * g.cell[1], g.gmin[1] + (float)(hy + 1) * g.cell[1], o.y, w.idy, d.y);
    const float ez = slab_exit(g.gmin[2] + (float)lz * g.cell[2], g.gmin[2] + (float)(hz + 1) * g.cell[2], o.z, w.idz, d.z);
    const float seg_end = fminf(fminf(ex, ey), fminf(ez, w.t_end));
    bool local = false;
    if (LOCAL && g.hot > 0.0f && sk.x * (seg_end - w.t) > g.hot) {
      const float4 r = local_step<GEN>(lob, o, d, w.t, seg_end, sk.x, g.lin, tau);
      if (r.w > 0.5f) {
        ++steps;
        if (r.w < 1.5f) {
          w.t = r.x;
          w.sbar = r.y;
          return kWalkHit;
        }
        tau = r.z;
        w.t = fmaxf(w.t, r.x);
        if (r.x < seg_end) continue;  // next piece in the same cell
        local = true;
      }
    }
    if (!local) {
      const float need = sk.x * (seg_end - w.t);
      ++steps;
      if (tau < need) {
        w.t += tau / sk.x;
        w.sbar = sk.x;
        return kWalkHit;
      }
      tau -= fmaxf(need, 0.0f);
      w.t = fmaxf(w.t, seg_end);
    }
    if (seg_end >= w.t_end) return kWalkExit;
    // step to the cell beyond the exit face; after a cube jump the other axes are
    // re-derived from the exit point (rounding there only yields empty segments)
    if (ex <= ey && ex <= ez) {
      w.cx = d.x > 0.0f ? hx + 1 : lx - 1;
      if ((unsigned)w.cx >= (unsigned)g.dims[0]) return kWalkExit;
      if (r > 0) {
        w.cy = cell_index(fmaf(w.t, d.y, o.y), g.gmin[1], g.inv_cell[1], g.dims[1]);
        w.cz = cell_index(fmaf(w.t, d.z, o.z), g.gmin[2], g.inv_cell[2], g.dims[2]);
      }
    } else if (ey <= ez) {
      w.cy = d.y > 0.0f ? hy + 1 : ly - 1;
      if ((unsigned)w.cy >= (unsigned)g.dims[1]) return kWalkExit;
      if (r > 0) {
        w.cx = cell_index(fmaf(w.t, d.x, o.x), g.gmin[0], g.inv_cell[0], g.dims[0]);
        w.cz = cell_index(fmaf(w.t, d.z, o.z), g.gmin[2], g.inv_cell[2], g.dims[2]);
      }
    } else {
      w.cz = d.z > 0.0f ? hz + 1 : lz - 1;
      if ((unsigned)w.cz >= (unsigned)g.dims[2]) return kWalkExit;
      if (r > 0) {
        w.cx = cell_index(fmaf(w.t, d.x, o.x), g.gmin[0], g.inv_cell[0], g.dims[0]);
        w.cy = cell_index(fmaf(w.t, d.y, o.y), g.gmin[1], g.inv_cell[1], g.dims[1]);
      }
    }
  }
  return kWalkExit;
}

// ---------------------------------------------------------------- traversal of a scene
// A scene of several objects (SceneDev::split) is walked interval by interval: the
// faces of the objects' boxes cut the ray; an interval inside exactly one box walks that
// object's own grid (og: its node spacing, its local majorants), an interval inside
// several boxes walks the union grid (their majorants added), and intervals in no box
// are skipped.  The optical-depth budget tau carries from one interval to the next, so
// the tentative collisions are those of one delta-tracking walk against a piecewise
// majorant (unbiased, as with any majorant).  The union grid alone has the resolution of
// the finest grid over the whole union box, which coarsens it (brick doubling below
// 64 Mi cells) where the objects' own spacings differ.  Other scenes walk the union grid
// (a single object's own).

// [a, b]: the ray's parameter range inside the object's box (b < a when it misses).
__device__ __forceinline__ void box_span(const ObjectDev& ob, V3 o, V3 d, float& a, float& b) {
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  a = -INFINITY;
  b = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (dd[k] == 0.0f) {
      if (oo[k] < ob.bmin[k] || oo[k] > ob.bmax[k]) b = -INFINITY;
    } else {
      const float inv = 1.0f / dd[k];
      float t0 = (ob.bmin[k] - oo[k]) * inv, t1 = (ob.bmax[k] - oo[k]) * inv;
      if (t0 > t1) {
        const float tmp = t0;
        t0 = t1;
        t1 = tmp;
      }
      a = fmaxf(a, t0);
      b = fminf(b, t1);
    }
  }
}

// The first non-empty traversal interval at or after t (below tmax): walk w started on
// its grid, gid = the object whose box alone covers it, or -1 (several: the union
// grid).  False when no box lies ahead.  og: the objects' grids (S.og, or a copy of it
// in shared memory, which the walk reads with a per-lane index at every step).
__device__ __forceinline__ bool trace_interval(const SceneDev& S, const MajorantDev* og, V3 o, V3 d, float t, float tmax,
                                               Walk& w, int& gid) {
  for (int it = 0; it <= 2 * kMaxObjects; ++it) {  // each pass moves t past one box face
    float t_next = tmax;
    int n_in = 0, who = 0;
    for (int k = 0; k < S.n_objs; ++k) {
      float a, b;
      box_span(S.obj[k], o, d, a, b);
      if (!(b > a) || b <= t) continue;
      if (a <= t) {
        ++n_in;
        who = k;
        t_next = fminf(t_next, b);
      } else {
        t_next = fminf(t_next, a);
      }
    }
    if (!(t < t_next)) return false;
    if (n_in > 0) {
      gid = n_in == 1 ? who : -1;
      if (walk_begin(gid < 0 ? S.mg : og[gid], o, d, t, t_next, w)) return true;
    }
    t = t_next;
  }
  return false;
}

// Kinds of the path kernels (template parameter TRAV), as bits: kTravLocal compiles local
// majorants in (a thin object), kTravSplitBit the per-object intervals, kTravMulti the code
// of scenes of several objects (extinctions added, the scattering object chosen; without it
// a kernel holds the single-object paths only, which keeps the adjoint's code smaller).  A
// kernel of kind k serves every scene whose kind is a subset of k.
enum : int {
  kTravLocal = 1, kTravSplitBit = 2, kTravMulti = 4,
  kTravGrid = 0, kTravSplit = kTravSplitBit | kTravMulti, kTravSplitLocal = kTravSplit | kTravLocal
};

__host__ __device__ inline int trav_of(const SceneDev& S) {
  int k = kTravGrid;
  if (S.n_objs > 1) k |= kTravMulti;
  if (S.split) {
    k |= kTravSplit;
    for (int i = 0; i < S.n_objs; ++i)
      if (S.og[i].hot > 0.0f) k |= kTravLocal;
  } else if (S.mg.hot > 0.0f) {
    k |= kTravLocal;
  }
  return k;
}

// Starts the traversal of the ray over [0, tmax].
template <bool SPLIT>
__device__ __forceinline__ bool trace_begin(const SceneDev& S, const MajorantDev* og, V3 o, V3 d, float tmax, Walk& w,
                                            int& gid) {
  gid = -1;
  if (SPLIT && S.split) return trace_interval(S, og, o, d, 0.0f, tmax, w, gid);
  return walk_begin(S.mg, o, d, 0.0f, tmax, w);
}

// Advances the traversal to the next tentative collision (kWalkHit: w.t and w.sbar set)
// or to the end of the ray (kWalkExit), consuming tau.  SPLIT compiles the per-object
// intervals in (with LOCAL: objects' grids may have local majorants).
template <bool LOCAL, bool SPLIT, bool GEN>
__device__ __forceinline__ int trace_advance(const SceneDev& S, const MajorantDev* og, V3 o, V3 d, float tmax, Walk& w,
                                             int& gid, float& tau, uint32_t& steps) {
  for (int it = 0; it <= 2 * kMaxObjects + 1; ++it) {
    const bool own = SPLIT && gid >= 0;
    if (walk_advance<LOCAL, GEN>(own ? og[gid] : S.mg, S.obj[own ? gid : 0], o, d, w, tau, steps) == kWalkHit)
      return kWalkHit;
    if (!SPLIT || !S.split || !trace_interval(S, og, o, d, w.t_end, tmax, w, gid)) return kWalkExit;
  }
  return kWalkExit;
}

// One ratio-tracking step (NEE transmittance): T *= 1 - sigma_t/majorant.  Below
// kRatioRR the estimate plays Russian roulette: it survives with probability
// T/kRatioRR and is then set to kRatioRR, else it ends at 0.  Unbiased (the
// expectation of the new T is the old T), and it ends shadow rays that cross
// dense interiors after a few steps instead of a step per unit majorant depth.
// Threshold 0.5 (measured on the 128^3 heterogeneous workload against 0.1 and
// 0.25: 11% less render time for 1.5% more per-pixel variance).
// Returns false when the estimate reached 0.
constexpr float kRatioRR = 0.5f;

__device__ __forceinline__ bool ratio_step(float& T, float st, float sbar, Rng& rng) {
  T *= fmaxf(0.0f, 1.0f - st / sbar);
  if (T < kRatioRR) {
    if (T <= 0.0f) return false;
    if (rng.next() * kRatioRR < T) {
      T = kRatioRR;
    } else {
      T = 0.0f;
      return false;
    }
  }
  return true;
}

// Total extinction of the scene at x (objects add) and the field of the object
// that an extinction-proportional choice with uniform u picks (index in *k).
__device__ __forceinline__ float scene_sigma_t(const SceneDev& s, V3 x, V3 d) {
  float tot = 0.0f;
  for (int k = 0; k < s.n_objs; ++k) {
    if (!inside(s.obj[k], x)) continue;
    Field f;
    Local l;
    tot += sigma_t_object(s.obj[k], x, d, f, l);
  }
  return tot;
}

}  // namespace gpss
