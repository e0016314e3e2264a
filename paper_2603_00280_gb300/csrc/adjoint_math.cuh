// adjoint_math.cuh -- partial derivatives of the extinction and of the phase-function
// factors, and their scatter to grid nodes (used by the adjoint instance of the path
// kernel).  Derivations (u = mu/sigma, lambda = phi/Phi, a = d.grad mu/alpha,
// alpha = sqrt2 sigma/l, q = m.grad mu/alpha, M_k the NDF moments):
//   d sigma_t/d mu      = sigma(d) lambda'(u)/sigma^2,   lambda' = -lambda (u + lambda)
//   d sigma_t/d grad mu = -rho erfc(a)/2 d
//   d sigma_t/d sigma   = -sigma(d) (lambda' u + lambda)/sigma^2 + rho e^{-a^2}/(2 sqrt pi) alpha/sigma
//   d sigma_t/d l       = -rho e^{-a^2}/(2 sqrt pi) alpha/l
//   d ln D/d grad mu    = (2 M4/(alpha M3)) m - (2/alpha^2) grad mu
//   d ln D/d alpha      = 1/alpha + 2|grad mu|^2/alpha^3 - 2 q M4/(alpha M3)
//   d ln sigma(d)/d grad mu = -erfc(a)/(2 sigma(d)) d,   d ln sigma(d)/d alpha = e^{-a^2}/(2 sqrt pi sigma(d))
// A vertex with incoming d contributes W_nee d ln(F D(m_nee)/sigma(d)) + W_ph d ln(F D(m_ph)/sigma(d)):
// the sigma(d) part is shared, weighted by W_nee + W_ph.
#pragma once

#include "gpss_device.cuh"

namespace gpss {

// psi(a) and the two ratios erfc(a)/psi(a), (e^{-a^2}/(2 sqrt pi))/psi(a), without
// underflow for large a (continued fraction as in psi(); for a > 2 the ratios follow
// from K alone and from erfcx).
__device__ __forceinline__ void psi_ratios(float a, float& ps, float& ec_over, float& ea_over) {
  const float ex = exp_neg_sq(a);
  const float E = erfcxf(fabsf(a));
  const float ec = erfc_from(a, ex, E);
  if (a <= 2.0f) {
    const float ea = 0.5f * kInvSqrtPi * ex;
    ps = fmaf(-0.5f * a, ec, ea);
    ec_over = ec / ps;
    ea_over = ea / ps;
  } else {
    const float r = mills_cf(kSqrt2 * a);
    ps = ec * r * (0.5f * kInvSqrt2);
    ec_over = 2.0f * kSqrt2 / r;
    ea_over = kSqrt2 * kInvSqrtPi / (E * r);
  }
}

// Extinction of one object and its partials at a field sample.
struct DSig {
  float st, dmu, dvar, dl;
  V3 dg;
};

// st is evaluated by the forward's own expressions (local_of, projected_area), so that
// the adjoint's tentative-collision decisions replay the forward's bit for bit; the
// partials reuse sigma, alpha and rho from it.
__device__ __forceinline__ DSig dsigma_t(const ObjectDev& o, const Field& f, V3 d) {
  const Local l = local_of(o, f);
  const float sig = l.sigma, alpha = l.alpha, rho = l.rho;  // alpha = sqrt2 sigma/(s(x) l)
  const float u = f.mu / sig;
  const float lam = rho * sig;
  const float lamp = -lam * (u + lam);
  float ps, ec_over, ea_over;
  psi_ratios(dot(d, f.g) / alpha, ps, ec_over, ea_over);
  const float S = alpha * ps;
  DSig r;
  r.st = rho * projected_area(d, f, alpha);
  r.dmu = S * lamp / f.var;
  // sigma(d) = alpha psi(d.grad mu/alpha): the alpha cancels, d sigma(d)/d grad mu = psi'(a) d
  // = -erfc(a)/2 d, with erfc(a) = ec_over psi
  r.dg = (-0.5f * rho * ps * ec_over) * d;
  const float dsig = S * (-(lamp * u + lam) / f.var) + rho * ps * ea_over * alpha / sig;
  r.dvar = dsig / (2.0f * sig);
  // d/dl of the object's l (l(x) = s(x) l, alpha proportional to 1/l): 1/l = alpha_scale/sqrt2
  r.dl = -rho * ps * ea_over * alpha * (o.alpha_scale * kInvSqrt2);
  return r;
}

// d ln D(m) with respect to grad mu and alpha (the variance and l act through alpha).
struct DLogNdf {
  V3 dg;
  float dalpha;
};

static __device__ __noinline__ DLogNdf dlog_ndf(V3 m, Field f, float alpha) {
  float r4;
  ndf_iso(m, f.g, alpha, &r4);
  const float inv_a = 1.0f / alpha;
  const float q = dot(m, f.g) * inv_a;
  DLogNdf r;
  r.dg = fma3(-2.0f * inv_a * inv_a, f.g, (2.0f * r4 * inv_a) * m);
  r.dalpha = inv_a + 2.0f * dot(f.g, f.g) * inv_a * inv_a * inv_a - 2.0f * r4 * q * inv_a;
  return r;
}

// Scatters c_mu * dmu/d(node) + c_g . d(grad mu)/d(node) and c_var * dvar/d(node) into the
// interleaved (d mean, d variance) gradient buffer: one 8-byte atomic per node.
static __device__ __noinline__ void scatter_field(const ObjectDev& o, V3 x, float cmu, V3 cg, float cvar,
                                                  float2* __restrict__ dmv) {
  float wx, wy, wz;
  const int b = cell_of(o, x, wx, wy, wz);
  const int sy = o.n[0], sz = o.n[0] * o.n[1];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const float ax = cx ? wx : 1.0f - wx, ay = cy ? wy : 1.0f - wy, az = cz ? wz : 1.0f - wz;
    const float sx = cx ? 1.0f : -1.0f, syy = cy ? 1.0f : -1.0f, szz = cz ? 1.0f : -1.0f;
    const float w = ax * ay * az;
    const float gx = sx * ay * az * o.inv_h[0], gy = ax * syy * az * o.inv_h[1], gz = ax * ay * szz * o.inv_h[2];
    const int idx = b + cx + sy * cy + sz * cz;
    atomicAdd(dmv + idx, make_float2(fmaf(cmu, w, fmaf(cg.x, gx, fmaf(cg.y, gy, cg.z * gz))), cvar * w));
  }
}

// Scatters c * d(value at x)/d(node) of a trilinearly interpolated scalar node grid.
static __device__ __noinline__ void scatter_scalar(const ObjectDev& o, V3 x, float c, float* __restrict__ d) {
  float wx, wy, wz;
  const int b = cell_of(o, x, wx, wy, wz);
  const int sy = o.n[0], sz = o.n[0] * o.n[1];
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
    const float w = (cx ? wx : 1.0f - wx) * (cy ? wy : 1.0f - wy) * (cz ? wz : 1.0f - wz);
    atomicAdd(d + b + cx + sy * cy + sz * cz, c * w);
  }
}

static __device__ __noinline__ void scatter_albedo(const ObjectDev& o, V3 x, V3 c, float* __restrict__ dalb) {
  float wx, wy, wz;
  const int b = cell_of(o, x, wx, wy, wz);
  const int sy = o.n[0], sz = o.n[0] * o.n[1];
  const int plane = sz * o.n[2];
  const float cc[3] = {c.x, c.y, c.z};
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
    const float w = (cx ? wx : 1.0f - wx) * (cy ? wy : 1.0f - wy) * (cz ? wz : 1.0f - wz);
    const int idx = b + cx + sy * cy + sz * cz;
    if (o.channels == 1) {
      atomicAdd(dalb + idx, (cc[0] + cc[1] + cc[2]) * w);
    } else {
      for (int ch = 0; ch < 3; ++ch) atomicAdd(dalb + ch * plane + idx, cc[ch] * w);
    }
  }
}

}  // namespace gpss
