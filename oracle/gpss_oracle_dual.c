/*
 * gpss_oracle_dual.c -- FP64 oracle: forward-mode dual numbers over the field,
 * the extinction, the projected area, the NDF and the phase function, for the
 * oracle's adjoint (orc_render_grad).  TEST INFRASTRUCTURE ONLY (see
 * gpss_oracle.h).
 *
 * Nothing here is a hand-derived partial of the method: every derivative is
 * carried by the dual arithmetic through the same chain of definitions the
 * forward oracle evaluates --
 *   field (trilinear mu, grad mu, sigma^2, s(x), F)            (Sec. 4, O1)
 *   -> rho = lambda(mu/sigma)/sigma                            (Eq. macro_sigma_t)
 *   -> sigma(d) = alpha/(2 sqrt pi) e^{-a^2} - (d.g/2) erfc(a) (Eq. generalized_lambda times cos)
 *   -> D(m) = int_0^inf t^3 P(t m) dt                          (Eq. gdf_to_ndf, Eq. gdf)
 *   -> p = F D(m)/(4 sigma(d))                                 (Eq. phase, Eq. microfacet_vndf)
 * The only calculus written out is the derivative of each elementary function
 * (exp, log, sqrt, erfc, erfcx).
 *
 * The adjoint supports the isotropic GPSS (Sec. 4.2 with alpha_x = alpha_y =
 * alpha_z), stationary or with a correlation-scale grid s(x) (l(x) = l s(x)).
 *
 * Slots of the derivative vector (the parameters one field sample depends on):
 *   0..7    mean at the 8 corners of the sample's cell (corner k = (k&1, k>>1&1, k>>2))
 *   8..15   variance at the corners
 *   16..23  correlation-scale factor at the corners
 *   24      the object's length scale l
 *   25..32  albedo at the corners (one channel at a time)
 */
#include "gpss_oracle.h"
#include "gpss_oracle_internal.h"

#include <math.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* dual arithmetic                                                            */
/* ------------------------------------------------------------------------ */
orc_dual orc_dconst(double v) {
  orc_dual r;
  memset(&r, 0, sizeof(r));
  r.v = v;
  return r;
}

static orc_dual dadd(orc_dual a, orc_dual b) {
  for (int i = 0; i < ORC_ND; ++i) a.d[i] += b.d[i];
  a.v += b.v;
  return a;
}

static orc_dual dsub(orc_dual a, orc_dual b) {
  for (int i = 0; i < ORC_ND; ++i) a.d[i] -= b.d[i];
  a.v -= b.v;
  return a;
}

static orc_dual dscale(orc_dual a, double s) {
  for (int i = 0; i < ORC_ND; ++i) a.d[i] *= s;
  a.v *= s;
  return a;
}

static orc_dual dmul(orc_dual a, orc_dual b) {
  orc_dual r;
  r.v = a.v * b.v;
  for (int i = 0; i < ORC_ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}

static orc_dual ddiv(orc_dual a, orc_dual b) {
  orc_dual r;
  r.v = a.v / b.v;
  for (int i = 0; i < ORC_ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}

/* f(a) with f(a.v) = v and f'(a.v) = dv */
static orc_dual dapply(orc_dual a, double v, double dv) {
  orc_dual r;
  r.v = v;
  for (int i = 0; i < ORC_ND; ++i) r.d[i] = dv * a.d[i];
  return r;
}

static orc_dual dsqrt(orc_dual a) {
  double v = sqrt(a.v);
  return dapply(a, v, 0.5 / v);
}

static orc_dual dexp(orc_dual a) {
  double v = exp(a.v);
  return dapply(a, v, v);
}

/* erfc'(x) = -2/sqrt(pi) e^{-x^2} */
static orc_dual derfc(orc_dual a) {
  return dapply(a, erfc(a.v), -2.0 / ORC_SQRTPI * exp(-a.v * a.v));
}

/* erfcx'(x) = 2 x erfcx(x) - 2/sqrt(pi).  For x >= 26 that difference cancels;
 * there it is summed from the tail of the A&S 7.1.23 series behind orc_erfcx:
 * 2 x erfcx(x) = (2/sqrt pi) sum_m (-1)^m (2m-1)!!/(2x^2)^m, so the derivative is
 * the same sum without its m = 0 term. */
static double erfcx_deriv(double x) {
  if (x < 26.0) return 2.0 * x * orc_erfcx(x) - 2.0 / ORC_SQRTPI;
  double z2 = 2.0 * x * x, term = 1.0, sum = 0.0;
  for (int m = 1; m < 60; ++m) {
    term *= -(2.0 * m - 1.0) / z2;
    sum += term;
    if (fabs(term) < 1e-18 * fabs(sum)) break;
  }
  return 2.0 / ORC_SQRTPI * sum;
}

static orc_dual derfcx(orc_dual a) { return dapply(a, orc_erfcx(a.v), erfcx_deriv(a.v)); }

/* ------------------------------------------------------------------------ */
/* field sample with its dependence on the corner values (O1)                */
/* ------------------------------------------------------------------------ */
int orc_dual_field(const orc_object* o, const double x[3], orc_dfield* f) {
  const int n[3] = {o->nx, o->ny, o->nz};
  int i[3];
  double w[3], h[3];
  for (int a = 0; a < 3; ++a) {
    if (!(x[a] >= o->bmin[a] && x[a] <= o->bmax[a])) return 0;
    h[a] = (o->bmax[a] - o->bmin[a]) / (double)(n[a] - 1);
    double fr = (x[a] - o->bmin[a]) / h[a];
    int ia = (int)floor(fr);
    if (ia < 0) ia = 0;
    if (ia > n[a] - 2) ia = n[a] - 2;
    double wa = fr - ia;
    i[a] = ia;
    w[a] = wa < 0.0 ? 0.0 : (wa > 1.0 ? 1.0 : wa);
  }
  f->mu = orc_dconst(0.0);
  f->var = orc_dconst(0.0);
  f->cs = orc_dconst(o->cscale ? 0.0 : 1.0);
  for (int a = 0; a < 3; ++a) f->g[a] = orc_dconst(0.0);
  for (int c = 0; c < 3; ++c) f->F[c] = orc_dconst(0.0);
  const size_t plane = (size_t)n[0] * n[1] * n[2];
  for (int k = 0; k < 8; ++k) {
    int cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
    size_t idx = (size_t)(i[0] + cx) + (size_t)n[0] * ((size_t)(i[1] + cy) + (size_t)n[1] * (i[2] + cz));
    f->node[k] = (int64_t)idx;
    double wx = cx ? w[0] : 1.0 - w[0];
    double wy = cy ? w[1] : 1.0 - w[1];
    double wz = cz ? w[2] : 1.0 - w[2];
    double wt = wx * wy * wz;
    /* the interpolant and its x-, y-, z-derivatives are linear in the corner values */
    double gx = (cx ? 1.0 : -1.0) / h[0] * wy * wz;
    double gy = (cy ? 1.0 : -1.0) / h[1] * wx * wz;
    double gz = (cz ? 1.0 : -1.0) / h[2] * wx * wy;
    double mv = (double)o->mean[idx], vv = (double)o->var[idx];
    f->mu.v += wt * mv;
    f->mu.d[ORC_SLOT_MEAN + k] = wt;
    f->g[0].v += gx * mv;
    f->g[0].d[ORC_SLOT_MEAN + k] = gx;
    f->g[1].v += gy * mv;
    f->g[1].d[ORC_SLOT_MEAN + k] = gy;
    f->g[2].v += gz * mv;
    f->g[2].d[ORC_SLOT_MEAN + k] = gz;
    f->var.v += wt * vv;
    f->var.d[ORC_SLOT_VAR + k] = wt;
    if (o->cscale) {
      f->cs.v += wt * (double)o->cscale[idx];
      f->cs.d[ORC_SLOT_CS + k] = wt;
    }
    for (int c = 0; c < o->channels; ++c) {
      f->F[c].v += wt * (double)o->albedo[c * plane + idx];
      f->F[c].d[ORC_SLOT_ALB + k] = wt;
    }
  }
  if (o->channels == 1) f->F[1] = f->F[2] = f->F[0];
  /* alpha = sqrt(2) sigma / (l s(x))  (Eq. roughness) */
  orc_dual l = orc_dconst(o->length_scale);
  l.d[ORC_SLOT_L] = 1.0;
  f->sigma = dsqrt(f->var);
  f->alpha = ddiv(dscale(f->sigma, ORC_SQRT2), dmul(l, f->cs));
  return 1;
}

/* rho = lambda(mu/sigma)/sigma, lambda(u) = sqrt(2/pi)/erfcx(-u/sqrt2) (Eq. macro_sigma_t).
 * Beyond u = 28 (more than 28 standard deviations outside the mean surface)
 * lambda(u) < 1e-170 and erfcx(-u/sqrt2) heads for overflow: the density and its
 * derivatives are taken as 0 there (the forward oracle's lambda is 0 from u = 37.6). */
static orc_dual drho(const orc_dfield* f) {
  orc_dual u = ddiv(f->mu, f->sigma);
  if (u.v > 28.0) return orc_dconst(0.0);
  orc_dual lam = ddiv(orc_dconst(sqrt(2.0 / ORC_PI)), derfcx(dscale(u, -1.0 / ORC_SQRT2)));
  return ddiv(lam, f->sigma);
}

/* sigma(d) = E[max(0, -d.g)], g ~ N(grad mu, alpha^2/2 I):
 * alpha/(2 sqrt pi) e^{-a^2} - (d.grad mu)/2 erfc(a), a = d.grad mu/alpha  (the same
 * multiplied-out Eq. generalized_lambda as orc_projected_area_world) */
orc_dual orc_dual_projected_area(const orc_dfield* f, const double d[3]) {
  orc_dual dg = dadd(dadd(dscale(f->g[0], d[0]), dscale(f->g[1], d[1])), dscale(f->g[2], d[2]));
  orc_dual a = ddiv(dg, f->alpha);
  orc_dual t1 = dmul(dscale(f->alpha, 1.0 / (2.0 * ORC_SQRTPI)), dexp(dscale(dmul(a, a), -1.0)));
  orc_dual t2 = dmul(dscale(dg, 0.5), derfc(a));
  return dsub(t1, t2);
}

orc_dual orc_dual_sigma_t(const orc_dfield* f, const double d[3]) {
  return dmul(drho(f), orc_dual_projected_area(f, d));
}

/* ------------------------------------------------------------------------ */
/* NDF by quadrature of its definition, carried through the duals:           */
/*   D(m) = int_0^inf t^3 P(t m) dt,                                          */
/*   P(g') = exp(-|g' - grad mu|^2/alpha^2)/(pi^{3/2} alpha^3)  (Eq. gdf, isotropic) */
/* The integral of the dual integrand is the dual of the integral (the range */
/* does not depend on the parameters).  Adaptive Gauss-Legendre on the whole */
/* vector: a panel is split until every component agrees between one panel  */
/* and its two halves.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_dual mg, gg, inv_a2, norm; /* m.grad mu, |grad mu|^2, 1/alpha^2, 1/(pi^1.5 alpha^3) */
} dndf_ctx;

static orc_dual ndf_integrand(double t, void* vp) {
  const dndf_ctx* c = (const dndf_ctx*)vp;
  /* t^3 norm exp(-(t^2 - 2 t m.g + |g|^2)/alpha^2) */
  orc_dual q = dadd(dsub(orc_dconst(t * t), dscale(c->mg, 2.0 * t)), c->gg);
  orc_dual e = dexp(dscale(dmul(q, c->inv_a2), -1.0));
  return dscale(dmul(c->norm, e), t * t * t);
}

static orc_dual gl_panel(orc_dfn f, void* ctx, double a, double b) {
  const double *gx, *gw;
  int n = orc_gl_nodes(&gx, &gw);
  double mid = 0.5 * (a + b), h = 0.5 * (b - a);
  orc_dual s = orc_dconst(0.0);
  for (int i = 0; i < n; ++i) s = dadd(s, dscale(f(mid + h * gx[i], ctx), gw[i]));
  return dscale(s, h);
}

static double dual_err(const orc_dual* a, const orc_dual* b, const orc_dual* scale) {
  /* largest component difference relative to that component's scale */
  double e = fabs(a->v - b->v) / (fabs(scale->v) + 1e-300);
  double dmax = 0.0;
  for (int i = 0; i < ORC_ND; ++i) dmax = fmax(dmax, fabs(scale->d[i]));
  for (int i = 0; i < ORC_ND; ++i) {
    double s = fabs(scale->d[i]) + 1e-6 * dmax + 1e-300;
    e = fmax(e, fabs(a->d[i] - b->d[i]) / s);
  }
  return e;
}

static orc_dual dual_adapt(orc_dfn f, void* ctx, double a, double b, orc_dual whole, const orc_dual* scale,
                           int depth) {
  double m = 0.5 * (a + b);
  orc_dual l = gl_panel(f, ctx, a, m), r = gl_panel(f, ctx, m, b);
  orc_dual both = dadd(l, r);
  if (depth >= 20 || dual_err(&both, &whole, scale) <= 1e-11) return both;
  return dadd(dual_adapt(f, ctx, a, m, l, scale, depth + 1), dual_adapt(f, ctx, m, b, r, scale, depth + 1));
}

orc_dual orc_integrate_dual(orc_dfn f, void* ctx, const double* bp, int nb) {
  orc_dual pan[64], scale = orc_dconst(0.0), total = orc_dconst(0.0);
  if (nb > 65) nb = 65;
  for (int i = 0; i + 1 < nb; ++i) {
    pan[i] = gl_panel(f, ctx, bp[i], bp[i + 1]);
    scale.v += fabs(pan[i].v);
    for (int k = 0; k < ORC_ND; ++k) scale.d[k] += fabs(pan[i].d[k]);
  }
  for (int i = 0; i + 1 < nb; ++i) total = dadd(total, dual_adapt(f, ctx, bp[i], bp[i + 1], pan[i], &scale, 0));
  return total;
}

orc_dual orc_dual_ndf(const orc_dfield* f, const double m_in[3]) {
  double m[3] = {m_in[0], m_in[1], m_in[2]};
  double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int a = 0; a < 3; ++a) m[a] /= len;
  dndf_ctx c;
  c.mg = dadd(dadd(dscale(f->g[0], m[0]), dscale(f->g[1], m[1])), dscale(f->g[2], m[2]));
  c.gg = dadd(dadd(dmul(f->g[0], f->g[0]), dmul(f->g[1], f->g[1])), dmul(f->g[2], f->g[2]));
  orc_dual a2 = dmul(f->alpha, f->alpha);
  c.inv_a2 = ddiv(orc_dconst(1.0), a2);
  c.norm = ddiv(orc_dconst(1.0 / pow(ORC_PI, 1.5)), dmul(a2, f->alpha));
  /* the integrand peaks near the root of d/dt [3 ln t - (t - m.g)^2/alpha^2]; panels
   * at multiples of alpha about it (as the forward oracle's D) */
  double al = f->alpha.v, B = c.mg.v;
  double tmode = 0.5 * (B + sqrt(B * B + 6.0 * al * al));
  static const double ks[] = {-16.0, -8.0, -4.0, -2.0, -1.0, 0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 40.0};
  double bp[16];
  int nb = 0;
  bp[nb++] = 0.0;
  for (size_t i = 0; i < sizeof(ks) / sizeof(ks[0]); ++i) {
    double t = tmode + ks[i] * al;
    if (t > bp[nb - 1]) bp[nb++] = t;
  }
  return orc_integrate_dual(ndf_integrand, &c, bp, nb);
}

/* ln of the conductor phase function without F: ln(D(m)/(4 sigma(d))), m = (d2 - d)/|d2 - d|
 * (Eq. phase); returns 0 where p = 0 (the sample has no gradient then). */
int orc_dual_log_phase(const orc_dfield* f, const double d[3], const double d2[3], orc_dual* out) {
  double m[3] = {d2[0] - d[0], d2[1] - d[1], d2[2] - d[2]};
  double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  if (!(len > 0.0)) return 0;
  for (int a = 0; a < 3; ++a) m[a] /= len;
  if (d[0] * m[0] + d[1] * m[1] + d[2] * m[2] >= 0.0) return 0;
  orc_dual D = orc_dual_ndf(f, m);
  orc_dual sd = orc_dual_projected_area(f, d);
  if (!(D.v > 0.0) || !(sd.v > 0.0)) return 0;
  orc_dual r;
  r.v = log(D.v) - log(sd.v) - log(4.0);
  for (int i = 0; i < ORC_ND; ++i) r.d[i] = D.d[i] / D.v - sd.d[i] / sd.v;
  *out = r;
  return 1;
}

int orc_dual_eval(const orc_object* o, int what, const double x[3], const double d[3], const double d2[3],
                  double* out_v, double* out_d, int64_t* node) {
  orc_dfield f;
  if (!orc_dual_field(o, x, &f)) return 0;
  orc_dual r;
  if (what == 0) {
    r = orc_dual_sigma_t(&f, d);
  } else if (what == 1) {
    r = orc_dual_projected_area(&f, d);
  } else if (what == 2) {
    r = orc_dual_ndf(&f, d2);
  } else if (what == 3) {
    if (!orc_dual_log_phase(&f, d, d2, &r)) return 0;
  } else {
    return 0;
  }
  *out_v = r.v;
  for (int i = 0; i < ORC_ND; ++i) out_d[i] = r.d[i];
  for (int k = 0; k < 8; ++k) node[k] = f.node[k];
  return 1;
}
