/*
 * gpss_oracle_medium.c -- FP64 oracle: special functions, grid fields, the
 * GPSS extinction, NDF and phase function.  TEST INFRASTRUCTURE ONLY (see
 * gpss_oracle.h).  Each function names the passage of the paper it follows.
 */
#include "gpss_oracle.h"
#include "gpss_oracle_internal.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Special functions.  phi/Phi are the notation of Sec. 3 (Table notations). */
/* ------------------------------------------------------------------------ */

/* exp(x^2) evaluated with x^2 split so that the large part is exact. */
static double exp_sq(double x) {
  double xh = floor(x * 1048576.0) / 1048576.0; /* 20 fractional bits: xh^2 exact */
  double xl = x - xh;
  return exp(xh * xh) * exp((x + xh) * xl);
}

/* Scaled complementary error function exp(x^2) erfc(x).  For x >= 26 the
 * asymptotic expansion of Abramowitz & Stegun 7.1.23 is summed; below that
 * the product of exp(x^2) and the C library's erfc is used directly. */
double orc_erfcx(double x) {
  if (x < 0.0) {
    if (x < -26.6) return INFINITY;
    return 2.0 * exp_sq(x) - orc_erfcx(-x);
  }
  if (x < 26.0) return exp_sq(x) * erfc(x);
  double z2 = 2.0 * x * x, term = 1.0, sum = 1.0;
  for (int m = 1; m < 60; ++m) {
    term *= -(2.0 * m - 1.0) / z2;
    sum += term;
    if (fabs(term) < 1e-18) break;
  }
  return sum / (x * ORC_SQRTPI);
}

/* ln Phi(u) for the standard normal CDF Phi. */
double orc_log_ndtr(double u) {
  if (u > 0.0) return log1p(-0.5 * erfc(u / ORC_SQRT2));
  if (u > -20.0) return log(0.5 * erfc(-u / ORC_SQRT2));
  double t = -u / ORC_SQRT2;
  return -t * t + log(0.5 * orc_erfcx(t));
}

/* Inverse Mills ratio lambda(u) = phi(u)/Phi(u) = sqrt(2/pi)/erfcx(-u/sqrt2).
 * The density of Eq. macro_sigma_t is rho(f) = lambda(f/sigma)/sigma. */
double orc_inv_mills(double u) {
  double e = orc_erfcx(-u / ORC_SQRT2);
  if (isinf(e)) return 0.0;
  return sqrt(2.0 / ORC_PI) / e;
}

/* erf^{-1} by bisection on the C library's erf (slow, exact to ~1 ulp). */
double orc_erfinv(double v) {
  if (v <= -1.0) return -INFINITY;
  if (v >= 1.0) return INFINITY;
  double lo = -7.0, hi = 7.0;
  for (int i = 0; i < 200 && hi - lo > 1e-16 * (1.0 + fabs(lo)); ++i) {
    double mid = 0.5 * (lo + hi);
    if (erf(mid) < v) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw (SC'11).       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four uniforms in (0,1) for counter (pixel, sample, bounce|purpose<<16, draw). */
void orc_uniform4(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t bounce,
                  uint32_t purpose, uint32_t draw, double u[4]) {
  uint32_t ctr[4] = {pixel, sample, (bounce & 0xFFFFu) | (purpose << 16), draw};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = ((double)r[i] + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Grid fields.  Node-centred grids spanning the box, trilinear interpolation;
 * the gradient is that of the interpolant.  The paper's mean function is a
 * signed distance field whose normalised gradient is the normal (Sec. 4).   */
/* ------------------------------------------------------------------------ */
int orc_field(const orc_object* o, const double x[3], double* mu, double grad[3],
              double* var, double albedo[3]) {
  const int n[3] = {o->nx, o->ny, o->nz};
  int i[3];
  double w[3], h[3];
  for (int a = 0; a < 3; ++a) {
    if (!(x[a] >= o->bmin[a] && x[a] <= o->bmax[a])) return 0;
    h[a] = (o->bmax[a] - o->bmin[a]) / (double)(n[a] - 1);
    double f = (x[a] - o->bmin[a]) / h[a];
    int ia = (int)floor(f);
    if (ia < 0) ia = 0;
    if (ia > n[a] - 2) ia = n[a] - 2;
    double wa = f - ia;
    if (wa < 0.0) wa = 0.0;
    if (wa > 1.0) wa = 1.0;
    i[a] = ia;
    w[a] = wa;
  }
  double m = 0.0, v = 0.0, g[3] = {0.0, 0.0, 0.0}, al[3] = {0.0, 0.0, 0.0};
  const size_t plane = (size_t)n[0] * n[1] * n[2];
  for (int c = 0; c < 8; ++c) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    size_t idx = (size_t)(i[0] + cx) + (size_t)n[0] * ((size_t)(i[1] + cy) + (size_t)n[1] * (i[2] + cz));
    double wx = cx ? w[0] : 1.0 - w[0];
    double wy = cy ? w[1] : 1.0 - w[1];
    double wz = cz ? w[2] : 1.0 - w[2];
    double sx = cx ? 1.0 : -1.0, sy = cy ? 1.0 : -1.0, sz = cz ? 1.0 : -1.0;
    double wt = wx * wy * wz;
    double mv = (double)o->mean[idx];
    m += wt * mv;
    v += wt * (double)o->var[idx];
    g[0] += sx / h[0] * wy * wz * mv;
    g[1] += sy / h[1] * wx * wz * mv;
    g[2] += sz / h[2] * wx * wy * mv;
    for (int ch = 0; ch < o->channels; ++ch) al[ch] += wt * (double)o->albedo[ch * plane + idx];
  }
  if (o->channels == 1) al[1] = al[2] = al[0];
  if (mu) *mu = m;
  if (var) *var = v;
  if (grad) { grad[0] = g[0]; grad[1] = g[1]; grad[2] = g[2]; }
  if (albedo) { albedo[0] = al[0]; albedo[1] = al[1]; albedo[2] = al[2]; }
  return 1;
}

/* Trilinear interpolation of a node grid (plane `c` of a multi-plane grid) at x,
 * which lies in the box (same cell rule as orc_field). */
static double interp_plane(const orc_object* o, const float* grid, int c, const double x[3]) {
  const int n[3] = {o->nx, o->ny, o->nz};
  int i[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    double h = (o->bmax[a] - o->bmin[a]) / (double)(n[a] - 1);
    double f = (x[a] - o->bmin[a]) / h;
    int ia = (int)floor(f);
    if (ia < 0) ia = 0;
    if (ia > n[a] - 2) ia = n[a] - 2;
    double wa = f - ia;
    i[a] = ia;
    w[a] = wa < 0.0 ? 0.0 : (wa > 1.0 ? 1.0 : wa);
  }
  const size_t plane = (size_t)n[0] * n[1] * n[2];
  double v = 0.0;
  for (int k = 0; k < 8; ++k) {
    int cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
    size_t idx = (size_t)(i[0] + cx) + (size_t)n[0] * ((size_t)(i[1] + cy) + (size_t)n[1] * (i[2] + cz));
    double wt = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) * (cz ? w[2] : 1.0 - w[2]);
    v += wt * (double)grid[c * plane + idx];
  }
  return v;
}

static void basis(const double z[3], double t1[3], double t2[3]);

int orc_point(const orc_object* o, const double x[3], orc_fpt* p) {
  if (!orc_field(o, x, &p->mu, p->g, &p->var, p->F)) return 0;
  p->sigma = sqrt(p->var);
  p->G = sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);
  for (int a = 0; a < 3; ++a) p->nhat[a] = p->G > 0.0 ? p->g[a] / p->G : 0.0;
  p->ndf = o->ndf;
  /* correlation lengths at x: l_a s(x) (Eq. roughness per axis of the local frame) */
  double s = o->cscale ? interp_plane(o, o->cscale, 0, x) : 1.0;
  double lt = o->length_scale * s;
  double lb = (o->length_scale_b > 0.0 ? o->length_scale_b : o->length_scale) * s;
  double ln = (o->length_scale_n > 0.0 ? o->length_scale_n : o->length_scale) * s;
  p->alpha = ORC_SQRT2 * p->sigma / lt;
  p->ax = p->alpha;
  p->ay = ORC_SQRT2 * p->sigma / lb;
  p->az = ORC_SQRT2 * p->sigma / ln;
  p->aniso = (lb != lt || ln != lt);
  /* frame: n from the mean gradient, t from the tangent field */
  if (p->G > 0.0) {
    for (int a = 0; a < 3; ++a) p->fn[a] = p->nhat[a];
  } else {
    p->fn[0] = 0.0; p->fn[1] = 0.0; p->fn[2] = 1.0;
  }
  double t[3] = {0.0, 0.0, 0.0};
  if (o->tangent)
    for (int a = 0; a < 3; ++a) t[a] = interp_plane(o, o->tangent, a, x);
  double tn = t[0] * p->fn[0] + t[1] * p->fn[1] + t[2] * p->fn[2];
  double tp[3] = {t[0] - tn * p->fn[0], t[1] - tn * p->fn[1], t[2] - tn * p->fn[2]};
  double l2 = tp[0] * tp[0] + tp[1] * tp[1] + tp[2] * tp[2];
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  if (l2 > 1e-12 * t2 && l2 > 0.0) {
    double il = 1.0 / sqrt(l2);
    for (int a = 0; a < 3; ++a) p->ft[a] = tp[a] * il;
    p->fb[0] = p->fn[1] * p->ft[2] - p->fn[2] * p->ft[1];
    p->fb[1] = p->fn[2] * p->ft[0] - p->fn[0] * p->ft[2];
    p->fb[2] = p->fn[0] * p->ft[1] - p->fn[1] * p->ft[0];
  } else {
    basis(p->fn, p->ft, p->fb);
  }
  return 1;
}

/* components of v in the kernel frame (t, b, n) */
static void kernel_frame_coords(const orc_fpt* p, const double v[3], double out[3]) {
  out[0] = v[0] * p->ft[0] + v[1] * p->ft[1] + v[2] * p->ft[2];
  out[1] = v[0] * p->fb[0] + v[1] * p->fb[1] + v[2] * p->fb[2];
  out[2] = v[0] * p->fn[0] + v[1] * p->fn[1] + v[2] * p->fn[2];
}

/* ------------------------------------------------------------------------ */
/* Projected area (Eq. generalized_lambda and the line sigma = Lambda cos):  */
/* Lambda(w) cos(theta) with a = cos(theta)/alpha_perp multiplied out:      */
/*   sigma(w) = alpha_e/(2 sqrt(pi)) exp(-a^2) - (1/2) G w_z erfc(a),       */
/*   alpha_e^2 = alpha_x^2 w_x^2 + alpha_y^2 w_y^2 + alpha_z^2 w_z^2,       */
/*   a = G w_z / alpha_e,                                                    */
/* where G is the length of the mean gradient (the paper's G = 1).          */
/* ------------------------------------------------------------------------ */
double orc_projected_area_local(const double w[3], double G, double ax, double ay, double az) {
  double ae = sqrt(ax * ax * w[0] * w[0] + ay * ay * w[1] * w[1] + az * az * w[2] * w[2]);
  double proj = G * w[2];
  double a = proj / ae;
  return ae / (2.0 * ORC_SQRTPI) * exp(-a * a) - 0.5 * proj * erfc(a);
}

/* ------------------------------------------------------------------------ */
/* Height-field macrofacet (Sec. 4.1, Eq. macro_sigma_t): Smith's Lambda of   */
/* the chosen NDF for a direction in the upper hemisphere (cos theta = c > 0):*/
/*   Beckmann: a = c/(alpha sin theta), Lambda = (e^{-a^2}/(a sqrt pi) - erfc a)/2 */
/*   GGX:      Lambda = (-1 + sqrt(1 + alpha^2 tan^2 theta))/2                */
/* sigma(w) = Lambda(w) w_z for w_z >= 0 and (1 + Lambda(-w)) |w_z| below.    */
/* ------------------------------------------------------------------------ */
static double smith_lambda(double c, int ndf, double alpha) {
  double s = sqrt(fmax(0.0, 1.0 - c * c));
  if (ndf == ORC_NDF_GGX) {
    if (c <= 0.0) return INFINITY;
    double t = s / c;
    return 0.5 * (-1.0 + sqrt(1.0 + alpha * alpha * t * t));
  }
  if (s == 0.0) return 0.0;
  double a = c / (alpha * s);
  if (a <= 0.0) return INFINITY;
  return 0.5 * (exp(-a * a) / (a * ORC_SQRTPI) - erfc(a));
}

double orc_projected_area_hf(const double w[3], int ndf, double alpha) {
  double c = w[2] / sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double s = sqrt(fmax(0.0, 1.0 - c * c));
  double cu = fabs(c);
  if (cu < 1e-12) {
    /* grazing: Lambda cos -> alpha/(2 sqrt pi) (Beckmann), alpha/2 (GGX) */
    return ndf == ORC_NDF_GGX ? 0.5 * alpha * s : alpha * s / (2.0 * ORC_SQRTPI);
  }
  double lam = smith_lambda(cu, ndf, alpha);
  return c >= 0.0 ? lam * cu : (1.0 + lam) * cu;
}

double orc_ndf_hf(const double m[3], int ndf, double alpha) {
  double c = m[2] / sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  if (c <= 0.0) return 0.0;
  double c2 = c * c, t2 = (1.0 - c2) / c2, a2 = alpha * alpha;
  if (ndf == ORC_NDF_GGX) {
    double q = a2 + t2;
    return a2 / (ORC_PI * c2 * c2 * q * q);
  }
  return exp(-t2 / a2) / (ORC_PI * a2 * c2 * c2);
}

/* components of v in a frame with the unit vector n as its z axis */
static void to_frame(const double v[3], const double n[3], double out[3]);

/* World-frame isotropic form for a field point: the mean gradient is g. */
double orc_projected_area_world(const double d[3], const orc_fpt* p) {
  if (p->ndf != ORC_NDF_GPSS) {
    double dl[3];
    to_frame(d, p->nhat, dl);
    return orc_projected_area_hf(dl, p->ndf, p->alpha);
  }
  if (p->aniso) {
    /* the paper's local frame: mean gradient (0, 0, G), roughness per axis */
    double dl[3];
    kernel_frame_coords(p, d, dl);
    return orc_projected_area_local(dl, p->G, p->ax, p->ay, p->az);
  }
  double dg = d[0] * p->g[0] + d[1] * p->g[1] + d[2] * p->g[2];
  double a = dg / p->alpha;
  return p->alpha / (2.0 * ORC_SQRTPI) * exp(-a * a) - 0.5 * dg * erfc(a);
}

/* ------------------------------------------------------------------------ */
/* NDF from its definition (Eq. gdf_to_ndf):  D(m) = int_0^inf t^3 P(t m) dt, */
/* P the Gaussian density of the gradient (Eq. gdf) with mean (0,0,G) and     */
/* covariance diag(alpha_a^2/2).  Evaluated by adaptive Gauss-Legendre        */
/* quadrature on a finite range around the peak of the integrand.             */
/* ------------------------------------------------------------------------ */
typedef struct { double m[3], G, ax, ay, az, norm; } ndf_ctx;

static double ndf_integrand(double t, void* vp) {
  const ndf_ctx* c = (const ndf_ctx*)vp;
  double ex = t * c->m[0] / c->ax, ey = t * c->m[1] / c->ay, ez = (t * c->m[2] - c->G) / c->az;
  return t * t * t * c->norm * exp(-(ex * ex + ey * ey + ez * ez));
}

double orc_ndf_local(const double m[3], double G, double ax, double ay, double az) {
  ndf_ctx c;
  double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int a = 0; a < 3; ++a) c.m[a] = m[a] / len;
  c.G = G; c.ax = ax; c.ay = ay; c.az = az;
  c.norm = 1.0 / (pow(ORC_PI, 1.5) * ax * ay * az);
  double A = c.m[0] * c.m[0] / (ax * ax) + c.m[1] * c.m[1] / (ay * ay) + c.m[2] * c.m[2] / (az * az);
  double B = G * c.m[2] / (az * az);
  double w = 1.0 / sqrt(A);
  double tmode = (B + sqrt(B * B + 6.0 * A)) / (2.0 * A);
  static const double ks[] = {-16.0, -8.0, -4.0, -2.0, -1.0, 0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 40.0};
  double bp[16];
  int nb = 0;
  bp[nb++] = 0.0;
  for (size_t i = 0; i < sizeof(ks) / sizeof(ks[0]); ++i) {
    double t = tmode + ks[i] * w;
    if (t > bp[nb - 1]) bp[nb++] = t;
  }
  double rough = 0.0;
  for (int i = 0; i + 1 < nb; ++i) rough += orc_integrate_rough(ndf_integrand, &c, bp[i], bp[i + 1]);
  double tol = 1e-13 * fabs(rough) / nb + 1e-300;
  double total = 0.0;
  for (int i = 0; i + 1 < nb; ++i) total += orc_integrate(ndf_integrand, &c, bp[i], bp[i + 1], tol);
  return total;
}

/* World-frame NDF for a field point (isotropic kernel): rotate m so that the
 * mean gradient is the local z axis; only m . nhat matters. */
double orc_ndf_world(const double m[3], const orc_fpt* p) {
  if (p->ndf != ORC_NDF_GPSS) {
    double ml[3];
    to_frame(m, p->nhat, ml);
    return orc_ndf_hf(ml, p->ndf, p->alpha);
  }
  if (p->aniso) {
    double ml[3];
    kernel_frame_coords(p, m, ml);
    return orc_ndf_local(ml, p->G, p->ax, p->ay, p->az);
  }
  double c = 1.0;
  if (p->G > 0.0) c = m[0] * p->nhat[0] + m[1] * p->nhat[1] + m[2] * p->nhat[2];
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  double ml[3] = {sqrt(fmax(0.0, 1.0 - c * c)), 0.0, c};
  return orc_ndf_local(ml, p->G, p->alpha, p->alpha, p->alpha);
}

/* ------------------------------------------------------------------------ */
/* Extinction (Eq. generalized_sigma_t): sigma_t = rho * sigma(d),           */
/* rho = phi(mu;0,sigma^2)/Phi(mu;0,sigma^2) = lambda(mu/sigma)/sigma.       */
/* ------------------------------------------------------------------------ */
double orc_sigma_t_point(const orc_fpt* p, const double d[3]) {
  double rho = orc_inv_mills(p->mu / p->sigma) / p->sigma;
  return rho * orc_projected_area_world(d, p);
}

double orc_sigma_t_object(const orc_object* o, const double x[3], const double d[3]) {
  orc_fpt p;
  if (!orc_point(o, x, &p)) return 0.0;
  return orc_sigma_t_point(&p, d);
}

double orc_sigma_t(const orc_scene* s, const double x[3], const double d[3]) {
  double sum = 0.0;
  for (int k = 0; k < s->n_objs; ++k) sum += orc_sigma_t_object(&s->objs[k], x, d);
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Phase function (Eq. phase with Eq. microfacet_vndf):                      */
/*   p(d, d2) = F D(m) <-d, m> / (4 |d.m| sigma(d)),  m = (d2-d)/|d2-d|.      */
/* Sampling mixture (end of Sec. 4.2): with probability R a       */
/* Beckmann visible-normal sample (Heitz & d'Eon 2014), else m uniform on the */
/* hemisphere around -d.  Beckmann frame and roughness: z = sign(-d.n) n and  */
/* alpha_B = clamp(alpha/G, 1e-3, 16); z = -d when G < 1e-6.                  */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normalize3(double v[3]) {
  double l = sqrt(dot3(v, v));
  v[0] /= l; v[1] /= l; v[2] /= l;
}

/* Orthonormal tangents of a unit vector (any completion works). */
static void basis(const double z[3], double t1[3], double t2[3]) {
  double a[3] = {1.0, 0.0, 0.0};
  if (fabs(z[0]) > 0.6) { a[0] = 0.0; a[1] = 1.0; }
  double k = dot3(a, z);
  for (int i = 0; i < 3; ++i) t1[i] = a[i] - k * z[i];
  normalize3(t1);
  t2[0] = z[1] * t1[2] - z[2] * t1[1];
  t2[1] = z[2] * t1[0] - z[0] * t1[2];
  t2[2] = z[0] * t1[1] - z[1] * t1[0];
}

static void to_frame(const double v[3], const double n[3], double out[3]) {
  double t1[3], t2[3];
  basis(n, t1, t2);
  out[0] = dot3(v, t1);
  out[1] = dot3(v, t2);
  out[2] = dot3(v, n);
}

static void beck_frame(const orc_fpt* p, const double d[3], double z[3], double* aB) {
  if (p->G < 1e-6) {
    z[0] = -d[0]; z[1] = -d[1]; z[2] = -d[2];
    *aB = 16.0;
    return;
  }
  double s = (-dot3(d, p->nhat) >= 0.0) ? 1.0 : -1.0;
  for (int i = 0; i < 3; ++i) z[i] = s * p->nhat[i];
  double a = p->alpha / p->G;
  if (a < 1e-3) a = 1e-3;
  if (a > 16.0) a = 16.0;
  *aB = a;
}

/* Isotropic Beckmann NDF about z with roughness a. */
static double beck_D(const double m[3], const double z[3], double a) {
  double c = dot3(m, z);
  if (c <= 0.0) return 0.0;
  double c2 = c * c, t2 = (1.0 - c2) / c2;
  return exp(-t2 / (a * a)) / (ORC_PI * a * a * c2 * c2);
}

/* Beckmann visible-normal density <wi,m> D(m) / ((1+Lambda(wi)) cos(theta_i)). */
static double beck_vis_pdf(const double m[3], const double wi[3], const double z[3], double a) {
  double wm = dot3(wi, m);
  if (wm <= 0.0) return 0.0;
  double D = beck_D(m, z, a);
  if (D == 0.0) return 0.0;
  double ci = dot3(wi, z);
  if (ci < 0.0) ci = 0.0;
  double si = sqrt(fmax(0.0, 1.0 - ci * ci));
  double denom;
  if (si == 0.0) {
    denom = ci;
  } else {
    double ac = ci / (a * si);
    denom = 0.5 * ci * (1.0 + erf(ac)) + a * si * exp(-ac * ac) / (2.0 * ORC_SQRTPI);
  }
  return wm * D / denom;
}

/* Visible-normal sampling of the Beckmann NDF (Heitz & d'Eon 2014): stretch
 * the incident direction to unit roughness, sample the standard visible
 * slope distribution (x slope by inverting its CDF, y slope Gaussian),
 * rotate, unstretch and convert the slope to a normal. */
static void beck_sample_vis(const double wi[3], const double z[3], double a, double u1,
                            double u2, double m[3]) {
  double t1[3], t2[3];
  basis(z, t1, t2);
  double ws[3] = {a * dot3(wi, t1), a * dot3(wi, t2), dot3(wi, z)};
  normalize3(ws);
  double ct = ws[2], st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double cphi = 1.0, sphi = 0.0;
  if (st > 1e-12) { cphi = ws[0] / st; sphi = ws[1] / st; }
  double sx;
  if (st < 1e-9) {
    sx = orc_erfinv(2.0 * u1 - 1.0);
  } else {
    double cot = ct / st;
    /* C(x) = cot (1+erf x)/2 + exp(-x^2)/(2 sqrt pi), increasing on x <= cot */
    double total = 0.5 * cot * (1.0 + erf(cot)) + exp(-cot * cot) / (2.0 * ORC_SQRTPI);
    double target = u1 * total, lo = -40.0, hi = cot;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * (1.0 + fabs(hi)); ++it) {
      double mid = 0.5 * (lo + hi);
      double c = 0.5 * cot * (1.0 + erf(mid)) + exp(-mid * mid) / (2.0 * ORC_SQRTPI);
      if (c < target) lo = mid; else hi = mid;
    }
    sx = 0.5 * (lo + hi);
  }
  double sy = orc_erfinv(2.0 * u2 - 1.0);
  double x = (cphi * sx - sphi * sy) * a;
  double y = (sphi * sx + cphi * sy) * a;
  double ml[3] = {-x, -y, 1.0};
  normalize3(ml);
  for (int i = 0; i < 3; ++i) m[i] = ml[0] * t1[i] + ml[1] * t2[i] + ml[2] * z[i];
  normalize3(m);
}

static void uniform_hemi(const double wi[3], double u1, double u2, double m[3]) {
  double t1[3], t2[3];
  basis(wi, t1, t2);
  double c = u1, s = sqrt(fmax(0.0, 1.0 - c * c)), ph = 2.0 * ORC_PI * u2;
  for (int i = 0; i < 3; ++i) m[i] = s * cos(ph) * t1[i] + s * sin(ph) * t2[i] + c * wi[i];
  normalize3(m);
}

static double mixture_pdf_m(const orc_fpt* p, const double d[3], const double m[3], double R) {
  double wi[3] = {-d[0], -d[1], -d[2]};
  if (dot3(wi, m) <= 0.0) return 0.0;
  double z[3], aB;
  beck_frame(p, d, z, &aB);
  return R * beck_vis_pdf(m, wi, z, aB) + (1.0 - R) / (2.0 * ORC_PI);
}

int orc_phase_eval_point(const orc_fpt* p, const double d[3], const double d2[3], double R,
                         double p_out[3], double* pdf_out) {
  double m[3] = {d2[0] - d[0], d2[1] - d[1], d2[2] - d[2]};
  double len = sqrt(dot3(m, m));
  p_out[0] = p_out[1] = p_out[2] = 0.0;
  if (pdf_out) *pdf_out = 0.0;
  if (!(len > 0.0)) return 0;
  for (int i = 0; i < 3; ++i) m[i] /= len;
  double dm = dot3(d, m);
  if (dm >= 0.0) return 0;
  double sd = orc_projected_area_world(d, p);
  double val = orc_ndf_world(m, p) / (4.0 * sd);
  for (int c = 0; c < 3; ++c) p_out[c] = p->F[c] * val;
  /* the oracle samples height-field kinds uniformly on the hemisphere about -d */
  double pdf_m = p->ndf == ORC_NDF_GPSS ? mixture_pdf_m(p, d, m, R) : 1.0 / (2.0 * ORC_PI);
  if (pdf_out) *pdf_out = pdf_m / (4.0 * fabs(dm));
  return 1;
}

int orc_phase_eval(const orc_scene* s, int k, const double x[3], const double d[3],
                   const double d2[3], double R, double p_out[3], double* pdf_out) {
  orc_fpt p;
  if (k < 0 || k >= s->n_objs || !orc_point(&s->objs[k], x, &p)) {
    p_out[0] = p_out[1] = p_out[2] = 0.0;
    if (pdf_out) *pdf_out = 0.0;
    return 0;
  }
  return orc_phase_eval_point(&p, d, d2, R, p_out, pdf_out);
}

int orc_phase_sample_point(const orc_fpt* p, const double d[3], double R, const double u[3],
                           double d2[3], double w_out[3], double* pdf_out) {
  double wi[3] = {-d[0], -d[1], -d[2]};
  double m[3];
  if (p->ndf != ORC_NDF_GPSS) {
    uniform_hemi(wi, u[1], u[2], m);
  } else if (u[0] < R) {
    double z[3], aB;
    beck_frame(p, d, z, &aB);
    beck_sample_vis(wi, z, aB, u[1], u[2], m);
  } else {
    uniform_hemi(wi, u[1], u[2], m);
  }
  double dm = dot3(d, m);
  w_out[0] = w_out[1] = w_out[2] = 0.0;
  *pdf_out = 0.0;
  if (dm >= 0.0) return 0;
  for (int i = 0; i < 3; ++i) d2[i] = d[i] - 2.0 * dm * m[i];
  normalize3(d2);
  double pdf_m = p->ndf == ORC_NDF_GPSS ? mixture_pdf_m(p, d, m, R) : 1.0 / (2.0 * ORC_PI);
  if (!(pdf_m > 0.0)) return 0;
  double sd = orc_projected_area_world(d, p);
  double w = orc_ndf_world(m, p) * fabs(dm) / (sd * pdf_m);
  for (int c = 0; c < 3; ++c) w_out[c] = p->F[c] * w;
  *pdf_out = pdf_m / (4.0 * fabs(dm));
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Exact visible-normal sampling.  The visible-normal density                */
/* max(0, -d.m) D(m) / sigma(d) of Eq. microfacet_vndf is, by Eq. gdf_to_ndf   */
/* (D(m) = int t^3 P(t m) dt and dg = t^2 dt dm), the direction of a slope g  */
/* drawn with density proportional to max(0, -d.g) N(g; g0, Sigma).  With     */
/* Sigma = L L^T (L symmetric), v = L d, s = |v| and e = -v/s, -d.g = s (beta + */
/* e.xi) for g = g0 + L xi, beta = -d.g0/s: the component y = beta + e.xi has */
/* density proportional to y phi(y - beta) on y > 0, and the components of xi */
/* orthogonal to e are independent standard normals.  GPSS objects: g0 =     */
/* grad mu, Sigma = sum_a (alpha_a^2/2) f_a f_a^T in the kernel frame.  Beckmann */
/* height fields: the same with g0 = n and alpha_n = 0 (the Beckmann NDF is   */
/* the GPSS with infinite correlation along n, Sec. 4.1).  The sample's pdf  */
/* over d2 is p/F = D(m)/(4 sigma(d)) and its weight p/pdf is F.  (The paper  */
/* samples a mixture instead; this sampler gives the oracle bounded path      */
/* weights, so per-pixel sample variances are reliable.)                      */
/* ------------------------------------------------------------------------ */
static double std_pdf(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * ORC_PI); }

/* Mills ratio R(x) = (1 - Phi(x))/phi(x) = sqrt(pi/2) erfcx(x/sqrt2) */
static double mills(double x) { return sqrt(0.5 * ORC_PI) * orc_erfcx(x / ORC_SQRT2); }

/* Unnormalised CDF H(y) = int_0^y t phi(t - beta) dt = beta (Phi(y-beta) - Phi(-beta))
 * + phi(beta) - phi(y-beta); for beta < 0 divided by phi(beta) and written with the
 * Mills ratio (B = -beta): [1 - B R(B)] - E [1 - B R(y+B)], E = e^{-y^2/2 - y B}. */
static double vis_cdf(double y, double beta) {
  if (beta >= 0.0) {
    double dPhi = 0.5 * (erfc(-(y - beta) / ORC_SQRT2) - erfc(beta / ORC_SQRT2));
    return beta * dPhi + std_pdf(beta) - std_pdf(y - beta);
  }
  double B = -beta, E = exp(-0.5 * y * y - y * B);
  return (1.0 - B * mills(B)) - E * (1.0 - B * mills(y + B));
}

static double vis_total(double beta) {
  if (beta >= 0.0) return beta * 0.5 * erfc(-beta / ORC_SQRT2) + std_pdf(beta);
  double B = -beta;
  return 1.0 - B * mills(B);
}

/* y > 0 with density proportional to y phi(y - beta), at CDF value xi (bisection) */
static double visible_slope(double beta, double xi) {
  double target = xi * vis_total(beta);
  double lo = 0.0, hi = (beta > 0.0 ? beta : 0.0) + 40.0;
  for (int it = 0; it < 400 && hi - lo > 1e-15 * (1.0 + hi); ++it) {
    double mid = 0.5 * (lo + hi);
    if (vis_cdf(mid, beta) < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static int exact_supported(const orc_fpt* p) { return p->ndf == ORC_NDF_GPSS || p->ndf == ORC_NDF_BECKMANN; }

/* L v for the gradient covariance of the field point (see above) */
static void cov_sqrt_apply(const orc_fpt* p, const double v[3], double out[3]) {
  double a[3] = {p->ax, p->ay, p->az};
  if (p->ndf == ORC_NDF_BECKMANN) { a[0] = a[1] = p->alpha; a[2] = 0.0; }
  const double* f[3] = {p->ft, p->fb, p->fn};
  out[0] = out[1] = out[2] = 0.0;
  for (int k = 0; k < 3; ++k) {
    double c = a[k] / ORC_SQRT2 * dot3(f[k], v);
    for (int i = 0; i < 3; ++i) out[i] += c * f[k][i];
  }
}

/* pdf over d2 of the exact sampler: p/F = D(m) / (4 sigma(d)) */
double orc_phase_pdf_exact(const orc_fpt* p, const double d[3], const double d2[3]) {
  double m[3] = {d2[0] - d[0], d2[1] - d[1], d2[2] - d[2]};
  double len = sqrt(dot3(m, m));
  if (!(len > 0.0)) return 0.0;
  for (int i = 0; i < 3; ++i) m[i] /= len;
  if (dot3(d, m) >= 0.0) return 0.0;
  double sd = orc_projected_area_world(d, p);
  return sd > 0.0 ? orc_ndf_world(m, p) / (4.0 * sd) : 0.0;
}

int orc_phase_sample_exact_point(const orc_fpt* p, const double d[3], const double u[3], double d2[3],
                                 double w_out[3], double* pdf_out) {
  w_out[0] = w_out[1] = w_out[2] = 0.0;
  *pdf_out = 0.0;
  if (!exact_supported(p)) return 0;
  double g0[3];
  if (p->ndf == ORC_NDF_GPSS) {
    for (int i = 0; i < 3; ++i) g0[i] = p->g[i];
  } else {
    for (int i = 0; i < 3; ++i) g0[i] = p->fn[i];
  }
  double v[3], xi[3], e1[3], e2[3], g[3];
  cov_sqrt_apply(p, d, v);
  double s = sqrt(dot3(v, v));
  if (!(s > 0.0)) return 0;
  double e[3] = {-v[0] / s, -v[1] / s, -v[2] / s};
  double beta = -dot3(d, g0) / s;
  double y = visible_slope(beta, u[0]);
  basis(e, e1, e2);
  double z1 = ORC_SQRT2 * orc_erfinv(2.0 * u[1] - 1.0), z2 = ORC_SQRT2 * orc_erfinv(2.0 * u[2] - 1.0);
  for (int i = 0; i < 3; ++i) xi[i] = (y - beta) * e[i] + z1 * e1[i] + z2 * e2[i];
  cov_sqrt_apply(p, xi, g);
  for (int i = 0; i < 3; ++i) g[i] += g0[i];
  double gl = sqrt(dot3(g, g));
  if (!(gl > 0.0)) return 0;
  double m[3] = {g[0] / gl, g[1] / gl, g[2] / gl};
  double dm = dot3(d, m);
  if (dm >= 0.0) return 0;
  for (int i = 0; i < 3; ++i) d2[i] = d[i] - 2.0 * dm * m[i];
  normalize3(d2);
  double pdf = orc_phase_pdf_exact(p, d, d2);
  if (!(pdf > 0.0)) return 0;
  for (int c = 0; c < 3; ++c) w_out[c] = p->F[c];
  *pdf_out = pdf;
  return 1;
}

int orc_phase_sample_exact(const orc_scene* s, int k, const double x[3], const double d[3], const double u[3],
                           double d2[3], double w_out[3], double* pdf_out) {
  orc_fpt p;
  if (k < 0 || k >= s->n_objs || !orc_point(&s->objs[k], x, &p)) return 0;
  return orc_phase_sample_exact_point(&p, d, u, d2, w_out, pdf_out);
}

int orc_phase_sample(const orc_scene* s, int k, const double x[3], const double d[3],
                     double R, const double u[3], double d2[3], double w_out[3],
                     double* pdf_out) {
  orc_fpt p;
  if (k < 0 || k >= s->n_objs || !orc_point(&s->objs[k], x, &p)) return 0;
  return orc_phase_sample_point(&p, d, R, u, d2, w_out, pdf_out);
}

/* ------------------------------------------------------------------------ */
/* Adaptive Gauss-Legendre quadrature (12 nodes, interval halving).  Nodes  */
/* are computed at first use by Newton's method on the Legendre recurrence. */
/* ------------------------------------------------------------------------ */
#define ORC_NGL 12
static double gl_x[ORC_NGL], gl_w[ORC_NGL];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;

static void gl_init(void) {
  const int n = ORC_NGL;
  for (int i = 0; i < n; ++i) {
    double x = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

static double gl_rule(orc_fn f, void* ctx, double a, double b) {
  double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
  for (int i = 0; i < ORC_NGL; ++i) s += gl_w[i] * f(c + h * gl_x[i], ctx);
  return s * h;
}

static double gl_adapt(orc_fn f, void* ctx, double a, double b, double whole, double tol, int depth) {
  double m = 0.5 * (a + b);
  double l = gl_rule(f, ctx, a, m), r = gl_rule(f, ctx, m, b);
  double both = l + r;
  double err = fabs(both - whole);
  /* converged, below the round-off floor of the rule, or too deep */
  if (depth >= 24 || err <= tol || err <= 1e-14 * fabs(both)) return both;
  return gl_adapt(f, ctx, a, m, l, 0.5 * tol, depth + 1) + gl_adapt(f, ctx, m, b, r, 0.5 * tol, depth + 1);
}

int orc_gl_nodes(const double** x, const double** w) {
  pthread_once(&gl_once, gl_init);
  *x = gl_x;
  *w = gl_w;
  return ORC_NGL;
}

/* Integral of f over [a,b] to an absolute tolerance abs_tol. */
double orc_integrate(orc_fn f, void* ctx, double a, double b, double abs_tol) {
  pthread_once(&gl_once, gl_init);
  if (!(b > a)) return 0.0;
  double whole = gl_rule(f, ctx, a, b);
  return gl_adapt(f, ctx, a, b, whole, abs_tol, 0);
}

/* Rough (non-adaptive) estimate, used to scale tolerances. */
double orc_integrate_rough(orc_fn f, void* ctx, double a, double b) {
  pthread_once(&gl_once, gl_init);
  if (!(b > a)) return 0.0;
  return gl_rule(f, ctx, a, b);
}
