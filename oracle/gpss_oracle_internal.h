/* gpss_oracle_internal.h -- private declarations shared by the oracle's .c
 * files.  TEST INFRASTRUCTURE ONLY (see gpss_oracle.h). */
#ifndef GPSS_ORACLE_INTERNAL_H
#define GPSS_ORACLE_INTERNAL_H

#include <stdint.h>
#include "gpss_oracle.h"

#define ORC_PI 3.14159265358979323846
#define ORC_SQRT2 1.41421356237309504880
#define ORC_SQRTPI 1.77245385090551602730

typedef double (*orc_fn)(double, void*);

/* Field values of one object at one point, with derived quantities. */
typedef struct {
  double mu, g[3], var, F[3];
  double sigma;   /* sqrt(var)                         */
  double alpha;   /* sqrt(2) sigma / l  (Eq. roughness) */
  double G;       /* |grad mu|                          */
  double nhat[3]; /* grad mu / G (0 when G == 0)        */
  int ndf;        /* the object's NDF kind              */
  /* kernel: roughness per axis of the frame (t, b, n); aniso = not all equal */
  double ax, ay, az;
  double ft[3], fb[3], fn[3];
  int aniso;
} orc_fpt;

int orc_point(const orc_object* o, const double x[3], orc_fpt* p);
double orc_projected_area_world(const double d[3], const orc_fpt* p);
double orc_ndf_world(const double m[3], const orc_fpt* p);
double orc_sigma_t_point(const orc_fpt* p, const double d[3]);
int orc_phase_eval_point(const orc_fpt* p, const double d[3], const double d2[3], double R,
                         double p_out[3], double* pdf_out);
int orc_phase_sample_point(const orc_fpt* p, const double d[3], double R, const double u[3],
                           double d2[3], double w_out[3], double* pdf_out);
int orc_phase_sample_exact_point(const orc_fpt* p, const double d[3], const double u[3], double d2[3],
                                 double w_out[3], double* pdf_out);
double orc_phase_pdf_exact(const orc_fpt* p, const double d[3], const double d2[3]);
double orc_integrate(orc_fn f, void* ctx, double a, double b, double abs_tol);
double orc_integrate_rough(orc_fn f, void* ctx, double a, double b);
double orc_erfinv(double v);
void orc_uniform4(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t bounce,
                  uint32_t purpose, uint32_t draw, double u[4]);
/* Gauss-Legendre nodes and weights on [-1, 1] of the adaptive rule; returns the count. */
int orc_gl_nodes(const double** x, const double** w);

/* ---- forward-mode dual numbers (gpss_oracle_dual.c), for orc_render_grad ---- */
/* Derivative slots: the 8 cell corners of a field sample for the mean, the
 * variance and the correlation-scale factor, the object's length scale, and the
 * 8 corners of one albedo channel. */
#define ORC_ND 33
enum { ORC_SLOT_MEAN = 0, ORC_SLOT_VAR = 8, ORC_SLOT_CS = 16, ORC_SLOT_L = 24, ORC_SLOT_ALB = 25 };
typedef struct { double v; double d[ORC_ND]; } orc_dual;
typedef struct {
  orc_dual mu, g[3], var, cs, F[3]; /* trilinear fields and grad mu of the interpolant     */
  orc_dual sigma, alpha;            /* sqrt(var), sqrt(2) sigma/(l s(x))                    */
  int64_t node[8];                  /* node index of corner k (the slots' parameters)     */
} orc_dfield;
orc_dual orc_dconst(double v);
int orc_dual_field(const orc_object* o, const double x[3], orc_dfield* f);
orc_dual orc_dual_projected_area(const orc_dfield* f, const double d[3]);
orc_dual orc_dual_sigma_t(const orc_dfield* f, const double d[3]);
orc_dual orc_dual_ndf(const orc_dfield* f, const double m[3]);
int orc_dual_log_phase(const orc_dfield* f, const double d[3], const double d2[3], orc_dual* out);
/* Adaptive Gauss-Legendre integral of a dual-valued function over [a, b]: panels are
 * split until every component (value and each derivative) converges. */
typedef orc_dual (*orc_dfn)(double t, void* ctx);
orc_dual orc_integrate_dual(orc_dfn f, void* ctx, const double* breaks, int nbreaks);

#endif
