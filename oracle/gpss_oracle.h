/*
 * gpss_oracle.h -- FP64 CPU oracle for the GPSS macrofacet medium.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product library
 * (the CUDA path) never includes, links or calls it, and the two share no
 * source: this header and its .c files are written independently from the
 * paper ("Macrofacet Theory for Gaussian Process Statistical Surfaces").
 *
 * Everything is computed in double precision.  Input grids are FP32 (that is
 * the scene definition); they are widened on read.
 *
 * Reading of the paper used throughout (the paper's own notation in brackets):
 *  - A scene object is a GPSS f ~ GP(mu(x), kappa) with squared-exponential
 *    kernel (Eq. se_kernel).  mu and sigma^2 are node-centred grids, trilinearly
 *    interpolated; grad mu is the analytic gradient of that interpolant.
 *  - Under the independence assumption (Sec. 4.2) the gradient at a point is
 *    g ~ N(grad mu, (sigma/l)^2 I) independent of f ~ N(mu, sigma^2); with an
 *    anisotropic kernel its covariance is sigma^2 diag(1/l_t^2, 1/l_b^2, 1/l_n^2)
 *    in the local frame of Sec. 4.2 (mean gradient along z), and a non-stationary
 *    kernel scales every l by a factor grid s(x).
 *  - Extinction for a ray marching along d (omega_o in Eq. generalized_sigma_t):
 *      sigma_t(x,d) = rho(x) * sigma(d),
 *      rho   = phi(mu;0,sigma^2) / Phi(mu;0,sigma^2)      (Eq. macro_sigma_t)
 *      sigma(d) = Lambda(d) cos(theta)                    (Eq. generalized_lambda)
 *    with the mean gradient (0,0,1) of the paper generalised to grad mu.
 *  - NDF by its definition D(m) = int_0^inf t^3 P(t m) dt  (Eq. gdf_to_ndf).
 *  - Conductor phase function p = F D_d(m) / (4 |d.m|)      (Eq. phase, vndf),
 *    F = albedo (no angular Fresnel term is given in the paper).
 */
#ifndef GPSS_ORACLE_H
#define GPSS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;            /* nodes per axis (>= 2), x fastest            */
  double bmin[3], bmax[3];   /* object bounding box = node-grid extent       */
  const float* mean;         /* nx*ny*nz signed-distance mean mu             */
  const float* var;          /* nx*ny*nz variance sigma^2 (> 0)              */
  const float* albedo;       /* channels planes of nx*ny*nz, F in [0,1]      */
  int channels;              /* 1 or 3                                       */
  double length_scale;       /* SE correlation l_t (> 0)                      */
  int ndf;                   /* ORC_NDF_GPSS (Sec. 4.2) or a height-field     */
                             /* macrofacet NDF (Sec. 4.1)                     */
  /* Anisotropic / non-stationary kernel (0 / NULL: isotropic, stationary).
   * Gradient covariance sigma^2 diag(1/l_t^2, 1/l_b^2, 1/l_n^2) in the frame
   * (t, b, n): n = grad mu/|grad mu| (world z where grad mu = 0), t = the tangent
   * field minus its n component, normalised (any unit vector orthogonal to n where
   * that vanishes), b = n x t.  Every l is multiplied by the factor s(x).           */
  double length_scale_b;     /* l_b (0: l_t)                                  */
  double length_scale_n;     /* l_n (0: l_t)                                  */
  const float* tangent;      /* NULL or 3 planes of nx*ny*nz: t(x), trilinear  */
  const float* cscale;       /* NULL or nx*ny*nz: s(x) > 0, trilinear         */
} orc_object;

/* NDF of an object.  GPSS: the generalized macrofacet of Sec. 4.2 (default).
 * Height-field macrofacets (Sec. 4.1): the same density rho with Lambda(w) cos(theta)
 * and the phase function of a chosen microfacet NDF about n = grad mu/|grad mu|,
 * roughness alpha = sqrt(2) sigma / l: Beckmann (the fully anisotropic GPSS with
 * infinite correlation along n) or GGX (the paper's artist-friendly choice). */
enum { ORC_NDF_GPSS = 0, ORC_NDF_BECKMANN = 1, ORC_NDF_GGX = 2 };

enum { ORC_LIGHT_DIRECTIONAL = 0, ORC_LIGHT_SKY = 1, ORC_LIGHT_UNIFORM = 2 };

typedef struct {
  int type;
  double dir[3];             /* directional: unit vector pointing to the light */
  double radiance[3];        /* irradiance (directional) or radiance scale    */
} orc_light;

enum { ORC_CAMERA_ORTHO = 0, ORC_CAMERA_PERSPECTIVE = 1 };

typedef struct {
  int type;
  double eye[3], look_at[3], up[3];
  double fov_y_deg, ortho_w, ortho_h;
  int width, height;
} orc_camera;

typedef struct {
  const orc_object* objs;
  int n_objs;
  orc_light light;
} orc_scene;

typedef struct {
  int spp, max_bounces;
  uint64_t seed;
  double mix_R;              /* probability of the Beckmann vNDF component    */
  int row_begin, row_end, row_step;
  int col_begin, col_end;
  int threads;               /* <= 0: all hardware threads                    */
  int sampler;               /* ORC_SAMPLER_MIXTURE (the paper's) or _EXACT     */
} orc_render_opts;

/* Phase sampling of the path tracer: the paper's mixture (end of Sec. 4.2), or
 * exact visible-normal sampling where the object supports it (GPSS, Beckmann
 * height fields; GGX keeps uniform half vectors).  Same expectation. */
enum { ORC_SAMPLER_MIXTURE = 0, ORC_SAMPLER_EXACT = 1 };

typedef struct {
  uint64_t paths, vertices, truncated;
} orc_stats;

/* ---- special functions (Sec. 3 notation: phi, Phi) ---------------------- */
double orc_erfcx(double x);           /* exp(x^2) erfc(x)                        */
double orc_log_ndtr(double u);        /* ln Phi(u), standard normal              */
double orc_inv_mills(double u);       /* lambda(u) = phi(u)/Phi(u)               */

/* ---- Philox4x32-10 (Salmon et al. 2011), used for seeded sampling -------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- fields and medium -------------------------------------------------- */
/* Returns 1 and fills the outputs if x lies in the object's box, else 0. */
int orc_field(const orc_object* o, const double x[3], double* mu, double grad[3],
              double* var, double albedo[3]);
/* Projected area sigma(w) in the paper's local frame: mean gradient (0,0,G),
 * roughness alpha_x, alpha_y, alpha_z (Eq. generalized_lambda times cos). */
double orc_projected_area_local(const double w[3], double G, double ax, double ay, double az);
/* Height-field macrofacet (Sec. 4.1), local frame with n = z: the NDF (zero for
 * m_z <= 0) and the projected area Lambda(w) cos(theta) for the marching
 * direction w, continued below the horizon by Lambda(-w) = -1 - Lambda(w). */
double orc_ndf_hf(const double m[3], int ndf, double alpha);
double orc_projected_area_hf(const double w[3], int ndf, double alpha);
/* NDF by quadrature of its definition, local frame (Eq. gdf_to_ndf, gdf). */
double orc_ndf_local(const double m[3], double G, double ax, double ay, double az);
/* Extinction of one object / the whole scene (extinctions of objects add). */
double orc_sigma_t_object(const orc_object* o, const double x[3], const double d[3]);
double orc_sigma_t(const orc_scene* s, const double x[3], const double d[3]);
/* Phase function of object k at x: p (per channel, includes F) and the pdf
 * of the sampling mixture over outgoing directions (end of Sec. 4.2).     */
int orc_phase_eval(const orc_scene* s, int k, const double x[3], const double d[3],
                   const double d2[3], double R, double p_out[3], double* pdf_out);
/* Samples d2 with three uniforms; returns weight p/pdf (per channel) and pdf. */
int orc_phase_sample(const orc_scene* s, int k, const double x[3], const double d[3],
                     double R, const double u[3], double d2[3], double w_out[3],
                     double* pdf_out);
/* Exact visible-normal sample of object k's phase function (GPSS objects and
 * Beckmann height fields): d2 with pdf p/F, weight F (per channel).  Returns 0
 * where unsupported (GGX) or for a measure-zero failure. */
int orc_phase_sample_exact(const orc_scene* s, int k, const double x[3], const double d[3], const double u[3],
                           double d2[3], double w_out[3], double* pdf_out);
/* Optical depth and transmittance along o + t d, t in [0, tmax]. */
double orc_optical_depth(const orc_scene* s, const double o[3], const double d[3], double tmax);
double orc_transmittance(const orc_scene* s, const double o[3], const double d[3], double tmax);

/* ---- rendering ------------------------------------------------------------ */
/* Path tracer by regular tracking.  sum/sumsq are width*height*3 doubles
 * (accumulated over samples of the selected pixels; others untouched).    */
int orc_render(const orc_scene* s, const orc_camera* cam, const orc_render_opts* o,
               double* sum, double* sumsq, orc_stats* st);
/* Same paths rendered in scene a and scene b with identical random numbers;
 * accumulates the per-path difference L_a - L_b (common random numbers). */
int orc_render_diff(const orc_scene* a, const orc_scene* b, const orc_camera* cam,
                    const orc_render_opts* o, double* sum, double* sumsq, orc_stats* st);

/* Gradient of the expected image's loss by path replay of the same regular-
 * tracking estimator (the oracle's adjoint).  d_image: width*height*3 doubles,
 * dLoss/dpixel (the loss is sum over the selected pixels of d_image * image).
 * out: one entry per object.  Gradients are ACCUMULATED (+=); a NULL output is
 * not computed.  nodes != NULL restricts the outputs to those node indices
 * (x fastest; each output then has n_nodes entries, in that order, albedo
 * channels planes of n_nodes), else every node (nx*ny*nz).  Isotropic GPSS
 * objects only (stationary or with a correlation-scale grid).  Returns 0, 1 for
 * bad arguments, 2 for an unsupported object.  *mismatch (nullable): quadrature
 * points that fell outside their piece's field cell (expected 0). */
typedef struct {
  const int64_t* nodes;
  int64_t n_nodes;
  double* d_mean;
  double* d_var;
  double* d_albedo;
  double* d_cscale;          /* objects with a correlation-scale grid only       */
  double* d_l;               /* 1 double: the object's length scale l_t          */
} orc_grad_out;

int orc_render_grad(const orc_scene* s, const orc_camera* cam, const orc_render_opts* o,
                    const double* d_image, orc_grad_out* out, orc_stats* st, uint64_t* mismatch);

/* Dual-number evaluation at one point of object k (test access to the adjoint's
 * partials): value and the ORC_ND derivative slots (corner k of the cell: mean
 * k, variance 8+k, correlation scale 16+k, l 24, albedo channel 0 25+k) of
 * sigma_t(x, d) (what = 0), sigma(d) (1), D(m = d2) (2) or ln(D(m)/sigma(d)) of
 * the pair (d, d2) (3); node[8] receives the corners' node indices.  Returns 0
 * outside the object's box or where the quantity is undefined. */
int orc_dual_eval(const orc_object* o, int what, const double x[3], const double d[3], const double d2[3],
                  double* out_v, double* out_d, int64_t* node);

/* Camera ray through pixel (px,py) at sub-pixel jitter (jx,jy) in [0,1). */
void orc_camera_ray(const orc_camera* c, int px, int py, double jx, double jy,
                    double org[3], double dir[3]);

#ifdef __cplusplus
}
#endif
#endif
