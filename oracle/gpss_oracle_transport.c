/*
 * gpss_oracle_transport.c -- FP64 oracle: transmittance, free flight and the
 * path tracer.  TEST INFRASTRUCTURE ONLY (see gpss_oracle.h).
 *
 * The medium is the classic exponential medium of Sec. 4 (Eq. sm2tr):
 * Tr = exp(-int sigma_t dt).  The paper renders it with null scattering
 * (Sec. 5) and notes that any classic-medium technique applies; the oracle
 * deliberately uses a different one, regular tracking: the optical depth
 * tau(t) is integrated by adaptive quadrature between cell faces and the
 * free-flight distance is the root of tau(t) = -ln(u).  Its expectation is
 * that of every unbiased free-flight sampler of the same medium.
 */
#include "gpss_oracle.h"
#include "gpss_oracle_internal.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { P_CAMERA = 0, P_FLIGHT = 1, P_PHASE = 3 };

static void ray_at(const double o[3], const double d[3], double t, double x[3]) {
  for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
}

/* Slab test: [*ta, *tb] = parameter range inside the box, 0 if none. */
static int ray_box(const double o[3], const double d[3], const double bmin[3], const double bmax[3],
                   double* ta, double* tb) {
  double lo = -INFINITY, hi = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) {
      if (o[a] < bmin[a] || o[a] > bmax[a]) return 0;
      continue;
    }
    double t1 = (bmin[a] - o[a]) / d[a], t2 = (bmax[a] - o[a]) / d[a];
    if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
    if (t1 > lo) lo = t1;
    if (t2 < hi) hi = t2;
  }
  if (!(hi >= lo)) return 0;
  *ta = lo;
  *tb = hi;
  return 1;
}

typedef struct { double* v; int n, cap; } dlist;

static void dl_push(dlist* l, double x) {
  if (l->n == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 256;
    l->v = (double*)realloc(l->v, sizeof(double) * (size_t)l->cap);
  }
  l->v[l->n++] = x;
}

static int cmp_d(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Length over which the density of one cell can change by O(1): half the
 * smallest standard deviation over the largest mean-gradient bound. */
static double cell_feature_len(const orc_object* o, const double x[3]) {
  const int n[3] = {o->nx, o->ny, o->nz};
  int i[3];
  double h[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = (o->bmax[a] - o->bmin[a]) / (double)(n[a] - 1);
    int ia = (int)floor((x[a] - o->bmin[a]) / h[a]);
    if (ia < 0) ia = 0;
    if (ia > n[a] - 2) ia = n[a] - 2;
    i[a] = ia;
  }
  double vmin = INFINITY, ed[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 8; ++c) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    size_t idx = (size_t)(i[0] + cx) + (size_t)n[0] * ((size_t)(i[1] + cy) + (size_t)n[1] * (i[2] + cz));
    if (o->var[idx] < vmin) vmin = o->var[idx];
    if (!cx) ed[0] = fmax(ed[0], fabs((double)o->mean[idx + 1] - o->mean[idx]) / h[0]);
    if (!cy) ed[1] = fmax(ed[1], fabs((double)o->mean[idx + n[0]] - o->mean[idx]) / h[1]);
    if (!cz) ed[2] = fmax(ed[2], fabs((double)o->mean[idx + (size_t)n[0] * n[1]] - o->mean[idx]) / h[2]);
  }
  double G = sqrt(ed[0] * ed[0] + ed[1] * ed[1] + ed[2] * ed[2]);
  if (!(G > 0.0)) return INFINITY;
  return 0.5 * sqrt(vmin) / G;
}

/* Splits [t0,t1] of the ray into sub-intervals on which sigma_t is smooth
 * (cell faces of every object are break points) and short compared with
 * the density's feature length.  Intervals outside every object are dropped
 * (sigma_t = 0 there).  Returns the count; *out holds pairs (a,b). */
static int build_pieces(const orc_scene* s, const double o[3], const double d[3], double t0, double t1,
                        double** out) {
  dlist bp = {0, 0, 0};
  for (int k = 0; k < s->n_objs; ++k) {
    const orc_object* ob = &s->objs[k];
    double ta, tb;
    if (!ray_box(o, d, ob->bmin, ob->bmax, &ta, &tb)) continue;
    if (ta < t0) ta = t0;
    if (tb > t1) tb = t1;
    if (!(tb > ta)) continue;
    dl_push(&bp, ta);
    dl_push(&bp, tb);
    const int n[3] = {ob->nx, ob->ny, ob->nz};
    for (int a = 0; a < 3; ++a) {
      if (d[a] == 0.0) continue;
      double h = (ob->bmax[a] - ob->bmin[a]) / (double)(n[a] - 1);
      for (int i = 1; i < n[a] - 1; ++i) {
        double t = (ob->bmin[a] + i * h - o[a]) / d[a];
        if (t > ta && t < tb) dl_push(&bp, t);
      }
    }
  }
  dlist pieces = {0, 0, 0};
  if (bp.n >= 2) {
    qsort(bp.v, (size_t)bp.n, sizeof(double), cmp_d);
    for (int i = 0; i + 1 < bp.n; ++i) {
      double a = bp.v[i], b = bp.v[i + 1];
      if (!(b > a)) continue;
      double mid[3];
      ray_at(o, d, 0.5 * (a + b), mid);
      double feat = INFINITY;
      int inside = 0;
      for (int k = 0; k < s->n_objs; ++k) {
        const orc_object* ob = &s->objs[k];
        int in = 1;
        for (int ax = 0; ax < 3; ++ax) in &= (mid[ax] >= ob->bmin[ax] && mid[ax] <= ob->bmax[ax]);
        if (!in) continue;
        inside = 1;
        double f = cell_feature_len(ob, mid);
        if (f < feat) feat = f;
      }
      if (!inside) continue;
      int K = 1;
      if (isfinite(feat)) {
        double kk = ceil((b - a) / feat);
        K = kk < 1.0 ? 1 : (kk > 100000.0 ? 100000 : (int)kk);
      }
      for (int j = 0; j < K; ++j) {
        dl_push(&pieces, a + (b - a) * j / K);
        dl_push(&pieces, j + 1 == K ? b : a + (b - a) * (j + 1) / K);
      }
    }
  }
  free(bp.v);
  *out = pieces.v;
  return pieces.n / 2;
}

typedef struct { const orc_scene* s; const double* o; const double* d; } ray_ctx;

static double sigt_along(double t, void* vp) {
  const ray_ctx* c = (const ray_ctx*)vp;
  double x[3];
  ray_at(c->o, c->d, t, x);
  return orc_sigma_t(c->s, x, c->d);
}

double orc_optical_depth(const orc_scene* s, const double o[3], const double d[3], double tmax) {
  double* pc = NULL;
  int n = build_pieces(s, o, d, 0.0, tmax, &pc);
  ray_ctx c = {s, o, d};
  double rough = 0.0;
  for (int i = 0; i < n; ++i) rough += orc_integrate_rough(sigt_along, &c, pc[2 * i], pc[2 * i + 1]);
  double tol = (1e-13 * fabs(rough) + 1e-16) / (n > 0 ? n : 1);
  double tau = 0.0;
  for (int i = 0; i < n; ++i) tau += orc_integrate(sigt_along, &c, pc[2 * i], pc[2 * i + 1], tol);
  free(pc);
  return tau;
}

/* Eq. sm2tr.  exp(-tau) is exactly 0 in double precision once tau > 745.2, so
 * the integration stops when a low-order estimate of the optical depth so far
 * exceeds 1e4 (far beyond any error of that estimate): the value returned is the
 * same, and shadow rays into the dense interior of a surface-like shell do not
 * integrate the whole interior. */
double orc_transmittance(const orc_scene* s, const double o[3], const double d[3], double tmax) {
  double* pc = NULL;
  int n = build_pieces(s, o, d, 0.0, tmax, &pc);
  ray_ctx c = {s, o, d};
  double rough = 0.0;
  for (int i = 0; i < n; ++i) {
    rough += orc_integrate_rough(sigt_along, &c, pc[2 * i], pc[2 * i + 1]);
    if (rough > 1e4) {
      free(pc);
      return 0.0;
    }
  }
  double tol = (1e-13 * fabs(rough) + 1e-16) / (n > 0 ? n : 1);
  double tau = 0.0;
  for (int i = 0; i < n; ++i) tau += orc_integrate(sigt_along, &c, pc[2 * i], pc[2 * i + 1], tol);
  free(pc);
  return exp(-tau);
}

/* Regular tracking: the distance t with tau(t) = target, if it lies before
 * the ray leaves the scene.  The crossing sub-interval is resolved by a
 * Newton iteration safeguarded by bisection. */
static int free_flight(const orc_scene* s, const double o[3], const double d[3], double target,
                       double* t_hit) {
  double* pc = NULL;
  int n = build_pieces(s, o, d, 0.0, INFINITY, &pc);
  ray_ctx c = {s, o, d};
  double tol = 1e-15 + 1e-13 * target;
  double cum = 0.0;
  int hit = 0;
  for (int i = 0; i < n && !hit; ++i) {
    double a = pc[2 * i], b = pc[2 * i + 1];
    double I = orc_integrate(sigt_along, &c, a, b, tol / 16.0);
    if (cum + I < target) { cum += I; continue; }
    double lo = a, hi = b, t = a + (b - a) * (target - cum) / I;
    for (int it = 0; it < 200; ++it) {
      double F = cum + orc_integrate(sigt_along, &c, a, t, tol / 16.0) - target;
      if (fabs(F) <= tol) break;
      if (F > 0.0) hi = t; else lo = t;
      if (hi - lo <= 1e-15 * (1.0 + fabs(t))) break;
      double f = sigt_along(t, &c);
      double tn = f > 0.0 ? t - F / f : 0.5 * (lo + hi);
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      t = tn;
    }
    *t_hit = t;
    hit = 1;
  }
  free(pc);
  return hit;
}

/* Camera: forward f, right r = f x up, image-up u = r x f; pixel (0,0) is
 * the top-left corner; ndc x in [-1,1] left to right, y top to bottom. */
void orc_camera_ray(const orc_camera* c, int px, int py, double jx, double jy, double org[3],
                    double dir[3]) {
  double f[3], r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = c->look_at[a] - c->eye[a];
  double l = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int a = 0; a < 3; ++a) f[a] /= l;
  r[0] = f[1] * c->up[2] - f[2] * c->up[1];
  r[1] = f[2] * c->up[0] - f[0] * c->up[2];
  r[2] = f[0] * c->up[1] - f[1] * c->up[0];
  l = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= l;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  double x = 2.0 * (px + jx) / c->width - 1.0;
  double y = 1.0 - 2.0 * (py + jy) / c->height;
  if (c->type == ORC_CAMERA_ORTHO) {
    for (int a = 0; a < 3; ++a) {
      org[a] = c->eye[a] + x * 0.5 * c->ortho_w * r[a] + y * 0.5 * c->ortho_h * u[a];
      dir[a] = f[a];
    }
  } else {
    double th = tan(0.5 * c->fov_y_deg * ORC_PI / 180.0), asp = (double)c->width / c->height;
    for (int a = 0; a < 3; ++a) {
      org[a] = c->eye[a];
      dir[a] = f[a] + x * th * asp * r[a] + y * th * u[a];
    }
    l = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int a = 0; a < 3; ++a) dir[a] /= l;
  }
}

/* Environment radiance.  Procedural sky: for w_z >= 0 a linear blend from
 * white at the horizon to (0.35,0.55,1) at the zenith; (0.25,0.22,0.20)
 * below the horizon.  Uniform: constant.  Both scaled by the light's
 * radiance. */
static void env_radiance(const orc_light* L, const double w[3], double out[3]) {
  if (L->type == ORC_LIGHT_SKY) {
    if (w[2] >= 0.0) {
      double t = w[2];
      out[0] = (1.0 - t) + t * 0.35;
      out[1] = (1.0 - t) + t * 0.55;
      out[2] = (1.0 - t) + t * 1.00;
    } else {
      out[0] = 0.25; out[1] = 0.22; out[2] = 0.20;
    }
    for (int c = 0; c < 3; ++c) out[c] *= L->radiance[c];
  } else {
    for (int c = 0; c < 3; ++c) out[c] = L->radiance[c];
  }
}

static double power_heuristic(double a, double b) {
  double a2 = a * a, b2 = b * b;
  return a2 / (a2 + b2);
}

/* ------------------------------------------------------------------------ */
/* Adjoint (orc_render_grad).  Path replay: the path is traced a second time  */
/* with the same random numbers, knowing its total radiance L_tot.  With the  */
/* sampling densities, the extinction-proportional object choice and the MIS  */
/* weights held fixed (their derivatives cancel in expectation: the sampled    */
/* paths' densities do not enter the expected image, and MIS weights sum to   */
/* one), the derivative of the path's estimate is the sum over its factors f  */
/* of d ln f times the radiance the path collects downstream of f.  The       */
/* factors of the regular-tracking estimator are                               */
/*   flight to a real collision at t:  sigma_t,k(x_t) exp(-int_0^t sigma_t)  */
/*   escaping flight:                  exp(-int_0^inf sigma_t)               */
/*   NEE:                              p_k(d, w_L) exp(-int sigma_t along w_L) */
/*   phase sample:                     p_k(d, d')                             */
/* (p includes F).  d ln of an exponential factor is -int d sigma_t, which    */
/* the oracle integrates by quadrature along the segment (not by collisions). */
/* Every partial comes from the dual numbers of gpss_oracle_dual.c.           */
/* ------------------------------------------------------------------------ */
typedef struct {             /* one object's request (shared by the workers) */
  const int32_t* map;        /* node -> output slot (-1: not wanted); NULL: slot = node */
  int64_t n;                 /* output length of each field */
  int channels;
  int want_mean, want_var, want_alb, want_cs, want_l;
} greq;

typedef struct {             /* one worker's accumulators for one object */
  double *mean, *var, *alb, *cs;
  double l;
} gacc;

typedef struct {
  const greq* rq;            /* per object */
  gacc* acc;                 /* per object, this worker's */
  double gpix[3];            /* dLoss/dpixel / spp of the path's pixel */
  double Ltot[3];            /* the path's radiance (first pass) */
  uint64_t mismatch;         /* quadrature points that left the piece's field cell */
} gctx;

static int64_t slot_of(const greq* rq, int64_t node) { return rq->map ? (int64_t)rq->map[node] : node; }

/* Whether the extinction of a field sample with these corners matters to the request. */
static int cell_wanted(const greq* rq, const int64_t node[8]) {
  if (rq->want_l) return 1;
  if (!(rq->want_mean || rq->want_var || rq->want_cs)) return 0;
  for (int k = 0; k < 8; ++k)
    if (slot_of(rq, node[k]) >= 0) return 1;
  return 0;
}

/* accumulates W * dv (dv: derivative slots of a field sample with corners f->node) */
static void scatter_dual(const greq* rq, gacc* a, const orc_dfield* f, const double* dv, double W) {
  if (W == 0.0) return;
  for (int k = 0; k < 8; ++k) {
    int64_t j = slot_of(rq, f->node[k]);
    if (j < 0) continue;
    if (rq->want_mean) a->mean[j] += W * dv[ORC_SLOT_MEAN + k];
    if (rq->want_var) a->var[j] += W * dv[ORC_SLOT_VAR + k];
    if (rq->want_cs) a->cs[j] += W * dv[ORC_SLOT_CS + k];
  }
  if (rq->want_l) a->l += W * dv[ORC_SLOT_L];
}

/* accumulates sum_c Wc[c] d ln F_c (F_c the albedo channel c at the sample) */
static void scatter_albedo(const greq* rq, gacc* a, const orc_dfield* f, const double Wc[3]) {
  if (!rq->want_alb) return;
  for (int c = 0; c < 3; ++c) {
    if (Wc[c] == 0.0 || !(f->F[c].v > 0.0)) continue;
    int plane = rq->channels == 1 ? 0 : c;
    for (int k = 0; k < 8; ++k) {
      int64_t j = slot_of(rq, f->node[k]);
      if (j >= 0) a->alb[(size_t)plane * rq->n + j] += Wc[c] * f->F[c].d[ORC_SLOT_ALB + k] / f->F[c].v;
    }
  }
}

typedef struct {
  const orc_object* ob;
  const double* o;
  const double* d;
  int64_t node0;
  uint64_t* mismatch;
} seg_ctx;

static orc_dual dsig_along(double t, void* vp) {
  const seg_ctx* c = (const seg_ctx*)vp;
  double x[3];
  ray_at(c->o, c->d, t, x);
  orc_dfield f;
  if (!orc_dual_field(c->ob, x, &f) || f.node[0] != c->node0) {
    ++*c->mismatch;
    return orc_dconst(0.0);
  }
  return orc_dual_sigma_t(&f, c->d);
}

/* -W int_0^tmax d sigma_t ds along o + s d (the derivative of ln exp(-tau)):
 * per piece of build_pieces (each inside one field cell of every object) the
 * dual extinction of each object is integrated by adaptive quadrature. */
static void grad_segment(const orc_scene* s, gctx* g, const double o[3], const double d[3], double tmax,
                         double W) {
  if (W == 0.0) return;
  double* pc = NULL;
  int n = build_pieces(s, o, d, 0.0, tmax, &pc);
  for (int i = 0; i < n; ++i) {
    double a = pc[2 * i], b = pc[2 * i + 1], mid[3];
    ray_at(o, d, 0.5 * (a + b), mid);
    for (int k = 0; k < s->n_objs; ++k) {
      orc_dfield f;
      if (!orc_dual_field(&s->objs[k], mid, &f) || !cell_wanted(&g->rq[k], f.node)) continue;
      seg_ctx c = {&s->objs[k], o, d, f.node[0], &g->mismatch};
      double br[2] = {a, b};
      orc_dual I = orc_integrate_dual(dsig_along, &c, br, 2);
      scatter_dual(&g->rq[k], &g->acc[k], &f, I.d, -W);
    }
  }
  free(pc);
}

/* Wc[c] = dLoss/dpixel_c / spp times the radiance c the path collects from here on */
static double downstream(const gctx* g, const double L[3], double Wc[3]) {
  double W = 0.0;
  for (int c = 0; c < 3; ++c) {
    Wc[c] = g->gpix[c] * (g->Ltot[c] - L[c]);
    W += Wc[c];
  }
  return W;
}

/* d ln p_k(d, d2) with channel weights Wc at the field sample f */
static void grad_phase(const gctx* g, int k, const orc_dfield* f, const double d[3], const double d2[3],
                       const double Wc[3]) {
  double W = Wc[0] + Wc[1] + Wc[2];
  if (W == 0.0 && Wc[0] == 0.0 && Wc[1] == 0.0 && Wc[2] == 0.0) return;
  orc_dual lp;
  if (!orc_dual_log_phase(f, d, d2, &lp)) return;
  scatter_dual(&g->rq[k], &g->acc[k], f, lp.d, W);
  scatter_albedo(&g->rq[k], &g->acc[k], f, Wc);
}

/* One path: camera ray, then per real scattering vertex next-event
 * estimation and phase-function sampling (MIS with the environment).  At
 * most max_bounces real vertices; no continuation after the last.
 * g != NULL: the gradient replay of a path whose radiance g->Ltot is known. */
static void trace_path(const orc_scene* s, const orc_camera* cam, const orc_render_opts* op, int px,
                       int py, int sample, double L[3], uint64_t* nvert, int* truncated, gctx* g) {
  const uint32_t pixel = (uint32_t)(py * cam->width + px);
  const double inv4pi = 1.0 / (4.0 * ORC_PI);
  double u[4], o[3], d[3], beta[3] = {1.0, 1.0, 1.0}, prev_pdf = -1.0;
  L[0] = L[1] = L[2] = 0.0;
  *truncated = 0;
  orc_uniform4(op->seed, pixel, (uint32_t)sample, 0, P_CAMERA, 0, u);
  orc_camera_ray(cam, px, py, u[0], u[1], o, d);
  const int env = s->light.type != ORC_LIGHT_DIRECTIONAL;
  for (int bounce = 0;; ++bounce) {
    orc_uniform4(op->seed, pixel, (uint32_t)sample, (uint32_t)bounce, P_FLIGHT, 0, u);
    double t, Wc[3], Wseg = 0.0;
    if (g) Wseg = downstream(g, L, Wc);
    if (!free_flight(s, o, d, -log(u[0]), &t)) {
      if (env) {
        double Le[3], w = prev_pdf < 0.0 ? 1.0 : power_heuristic(prev_pdf, inv4pi);
        env_radiance(&s->light, d, Le);
        for (int c = 0; c < 3; ++c) L[c] += beta[c] * Le[c] * w;
      }
      if (g) grad_segment(s, g, o, d, INFINITY, Wseg);
      return;
    }
    double x[3];
    ray_at(o, d, t, x);
    (*nvert)++;
    /* scattering object chosen in proportion to its extinction */
    double sig[64], tot = 0.0;
    int nk = s->n_objs < 64 ? s->n_objs : 64;
    for (int k = 0; k < nk; ++k) tot += (sig[k] = orc_sigma_t_object(&s->objs[k], x, d));
    int kk = 0;
    double acc = 0.0, pick = u[1] * tot;
    for (kk = 0; kk < nk - 1; ++kk) {
      acc += sig[kk];
      if (pick < acc) break;
    }
    while (kk > 0 && sig[kk] == 0.0) --kk;
    orc_fpt p;
    if (!orc_point(&s->objs[kk], x, &p)) return;
    orc_dfield df;
    if (g) {
      /* flight factor sigma_t,k(x) exp(-int_0^t sigma_t): d ln = d sigma_t,k/sigma_t,k - int d sigma_t */
      orc_dual_field(&s->objs[kk], x, &df);
      orc_dual st = orc_dual_sigma_t(&df, d);
      if (st.v > 0.0) {
        double dv[ORC_ND];
        for (int i = 0; i < ORC_ND; ++i) dv[i] = st.d[i] / st.v;
        scatter_dual(&g->rq[kk], &g->acc[kk], &df, dv, Wseg);
      }
      grad_segment(s, g, o, d, t, Wseg);
    }
    /* next-event estimation: contribution C = beta p Tr Le (w / light pdf) */
    double pv[3], pdf_ph, C[3] = {0.0, 0.0, 0.0}, wl[3];
    if (!env) {
      for (int a = 0; a < 3; ++a) wl[a] = s->light.dir[a];
      orc_phase_eval_point(&p, d, wl, op->mix_R, pv, &pdf_ph);
      double Tr = orc_transmittance(s, x, wl, INFINITY);
      for (int c = 0; c < 3; ++c) C[c] = beta[c] * pv[c] * Tr * s->light.radiance[c];
    } else {
      double z = 1.0 - 2.0 * u[2], ph = 2.0 * ORC_PI * u[3], r = sqrt(fmax(0.0, 1.0 - z * z));
      wl[0] = r * cos(ph);
      wl[1] = r * sin(ph);
      wl[2] = z;
      orc_phase_eval_point(&p, d, wl, op->mix_R, pv, &pdf_ph);
      if (op->sampler == ORC_SAMPLER_EXACT && (p.ndf == ORC_NDF_GPSS || p.ndf == ORC_NDF_BECKMANN))
        pdf_ph = orc_phase_pdf_exact(&p, d, wl);  /* the phase sampler's pdf of w_L (MIS) */
      if (pv[0] > 0.0 || pv[1] > 0.0 || pv[2] > 0.0) {
        double Tr = orc_transmittance(s, x, wl, INFINITY);
        double Le[3], w = power_heuristic(inv4pi, pdf_ph);
        env_radiance(&s->light, wl, Le);
        for (int c = 0; c < 3; ++c) C[c] = beta[c] * pv[c] * Tr * Le[c] * w / inv4pi;
      }
    }
    if (g) {
      /* NEE factors p_k(d, w_L) and exp(-int sigma_t along w_L), weighted by C itself */
      double Wn[3];
      for (int c = 0; c < 3; ++c) Wn[c] = g->gpix[c] * C[c];
      grad_phase(g, kk, &df, d, wl, Wn);
      grad_segment(s, g, x, wl, INFINITY, Wn[0] + Wn[1] + Wn[2]);
    }
    for (int c = 0; c < 3; ++c) L[c] += C[c];
    if (bounce + 1 >= op->max_bounces) {
      *truncated = 1;
      return;
    }
    orc_uniform4(op->seed, pixel, (uint32_t)sample, (uint32_t)bounce, P_PHASE, 0, u);
    double d2[3], wgt[3], pdf;
    if (op->sampler == ORC_SAMPLER_EXACT && (p.ndf == ORC_NDF_GPSS || p.ndf == ORC_NDF_BECKMANN)) {
      if (!orc_phase_sample_exact_point(&p, d, u, d2, wgt, &pdf)) return;
    } else if (!orc_phase_sample_point(&p, d, op->mix_R, u, d2, wgt, &pdf)) {
      return;
    }
    if (g) {
      /* phase-sample factor p_k(d, d2), weighted by everything collected after this vertex's NEE */
      downstream(g, L, Wc);
      grad_phase(g, kk, &df, d, d2, Wc);
    }
    for (int c = 0; c < 3; ++c) beta[c] *= wgt[c];
    prev_pdf = pdf;
    for (int a = 0; a < 3; ++a) { o[a] = x[a]; d[a] = d2[a]; }
  }
}

typedef struct {
  const orc_scene* a;
  const orc_scene* b; /* NULL: plain render */
  const orc_camera* cam;
  const orc_render_opts* op;
  double* sum;
  double* sumsq;
  int next;
  int nrows;
  uint64_t paths, vertices, truncated;
  pthread_mutex_t mu;
} job_t;

static void* worker(void* vp) {
  job_t* j = (job_t*)vp;
  for (;;) {
    int r = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
    if (r >= j->nrows) break;
    int py = j->op->row_begin + r * j->op->row_step;
    uint64_t np = 0, nv = 0, nt = 0;
    for (int px = j->op->col_begin; px < j->op->col_end; ++px) {
      size_t pix = (size_t)py * j->cam->width + px;
      for (int s = 0; s < j->op->spp; ++s) {
        double La[3], Lb[3] = {0.0, 0.0, 0.0};
        int tr;
        trace_path(j->a, j->cam, j->op, px, py, s, La, &nv, &tr, NULL);
        nt += tr;
        if (j->b) {
          uint64_t nv2 = 0;
          int tr2;
          trace_path(j->b, j->cam, j->op, px, py, s, Lb, &nv2, &tr2, NULL);
        }
        for (int c = 0; c < 3; ++c) {
          double v = La[c] - Lb[c];
          j->sum[pix * 3 + c] += v;
          j->sumsq[pix * 3 + c] += v * v;
        }
        ++np;
      }
    }
    pthread_mutex_lock(&j->mu);
    j->paths += np;
    j->vertices += nv;
    j->truncated += nt;
    pthread_mutex_unlock(&j->mu);
  }
  return NULL;
}

static int run(const orc_scene* a, const orc_scene* b, const orc_camera* cam, const orc_render_opts* op,
               double* sum, double* sumsq, orc_stats* st) {
  if (!a || !cam || !op || !sum || !sumsq || op->spp <= 0 || op->max_bounces <= 0 || op->row_step <= 0)
    return 1;
  if (op->row_begin < 0 || op->row_end > cam->height || op->col_begin < 0 || op->col_end > cam->width)
    return 1;
  job_t j;
  memset(&j, 0, sizeof(j));
  j.a = a; j.b = b; j.cam = cam; j.op = op; j.sum = sum; j.sumsq = sumsq;
  j.nrows = op->row_end > op->row_begin ? (op->row_end - op->row_begin + op->row_step - 1) / op->row_step : 0;
  pthread_mutex_init(&j.mu, NULL);
  int nt = op->threads > 0 ? op->threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nt < 1) nt = 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, worker, &j);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&j.mu);
  if (st) {
    st->paths = j.paths;
    st->vertices = j.vertices;
    st->truncated = j.truncated;
  }
  return 0;
}

int orc_render(const orc_scene* s, const orc_camera* cam, const orc_render_opts* o, double* sum,
               double* sumsq, orc_stats* st) {
  return run(s, NULL, cam, o, sum, sumsq, st);
}

int orc_render_diff(const orc_scene* a, const orc_scene* b, const orc_camera* cam,
                    const orc_render_opts* o, double* sum, double* sumsq, orc_stats* st) {
  if (!b) return 1;
  return run(a, b, cam, o, sum, sumsq, st);
}

/* ------------------------------------------------------------------------ */
/* orc_render_grad: workers over pixel rows, each with its own accumulators. */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_scene* s;
  const orc_camera* cam;
  const orc_render_opts* op;
  const double* d_image;
  const greq* rq;
  orc_grad_out* out;
  int next, nrows;
  uint64_t paths, vertices, truncated, mismatch;
  pthread_mutex_t mu;
} gjob_t;

static double* zalloc(size_t n) { return n ? (double*)calloc(n, sizeof(double)) : NULL; }

static void* grad_worker(void* vp) {
  gjob_t* j = (gjob_t*)vp;
  const int no = j->s->n_objs;
  gacc acc[16];
  gctx g;
  memset(&g, 0, sizeof(g));
  g.rq = j->rq;
  g.acc = acc;
  for (int k = 0; k < no; ++k) {
    const greq* r = &j->rq[k];
    acc[k].mean = r->want_mean ? zalloc((size_t)r->n) : NULL;
    acc[k].var = r->want_var ? zalloc((size_t)r->n) : NULL;
    acc[k].alb = r->want_alb ? zalloc((size_t)r->n * r->channels) : NULL;
    acc[k].cs = r->want_cs ? zalloc((size_t)r->n) : NULL;
    acc[k].l = 0.0;
  }
  uint64_t np = 0, nv = 0, nt = 0;
  for (;;) {
    int r = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
    if (r >= j->nrows) break;
    int py = j->op->row_begin + r * j->op->row_step;
    for (int px = j->op->col_begin; px < j->op->col_end; ++px) {
      size_t pix = (size_t)py * j->cam->width + px;
      for (int c = 0; c < 3; ++c) g.gpix[c] = j->d_image[pix * 3 + c] / j->op->spp;
      int any = g.gpix[0] != 0.0 || g.gpix[1] != 0.0 || g.gpix[2] != 0.0;
      for (int smp = 0; smp < j->op->spp; ++smp) {
        double L[3];
        int tr;
        uint64_t v0 = 0;
        trace_path(j->s, j->cam, j->op, px, py, smp, L, &v0, &tr, NULL);
        nv += v0;
        nt += tr;
        ++np;
        if (!any || (L[0] == 0.0 && L[1] == 0.0 && L[2] == 0.0)) continue;
        for (int c = 0; c < 3; ++c) g.Ltot[c] = L[c];
        double L2[3];
        uint64_t v1 = 0;
        trace_path(j->s, j->cam, j->op, px, py, smp, L2, &v1, &tr, &g);
      }
    }
  }
  pthread_mutex_lock(&j->mu);
  for (int k = 0; k < no; ++k) {
    const greq* r = &j->rq[k];
    orc_grad_out* o = &j->out[k];
    for (int64_t i = 0; i < r->n; ++i) {
      if (acc[k].mean) o->d_mean[i] += acc[k].mean[i];
      if (acc[k].var) o->d_var[i] += acc[k].var[i];
      if (acc[k].cs) o->d_cscale[i] += acc[k].cs[i];
    }
    if (acc[k].alb)
      for (int64_t i = 0; i < r->n * r->channels; ++i) o->d_albedo[i] += acc[k].alb[i];
    if (r->want_l) *o->d_l += acc[k].l;
    free(acc[k].mean);
    free(acc[k].var);
    free(acc[k].alb);
    free(acc[k].cs);
  }
  j->paths += np;
  j->vertices += nv;
  j->truncated += nt;
  j->mismatch += g.mismatch;
  pthread_mutex_unlock(&j->mu);
  return NULL;
}

int orc_render_grad(const orc_scene* s, const orc_camera* cam, const orc_render_opts* op,
                    const double* d_image, orc_grad_out* out, orc_stats* st, uint64_t* mismatch) {
  if (!s || !cam || !op || !d_image || !out || op->spp <= 0 || op->max_bounces <= 0 || op->row_step <= 0)
    return 1;
  if (s->n_objs < 1 || s->n_objs > 16) return 1;
  if (op->row_begin < 0 || op->row_end > cam->height || op->col_begin < 0 || op->col_end > cam->width) return 1;
  for (int k = 0; k < s->n_objs; ++k) {
    const orc_object* ob = &s->objs[k];
    double lb = ob->length_scale_b > 0.0 ? ob->length_scale_b : ob->length_scale;
    double ln = ob->length_scale_n > 0.0 ? ob->length_scale_n : ob->length_scale;
    if (ob->ndf != ORC_NDF_GPSS || lb != ob->length_scale || ln != ob->length_scale || ob->tangent) return 2;
    if (out[k].d_cscale && !ob->cscale) return 1;
  }
  greq rq[16];
  int32_t* maps[16] = {NULL};
  int rc = 0;
  for (int k = 0; k < s->n_objs; ++k) {
    const orc_object* ob = &s->objs[k];
    const int64_t N = (int64_t)ob->nx * ob->ny * ob->nz;
    greq* r = &rq[k];
    memset(r, 0, sizeof(*r));
    r->channels = ob->channels;
    r->want_mean = out[k].d_mean != NULL;
    r->want_var = out[k].d_var != NULL;
    r->want_alb = out[k].d_albedo != NULL;
    r->want_cs = out[k].d_cscale != NULL;
    r->want_l = out[k].d_l != NULL;
    if (out[k].nodes) {
      maps[k] = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
      for (int64_t i = 0; i < N; ++i) maps[k][i] = -1;
      for (int64_t i = 0; i < out[k].n_nodes; ++i) {
        int64_t v = out[k].nodes[i];
        if (v < 0 || v >= N) rc = 1;
        else maps[k][v] = (int32_t)i;
      }
      r->map = maps[k];
      r->n = out[k].n_nodes;
    } else {
      r->n = N;
    }
  }
  if (rc == 0) {
    gjob_t j;
    memset(&j, 0, sizeof(j));
    j.s = s; j.cam = cam; j.op = op; j.d_image = d_image; j.rq = rq; j.out = out;
    j.nrows = op->row_end > op->row_begin ? (op->row_end - op->row_begin + op->row_step - 1) / op->row_step : 0;
    pthread_mutex_init(&j.mu, NULL);
    int nt = op->threads > 0 ? op->threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    if (nt > 256) nt = 256;
    pthread_t th[256];
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, grad_worker, &j);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&j.mu);
    if (st) {
      st->paths = j.paths;
      st->vertices = j.vertices;
      st->truncated = j.truncated;
    }
    if (mismatch) *mismatch = j.mismatch;
  }
  for (int k = 0; k < s->n_objs; ++k) free(maps[k]);
  return rc;
}
