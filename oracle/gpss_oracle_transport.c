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

/* One path: camera ray, then per real scattering vertex next-event
 * estimation and phase-function sampling (MIS with the environment).  At
 * most max_bounces real vertices; no continuation after the last. */
static void trace_path(const orc_scene* s, const orc_camera* cam, const orc_render_opts* op, int px,
                       int py, int sample, double L[3], uint64_t* nvert, int* truncated) {
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
    double t;
    if (!free_flight(s, o, d, -log(u[0]), &t)) {
      if (env) {
        double Le[3], w = prev_pdf < 0.0 ? 1.0 : power_heuristic(prev_pdf, inv4pi);
        env_radiance(&s->light, d, Le);
        for (int c = 0; c < 3; ++c) L[c] += beta[c] * Le[c] * w;
      }
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
    /* next-event estimation */
    double pv[3], pdf_ph;
    if (!env) {
      const double* wl = s->light.dir;
      orc_phase_eval_point(&p, d, wl, op->mix_R, pv, &pdf_ph);
      double Tr = orc_transmittance(s, x, wl, INFINITY);
      for (int c = 0; c < 3; ++c) L[c] += beta[c] * pv[c] * Tr * s->light.radiance[c];
    } else {
      double z = 1.0 - 2.0 * u[2], ph = 2.0 * ORC_PI * u[3], r = sqrt(fmax(0.0, 1.0 - z * z));
      double wl[3] = {r * cos(ph), r * sin(ph), z};
      orc_phase_eval_point(&p, d, wl, op->mix_R, pv, &pdf_ph);
      if (pv[0] > 0.0 || pv[1] > 0.0 || pv[2] > 0.0) {
        double Tr = orc_transmittance(s, x, wl, INFINITY);
        double Le[3], w = power_heuristic(inv4pi, pdf_ph);
        env_radiance(&s->light, wl, Le);
        for (int c = 0; c < 3; ++c) L[c] += beta[c] * pv[c] * Tr * Le[c] * w / inv4pi;
      }
    }
    if (bounce + 1 >= op->max_bounces) {
      *truncated = 1;
      return;
    }
    orc_uniform4(op->seed, pixel, (uint32_t)sample, (uint32_t)bounce, P_PHASE, 0, u);
    double d2[3], wgt[3], pdf;
    if (!orc_phase_sample_point(&p, d, op->mix_R, u, d2, wgt, &pdf)) return;
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
        trace_path(j->a, j->cam, j->op, px, py, s, La, &nv, &tr);
        nt += tr;
        if (j->b) {
          uint64_t nv2 = 0;
          int tr2;
          trace_path(j->b, j->cam, j->op, px, py, s, Lb, &nv2, &tr2);
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
