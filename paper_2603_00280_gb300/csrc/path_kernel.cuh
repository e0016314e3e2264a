// path_kernel.cuh -- the persistent path kernel k_path<ADJ, TRAV, GEN>:
//   ADJ = false  forward render (film accumulation);
//   ADJ = true   path-replay adjoint: the same paths, traced from the same random
//                numbers by the same code, with gradient scattering added;
//   TRAV         the traversal compiled in (trav_of): the union majorant grid alone,
//                with local majorants (a thin single object), or per-object intervals
//                (several objects; gpss_device.cuh, trace_advance);
//   GEN          height-field objects and anisotropic / non-stationary kernels
//                compiled in (otherwise every object is an isotropic stationary GPSS
//                and the kind and kernel dispatch folds away).
//
// Integrator (Sec. 5 of the paper: null scattering on the classic exponential
// medium of Sec. 4):
//   - free flight by delta tracking against the majorant (tentative collisions at
//     optical depth -ln(u) of the majorant, real with probability sigma_t/majorant);
//   - at each real vertex next-event estimation with a ratio-tracking shadow ray
//     (T *= 1 - sigma_t/majorant per tentative collision, Russian roulette below
//     T = kRatioRR = 0.5), MIS (power heuristic) against phase sampling for environment lights;
//   - phase sampling with the mixture of Sec. 4.2 (or exactly from the visible
//     normals); at most max_bounces real vertices, no continuation after the last,
//     no Russian roulette on paths.
//
// Execution model: one persistent thread per resident lane.  Each iteration of the
// main loop advances every active lane by ONE tentative collision of its current
// ray (free-flight or shadow ray), so the lanes of a warp run the same traversal +
// extinction code together.  Lanes that reach a real vertex wait; the warp serves
// its waiting lanes together once at least `shade_min` of them wait or no lane can
// step, so the long shading code runs with many lanes active.  (A warp-private
// pool that parked waiting paths in shared memory and handed their lanes other
// paths was measured slower: its state swap runs every iteration on the few lanes
// that just reached a vertex.)  Shading code and the Philox block are out of line,
// keeping the traversal loop small in the instruction cache.  A finished lane takes
// the next (sample, pixel) index from a warp-private chunk of the global work cursor
// (one atomic per chunk; ranks from __ballot_sync/__popc).  Path state lives in
// registers.  Path index = sample * npix + pixel.
//
// Adjoint (path replay backpropagation, Vicini et al. 2021; null-collision terms of
// differential delta/ratio tracking, Nimier-David et al. 2022): with the majorant,
// sampling and light pdfs, MIS weights and roulette probabilities held fixed, every
// factor of the estimator contributes d(log factor) times the radiance the path
// collects downstream of it.  The path radiance L is read from the forward render
// (12 bytes kept per path), so downstream radiance is L - L_so_far at every event:
//   - tentative collision of a flight: weight <g, L - L_so_far> times
//     d sigma_t,k / sigma_t,k (real, k the scattering object; with several objects
//     taken when the vertex is shaded and k chosen) or -d sigma_t/(majorant - sigma_t)
//     (null; every object's partials to its own nodes);
//   - shadow ray: replayed twice from its random numbers -- first for its final
//     transmittance T (nothing is stored by the forward render), then, when the
//     vertex's NEE contribution carries gradient, with each tentative collision
//     scattering -d sigma_t/(majorant - sigma_t) with weight <g, pend> T, pend = the
//     vertex's NEE contribution before T;
//   - vertex: d ln(F D(m_L)/sigma(d)) with weight <g, C_k> (C_k = pend T) and
//     d ln(F D(m)/sigma(d)) of the sampled direction with weight <g, radiance after
//     the vertex's NEE>, taken once the shadow ray's first pass gives T;
// where g = dLoss/dpixel / spp.  Each evaluation scatters to the 8 grid nodes it
// interpolates (float atomics); the length-scale gradient is reduced per warp and
// object.
#pragma once

#include "adjoint_math.cuh"
#include "gpss_internal.h"

namespace gpss {

constexpr int kPathBlock = 128;
constexpr int kChunk = 256;
constexpr uint32_t kMaxEventsPerPath = 1u << 24;  // runaway guard (counted as aborted)

struct PathArgs {
  int spp, max_bounces;
  uint64_t seed;
  float mix_R;
  int npix;
  long long total;
  float inv_spp;
  int shade_min;
  int exact_vndf;  // sample the phase function with the exact visible-normal sampler
};

struct AdjOut {
  const float* d_image;   // dLoss/dimage (H*W*3)
  const float* L_path;    // per-path radiance of the forward render (3 per path)
  float2* d_mv;           // interleaved (d mean, d variance) accumulation buffer, or null
  float* d_alb;
  float* d_l;             // one per object
  float* d_cs;            // d correlation-scale factor per node, or null
  long long node_off[kMaxObjects];  // object k's first node in d_mv and d_cs (objects in order)
  long long alb_off[kMaxObjects];   // object k's first albedo value in d_alb (channels x nodes each)
  // record = 1: the forward pass whose per-path radiance the adjoint replays, run by the
  // adjoint's own kernel with no gradient (d_image unused): film and per-path radiance
  // as a forward render.  The replay then executes the same machine code with the same
  // random numbers, so its decisions match the recorded ones bit for bit.
  int record;
};

// Per-lane work counters, reduced per warp at the end of the kernel.
struct LaneCounters {
  uint32_t paths, vert, null_, shadow, cells, trunc, abort;
  uint32_t max_events;  // most tentative collisions of one path
  float acc_l[kMaxObjects];  // adjoint: length-scale gradient per object
  uint32_t nonfinite;   // adjoint: contributions skipped as not finite
};

enum Mode : int { kFlight = 0, kShadow = 1, kShadowPre = 2 };  // kShadowPre: adjoint only

// Whether a scene needs the general kernel instances: some object is a height-field
// macrofacet or has an anisotropic or non-stationary kernel.
inline bool scene_general(const SceneDev& S) {
  for (int k = 0; k < S.n_objs; ++k)
    if (S.obj[k].ndf != kNdfGpss || S.obj[k].general) return true;
  return false;
}

// GEN = false: every object is an isotropic stationary GPSS, so a field sample's kind and
// kernel are constants and their dispatch folds away.
template <bool GEN>
__device__ __forceinline__ Field fetch_k(const ObjectDev& o, V3 x) {
  if constexpr (GEN) {
    return fetch(o, x);
  } else {
    Field f = fetch_iso(o, x);
    f.ndf = kNdfGpss;
    return f;
  }
}


// Total extinction at x (single object fast path; several objects add; MULTI = false:
// the kernel serves single-object scenes only).
template <bool GEN, bool MULTI>
__device__ __forceinline__ float sigma_t_at(const SceneDev& S, V3 x, V3 d) {
  if (!MULTI || S.n_objs == 1) {
    if (!inside(S.obj[0], x)) return 0.0f;
    const Field f = fetch_k<GEN>(S.obj[0], x);
    const Local l = local_of(S.obj[0], f);
    return l.rho * projected_area(d, f, l.alpha);
  }
  float tot = 0.0f;
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    const Field f = fetch_k<GEN>(S.obj[k], x);
    const Local l = local_of(S.obj[k], f);
    tot += l.rho * projected_area(d, f, l.alpha);
  }
  return tot;
}

// The scattering object, chosen in proportion to its extinction (reading Q13).
template <bool GEN>
static __device__ __noinline__ int choose_object(const SceneDev& S, V3 x, V3 d, float u) {
  float tot = 0.0f;
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    Field fk;
    Local lk;
    tot += sigma_t_object<GEN>(S.obj[k], x, d, fk, lk);
  }
  float acc = 0.0f;
  int last = 0;
  const float pick = u * tot;
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    Field fk;
    Local lk;
    const float st = sigma_t_object<GEN>(S.obj[k], x, d, fk, lk);
    if (st <= 0.0f) continue;
    last = k;
    acc += st;
    if (pick < acc) break;
  }
  return last;
}

// Adjoint: scatter the derivative of object k's extinction (partials ds) at x with
// weight w.  The correlation-scale factor s enters through l(x) = s(x) l: d/ds(x) =
// (d/dl) l/s(x).  (GEN = false: the object has no correlation-scale grid.)  Returns the
// length-scale part.
template <bool GEN>
__device__ __forceinline__ float adj_scatter_event(const ObjectDev& ob, int k, V3 x, const DSig& ds, float w, float cs,
                                                   const AdjOut& A, uint32_t& nonfinite) {
  if (w == 0.0f) return 0.0f;
  const float cmu = w * ds.dmu, cvar = w * ds.dvar, cl = w * ds.dl;
  const V3 cg = w * ds.dg;
  // a contribution that is not finite (an extinction evaluated at the edge of FP32
  // range) is skipped and counted, so that it cannot poison the gradient grids
  if (!isfinite(cmu + cvar + cl + cg.x + cg.y + cg.z)) {
    ++nonfinite;
    return 0.0f;
  }
  if (A.d_mv) scatter_field(ob, x, cmu, cg, cvar, A.d_mv + A.node_off[k]);
  if constexpr (GEN) {
    if (A.d_cs && ob.cscale) scatter_scalar(ob, x, cl * (kSqrt2 / ob.alpha_scale) / cs, A.d_cs + A.node_off[k]);
  }
  return cl;
}

// The partials of ln sigma_t (a real collision's factor): each divided by sigma_t before
// any weight multiplies it, so a tiny sigma_t cannot overflow the weight.
__device__ __forceinline__ DSig dlog_of(const DSig& ds) {
  const float inv = 1.0f / ds.st;
  DSig r = ds;
  r.dmu *= inv;
  r.dvar *= inv;
  r.dl *= inv;
  r.dg = inv * ds.dg;
  return r;
}

// Adjoint: w d sigma_t of every object at x (the total extinction's derivative, each
// object's partials scattered to its own nodes); the length-scale parts per object.
template <bool GEN>
__device__ __forceinline__ void adj_scatter_all(const SceneDev& S, V3 x, V3 d, float w, const AdjOut& A,
                                                LaneCounters& c) {
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    const Field f = fetch_k<GEN>(S.obj[k], x);
    const DSig ds = dsigma_t(S.obj[k], f, d);
    c.acc_l[k] += adj_scatter_event<GEN>(S.obj[k], k, x, ds, w, f.cs, A, c.nonfinite);
  }
}

// Adjoint: gradient of the vertex factors of object k at x (incoming direction d_in):
// the NEE factor F D(m_nee)/sigma(d_in) with weight Wnee and the sampled direction's
// factor F D(m)/sigma(d_in) with weight Wph (the sigma(d_in) part is shared).
template <bool GEN>
__device__ __forceinline__ float adj_vertex(const ObjectDev& ob, int k, V3 x, V3 d_in, V3 wl, V3 d_next, float Wnee,
                                            float Wph, V3 albedo_coef, const AdjOut& A, uint32_t& nonfinite) {
  const Field f = fetch_k<GEN>(ob, x);
  const float sig = sqrtf(f.var);
  const float alpha = sig * f.as;
  V3 cg = v3(0, 0, 0);
  float dalpha = 0.0f;
  if (Wnee != 0.0f) {
    const DLogNdf dn = dlog_ndf(normalize(wl - d_in), f, alpha);
    cg = fma3(Wnee, dn.dg, cg);
    dalpha = fmaf(Wnee, dn.dalpha, dalpha);
  }
  if (Wph != 0.0f) {
    const DLogNdf dn = dlog_ndf(normalize(d_next - d_in), f, alpha);
    cg = fma3(Wph, dn.dg, cg);
    dalpha = fmaf(Wph, dn.dalpha, dalpha);
  }
  const float W = Wnee + Wph;
  if (W != 0.0f) {
    // -W d ln sigma(d_in): sigma(d) = alpha psi(a), d ln/d grad mu = -erfc(a)/(2 alpha psi) d,
    // d ln/d alpha = e^{-a^2}/(2 sqrt(pi) alpha psi)
    const float inv_a = 1.0f / alpha;
    float ps, ec_over, ea_over;
    psi_ratios(dot(d_in, f.g) * inv_a, ps, ec_over, ea_over);
    cg = fma3(W * 0.5f * ec_over * inv_a, d_in, cg);
    dalpha = fmaf(-W, ea_over * inv_a, dalpha);
  }
  const float cvar = dalpha * alpha / (2.0f * f.var);
  // d/dl through alpha = sqrt2 sigma/(s(x) l); d/ds(x) = (d/dl) l/s(x)
  const float dl = -dalpha * alpha * (ob.alpha_scale * kInvSqrt2);
  if (!isfinite(cg.x + cg.y + cg.z + cvar + dl + albedo_coef.x + albedo_coef.y + albedo_coef.z)) {
    ++nonfinite;  // skipped and counted (see adj_scatter_event)
    return 0.0f;
  }
  if (A.d_mv && (Wnee != 0.0f || Wph != 0.0f)) scatter_field(ob, x, 0.0f, cg, cvar, A.d_mv + A.node_off[k]);
  if (A.d_alb && (albedo_coef.x != 0.0f || albedo_coef.y != 0.0f || albedo_coef.z != 0.0f))
    scatter_albedo(ob, x, albedo_coef, A.d_alb + A.alb_off[k]);
  if constexpr (GEN) {
    if (A.d_cs && ob.cscale && dl != 0.0f)
      scatter_scalar(ob, x, dl * (kSqrt2 / ob.alpha_scale) / f.cs, A.d_cs + A.node_off[k]);
  }
  return dl;
}

// ---------------------------------------------------------------- per-lane path state
// The part of a lane's state that the traversal loop does not touch -- throughput,
// radiance, the pending NEE contribution, the next direction, weight and pdf, the bounce,
// pixel and path index: read and written at vertices and at the ends of rays only.  In the
// forward kernels it lives in shared memory (one record per thread, 21 words: an odd
// stride, so a warp's accesses to one field hit 32 different banks) instead of registers,
// which at the 64-register cap spilled it to local memory, whose reloads missed L1 under
// the field gathers' traffic (5% less frame time).  The adjoint kernel, at 128 registers
// without spills, keeps it in registers (in shared memory it ran 4% slower).
struct LaneCold {
  V3 beta, L, pend, d_next, beta_next;
  float prev_pdf, pdf_next;
  int bounce;
  uint32_t pixel;
  uint32_t pidx_lo, pidx_hi;
};
static_assert(sizeof(LaneCold) == 21 * 4, "LaneCold: 21 words (odd stride)");

struct Lane {
  bool active, waiting, begin, cont, walk_ok;
  int gid;     // the grid of the traversal interval (trace_advance)
  bool vgrad;  // adjoint: waiting for the vertex gradient (shadow pre-pass done), not for shading
  LaneCold* c;  // the lane's record in shared memory
  int job;
  Rng rng;
  V3 o, d;
  float T;
  int mode;
  uint32_t events;
  Walk w;
  // adjoint state: the path's forward radiance, dLoss/dpixel / spp, the current
  // vertex's final shadow transmittance, its arriving direction and scattering object
  V3 Ltot, gpix;
  float Tfin;
  V3 d_in;
  int kobj;
};

__device__ __forceinline__ void lane_init(Lane& s) {
  s.active = s.waiting = s.begin = s.cont = s.walk_ok = s.vgrad = false;
  s.gid = -1;
  s.c->pidx_lo = s.c->pidx_hi = 0u;
  s.c->pixel = 0;
  s.job = 0;
}

// The order of a render's paths.  The image is cut into kTile x kTile pixel tiles, taken
// in row-major order, and all samples of one tile come before the next tile (samples
// outer, pixels inner); the pixels outside the full tiles (a right and a bottom strip,
// when a side is not a multiple of kTile) follow, samples outer.  The resident lanes
// then hold the paths of a few neighbouring tiles, whose camera rays and first vertices
// read the same field cells (L2 reuse on grids larger than L2).  A path keeps its
// (pixel, sample), hence its random numbers: the order changes only the order of the
// film's float sums.
constexpr int kTile = 16;

__device__ __forceinline__ void path_of(long long pidx, int width, int height, int spp, uint32_t& pixel, int& sample) {
  const int tx = width / kTile, ty = height / kTile;
  const long long per_tile = (long long)kTile * kTile * spp;
  const long long full = per_tile * tx * ty;
  if (pidx < full) {
    const long long tile = pidx / per_tile;
    const long long r = pidx - tile * per_tile;
    sample = (int)(r / (kTile * kTile));
    const int q = (int)(r - (long long)sample * (kTile * kTile));
    const int py = (int)(tile / tx) * kTile + q / kTile, px = (int)(tile % tx) * kTile + q % kTile;
    pixel = (uint32_t)py * (uint32_t)width + (uint32_t)px;
    return;
  }
  const long long rest = (long long)width * height - (long long)tx * ty * (kTile * kTile);  // > 0 here
  const long long r = pidx - full;
  sample = (int)(r / rest);
  int k = (int)(r - (long long)sample * rest);
  const int rw = width - tx * kTile, rh = ty * kTile;  // the right strip is rw x rh pixels
  if (k < rw * rh) {
    pixel = (uint32_t)(k / rw) * (uint32_t)width + (uint32_t)(tx * kTile + k % rw);
    return;
  }
  k -= rw * rh;
  pixel = (uint32_t)(rh + k / width) * (uint32_t)width + (uint32_t)(k % width);
}

// Starts path `pidx` (in the order of path_of) of a render; returns false when the
// adjoint has nothing to do for it (no gradient flows through its pixel).
template <bool ADJ>
__device__ __forceinline__ bool lane_start(Lane& s, const CameraDev& C, const PathArgs& P, const AdjOut& A,
                                           long long pidx) {
  s.c->pidx_lo = (uint32_t)pidx;
  s.c->pidx_hi = (uint32_t)((unsigned long long)pidx >> 32);
  int sample;
  path_of(pidx, C.width, C.height, P.spp, s.c->pixel, sample);
  if constexpr (ADJ) {
    if (A.record) {
      s.gpix = v3(0.0f, 0.0f, 0.0f);
      s.Ltot = v3(0.0f, 0.0f, 0.0f);
    } else {
      s.gpix = v3(A.d_image[3 * s.c->pixel] * P.inv_spp, A.d_image[3 * s.c->pixel + 1] * P.inv_spp,
                  A.d_image[3 * s.c->pixel + 2] * P.inv_spp);
      s.Ltot = v3(A.L_path[3 * pidx], A.L_path[3 * pidx + 1], A.L_path[3 * pidx + 2]);
      if (s.gpix.x == 0.0f && s.gpix.y == 0.0f && s.gpix.z == 0.0f) return false;
    }
  }
  s.rng.init(P.seed, s.c->pixel, (uint32_t)sample);
  s.rng.start(0, kPurposeCamera);
  const float jx = s.rng.next(), jy = s.rng.next();
  camera_ray(C, (int)(s.c->pixel % (uint32_t)C.width), (int)(s.c->pixel / (uint32_t)C.width), jx, jy, s.o, s.d);
  s.c->beta = v3(1.0f, 1.0f, 1.0f);
  s.c->L = v3(0.0f, 0.0f, 0.0f);
  s.c->prev_pdf = -1.0f;
  s.c->bounce = 0;
  s.mode = kFlight;
  s.events = 0;
  s.rng.start(0, kPurposeFlight);
  s.begin = true;
  s.waiting = false;
  s.vgrad = false;
  s.active = true;
  return true;
}

// Adjoint: the vertex's gradient once its NEE contribution C = pend T_fin is known (T_fin
// = the shadow ray's final transmittance, recomputed by the replay), and C added to the
// radiance so far.  wl: the NEE direction.
template <bool GEN>
__device__ __forceinline__ void adj_vertex_done(Lane& s, const SceneDev& S, const AdjOut& A, V3 wl, float Tfin,
                                                LaneCounters& c) {
  const V3 x = s.o;
  const V3 Ck = v3(s.c->pend.x * Tfin, s.c->pend.y * Tfin, s.c->pend.z * Tfin);
  if (s.gpix.x == 0.0f && s.gpix.y == 0.0f && s.gpix.z == 0.0f) {  // recording: no gradient
    s.c->L = s.c->L + Ck;
    return;
  }
  const V3 F = fetch_albedo(S.obj[s.kobj], x);
  const V3 after = s.Ltot - s.c->L - Ck;
  const float Wnee = dot(s.gpix, Ck);
  const float Wph = s.cont ? dot(s.gpix, after) : 0.0f;
  const V3 ac = v3(F.x > 0.0f ? s.gpix.x * (Ck.x + (s.cont ? after.x : 0.0f)) / F.x : 0.0f,
                   F.y > 0.0f ? s.gpix.y * (Ck.y + (s.cont ? after.y : 0.0f)) / F.y : 0.0f,
                   F.z > 0.0f ? s.gpix.z * (Ck.z + (s.cont ? after.z : 0.0f)) / F.z : 0.0f);
  c.acc_l[s.kobj] += adj_vertex<GEN>(S.obj[s.kobj], s.kobj, x, s.d_in, wl, s.c->d_next, Wnee, Wph, ac, A, c.nonfinite);
  s.c->L = s.c->L + Ck;
}

// After the shadow ray (or in place of it): the next flight, or the end of the path.
__device__ __forceinline__ bool lane_continue(Lane& s) {
  if (!s.cont) return true;
  s.mode = kFlight;
  s.d = s.c->d_next;
  s.c->beta = s.c->beta_next;
  s.c->prev_pdf = s.c->pdf_next;
  s.rng.start((uint32_t)s.c->bounce, kPurposeFlight);
  s.begin = true;
  return false;
}

// Ends the path at the lane's next step: with walk_ok = false and beta = 0 the step
// treats it as an escaped flight that adds nothing.
__device__ __forceinline__ void lane_end_at_next_step(Lane& s) {
  s.mode = kFlight;
  s.walk_ok = false;
  s.begin = false;
  s.c->beta = v3(0.0f, 0.0f, 0.0f);
}

// Adjoint, with the warp's shading (the vertex gradient is long, divergent code: taken
// in the traversal loop it would run for one lane at a time): the gradient of the vertex
// whose shadow pre-pass found T_fin, then the gradient pass of the same shadow ray (its
// random numbers replayed from the start of the NEE stream) if it carries any.
template <bool GEN>
__device__ __forceinline__ void lane_vertex_grad(Lane& s, const SceneDev& S, const AdjOut& A, LaneCounters& c) {
  s.waiting = false;
  s.vgrad = false;
  adj_vertex_done<GEN>(s, S, A, s.d, s.Tfin, c);
  if (s.Tfin > 0.0f && dot(s.gpix, s.c->pend) != 0.0f) {
    s.mode = kShadow;
    s.T = 1.0f;
    s.begin = true;
    s.rng.start((uint32_t)(s.c->bounce - 1), kPurposeNee);
    if (S.light.kind != kLightDirectional) {
      s.rng.next();
      s.rng.next();
    }
    return;
  }
  if (lane_continue(s)) lane_end_at_next_step(s);
}

// Shading of a real vertex: phase sampling, next-event estimation setup.
template <bool ADJ, bool GEN, bool MULTI>
__device__ __forceinline__ void lane_shade(Lane& s, const SceneDev& S, const PathArgs& P, const AdjOut& A,
                                           LaneCounters& c) {
  if constexpr (ADJ) {
    if (s.vgrad) {
      lane_vertex_grad<GEN>(s, S, A, c);
      return;
    }
  }
  const bool env = S.light.kind != kLightDirectional;
  s.waiting = false;
  const V3 x = fma3(s.w.t, s.d, s.o);
  const bool multi = MULTI && S.n_objs > 1;
  const int k = multi ? choose_object<GEN>(S, x, s.d, s.rng.next()) : 0;
  const Field f = fetch_k<GEN>(S.obj[k], x);
  const float alpha = sqrtf(f.var) * f.as;  // the density rho is not needed for shading
  const V3 F = fetch_albedo(S.obj[k], x);
  if constexpr (ADJ) {
    // several objects: the real collision's factor is the chosen object's sigma_t,k (the
    // choice probability sigma_t,k/sigma_t is held fixed), known only now
    if (multi) {
      const float W = dot(s.gpix, s.Ltot - s.c->L);
      if (W != 0.0f) {
        const DSig ds = dsigma_t(S.obj[k], f, s.d);
        if (ds.st > 0.0f) c.acc_l[k] += adj_scatter_event<GEN>(S.obj[k], k, x, dlog_of(ds), W, f.cs, A, c.nonfinite);
      }
    }
    s.d_in = s.d;
    s.kobj = k;
  }
  s.o = x;
  s.cont = s.c->bounce + 1 < P.max_bounces;
  float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
  if (s.cont) {
    s.rng.start((uint32_t)s.c->bounce, kPurposePhase);
    u0 = s.rng.next();
    u1 = s.rng.next();
    u2 = s.rng.next();
  } else {
    ++c.trunc;
  }
  s.rng.start((uint32_t)s.c->bounce, kPurposeNee);
  V3 wl, Le;
  if (!env) {
    wl = v3(S.light.dir[0], S.light.dir[1], S.light.dir[2]);
    Le = v3(S.light.radiance[0], S.light.radiance[1], S.light.radiance[2]);
  } else {
    const float z = 1.0f - 2.0f * s.rng.next();
    const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincospif(2.0f * s.rng.next(), &sp, &cp);
    wl = v3(r * cp, r * sp, z);
    Le = env_radiance(S.light, wl);
  }
  const VertexShade vs = shade_vertex_call(s.d, wl, f, alpha, P.mix_R, s.cont, P.exact_vndf != 0, u0, u1, u2);
  if (s.cont) {
    const PhaseSample& ps = vs.next;
    if (ps.ok) {
      s.c->d_next = ps.d2;
      s.c->beta_next = v3(s.c->beta.x * F.x * ps.w_over_F, s.c->beta.y * F.y * ps.w_over_F, s.c->beta.z * F.z * ps.w_over_F);
      s.c->pdf_next = ps.pdf;
    } else {
      s.cont = false;
    }
  }
  const PhaseEval& pe = vs.nee;
  const float lw = env ? power_heuristic(kInv4Pi, pe.pdf) * (4.0f * kPi) : 1.0f;
  const float scale = pe.p_over_F * lw;
  s.c->pend = v3(s.c->beta.x * F.x * scale * Le.x, s.c->beta.y * F.y * scale * Le.y, s.c->beta.z * F.z * scale * Le.z);
  ++s.c->bounce;
  if (scale > 0.0f) {
    // the shadow ray; the adjoint first replays it for its final transmittance (pre-pass)
    s.mode = ADJ ? kShadowPre : kShadow;
    s.d = wl;
    s.T = 1.0f;
    s.begin = true;
    return;
  }
  if constexpr (ADJ) adj_vertex_done<GEN>(s, S, A, wl, 0.0f, c);  // no NEE contribution
  if (s.cont) {
    lane_continue(s);
  } else {
    lane_end_at_next_step(s);  // no shadow ray and no continuation
  }
}

// One tentative collision of the lane's current ray; returns true when the path ends.
// Adjoint shadow rays run twice from the same random numbers: a pre-pass (kShadowPre)
// that only computes the ray's final transmittance T_fin, then -- when the vertex's
// NEE contribution pend T_fin carries gradient -- the gradient pass (kShadow) whose
// tentative collisions scatter -d sigma_t/(majorant - sigma_t) with weight <g, pend> T_fin.
template <bool ADJ, int TRAV, bool GEN>
__device__ __forceinline__ bool lane_step(Lane& s, const SceneDev& S, const MajorantDev* og, const PathArgs& P,
                                          const AdjOut& A, LaneCounters& c) {
  const bool env = S.light.kind != kLightDirectional;
  constexpr bool LOCAL = (TRAV & kTravLocal) != 0, SPLIT = (TRAV & kTravSplitBit) != 0,
                 MULTI = (TRAV & kTravMulti) != 0;
  if (s.begin) {
    s.walk_ok = trace_begin<SPLIT>(S, og, s.o, s.d, INFINITY, s.w, s.gid);
    s.begin = false;
  }
  bool hit = false;
  if (s.walk_ok) {
    float tau = -__logf(s.rng.next());
    hit = trace_advance<LOCAL, SPLIT, GEN>(S, og, s.o, s.d, INFINITY, s.w, s.gid, tau, c.cells) == kWalkHit;
  }
  if (hit) {
    ++s.events;
    const V3 x = fma3(s.w.t, s.d, s.o);
    if (ADJ && s.mode == kShadowPre) {
      ++c.shadow;
      if (!ratio_step(s.T, sigma_t_at<GEN, MULTI>(S, x, s.d), s.w.sbar, s.rng)) s.walk_ok = false;
    } else if (ADJ && (!MULTI || S.n_objs == 1)) {
      // the extinction by the forward's expression (the recording pass and the replay run
      // this same code), its partials only where a gradient is scattered
      float st = 0.0f, k_adj = 0.0f;
      bool real = false;
      Field f;
      const bool inobj = inside(S.obj[0], x);
      if (inobj) {
        f = fetch_k<GEN>(S.obj[0], x);
        const Local l = local_of(S.obj[0], f);
        st = l.rho * projected_area(s.d, f, l.alpha);
      }
      if (s.mode == kFlight) {
        real = s.rng.next() * s.w.sbar < st;
        const float W = dot(s.gpix, s.Ltot - s.c->L);
        if (W != 0.0f) k_adj = real ? W : -W / (s.w.sbar - st);  // real: times d ln sigma_t
        if (real) {
          ++c.vert;
          s.waiting = true;
        } else {
          ++c.null_;
        }
      } else {
        ++c.shadow;
        const float Wn = dot(s.gpix, s.c->pend) * s.Tfin;
        if (Wn != 0.0f) k_adj = -Wn / (s.w.sbar - st);
        if (!ratio_step(s.T, st, s.w.sbar, s.rng)) s.walk_ok = false;
      }
      if (inobj && k_adj != 0.0f) {
        const DSig ds = dsigma_t(S.obj[0], f, s.d);
        c.acc_l[0] += adj_scatter_event<GEN>(S.obj[0], 0, x, real ? dlog_of(ds) : ds, k_adj, f.cs, A, c.nonfinite);
      }
    } else {
      const float st = sigma_t_at<GEN, MULTI>(S, x, s.d);
      float k_adj = 0.0f;  // adjoint (several objects): weight of every object's d sigma_t here
      if (s.mode == kFlight) {
        const bool real = s.rng.next() * s.w.sbar < st;
        if constexpr (ADJ) {
          // a real collision's gradient waits for the object choice at shading
          const float W = dot(s.gpix, s.Ltot - s.c->L);
          if (!real && W != 0.0f) k_adj = -W / (s.w.sbar - st);
        }
        if (real) {
          ++c.vert;
          s.waiting = true;  // real scattering vertex: parked and shaded with the warp's pool
        } else {
          ++c.null_;
        }
      } else {
        ++c.shadow;
        if constexpr (ADJ) {
          const float Wn = dot(s.gpix, s.c->pend) * s.Tfin;
          if (Wn != 0.0f) k_adj = -Wn / (s.w.sbar - st);
        }
        if (!ratio_step(s.T, st, s.w.sbar, s.rng)) s.walk_ok = false;  // T = 0: the shadow ray ends here
      }
      if constexpr (ADJ) {
        if (k_adj != 0.0f) adj_scatter_all<GEN>(S, x, s.d, k_adj, A, c);
      }
    }
    if (s.events >= kMaxEventsPerPath) {
      ++c.abort;
      s.waiting = false;
      return true;
    }
    return false;
  }
  if (s.mode == kFlight) {
    if (env) {
      const V3 Le = env_radiance(S.light, s.d);
      const float wm = s.c->prev_pdf < 0.0f ? 1.0f : power_heuristic(s.c->prev_pdf, kInv4Pi);
      s.c->L = v3(fmaf(s.c->beta.x * Le.x, wm, s.c->L.x), fmaf(s.c->beta.y * Le.y, wm, s.c->L.y), fmaf(s.c->beta.z * Le.z, wm, s.c->L.z));
    }
    return true;
  }
  if constexpr (ADJ) {
    if (s.mode == kShadowPre) {
      // T_fin known: the lane waits for the warp's shading, which takes the vertex's
      // gradient and starts the gradient pass (lane_vertex_grad); a recording path (no
      // gradient) has neither and goes on at once (scheduling only: the path's arithmetic
      // and random numbers are the same either way)
      s.Tfin = s.T;
      if (s.gpix.x == 0.0f && s.gpix.y == 0.0f && s.gpix.z == 0.0f) {
        s.c->L = s.c->L + v3(s.c->pend.x * s.Tfin, s.c->pend.y * s.Tfin, s.c->pend.z * s.Tfin);
        return lane_continue(s);
      }
      s.vgrad = true;
      s.waiting = true;
      return false;
    }
  } else {
    s.c->L = v3(fmaf(s.c->pend.x, s.T, s.c->L.x), fmaf(s.c->pend.y, s.T, s.c->L.y), fmaf(s.c->pend.z, s.T, s.c->L.z));
  }
  return lane_continue(s);
}

// Film accumulation (forward) or the replay check (adjoint) of a finished path.
template <bool ADJ>
__device__ __forceinline__ void lane_finish(Lane& s, const PathArgs& P, float* __restrict__ image,
                                            float* __restrict__ sqsum, float* __restrict__ path_radiance,
                                            bool record, LaneCounters& c) {
  if (!ADJ || record) {
    float* px = image + 3 * (size_t)s.c->pixel;
    atomicAdd(px + 0, s.c->L.x * P.inv_spp);
    atomicAdd(px + 1, s.c->L.y * P.inv_spp);
    atomicAdd(px + 2, s.c->L.z * P.inv_spp);
    if (sqsum) {
      float* q = sqsum + 3 * (size_t)s.c->pixel;
      atomicAdd(q + 0, s.c->L.x * s.c->L.x);
      atomicAdd(q + 1, s.c->L.y * s.c->L.y);
      atomicAdd(q + 2, s.c->L.z * s.c->L.z);
    }
    if (path_radiance) {
      const long long pidx = (long long)(((unsigned long long)s.c->pidx_hi << 32) | s.c->pidx_lo);
      float* pr = path_radiance + 3 * pidx;
      pr[0] = s.c->L.x;
      pr[1] = s.c->L.y;
      pr[2] = s.c->L.z;
    }
  } else {
    // the replay must reproduce the forward path; count any that does not
    const V3 e = s.c->L - s.Ltot;
    const float tol = 1e-3f * (fabsf(s.Ltot.x) + fabsf(s.Ltot.y) + fabsf(s.Ltot.z)) + 1e-6f;
    if (fabsf(e.x) + fabsf(e.y) + fabsf(e.z) > tol) ++c.abort;
  }
  ++c.paths;
  c.max_events = max(c.max_events, s.events);
  s.active = false;
}

// Warp-converged chunked work distribution: lanes without a path take the next
// indices of the warp's chunk of the global cursor (one atomic per `chunk`).
struct WarpCursor {
  long long next, end;
  bool exhausted;
};

__device__ __forceinline__ long long warp_take(WarpCursor& wc, bool want, unsigned need, int lane,
                                               unsigned long long* cursor, long long total, int chunk) {
  const int n_need = __popc(need);
  const int rank = __popc(need & ((1u << lane) - 1u));
  const long long avail = wc.end - wc.next;
  long long mine = -1;
  if (avail >= n_need) {
    if (want) mine = wc.next + rank;
    wc.next += n_need;
  } else {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)chunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (want) mine = rank < avail ? wc.next + rank : (long long)base + (rank - avail);
    wc.next = (long long)base + (n_need - avail);
    wc.end = (long long)base + chunk;
    if ((long long)base >= total) wc.exhausted = true;
  }
  return mine;
}

__device__ __forceinline__ void flush_counters(const LaneCounters& c, unsigned long long* counters, float* d_l,
                                               int n_objs) {
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  if (d_l) {
    for (int k = 0; k < n_objs; ++k) {
      float a = c.acc_l[k];
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(FULL, a, off);
      if (lane == 0 && a != 0.0f) atomicAdd(d_l + k, a);
    }
  }
  const uint32_t vals[7] = {c.paths, c.vert, c.null_, c.shadow, c.cells, c.trunc, c.abort};
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
    if (lane == 0 && v) atomicAdd(counters + i, v);
  }
  unsigned long long nf = c.nonfinite;
  for (int off = 16; off > 0; off >>= 1) nf += __shfl_down_sync(FULL, nf, off);
  if (lane == 0 && nf) atomicAdd(counters + kCntNonFinite, nf);
  uint32_t me = c.max_events;
  for (int off = 16; off > 0; off >>= 1) me = max(me, __shfl_down_sync(FULL, me, off));
  if (lane == 0 && me) atomicMax(counters + kCntMaxEvents, (unsigned long long)me);
}

// ---------------------------------------------------------------- the path loop
// One warp's persistent loop over the paths of a work source W, which provides:
//   take(s, need, lane)  new paths for the lanes in `need` (warp-collective);
//   exhausted()          no new path is left (warp-uniform);
//   scene(s), args(s)    the scene and options of a path (its job's, in a batch);
//   grids(s)             the objects' own majorant grids of that scene (per-object traversal);
//   finish(s, c)         film accumulation / replay check of a finished path;
//   adj()                the adjoint's buffers.
// Each iteration: (1) lanes without a path take new ones; (2) once at least shade_min
// lanes wait at a real vertex (or no other lane can step) the warp shades them
// together; (3) every other lane with a path advances it by one tentative collision.
template <bool ADJ, int TRAV, bool GEN, class W>
__device__ __forceinline__ void path_loop(W& src, int shade_min, LaneCold* cold, LaneCounters& c) {
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  Lane s;
  LaneCold own;  // the adjoint kernel (128 registers, no spills) keeps the record in registers
  if constexpr (ADJ) {
    s.c = &own;
  } else {
    s.c = cold + threadIdx.x;
  }
  lane_init(s);
  for (;;) {
    const unsigned need = __ballot_sync(FULL, !s.active);
    if (need && !src.exhausted()) src.take(s, need, lane);
    const unsigned act = __ballot_sync(FULL, s.active);
    if (act == 0u) {
      if (src.exhausted()) break;
      continue;
    }
    const unsigned wait_mask = __ballot_sync(FULL, s.waiting);
    if (wait_mask && (__popc(wait_mask) >= shade_min || wait_mask == act)) {
      if (s.waiting) lane_shade<ADJ, GEN, (TRAV & kTravMulti) != 0>(s, src.scene(s), src.args(s), src.adj(), c);
    }
    if (!s.active || s.waiting) continue;
    if (lane_step<ADJ, TRAV, GEN>(s, src.scene(s), src.grids(s), src.args(s), src.adj(), c)) src.finish(s, c);
  }
}

// ---------------------------------------------------------------- single-render kernel
// Work source of one render: path indices [0, total) from the global cursor.
template <bool ADJ>
struct RenderSource {
  const SceneDev& S;
  const CameraDev& C;
  const PathArgs& P;
  const AdjOut& A;
  float* image;
  float* sqsum;
  float* path_radiance;
  unsigned long long* cursor;
  const MajorantDev* og;  // the objects' grids, copied to shared memory
  WarpCursor wc;
  __device__ __forceinline__ void take(Lane& s, unsigned need, int lane) {
    const long long mine = warp_take(wc, !s.active, need, lane, cursor, P.total, kChunk);
    if (!s.active && mine >= 0 && mine < P.total) lane_start<ADJ>(s, C, P, A, mine);
  }
  __device__ __forceinline__ bool exhausted() const { return wc.exhausted || wc.next >= P.total; }
  __device__ __forceinline__ const SceneDev& scene(const Lane&) const { return S; }
  __device__ __forceinline__ const MajorantDev* grids(const Lane&) const { return og; }
  __device__ __forceinline__ const PathArgs& args(const Lane&) const { return P; }
  __device__ __forceinline__ const AdjOut& adj() const { return A; }
  __device__ __forceinline__ void finish(Lane& s, LaneCounters& c) {
    lane_finish<ADJ>(s, P, image, sqsum, path_radiance, A.record != 0, c);
  }
};

// TRAV: the scene's traversal (trav_of).  GEN: some object is a
// height-field macrofacet or has an anisotropic or non-stationary kernel (the adjoint
// supports the isotropic GPSS, stationary or with a correlation-scale grid).
template <bool ADJ, int TRAV, bool GEN>
__global__ void __launch_bounds__(kPathBlock, ADJ ? 4 : 8)
    k_path(const __grid_constant__ SceneDev S, const __grid_constant__ CameraDev C, const __grid_constant__ PathArgs P,
           float* __restrict__ image, float* __restrict__ sqsum, float* __restrict__ path_radiance,
           unsigned long long* __restrict__ counters, const __grid_constant__ AdjOut A) {
  // the objects' grids in shared memory: the per-object walk reads them with a per-lane
  // object index at every step (a parameter-space read would be an indexed constant load)
  __shared__ MajorantDev s_og[kMaxObjects];
  if constexpr ((TRAV & kTravSplitBit) != 0) {
    if (threadIdx.x < kMaxObjects) s_og[threadIdx.x] = S.og[threadIdx.x];
    __syncthreads();
  }
  __shared__ LaneCold s_cold[kPathBlock];
  RenderSource<ADJ> src{S, C, P, A, image, sqsum, path_radiance, counters + kCntNum, s_og, WarpCursor{0, 0, false}};
  LaneCounters c{0, 0, 0, 0, 0, 0, 0, 0, {0.0f, 0.0f, 0.0f, 0.0f}, 0};
  path_loop<ADJ, TRAV, GEN>(src, P.shade_min, s_cold, c);
  flush_counters(c, counters, ADJ ? A.d_l : nullptr, S.n_objs);
}

}  // namespace gpss
