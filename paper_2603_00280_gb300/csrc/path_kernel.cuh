// path_kernel.cuh -- the persistent path kernel, in two instances:
//   ADJ = false  forward render (film accumulation);
//   ADJ = true   path-replay adjoint: the same paths, traced from the same random
//                numbers by the same code, with gradient scattering added.
//
// Integrator (Sec. 5 of the paper: null scattering on the classic exponential
// medium of Sec. 4):
//   - free flight by delta tracking against the majorant (tentative collisions at
//     optical depth -ln(u) of the majorant, real with probability sigma_t/majorant);
//   - at each real vertex next-event estimation with a ratio-tracking shadow ray
//     (T *= 1 - sigma_t/majorant per tentative collision, Russian roulette below
//     T = 0.1), MIS (power heuristic) against phase sampling for environment lights;
//   - phase sampling with the mixture of Sec. 4.2.2; at most max_bounces real
//     vertices, no continuation after the last, no Russian roulette on paths.
//
// Execution model: one persistent thread per resident lane.  Each iteration of the
// main loop advances every active lane by ONE tentative collision of its current
// ray (free-flight or shadow ray), so the lanes of a warp run the same traversal +
// extinction code together.  Lanes that reach a real vertex (or, in the adjoint, a
// vertex whose gradient is due) wait; the warp serves its waiting lanes together
// once at least `shade_min` of them wait or no lane can step, so the long shading
// code runs with many lanes active.  Shading code and the Philox block are out of
// line, keeping the traversal loop small in the instruction cache.  A finished
// lane takes the next (sample, pixel) index from a warp-private chunk of the
// global work cursor (one atomic per chunk; ranks from __ballot_sync/__popc).  Path
// state lives in registers.  Path index = sample * npix + pixel.
//
// Adjoint (path replay backpropagation, Vicini et al. 2021; null-collision terms of
// differential delta/ratio tracking, Nimier-David et al. 2022): with the majorant,
// sampling and light pdfs, MIS weights and roulette probabilities held fixed, every
// factor of the estimator contributes d(log factor) times the radiance the path
// collects downstream of it.  The path radiance L is read from the forward render
// (kept per path, with each vertex's final shadow transmittance), so downstream
// radiance is L - L_so_far at every event:
//   - tentative collision of a flight: weight <g, L - L_so_far> times
//     d sigma_t / sigma_t (real) or -d sigma_t/(majorant - sigma_t) (null);
//   - shadow ray: each tentative collision scatters -d sigma_t/(majorant - sigma_t)
//     with weight <g, pend> T, pend = the vertex's NEE contribution before T and T
//     the ray's final transmittance, recorded per vertex by the forward render;
//   - vertex: d ln(F D(m_L)/sigma(d)) with weight <g, C_k> (C_k = pend T) and
//     d ln(F D(m)/sigma(d)) of the sampled direction with weight <g, radiance after
//     the vertex's NEE>;
// where g = dLoss/dpixel / spp.  Each evaluation scatters to the 8 grid nodes it
// interpolates (float atomics); the length-scale gradient is reduced per warp.
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
};

struct AdjOut {
  const float* d_image;   // dLoss/dimage (H*W*3)
  const float* L_path;    // per-path radiance of the forward render (3 per path)
  const float* T_path;    // per-vertex final shadow transmittance (max_bounces per path)
  float* d_mean;
  float* d_var;
  float* d_alb;
  float* d_l;
};

enum Mode : int { kFlight = 0, kShadow = 1 };

// Total extinction at x (single object fast path; several objects add).
__device__ __forceinline__ float sigma_t_at(const SceneDev& S, V3 x, V3 d) {
  if (S.n_objs == 1) {
    if (!inside(S.obj[0], x)) return 0.0f;
    Field f;
    Local l;
    return sigma_t_object(S.obj[0], x, d, f, l);
  }
  return scene_sigma_t(S, x, d);
}

// The scattering object, chosen in proportion to its extinction (reading Q13),
// and its field at x.
static __device__ __noinline__ int choose_object(const SceneDev& S, V3 x, V3 d, float u, Field& f, Local& l) {
  float tot = 0.0f;
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    Field fk;
    Local lk;
    tot += sigma_t_object(S.obj[k], x, d, fk, lk);
  }
  float acc = 0.0f;
  int last = 0;
  const float pick = u * tot;
  for (int k = 0; k < S.n_objs; ++k) {
    if (!inside(S.obj[k], x)) continue;
    Field fk;
    Local lk;
    const float st = sigma_t_object(S.obj[k], x, d, fk, lk);
    if (st <= 0.0f) continue;
    last = k;
    f = fk;
    l = lk;
    acc += st;
    if (pick < acc) break;
  }
  return last;
}

// Adjoint: scatter the derivative of the extinction (partials ds) at x with weight k.
__device__ __forceinline__ float adj_scatter_event(const ObjectDev& ob, V3 x, const DSig& ds, float k, float* d_mean,
                                                   float* d_var) {
  if (!isfinite(k) || k == 0.0f) return 0.0f;
  scatter_field(ob, x, k * ds.dmu, k * ds.dg, k * ds.dvar, d_mean, d_var);
  return k * ds.dl;
}

// Adjoint: gradient of the vertex factors at x (incoming direction d_in).
static __device__ __noinline__ float adj_vertex(const ObjectDev& ob, V3 x, V3 d_in, V3 wl, V3 d_next, float Wnee,
                                                float Wph, V3 albedo_coef, const AdjOut A) {
  const Field f = fetch(ob, x);
  V3 cg = v3(0, 0, 0);
  float cvar = 0.0f, dl = 0.0f;
  if (Wnee != 0.0f) {
    const DPhase dp = dlog_phase(d_in, normalize(wl - d_in), f, ob.alpha_scale);
    cg = fma3(Wnee, dp.dg, cg);
    cvar += Wnee * dp.dvar;
    dl += Wnee * dp.dl;
  }
  if (Wph != 0.0f) {
    const DPhase dp = dlog_phase(d_in, normalize(d_next - d_in), f, ob.alpha_scale);
    cg = fma3(Wph, dp.dg, cg);
    cvar += Wph * dp.dvar;
    dl += Wph * dp.dl;
  }
  if ((A.d_mean || A.d_var) && (Wnee != 0.0f || Wph != 0.0f)) scatter_field(ob, x, 0.0f, cg, cvar, A.d_mean, A.d_var);
  if (A.d_alb && (albedo_coef.x != 0.0f || albedo_coef.y != 0.0f || albedo_coef.z != 0.0f))
    scatter_albedo(ob, x, albedo_coef, A.d_alb);
  return dl;
}

template <bool ADJ>
__global__ void __launch_bounds__(kPathBlock, ADJ ? 4 : 5) k_path(const SceneDev S, const CameraDev C, const PathArgs P,
                                                    float* __restrict__ image, float* __restrict__ sqsum,
                                                    float* __restrict__ path_radiance, float* __restrict__ path_T,
                                                    unsigned long long* __restrict__ counters, const AdjOut A) {
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  unsigned long long* cursor = counters + kCntNum;
  const bool env = S.light.kind != kLightDirectional;

  long long chunk_next = 0, chunk_end = 0;
  bool exhausted = false;

  bool active = false, waiting = false, begin = false;
  long long pidx = 0;
  uint32_t pixel = 0;
  Rng rng;
  V3 o{}, d{}, beta{}, L{}, pend{}, d_next{}, beta_next{};
  float prev_pdf = -1.0f, T = 1.0f, pdf_next = 0.0f;
  int bounce = 0, mode = kFlight;
  bool cont = false, walk_ok = false;
  uint32_t events = 0;
  Walk w;
  // adjoint state
  bool vgrad = false;
  V3 Ltot{}, gpix{}, d_in{};
  float Tfin = 0.0f, acc_l = 0.0f;

  uint32_t c_paths = 0, c_vert = 0, c_null = 0, c_shadow = 0, c_cells = 0, c_trunc = 0, c_abort = 0;

  for (;;) {
    // ------------------------------------------------ regeneration (warp-converged)
    const unsigned need = __ballot_sync(FULL, !active);
    if (need && !exhausted) {
      const int n_need = __popc(need);
      const int rank = __popc(need & ((1u << lane) - 1u));
      long long avail = chunk_end - chunk_next;
      long long mine = -1;
      if (avail >= n_need) {
        if (!active) mine = chunk_next + rank;
        chunk_next += n_need;
      } else {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)kChunk);
        base = __shfl_sync(FULL, base, 0);
        if (!active) mine = rank < avail ? chunk_next + rank : (long long)base + (rank - avail);
        chunk_next = (long long)base + (n_need - avail);
        chunk_end = (long long)base + kChunk;
        if ((long long)base >= P.total) exhausted = true;
      }
      if (!active && mine >= 0 && mine < P.total) {
        pidx = mine;
        const int sample = (int)(mine / P.npix);
        pixel = (uint32_t)(mine - (long long)sample * P.npix);
        bool skip = false;
        if constexpr (ADJ) {
          gpix = v3(A.d_image[3 * pixel] * P.inv_spp, A.d_image[3 * pixel + 1] * P.inv_spp,
                    A.d_image[3 * pixel + 2] * P.inv_spp);
          Ltot = v3(A.L_path[3 * pidx], A.L_path[3 * pidx + 1], A.L_path[3 * pidx + 2]);
          skip = gpix.x == 0.0f && gpix.y == 0.0f && gpix.z == 0.0f;  // no gradient flows through this pixel
          vgrad = false;
        }
        if (!skip) {
          rng.init(P.seed, pixel, (uint32_t)sample);
          rng.start(0, kPurposeCamera);
          const float jx = rng.next(), jy = rng.next();
          camera_ray(C, (int)(pixel % (uint32_t)C.width), (int)(pixel / (uint32_t)C.width), jx, jy, o, d);
          beta = v3(1.0f, 1.0f, 1.0f);
          L = v3(0.0f, 0.0f, 0.0f);
          prev_pdf = -1.0f;
          bounce = 0;
          mode = kFlight;
          events = 0;
          rng.start(0, kPurposeFlight);
          begin = true;
          waiting = false;
          active = true;
        }
      }
    }
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) {
      if (exhausted || chunk_next >= P.total) break;
      continue;
    }

    // ------------------------------------------------ deferred shading (and vertex gradients)
    const unsigned wait_mask = __ballot_sync(FULL, waiting || vgrad);
    if (wait_mask && (__popc(wait_mask) >= P.shade_min || wait_mask == act)) {
      if constexpr (ADJ) {
        if (vgrad) {
          vgrad = false;
          const ObjectDev& ob = S.obj[0];
          const V3 Ck = v3(pend.x * Tfin, pend.y * Tfin, pend.z * Tfin);
          const V3 after = Ltot - L - Ck;
          const V3 F = fetch_albedo(ob, o);
          const float Wnee = dot(gpix, Ck);
          const float Wph = cont ? dot(gpix, after) : 0.0f;
          const V3 ac = v3(F.x > 0.0f ? gpix.x * (Ck.x + (cont ? after.x : 0.0f)) / F.x : 0.0f,
                           F.y > 0.0f ? gpix.y * (Ck.y + (cont ? after.y : 0.0f)) / F.y : 0.0f,
                           F.z > 0.0f ? gpix.z * (Ck.z + (cont ? after.z : 0.0f)) / F.z : 0.0f);
          acc_l += adj_vertex(ob, o, d_in, d, d_next, Wnee, Wph, ac, A);
          L = L + Ck;
          if (cont) {
            mode = kFlight;
            d = d_next;
            beta = beta_next;
            prev_pdf = pdf_next;
            rng.start((uint32_t)bounce, kPurposeFlight);
            begin = true;
          } else {
            walk_ok = false;  // treated below as an escaped flight that adds nothing
            mode = kFlight;
            begin = false;
            beta = v3(0.0f, 0.0f, 0.0f);
          }
        }
      }
      if (waiting) {
        waiting = false;
        const V3 x = fma3(w.t, d, o);
        Field f;
        Local l;
        int k = 0;
        if (S.n_objs > 1) {
          k = choose_object(S, x, d, rng.next(), f, l);
        } else {
          f = fetch(S.obj[0], x);
          l = local_of(S.obj[0], f);
        }
        const V3 F = fetch_albedo(S.obj[k], x);
        o = x;
        cont = bounce + 1 < P.max_bounces;
        if (cont) {
          rng.start((uint32_t)bounce, kPurposePhase);
          const float u0 = rng.next(), u1 = rng.next(), u2 = rng.next();
          const PhaseSample ps = phase_sample_call(d, f, l.alpha, P.mix_R, u0, u1, u2);
          if (ps.ok) {
            d_next = ps.d2;
            beta_next = v3(beta.x * F.x * ps.w_over_F, beta.y * F.y * ps.w_over_F, beta.z * F.z * ps.w_over_F);
            pdf_next = ps.pdf;
          } else {
            cont = false;
          }
        } else {
          ++c_trunc;
        }
        rng.start((uint32_t)bounce, kPurposeNee);
        V3 wl, Le;
        if (!env) {
          wl = v3(S.light.dir[0], S.light.dir[1], S.light.dir[2]);
          Le = v3(S.light.radiance[0], S.light.radiance[1], S.light.radiance[2]);
        } else {
          const float z = 1.0f - 2.0f * rng.next();
          const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
          float sp, cp;
          sincospif(2.0f * rng.next(), &sp, &cp);
          wl = v3(r * cp, r * sp, z);
          Le = env_radiance(S.light, wl);
        }
        const PhaseEval pe = phase_eval_call(d, wl, f, l.alpha, P.mix_R);
        const float lw = env ? power_heuristic(kInv4Pi, pe.pdf) * (4.0f * kPi) : 1.0f;
        const float scale = pe.p_over_F * lw;
        pend = v3(beta.x * F.x * scale * Le.x, beta.y * F.y * scale * Le.y, beta.z * F.z * scale * Le.z);
        if constexpr (ADJ) {
          d_in = d;
          Tfin = scale > 0.0f ? A.T_path[(size_t)pidx * P.max_bounces + bounce] : 0.0f;
        } else {
          if (path_T && !(scale > 0.0f)) path_T[(size_t)pidx * P.max_bounces + bounce] = 0.0f;
        }
        ++bounce;
        if (scale > 0.0f) {
          mode = kShadow;
          d = wl;
          T = 1.0f;
          begin = true;
        } else if (ADJ) {
          d = wl;
          vgrad = true;  // the vertex's phase-sampling factor still has a gradient
        } else if (cont) {
          mode = kFlight;
          d = d_next;
          beta = beta_next;
          prev_pdf = pdf_next;
          rng.start((uint32_t)bounce, kPurposeFlight);
          begin = true;
        } else {
          // no shadow ray and no continuation: with walk_ok = false and beta = 0 the
          // step below treats the lane as an escaped flight that adds nothing
          mode = kFlight;
          walk_ok = false;
          begin = false;
          beta = v3(0.0f, 0.0f, 0.0f);
        }
      }
    }
    if (!active || waiting || vgrad) continue;

    // ------------------------------------------------ one tentative collision
    if (begin) {
      walk_ok = walk_begin(S.mg, o, d, INFINITY, w);
      begin = false;
    }
    bool hit = false;
    if (walk_ok) hit = walk_advance(S.mg, o, d, w, -__logf(rng.next()), c_cells);
    bool finish = false;
    if (hit) {
      ++events;
      const V3 x = fma3(w.t, d, o);
      float st;
      DSig ds;
      bool inobj = false;
      if constexpr (ADJ) {
        // extinction and its partials from one evaluation (the decision uses the same value)
        inobj = inside(S.obj[0], x);
        st = 0.0f;
        if (inobj) {
          const Field f = fetch(S.obj[0], x);
          ds = dsigma_t(S.obj[0], f, d);
          st = ds.st;
        }
      } else {
        st = sigma_t_at(S, x, d);
      }
      if (mode == kFlight) {
        const bool real = rng.next() * w.sbar < st;
        if constexpr (ADJ) {
          const float W = dot(gpix, Ltot - L);
          if (W != 0.0f && inobj)
            acc_l += adj_scatter_event(S.obj[0], x, ds, real ? W / st : -W / (w.sbar - st), A.d_mean, A.d_var);
        }
        if (real) {
          ++c_vert;
          waiting = true;  // real scattering vertex: shaded with the warp's other waiting lanes
        } else {
          ++c_null;
        }
      } else {
        ++c_shadow;
        if constexpr (ADJ) {
          const float Wn = dot(gpix, pend) * Tfin;
          if (Wn != 0.0f && inobj)
            acc_l += adj_scatter_event(S.obj[0], x, ds, -Wn / (w.sbar - st), A.d_mean, A.d_var);
        }
        if (!ratio_step(T, st, w.sbar, rng)) walk_ok = false;  // T = 0: the shadow ray ends here
      }
      if (events >= kMaxEventsPerPath) {
        ++c_abort;
        finish = true;
        waiting = false;
      }
    } else {
      if (mode == kFlight) {
        if (env) {
          const V3 Le = env_radiance(S.light, d);
          const float wm = prev_pdf < 0.0f ? 1.0f : power_heuristic(prev_pdf, kInv4Pi);
          L = v3(fmaf(beta.x * Le.x, wm, L.x), fmaf(beta.y * Le.y, wm, L.y), fmaf(beta.z * Le.z, wm, L.z));
        }
        finish = true;
      } else if (ADJ) {
        vgrad = true;  // shadow ray done: the vertex gradient is due
      } else {
        L = v3(fmaf(pend.x, T, L.x), fmaf(pend.y, T, L.y), fmaf(pend.z, T, L.z));
        if (path_T) path_T[(size_t)pidx * P.max_bounces + (bounce - 1)] = T;
        if (cont) {
          mode = kFlight;
          d = d_next;
          beta = beta_next;
          prev_pdf = pdf_next;
          rng.start((uint32_t)bounce, kPurposeFlight);
          begin = true;
        } else {
          finish = true;
        }
      }
    }
    if (finish) {
      if constexpr (!ADJ) {
        float* px = image + 3 * (size_t)pixel;
        atomicAdd(px + 0, L.x * P.inv_spp);
        atomicAdd(px + 1, L.y * P.inv_spp);
        atomicAdd(px + 2, L.z * P.inv_spp);
        if (sqsum) {
          float* q = sqsum + 3 * (size_t)pixel;
          atomicAdd(q + 0, L.x * L.x);
          atomicAdd(q + 1, L.y * L.y);
          atomicAdd(q + 2, L.z * L.z);
        }
        if (path_radiance) {
          float* pr = path_radiance + 3 * pidx;
          pr[0] = L.x;
          pr[1] = L.y;
          pr[2] = L.z;
        }
      } else {
        // the replay must reproduce the forward path; count any that does not
        const V3 e = L - Ltot;
        const float tol = 1e-3f * (fabsf(Ltot.x) + fabsf(Ltot.y) + fabsf(Ltot.z)) + 1e-6f;
        if (fabsf(e.x) + fabsf(e.y) + fabsf(e.z) > tol) ++c_abort;
      }
      ++c_paths;
      active = false;
    }
  }

  // ------------------------------------------------ counters: warp reduce, one atomic per warp
  if constexpr (ADJ) {
    for (int off = 16; off > 0; off >>= 1) acc_l += __shfl_down_sync(FULL, acc_l, off);
    if (lane == 0 && A.d_l && acc_l != 0.0f) atomicAdd(A.d_l, acc_l);
  }
  uint32_t vals[7] = {c_paths, c_vert, c_null, c_shadow, c_cells, c_trunc, c_abort};
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
    if (lane == 0 && v) atomicAdd(counters + i, v);
  }
}

}  // namespace gpss
