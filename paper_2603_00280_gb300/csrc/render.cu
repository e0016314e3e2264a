// render.cu -- forward path tracing of the GPSS medium (persistent kernel).
//
// Integrator (Sec. 5 of the paper: null scattering on the classic exponential
// medium of Sec. 4):
//   - free flight by delta tracking against the majorant grid: tentative
//     collisions at optical depth -ln(u) of the majorant, accepted as real with
//     probability sigma_t / majorant;
//   - at each real vertex, next-event estimation with a ratio-tracking shadow ray
//     (T *= 1 - sigma_t/majorant at each tentative collision, Russian roulette
//     below T = 0.1), MIS (power heuristic) against phase sampling for
//     environment lights;
//   - phase sampling with the mixture of Sec. 4.2.2; at most max_bounces real
//     vertices, no continuation after the last, no Russian roulette on paths.
//
// Execution model: one persistent thread per resident lane.  Each iteration of
// the main loop advances every active lane by ONE tentative collision of its
// current ray (the free-flight ray or the shadow ray), so all lanes of a warp run
// the same traversal + extinction code together.  A lane whose flight ends in a
// real collision waits; the warp shades its waiting lanes together once at least
// `shade_min` of them wait (or no lane can step), so the long shading code runs
// with many lanes active.  Shading functions and the Philox block are out of
// line, keeping the traversal loop small in the instruction cache.  A lane whose
// path has finished takes the next (sample, pixel) index from a warp-private
// chunk of the global work cursor (one atomic per chunk; ranks from
// __ballot_sync/__popc).  Path state lives in registers.  Path index =
// sample * npix + pixel, so a chunk covers adjacent pixels at the same sample.
#include "gpss_internal.h"

namespace gpss {

constexpr int kRenderBlock = 128;
constexpr int kChunk = 256;
constexpr uint32_t kMaxEventsPerPath = 1u << 24;  // runaway guard (counted as aborted)

struct RenderArgs {
  int spp, max_bounces;
  uint64_t seed;
  float mix_R;
  int npix;
  long long total;
  float inv_spp;
  int shade_min;
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

__global__ void __launch_bounds__(kRenderBlock) k_render(const SceneDev S, const CameraDev C, const RenderArgs P,
                                                        float* __restrict__ image, float* __restrict__ sqsum,
                                                        float* __restrict__ path_radiance,
                                                        unsigned long long* __restrict__ counters) {
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
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) {
      if (exhausted || chunk_next >= P.total) break;
      continue;
    }

    // ------------------------------------------------ deferred shading of real vertices
    const unsigned wait_mask = __ballot_sync(FULL, waiting);
    if (wait_mask && (__popc(wait_mask) >= P.shade_min || wait_mask == act) && waiting) {
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
      float lpdf_w;  // MIS weight / light pdf (directional: 1)
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
      if (!env) {
        lpdf_w = 1.0f;
      } else {
        lpdf_w = power_heuristic(kInv4Pi, pe.pdf) * (4.0f * kPi);
      }
      const float scale = pe.p_over_F * lpdf_w;
      pend = v3(beta.x * F.x * scale * Le.x, beta.y * F.y * scale * Le.y, beta.z * F.z * scale * Le.z);
      ++bounce;
      if (scale > 0.0f) {
        mode = kShadow;
        d = wl;
        T = 1.0f;
        begin = true;
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
        d = v3(0.0f, 0.0f, 0.0f);
        beta = v3(0.0f, 0.0f, 0.0f);
      }
    }
    if (!active || waiting) continue;

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
      const float st = sigma_t_at(S, fma3(w.t, d, o), d);
      if (mode == kFlight) {
        if (rng.next() * w.sbar < st) {
          ++c_vert;
          waiting = true;      // real scattering vertex: shaded with the warp's other waiting lanes
        } else {
          ++c_null;
        }
      } else {
        ++c_shadow;
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
      } else {
        L = v3(fmaf(pend.x, T, L.x), fmaf(pend.y, T, L.y), fmaf(pend.z, T, L.z));
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
      ++c_paths;
      active = false;
    }
  }

  // ------------------------------------------------ counters: warp reduce, one atomic per warp
  uint32_t vals[7] = {c_paths, c_vert, c_null, c_shadow, c_cells, c_trunc, c_abort};
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
    if (lane == 0 && v) atomicAdd(counters + i, v);
  }
}

int render_block_size() { return kRenderBlock; }

int render_grid_size(int device, int block) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render, block, 0);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

cudaError_t launch_render(const SceneDev& S, const CameraDev& C, const gpss_render_opts& o, float* image,
                          float* sqsum, float* path_radiance, unsigned long long* counters, int grid, int block,
                          int shade_min, cudaStream_t st) {
  RenderArgs P;
  P.spp = o.spp;
  P.max_bounces = o.max_bounces;
  P.seed = o.seed;
  P.mix_R = o.mix_R;
  P.npix = C.width * C.height;
  P.total = (long long)P.npix * o.spp;
  P.inv_spp = 1.0f / (float)o.spp;
  P.shade_min = shade_min;
  k_render<<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters);
  return cudaGetLastError();
}

}  // namespace gpss
