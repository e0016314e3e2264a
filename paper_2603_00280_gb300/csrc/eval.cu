// eval.cu -- per-query evaluators of the medium (parity checks against the
// oracle).  They call the same device functions as the renderer.
#include "gpss_internal.h"

namespace gpss {

__device__ __forceinline__ V3 ld3(const float* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ void st3(float* p, int i, V3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}

__global__ void k_eval_sigma_t(const SceneDev S, int n, const float* pos, const float* dir, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = scene_sigma_t(S, ld3(pos, i), ld3(dir, i));
}

__global__ void k_eval_local_majorant(const SceneDev S, int n, const float* org, const float* dir, const float* t0,
                                      const float* tmax, float* t_end, float* sbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 pc = local_majorant(S.obj[0], ld3(org, i), ld3(dir, i), t0[i], tmax[i]);
  t_end[i] = pc.x;
  sbar[i] = pc.y;
}

__global__ void k_eval_local_piece(const SceneDev S, int n, const float* org, const float* dir, const float* t0,
                                   const float* tmax, const float* tau, float* t_end, int* lin, float* depth,
                                   float* t_hit, float* sbar_hit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const LocalPiece p = local_piece(S.obj[0], ld3(org, i), ld3(dir, i), t0[i], tmax[i], true, INFINITY);
  t_end[i] = p.t_end;
  lin[i] = p.lin;
  if (!(p.t_end > t0[i])) {
    depth[i] = 0.0f;
    t_hit[i] = p.t_end;
    sbar_hit[i] = 0.0f;
    return;
  }
  const float D = p.lin ? lin_depth(p, t0[i], p.t_end) : p.sbar * (p.t_end - t0[i]);
  depth[i] = D;
  float sb = p.sbar;
  float th = p.t_end;
  if (tau[i] < D) {
    if (p.lin) {
      const float2 h = lin_collision(p, t0[i], p.t_end, tau[i]);
      th = h.x;
      sb = h.y;
    } else {
      th = t0[i] + tau[i] / p.sbar;
    }
  } else if (p.lin) {
    sb = lin_collision(p, t0[i], p.t_end, D).y;  // the majorant at the piece's end
  }
  t_hit[i] = th;
  sbar_hit[i] = sb;
}

__global__ void k_eval_phase(const SceneDev S, int k, int n, const float* pos, const float* din, const float* dout,
                             float R, float* p3, float* pdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 x = ld3(pos, i);
  const ObjectDev& o = S.obj[k];
  if (!inside(o, x)) {
    st3(p3, i, v3(0, 0, 0));
    pdf[i] = 0.0f;
    return;
  }
  const Field f = fetch(o, x);
  const Local l = local_of(o, f);
  float pF, pd;
  phase_eval(ld3(din, i), ld3(dout, i), f, l.alpha, R, pF, pd);
  const V3 F = fetch_albedo(o, x);
  st3(p3, i, pF * F);
  pdf[i] = pd;
}

__global__ void k_sample_phase_vndf(const SceneDev S, int k, int n, const float* pos, const float* din,
                                    const float* u3, float* dout, float* w3, float* pdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 x = ld3(pos, i);
  const ObjectDev& o = S.obj[k];
  V3 d2 = v3(0, 0, 0);
  float wF = 0.0f, pd = 0.0f;
  V3 F = v3(0, 0, 0);
  if (inside(o, x)) {
    const Field f = fetch(o, x);
    const float alpha = sqrtf(f.var) * f.as;
    const V3 d = ld3(din, i);
    const V3 u = ld3(u3, i);
    if (!phase_sample_vndf(projected_area(d, f, alpha), d, f, alpha, u.x, u.y, u.z, d2, wF, pd)) wF = 0.0f;
    F = fetch_albedo(o, x);
  }
  st3(dout, i, d2);
  st3(w3, i, wF * F);
  pdf[i] = pd;
}

__global__ void k_sample_phase(const SceneDev S, int k, int n, const float* pos, const float* din, const float* u3,
                               float R, float* dout, float* w3, float* pdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 x = ld3(pos, i);
  const ObjectDev& o = S.obj[k];
  V3 d2 = v3(0, 0, 0);
  float wF = 0.0f, pd = 0.0f;
  V3 F = v3(0, 0, 0);
  if (inside(o, x)) {
    const Field f = fetch(o, x);
    const Local l = local_of(o, f);
    const V3 u = ld3(u3, i);
    if (!phase_sample(ld3(din, i), f, l.alpha, R, u.x, u.y, u.z, d2, wF, pd)) wF = 0.0f;
    F = fetch_albedo(o, x);
  }
  st3(dout, i, d2);
  st3(w3, i, wF * F);
  pdf[i] = pd;
}

__global__ void k_eval_ndf(int n, const float* m3, float G, float ax, float ay, float az, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = ndf_local(ld3(m3, i), G, ax, ay, az);
}

__global__ void k_eval_proj(int n, const float* w3, float G, float ax, float ay, float az, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = projected_area_local(ld3(w3, i), G, ax, ay, az);
}

// Deterministic transmittance: the ray is split at every face of every object's
// field cells; each cell segment is further split into pieces no longer than
// half the density's feature length sigma_min/|grad mu|_max of the cell, and each
// piece is integrated with 8-point Gauss-Legendre.  Accumulated in FP64.
__constant__ float c_gl8_x[8] = {-0.9602898564975363f, -0.7966664774136267f, -0.5255324099163290f,
                                 -0.1834346424956498f, 0.1834346424956498f,  0.5255324099163290f,
                                 0.7966664774136267f,  0.9602898564975363f};
__constant__ float c_gl8_w[8] = {0.1012285362903763f, 0.2223810344533745f, 0.3137066458778873f,
                                 0.3626837833783620f, 0.3626837833783620f, 0.3137066458778873f,
                                 0.2223810344533745f, 0.1012285362903763f};

__device__ double object_optical_depth(const ObjectDev& ob, V3 o, V3 d, float tmax) {
  // clip to the object box
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  float t0 = 0.0f, t1 = tmax;
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0f) {
      if (oo[a] < ob.bmin[a] || oo[a] > ob.bmax[a]) return 0.0;
    } else {
      float ta = (ob.bmin[a] - oo[a]) / dd[a], tb = (ob.bmax[a] - oo[a]) / dd[a];
      if (ta > tb) { const float tmp = ta; ta = tb; tb = tmp; }
      t0 = fmaxf(t0, ta);
      t1 = fminf(t1, tb);
    }
  }
  if (!(t1 > t0)) return 0.0;
  // walk field cells
  float h[3], tm[3], td[3];
  int idx[3], st[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = 1.0f / ob.inv_h[a];
    const float p = fmaf(t0, dd[a], oo[a]);
    int i = (int)floorf((p - ob.bmin[a]) * ob.inv_h[a]);
    i = min(max(i, 0), ob.n[a] - 2);
    idx[a] = i;
    if (dd[a] > 0.0f) {
      st[a] = 1;
      tm[a] = (ob.bmin[a] + (i + 1) * h[a] - oo[a]) / dd[a];
      td[a] = h[a] / dd[a];
    } else if (dd[a] < 0.0f) {
      st[a] = -1;
      tm[a] = (ob.bmin[a] + i * h[a] - oo[a]) / dd[a];
      td[a] = -h[a] / dd[a];
    } else {
      st[a] = 0;
      tm[a] = INFINITY;
      td[a] = INFINITY;
    }
  }
  double tau = 0.0;
  float t = t0;
  for (int guard = 0; guard < 1 << 20; ++guard) {
    const float tn = fminf(fminf(tm[0], tm[1]), fminf(tm[2], t1));
    if (tn > t) {
      // feature length of this cell
      const int b = idx[0] + ob.n[0] * (idx[1] + ob.n[1] * idx[2]);
      const int sy = ob.n[0], sz = ob.n[0] * ob.n[1];
      float vmin = INFINITY, ex = 0.0f, ey = 0.0f, ez = 0.0f;
      for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const int j = b + cx + sy * cy + sz * cz;
        const float2 v = ob.mv[j];
        vmin = fminf(vmin, v.y);
        if (!cx) ex = fmaxf(ex, fabsf(ob.mv[j + 1].x - v.x));
        if (!cy) ey = fmaxf(ey, fabsf(ob.mv[j + sy].x - v.x));
        if (!cz) ez = fmaxf(ez, fabsf(ob.mv[j + sz].x - v.x));
      }
      const float gx = ex * ob.inv_h[0], gy = ey * ob.inv_h[1], gz = ez * ob.inv_h[2];
      const float G = sqrtf(gx * gx + gy * gy + gz * gz);
      const float feat = G > 0.0f ? 0.5f * sqrtf(vmin) / G : INFINITY;
      int K = 1;
      if (isfinite(feat)) K = min(max((int)ceilf((tn - t) / feat), 1), 4096);
      const float hseg = (tn - t) / (float)K;
      for (int s = 0; s < K; ++s) {
        const float a0 = t + s * hseg;
        double acc = 0.0;
        for (int q = 0; q < 8; ++q) {
          const float tq = a0 + 0.5f * hseg * (1.0f + c_gl8_x[q]);
          const V3 x = fma3(tq, d, o);
          Field f;
          Local l;
          acc += (double)c_gl8_w[q] * (double)sigma_t_object(ob, x, d, f, l);
        }
        tau += acc * 0.5 * (double)hseg;
      }
    }
    t = tn;
    if (tn >= t1) break;
    int a = (tm[0] <= tm[1] && tm[0] <= tm[2]) ? 0 : (tm[1] <= tm[2] ? 1 : 2);
    idx[a] += st[a];
    tm[a] += td[a];
    if (idx[a] < 0 || idx[a] > ob.n[a] - 2) break;
  }
  return tau;
}

__global__ void k_eval_tr(const SceneDev S, int n, const float* org, const float* dir, const float* tmax, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 o = ld3(org, i), d = ld3(dir, i);
  double tau = 0.0;
  for (int k = 0; k < S.n_objs; ++k) tau += object_optical_depth(S.obj[k], o, d, tmax[i]);
  out[i] = (float)exp(-tau);
}

// Ratio tracking with the renderer's majorant traversal and extinction.
__global__ void k_estimate_tr(const __grid_constant__ SceneDev S, int n, const float* org, const float* dir, const float* tmax,
                              int samples, uint64_t seed, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 o = ld3(org, i), d = ld3(dir, i);
  double acc = 0.0;
  uint32_t cells = 0;
  for (int s = 0; s < samples; ++s) {
    Rng rng;
    rng.init(seed, (uint32_t)i, (uint32_t)s);
    rng.start(0, kPurposeNee);
    Walk w;
    int gid;
    float T = 1.0f;
    if (trace_begin<true>(S, S.og, o, d, tmax[i], w, gid)) {
      for (float tau = -__logf(rng.next());
           trace_advance<true, true, true>(S, S.og, o, d, tmax[i], w, gid, tau, cells) == kWalkHit;
           tau = -__logf(rng.next())) {
        const V3 x = fma3(w.t, d, o);
        const float st = scene_sigma_t(S, x, d);
        if (!ratio_step(T, st, w.sbar, rng)) break;
      }
    }
    acc += T;
  }
  out[i] = (float)(acc / samples);
}

// Delta-tracking free-flight distance (the renderer's flight loop without scattering).
__global__ void k_free_flight(const __grid_constant__ SceneDev S, int n, const float* org, const float* dir, int samples,
                              uint64_t seed, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V3 o = ld3(org, i), d = ld3(dir, i);
  uint32_t cells = 0;
  for (int s = 0; s < samples; ++s) {
    Rng rng;
    rng.init(seed, (uint32_t)i, (uint32_t)s);
    rng.start(0, kPurposeFlight);
    Walk w;
    int gid;
    float t_hit = INFINITY;
    if (trace_begin<true>(S, S.og, o, d, INFINITY, w, gid)) {
      for (float tau = -__logf(rng.next());
           trace_advance<true, true, true>(S, S.og, o, d, INFINITY, w, gid, tau, cells) == kWalkHit;
           tau = -__logf(rng.next())) {
        const V3 x = fma3(w.t, d, o);
        const float st = scene_sigma_t(S, x, d);
        if (rng.next() * w.sbar < st) {
          t_hit = w.t;
          break;
        }
      }
    }
    out[(size_t)i * samples + s] = t_hit;
  }
}

__global__ void k_philox(int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox4x32_10(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, key[2 * i], key[2 * i + 1]);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

}  // namespace gpss

// ------------------------------------------------------------------ C-ABI wrappers
using namespace gpss;

static inline int nb(int n) { return (n + 127) / 128; }

#define CHECK_N(n)                                       \
  if ((n) < 0 || (n) > (1 << 28)) {                      \
    set_error("n must be in [0, 2^28]");                 \
    return GPSS_ERR_INVALID_ARG;                         \
  }                                                      \
  if ((n) == 0) return GPSS_OK;

extern "C" gpss_status gpss_eval_sigma_t(gpss_scene s, int n, const float* pos3, const float* dir3, float* out,
                                         gpss_stream stream) {
  if (!s || !pos3 || !dir3 || !out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_eval_sigma_t<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, pos3, dir3, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_sigma_t");
}

extern "C" gpss_status gpss_eval_local_piece(gpss_scene s, int n, const float* org3, const float* dir3,
                                             const float* t0, const float* t_max, const float* tau, float* t_end,
                                             int* lin, float* depth, float* t_hit, float* sbar_hit,
                                             gpss_stream stream) {
  if (!s || !org3 || !dir3 || !t0 || !t_max || !tau || !t_end || !lin || !depth || !t_hit || !sbar_hit) {
    set_error("null argument");
    return GPSS_ERR_INVALID_ARG;
  }
  CHECK_N(n);
  k_eval_local_piece<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, org3, dir3, t0, t_max, tau, t_end,
                                                             lin, depth, t_hit, sbar_hit);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_local_piece");
}

extern "C" gpss_status gpss_eval_local_majorant(gpss_scene s, int n, const float* org3, const float* dir3,
                                                const float* t0, const float* t_max, float* t_end, float* sbar,
                                                gpss_stream stream) {
  if (!s || !org3 || !dir3 || !t0 || !t_max || !t_end || !sbar) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_eval_local_majorant<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, org3, dir3, t0, t_max, t_end, sbar);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_local_majorant");
}

extern "C" gpss_status gpss_eval_phase(gpss_scene s, int object, int n, const float* pos3, const float* d_in3,
                                       const float* d_out3, float mix_R, float* p3_out, float* pdf_out,
                                       gpss_stream stream) {
  if (!s || !pos3 || !d_in3 || !d_out3 || !p3_out || !pdf_out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (object < 0 || object >= s->n_objs) { set_error("object index out of range"); return GPSS_ERR_INVALID_ARG; }
  if (!(mix_R > 0.0f && mix_R < 1.0f)) { set_error("mix_R must lie in (0,1)"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_eval_phase<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), object, n, pos3, d_in3, d_out3, mix_R, p3_out,
                                                        pdf_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_phase");
}

extern "C" gpss_status gpss_sample_phase(gpss_scene s, int object, int n, const float* pos3, const float* d_in3,
                                         const float* u3, float mix_R, float* d_out3, float* w3_out, float* pdf_out,
                                         gpss_stream stream) {
  if (!s || !pos3 || !d_in3 || !u3 || !d_out3 || !w3_out || !pdf_out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (object < 0 || object >= s->n_objs) { set_error("object index out of range"); return GPSS_ERR_INVALID_ARG; }
  if (!(mix_R > 0.0f && mix_R < 1.0f)) { set_error("mix_R must lie in (0,1)"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_sample_phase<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), object, n, pos3, d_in3, u3, mix_R, d_out3,
                                                          w3_out, pdf_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "sample_phase");
}

extern "C" gpss_status gpss_sample_phase_vndf(gpss_scene s, int object, int n, const float* pos3,
                                              const float* d_in3, const float* u3, float* d_out3, float* w3_out,
                                              float* pdf_out, gpss_stream stream) {
  if (!s || !pos3 || !d_in3 || !u3 || !d_out3 || !w3_out || !pdf_out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (object < 0 || object >= s->n_objs) { set_error("object index out of range"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_sample_phase_vndf<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), object, n, pos3, d_in3, u3, d_out3,
                                                               w3_out, pdf_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "sample_phase_vndf");
}

static bool positive_finite(float v) { return v > 0.0f && v < 3.0e38f; }

extern "C" gpss_status gpss_eval_ndf(int n, const float* m3, float G, float ax, float ay, float az, float* out,
                                     gpss_stream stream) {
  if (!m3 || !out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (!(G >= 0.0f) || !positive_finite(ax) || !positive_finite(ay) || !positive_finite(az)) {
    set_error("G must be >= 0 and roughness > 0");
    return GPSS_ERR_INVALID_ARG;
  }
  CHECK_N(n);
  k_eval_ndf<<<nb(n), 128, 0, (cudaStream_t)stream>>>(n, m3, G, ax, ay, az, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_ndf");
}

extern "C" gpss_status gpss_eval_projected_area(int n, const float* w3, float G, float ax, float ay, float az,
                                                float* out, gpss_stream stream) {
  if (!w3 || !out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (!(G >= 0.0f) || !positive_finite(ax) || !positive_finite(ay) || !positive_finite(az)) {
    set_error("G must be >= 0 and roughness > 0");
    return GPSS_ERR_INVALID_ARG;
  }
  CHECK_N(n);
  k_eval_proj<<<nb(n), 128, 0, (cudaStream_t)stream>>>(n, w3, G, ax, ay, az, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_projected_area");
}

extern "C" gpss_status gpss_eval_transmittance(gpss_scene s, int n, const float* org3, const float* dir3,
                                               const float* tmax, float* out, gpss_stream stream) {
  if (!s || !org3 || !dir3 || !tmax || !out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_eval_tr<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, org3, dir3, tmax, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "eval_transmittance");
}

extern "C" gpss_status gpss_estimate_transmittance(gpss_scene s, int n, const float* org3, const float* dir3,
                                                   const float* tmax, int samples, uint64_t seed, float* mean_out,
                                                   gpss_stream stream) {
  if (!s || !org3 || !dir3 || !tmax || !mean_out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (samples < 1) { set_error("samples must be >= 1"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_estimate_tr<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, org3, dir3, tmax, samples, seed, mean_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "estimate_transmittance");
}

extern "C" gpss_status gpss_sample_free_flight(gpss_scene s, int n, const float* org3, const float* dir3, int samples,
                                               uint64_t seed, float* out, gpss_stream stream) {
  if (!s || !org3 || !dir3 || !out) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  if (samples < 1) { set_error("samples must be >= 1"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_free_flight<<<nb(n), 128, 0, (cudaStream_t)stream>>>(scene_dev(s), n, org3, dir3, samples, seed, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "sample_free_flight");
}

extern "C" gpss_status gpss_philox4x32_10(int n, const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4,
                                          gpss_stream stream) {
  if (!ctr4 || !key2 || !out4) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  CHECK_N(n);
  k_philox<<<nb(n), 128, 0, (cudaStream_t)stream>>>(n, ctr4, key2, out4);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPSS_OK : cuda_fail(e, "philox");
}
