// scene.cu -- scene upload (grids -> library layout) and the majorant grid.
//
// Layout in HBM per object: (mean, variance) interleaved as float2 per node so
// one 8-byte gather serves both fields of a corner; albedo as separate planes
// (read only at real collisions).  The majorant grid is a separate float grid
// over the union of the object boxes whose cells are `brick` x the finest field
// cell; for one object it is aligned with the field cells.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gpss_internal.h"

namespace gpss {

// Interleaves (mean, variance) per node, validates both, and lowers *vmin_bits
// to the bits of the smallest variance (positive floats order like their bits).
__global__ void k_interleave(const float* __restrict__ mean, const float* __restrict__ var, float2* __restrict__ mv,
                             size_t n, int* flags, unsigned* vmin_bits) {
  float vmin = INFINITY;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float m = mean[i], v = var[i];
    if (!isfinite(m)) atomicOr(flags, 1);
    if (!(v > 0.0f) || !isfinite(v)) atomicOr(flags, 2);
    else vmin = fminf(vmin, v);
    mv[i] = make_float2(m, v);
  }
  for (int off = 16; off > 0; off >>= 1) vmin = fminf(vmin, __shfl_xor_sync(0xFFFFFFFFu, vmin, off));
  if ((threadIdx.x & 31) == 0 && vmin < INFINITY) atomicMin(vmin_bits, __float_as_uint(vmin));
}

__global__ void k_check_albedo(const float* __restrict__ a, size_t n, int* flags) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = a[i];
    if (!(v >= 0.0f && v <= 1.0f)) atomicOr(flags, 4);
  }
}

// Correlation-scale factors must be finite and > 0 (bit 8), tangent components finite (bit 16).
__global__ void k_check_kernel_grid(const float* __restrict__ a, size_t n, int positive, int* flags) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = a[i];
    if (positive ? !(v > 0.0f && isfinite(v)) : !isfinite(v)) atomicOr(flags, positive ? 8 : 16);
  }
}

// Upper bound of sigma_t over a majorant cell, over all directions (row A3):
//   mu >= mu_lo, var in [v_lo, v_hi], |grad mu| <= G_hi (each gradient component of
//   the trilinear interpolant is a convex combination of edge differences / h);
//   lambda is decreasing, so rho <= lambda(mu_lo/sigma_hi)/sigma_lo for mu_lo >= 0 and
//   lambda(mu_lo/sigma_lo)/sigma_lo otherwise;  sigma(d) = E[max(0,-d.g)] <= G_hi +
//   alpha_hi/(2 sqrt(pi)) (height-field NDFs: 1 + alpha_hi/(2 sqrt(pi)) or 1 + alpha_hi/2),
//   alpha_hi = sqrt2 sigma_hi max(1/l_t, 1/l_b, 1/l_n)/s_lo with s_lo the smallest
//   correlation-scale factor of the cell's nodes (interpolated s stays above it).
//   Objects' bounds add.  A 1e-3 relative margin covers FP32
//   rounding of the per-sample evaluation.
__global__ void k_majorant(SceneDev S, MajorantDev g, float* __restrict__ maj) {
  const long long ncell = (long long)g.dims[0] * g.dims[1] * g.dims[2];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(c % g.dims[0]);
    const int cj = (int)((c / g.dims[0]) % g.dims[1]);
    const int ck = (int)(c / ((long long)g.dims[0] * g.dims[1]));
    const int cidx[3] = {ci, cj, ck};
    float total = 0.0f;
    for (int k = 0; k < S.n_objs; ++k) {
      const ObjectDev& o = S.obj[k];
      int lo[3], hi[3];
      bool overlap = true;
      for (int a = 0; a < 3; ++a) {
        const float wlo = g.gmin[a] + cidx[a] * g.cell[a];
        const float whi = wlo + g.cell[a];
        if (whi < o.bmin[a] || wlo > o.bmax[a]) { overlap = false; break; }
        const float flo = (wlo - o.bmin[a]) * o.inv_h[a];
        const float fhi = (whi - o.bmin[a]) * o.inv_h[a];
        int i0 = (int)floorf(flo + 1e-3f);
        int i1 = (int)ceilf(fhi - 1e-3f) - 1;
        i0 = min(max(i0, 0), o.n[a] - 2);
        i1 = min(max(i1, i0), o.n[a] - 2);
        lo[a] = i0;
        hi[a] = i1 + 1;  // node range
      }
      if (!overlap) continue;
      float mu_lo = INFINITY, v_lo = INFINITY, v_hi = 0.0f, ex = 0.0f, ey = 0.0f, ez = 0.0f, c_lo = 1.0f;
      if (o.cscale) c_lo = INFINITY;
      const int sy = o.n[0], sz = o.n[0] * o.n[1];
      for (int kk = lo[2]; kk <= hi[2]; ++kk)
        for (int jj = lo[1]; jj <= hi[1]; ++jj)
          for (int ii = lo[0]; ii <= hi[0]; ++ii) {
            const int idx = ii + sy * jj + sz * kk;
            const float2 v = o.mv[idx];
            mu_lo = fminf(mu_lo, v.x);
            v_lo = fminf(v_lo, v.y);
            v_hi = fmaxf(v_hi, v.y);
            if (ii < hi[0]) ex = fmaxf(ex, fabsf(o.mv[idx + 1].x - v.x));
            if (jj < hi[1]) ey = fmaxf(ey, fabsf(o.mv[idx + sy].x - v.x));
            if (kk < hi[2]) ez = fmaxf(ez, fabsf(o.mv[idx + sz].x - v.x));
            if (o.cscale) c_lo = fminf(c_lo, o.cscale[idx]);
          }
      const float gx = ex * o.inv_h[0], gy = ey * o.inv_h[1], gz = ez * o.inv_h[2];
      const float G_hi = sqrtf(gx * gx + gy * gy + gz * gz);
      const float s_lo = sqrtf(v_lo), s_hi = sqrtf(v_hi);
      const float u = mu_lo >= 0.0f ? mu_lo / s_hi : mu_lo / s_lo;
      const float rho_ub = inv_mills(u) / s_lo;
      // height-field macrofacets: sigma(d) <= max(0, -d.n) + alpha/(2 sqrt pi) (Beckmann),
      // <= max(0, -d.n) + alpha/2 (GGX), with |n| = 1
      const float a_hi = s_hi * o.alpha_scale * o.amax / c_lo;
      const float area_ub = o.ndf == kNdfGpss ? G_hi + a_hi * (0.5f * kInvSqrtPi)
                          : 1.0f + a_hi * (o.ndf == kNdfGgx ? 0.5f : 0.5f * kInvSqrtPi);
      total += rho_ub * area_ub;
    }
    maj[c] = total * 1.001f;
  }
}

// Skip grid (see MajorantDev): running max filters over cubes of radius
// 1, 2, 4, ... cells, built separably; the radius-2r max along an axis is the max
// of the radius-r maxima at offsets -r and +r (indices clamped at the grid edge,
// so a cube is clipped to the grid).
__global__ void k_max_axis(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, int axis,
                           int off, int with_center) {
  const long long n = (long long)nx * ny * nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const int dim = axis == 0 ? nx : axis == 1 ? ny : nz;
    const int p = axis == 0 ? i : axis == 1 ? j : k;
    const long long stride = axis == 0 ? 1 : axis == 1 ? nx : (long long)nx * ny;
    const int lo = max(p - off, 0), hi = min(p + off, dim - 1);
    float m = fmaxf(in[c + (lo - p) * stride], in[c + (hi - p) * stride]);
    if (with_center) m = fmaxf(m, in[c]);
    out[c] = m;
  }
}

__global__ void k_skip_init(const float* __restrict__ maj, float2* __restrict__ skip, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    skip[c] = make_float2(maj[c], 0.0f);
}

__global__ void k_skip_select(const float* __restrict__ mr, float2* __restrict__ skip, long long n, int r, float limit) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const float m = mr[c];
    if (m * (float)r <= limit && skip[c].y == (float)(r >> 1)) skip[c] = make_float2(m, (float)r);
  }
}

static int blocks_for(size_t n, int block) {
  size_t b = (n + block - 1) / block;
  return (int)(b < 65536 ? (b ? b : 1) : 65536);
}

gpss_status scene_upload(gpss_scene s, const gpss_object_desc* objs, int n, cudaStream_t st) {
  // flags[0]: validation bits; flags[1 + k]: bits of object k's smallest variance
  // (0x7f7f7f7f = 3.4e38 before the minimum)
  cudaError_t e = cudaMemsetAsync(s->flags, 0x7f, kSceneFlagWords * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->flags, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset flags");
  for (int k = 0; k < n; ++k) {
    ObjectHost& o = s->obj[k];
    const size_t nodes = o.nodes;
    e = cudaMemcpyAsync(s->tmp_planes, objs[k].mean, nodes * sizeof(float), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy mean");
    e = cudaMemcpyAsync(s->tmp_planes + nodes, objs[k].variance, nodes * sizeof(float), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy variance");
    k_interleave<<<blocks_for(nodes, 256), 256, 0, st>>>(s->tmp_planes, s->tmp_planes + nodes, o.mv, nodes, s->flags,
                                                         (unsigned*)(s->flags + 1 + k));
    e = cudaMemcpyAsync(o.albedo, objs[k].albedo, nodes * o.channels * sizeof(float), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy albedo");
    k_check_albedo<<<blocks_for(nodes * o.channels, 256), 256, 0, st>>>(o.albedo, nodes * o.channels, s->flags);
    if (o.cscale) {
      e = cudaMemcpyAsync(o.cscale, objs[k].correlation_scale, nodes * sizeof(float), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy correlation scale");
      k_check_kernel_grid<<<blocks_for(nodes, 256), 256, 0, st>>>(o.cscale, nodes, 1, s->flags);
    }
    if (o.tangent) {
      e = cudaMemcpyAsync(o.tangent, objs[k].tangent, 3 * nodes * sizeof(float), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy tangent field");
      k_check_kernel_grid<<<blocks_for(3 * nodes, 256), 256, 0, st>>>(o.tangent, 3 * nodes, 0, s->flags);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "upload kernels");
  int fl[kSceneFlagWords];
  e = cudaMemcpyAsync(fl, s->flags, sizeof(fl), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "read flags");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "upload");
  const int flags = fl[0];
  if (flags & 1) { set_error("mean contains non-finite values"); return GPSS_ERR_INVALID_ARG; }
  if (flags & 2) { set_error("variance must be finite and > 0"); return GPSS_ERR_INVALID_ARG; }
  if (flags & 4) { set_error("albedo must lie in [0,1]"); return GPSS_ERR_INVALID_ARG; }
  if (flags & 8) { set_error("correlation_scale must be finite and > 0"); return GPSS_ERR_INVALID_ARG; }
  if (flags & 16) { set_error("tangent must be finite"); return GPSS_ERR_INVALID_ARG; }
  // thin: some object's smallest standard deviation lies below its grid spacing,
  // where the grid majorant of the cells at its shell is loose
  s->thin = false;
  for (int k = 0; k < n; ++k) {
    float vmin;
    std::memcpy(&vmin, &fl[1 + k], sizeof(float));
    ObjectHost& o = s->obj[k];
    o.sigma_min = std::sqrt(vmin);
    float h = INFINITY;
    for (int a = 0; a < 3; ++a) h = std::fmin(h, (o.bmax[a] - o.bmin[a]) / (float)(o.n[a] - 1));
    o.thin = h > o.sigma_min;
    if (o.thin) s->thin = true;
  }
  return GPSS_OK;
}

// Skip grid of one majorant grid g (majorants maj, result skip) with the scene's levels
// and kappa; s->skip_tmp holds 3 x the cells of the largest grid.
static void build_skip_grid(gpss_scene s, const MajorantDev& g, const float* maj, float2* skip, cudaStream_t st) {
  const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  const long long n = (long long)nx * ny * nz;
  const int nb = blocks_for((size_t)n, 256);
  k_skip_init<<<nb, 256, 0, st>>>(maj, skip, n);
  if (s->skip_levels > 0) {
    float* P = s->skip_tmp;
    float* Q = P + n;
    float* R = Q + n;
    const float hmin = fminf(fminf(g.cell[0], g.cell[1]), g.cell[2]);
    const float limit = s->kappa / hmin;  // M_r * r * h_min <= kappa
    for (int lev = 0; lev < s->skip_levels; ++lev) {
      const int r = 1 << lev;
      const int off = lev == 0 ? 1 : r >> 1;
      const float* src = lev == 0 ? maj : P;
      k_max_axis<<<nb, 256, 0, st>>>(src, Q, nx, ny, nz, 0, off, lev == 0);
      k_max_axis<<<nb, 256, 0, st>>>(Q, R, nx, ny, nz, 1, off, lev == 0);
      k_max_axis<<<nb, 256, 0, st>>>(R, P, nx, ny, nz, 2, off, lev == 0);
      k_skip_select<<<nb, 256, 0, st>>>(P, skip, n, r, limit);
    }
  }
}

gpss_status build_skip(gpss_scene s, cudaStream_t st) {
  build_skip_grid(s, s->mg, s->maj, s->skip, st);
  if (s->n_objs > 1)
    for (int k = 0; k < s->n_objs; ++k) build_skip_grid(s, s->obj[k].og, s->obj[k].omaj, s->obj[k].oskip, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "skip grid kernels");
  return GPSS_OK;
}

SceneDev scene_dev(const gpss_scene_s* s) {
  SceneDev d;
  memset(&d, 0, sizeof(d));
  d.n_objs = s->n_objs;
  for (int k = 0; k < s->n_objs; ++k) {
    const ObjectHost& h = s->obj[k];
    ObjectDev& o = d.obj[k];
    for (int a = 0; a < 3; ++a) {
      o.bmin[a] = h.bmin[a];
      o.bmax[a] = h.bmax[a];
      o.n[a] = h.n[a];
      o.inv_h[a] = (float)(h.n[a] - 1) / (h.bmax[a] - h.bmin[a]);
    }
    o.channels = h.channels;
    o.ndf = h.ndf;
    o.alpha_scale = kSqrt2 / h.length_scale;
    o.mv = h.mv;
    o.albedo = h.albedo;
    o.kb = h.length_scale / h.length_scale_b;
    o.kn = h.length_scale / h.length_scale_n;
    o.amax = fmaxf(1.0f, fmaxf(o.kb, o.kn));
    o.cscale = h.cscale;
    o.tangent = h.tangent;
    o.general = (o.kb != 1.0f || o.kn != 1.0f || o.cscale || o.tangent) ? 1 : 0;
  }
  d.mg = s->mg;
  d.mg.maj = s->maj;
  d.mg.skip = s->skip;
  d.mg.hot = (s->n_objs == 1 && s->thin) ? s->hot : 0.0f;
  d.mg.lin = s->lin_flight ? 1 : 0;
  d.split = (s->n_objs > 1 && s->object_grids) ? 1 : 0;
  if (s->n_objs > 1)
    for (int k = 0; k < s->n_objs; ++k) {
      d.og[k] = s->obj[k].og;
      d.og[k].hot = s->obj[k].thin ? s->hot : 0.0f;
      d.og[k].lin = s->lin_flight ? 1 : 0;
    }
  d.light = s->light;
  return d;
}

gpss_status build_majorant(gpss_scene s, cudaStream_t st) {
  const SceneDev S = scene_dev(s);
  const long long ncell = (long long)s->mg.dims[0] * s->mg.dims[1] * s->mg.dims[2];
  k_majorant<<<blocks_for((size_t)ncell, 128), 128, 0, st>>>(S, s->mg, s->maj);
  if (s->n_objs > 1)
    for (int k = 0; k < s->n_objs; ++k) {
      // object k alone over its own grid
      SceneDev Sk = S;
      Sk.n_objs = 1;
      Sk.obj[0] = S.obj[k];
      const MajorantDev& g = s->obj[k].og;
      const long long oc = (long long)g.dims[0] * g.dims[1] * g.dims[2];
      k_majorant<<<blocks_for((size_t)oc, 128), 128, 0, st>>>(Sk, g, s->obj[k].omaj);
    }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "majorant kernel");
  return build_skip(s, st);
}

}  // namespace gpss
