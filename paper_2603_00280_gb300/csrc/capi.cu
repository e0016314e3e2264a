// capi.cu -- C-ABI: scene lifecycle, forward render, errors.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "gpss_internal.h"

namespace gpss {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void fill_stats(gpss_stats* st, const unsigned long long* c, float ms) {
  st->paths = c[kCntPaths];
  st->vertices = c[kCntVertices];
  st->null_collisions = c[kCntNull];
  st->shadow_steps = c[kCntShadow];
  st->majorant_cells = c[kCntCells];
  st->truncated = c[kCntTruncated];
  st->aborted = c[kCntAborted];
  st->max_path_events = c[kCntMaxEvents];
  st->ms = ms;
  st->nonfinite = c[kCntNonFinite];
}

gpss_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return GPSS_ERR_OOM;
  return GPSS_ERR_CUDA;
}

static bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool camera_dev(const gpss_camera* c, CameraDev* out) {
  if (!c || c->width < 1 || c->height < 1 || c->width > 65536 || c->height > 65536) {
    set_error("camera size must be in [1, 65536]");
    return false;
  }
  if (!finite3(c->eye) || !finite3(c->look_at) || !finite3(c->up)) {
    set_error("camera vectors must be finite");
    return false;
  }
  double f[3], r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = (double)c->look_at[a] - c->eye[a];
  double lf = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(lf > 0)) { set_error("camera look_at equals eye"); return false; }
  for (int a = 0; a < 3; ++a) f[a] /= lf;
  r[0] = f[1] * c->up[2] - f[2] * c->up[1];
  r[1] = f[2] * c->up[0] - f[0] * c->up[2];
  r[2] = f[0] * c->up[1] - f[1] * c->up[0];
  double lr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(lr > 1e-12)) { set_error("camera up is parallel to the view direction"); return false; }
  for (int a = 0; a < 3; ++a) r[a] /= lr;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  CameraDev d;
  d.ortho = c->type == GPSS_CAMERA_ORTHO;
  if (c->type != GPSS_CAMERA_ORTHO && c->type != GPSS_CAMERA_PERSPECTIVE) { set_error("unknown camera type"); return false; }
  for (int a = 0; a < 3; ++a) {
    d.eye[a] = c->eye[a];
    d.fwd[a] = (float)f[a];
    d.right[a] = (float)r[a];
    d.up[a] = (float)u[a];
  }
  if (d.ortho) {
    if (!(c->ortho_w > 0 && c->ortho_h > 0)) { set_error("ortho film size must be > 0"); return false; }
    d.half_w = 0.5f * c->ortho_w;
    d.half_h = 0.5f * c->ortho_h;
  } else {
    if (!(c->fov_y_deg > 0 && c->fov_y_deg < 179)) { set_error("fov_y_deg must lie in (0, 179)"); return false; }
    const double th = std::tan(0.5 * c->fov_y_deg * 3.14159265358979323846 / 180.0);
    d.half_w = (float)(th * c->width / c->height);
    d.half_h = (float)th;
  }
  d.width = c->width;
  d.height = c->height;
  *out = d;
  return true;
}

static gpss_status check_objects(const gpss_object_desc* objs, int n) {
  if (!objs || n < 1 || n > kMaxObjects) {
    set_error("n_objs must be in [1, %d]", kMaxObjects);
    return GPSS_ERR_INVALID_ARG;
  }
  for (int k = 0; k < n; ++k) {
    const gpss_object_desc& o = objs[k];
    if (o.nx < 2 || o.ny < 2 || o.nz < 2 || o.nx > 4096 || o.ny > 4096 || o.nz > 4096) {
      set_error("object %d: nodes per axis must be in [2, 4096]", k);
      return GPSS_ERR_INVALID_ARG;
    }
    if ((double)o.nx * o.ny * o.nz > 1.0e9) { set_error("object %d: grid too large", k); return GPSS_ERR_INVALID_ARG; }
    for (int a = 0; a < 3; ++a)
      if (!(std::isfinite(o.bbox_min[a]) && std::isfinite(o.bbox_max[a]) && o.bbox_max[a] > o.bbox_min[a])) {
        set_error("object %d: empty or non-finite box", k);
        return GPSS_ERR_INVALID_ARG;
      }
    if (!o.mean || !o.variance || !o.albedo) { set_error("object %d: null grid pointer", k); return GPSS_ERR_INVALID_ARG; }
    if (o.albedo_channels != 1 && o.albedo_channels != 3) {
      set_error("object %d: albedo_channels must be 1 or 3", k);
      return GPSS_ERR_INVALID_ARG;
    }
    if (!(o.length_scale > 0.0f) || !std::isfinite(o.length_scale)) {
      set_error("object %d: length_scale must be finite and > 0", k);
      return GPSS_ERR_INVALID_ARG;
    }
    if (o.ndf != GPSS_NDF_GPSS && o.ndf != GPSS_NDF_BECKMANN && o.ndf != GPSS_NDF_GGX) {
      set_error("object %d: unknown ndf %d", k, o.ndf);
      return GPSS_ERR_INVALID_ARG;
    }
    for (float l : {o.length_scale_b, o.length_scale_n})
      if (!(l == 0.0f || (l > 0.0f && std::isfinite(l)))) {
        set_error("object %d: length_scale_b / length_scale_n must be 0 or finite and > 0", k);
        return GPSS_ERR_INVALID_ARG;
      }
    const float lb = o.length_scale_b > 0.0f ? o.length_scale_b : o.length_scale;
    const float ln = o.length_scale_n > 0.0f ? o.length_scale_n : o.length_scale;
    if (lb != o.length_scale && !o.tangent) {
      set_error("object %d: length_scale_b != length_scale needs a tangent field", k);
      return GPSS_ERR_INVALID_ARG;
    }
    if (o.ndf != GPSS_NDF_GPSS && (lb != o.length_scale || ln != o.length_scale || o.tangent)) {
      set_error("object %d: height-field macrofacets take an isotropic kernel", k);
      return GPSS_ERR_INVALID_ARG;
    }
  }
  return GPSS_OK;
}

// Resolves an object's kernel description and makes its optional device grids match
// the descriptor (allocated where it has them, freed where it no longer does).
static gpss_status set_kernel(ObjectHost& o, const gpss_object_desc& d) {
  o.length_scale = d.length_scale;
  o.length_scale_b = d.length_scale_b > 0.0f ? d.length_scale_b : d.length_scale;
  o.length_scale_n = d.length_scale_n > 0.0f ? d.length_scale_n : d.length_scale;
  cudaError_t e = cudaSuccess;
  if (d.correlation_scale && !o.cscale) e = cudaMalloc(&o.cscale, o.nodes * sizeof(float));
  if (!d.correlation_scale && o.cscale) { cudaFree(o.cscale); o.cscale = nullptr; }
  if (e == cudaSuccess && d.tangent && !o.tangent) e = cudaMalloc(&o.tangent, 3 * o.nodes * sizeof(float));
  if (!d.tangent && o.tangent) { cudaFree(o.tangent); o.tangent = nullptr; }
  if (e != cudaSuccess) return cuda_fail(e, "kernel grid allocation");
  return GPSS_OK;
}

static gpss_status check_light(const gpss_light_desc* L) {
  if (!L) return GPSS_OK;
  if (L->type < 0 || L->type > 2) { set_error("unknown light type"); return GPSS_ERR_INVALID_ARG; }
  if (!finite3(L->dir) || !finite3(L->radiance)) { set_error("light values must be finite"); return GPSS_ERR_INVALID_ARG; }
  if (L->type == GPSS_LIGHT_DIRECTIONAL) {
    const double n = std::sqrt((double)L->dir[0] * L->dir[0] + (double)L->dir[1] * L->dir[1] + (double)L->dir[2] * L->dir[2]);
    if (!(n > 0)) { set_error("directional light needs a non-zero direction"); return GPSS_ERR_INVALID_ARG; }
  }
  return GPSS_OK;
}

gpss_status check_opts(const gpss_render_opts* o) {
  if (!o) { set_error("null options"); return GPSS_ERR_INVALID_ARG; }
  if (o->spp < 1) { set_error("spp must be >= 1"); return GPSS_ERR_INVALID_ARG; }
  if (o->max_bounces < 1 || o->max_bounces > 65535) { set_error("max_bounces must be in [1, 65535]"); return GPSS_ERR_INVALID_ARG; }
  if (!(o->mix_R > 0.0f && o->mix_R < 1.0f)) { set_error("mix_R must lie in (0,1)"); return GPSS_ERR_INVALID_ARG; }
  if (o->flags & ~(GPSS_FLAG_KEEP_PATH_RADIANCE | GPSS_FLAG_EXACT_VNDF)) { set_error("unknown flags"); return GPSS_ERR_INVALID_ARG; }
  return GPSS_OK;
}

static void free_scene(gpss_scene s) {
  if (!s) return;
  for (int k = 0; k < kMaxObjects; ++k) {
    cudaFree(s->obj[k].mv);
    cudaFree(s->obj[k].albedo);
    cudaFree(s->obj[k].cscale);
    cudaFree(s->obj[k].tangent);
    cudaFree(s->obj[k].omaj);
    cudaFree(s->obj[k].oskip);
  }
  cudaFree(s->maj);
  cudaFree(s->skip);
  cudaFree(s->skip_tmp);
  cudaFree(s->counters);
  cudaFree(s->tmp_planes);
  cudaFree(s->flags);
  cudaFree(s->grad_mv);
  cudaFree(s->film);
  cudaFree(s->path_radiance);
  delete s;
}

static gpss_status setup_majorant(gpss_scene s) {
  float hmin[3] = {INFINITY, INFINITY, INFINITY}, lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < s->n_objs; ++k)
    for (int a = 0; a < 3; ++a) {
      const ObjectHost& o = s->obj[k];
      hmin[a] = std::fmin(hmin[a], (o.bmax[a] - o.bmin[a]) / (float)(o.n[a] - 1));
      lo[a] = std::fmin(lo[a], o.bmin[a]);
      hi[a] = std::fmax(hi[a], o.bmax[a]);
    }
  int brick = s->brick;
  for (;;) {
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) {
      const float cell = hmin[a] * brick;
      s->mg.gmin[a] = lo[a];
      s->mg.cell[a] = cell;
      s->mg.inv_cell[a] = 1.0f / cell;
      s->mg.dims[a] = std::max(1, (int)std::ceil((hi[a] - lo[a]) / cell - 1e-4f));
      cells *= s->mg.dims[a];
    }
    if (cells <= 1.0 * (1 << 26) || brick >= 64) break;
    brick *= 2;  // keep the majorant grid below 64 Mi cells
  }
  s->brick = brick;
  const size_t ncell = (size_t)s->mg.dims[0] * s->mg.dims[1] * s->mg.dims[2];
  cudaError_t e = cudaMalloc(&s->maj, ncell * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "majorant allocation");
  s->mg.maj = s->maj;
  if ((e = cudaMalloc(&s->skip, ncell * sizeof(float2))) != cudaSuccess) return cuda_fail(e, "skip grid allocation");
  s->mg.skip = s->skip;
  size_t tmp_cells = ncell;
  if (s->n_objs > 1) {
    // each object's own grid: its box at its node spacing (x the brick that keeps it
    // below 64 Mi cells)
    for (int k = 0; k < s->n_objs; ++k) {
      ObjectHost& o = s->obj[k];
      MajorantDev& g = o.og;
      g = MajorantDev{};
      for (int b = 1;; b *= 2) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) {
          const float cell = (o.bmax[a] - o.bmin[a]) / (float)(o.n[a] - 1) * b;
          g.gmin[a] = o.bmin[a];
          g.cell[a] = cell;
          g.inv_cell[a] = 1.0f / cell;
          g.dims[a] = std::max(1, (int)std::ceil((o.bmax[a] - o.bmin[a]) / cell - 1e-4f));
          cells *= g.dims[a];
        }
        if (cells <= 1.0 * (1 << 26) || b >= 64) break;
      }
      const size_t oc = (size_t)g.dims[0] * g.dims[1] * g.dims[2];
      if ((e = cudaMalloc(&o.omaj, oc * sizeof(float))) != cudaSuccess ||
          (e = cudaMalloc(&o.oskip, oc * sizeof(float2))) != cudaSuccess)
        return cuda_fail(e, "object majorant allocation");
      g.maj = o.omaj;
      g.skip = o.oskip;
      tmp_cells = std::max(tmp_cells, oc);
    }
  }
  if ((e = cudaMalloc(&s->skip_tmp, 3 * tmp_cells * sizeof(float))) != cudaSuccess)
    return cuda_fail(e, "skip scratch allocation");
  return GPSS_OK;
}

}  // namespace gpss

using namespace gpss;

extern "C" const char* gpss_last_error(void) { return gpss::g_err; }

extern "C" int gpss_version(void) { return (1 << 16) | 0; }

extern "C" gpss_status gpss_scene_create(const gpss_object_desc* objs, int n_objs, const gpss_light_desc* light,
                                         int majorant_brick, gpss_stream stream, gpss_scene* out) {
  if (!out) { set_error("null output handle"); return GPSS_ERR_INVALID_ARG; }
  *out = nullptr;
  gpss_status st = check_objects(objs, n_objs);
  if (st != GPSS_OK) return st;
  if ((st = check_light(light)) != GPSS_OK) return st;
  if (majorant_brick < 0 || majorant_brick > 64) { set_error("majorant_brick must be in [0, 64]"); return GPSS_ERR_INVALID_ARG; }
  gpss_scene s = new (std::nothrow) gpss_scene_s();
  if (!s) { set_error("host allocation failed"); return GPSS_ERR_OOM; }
  cudaGetDevice(&s->device);
  s->n_objs = n_objs;
  s->brick = majorant_brick > 0 ? majorant_brick : 1;
  size_t max_nodes = 0;
  cudaError_t e;
  for (int k = 0; k < n_objs; ++k) {
    ObjectHost& o = s->obj[k];
    o.n[0] = objs[k].nx;
    o.n[1] = objs[k].ny;
    o.n[2] = objs[k].nz;
    for (int a = 0; a < 3; ++a) {
      o.bmin[a] = objs[k].bbox_min[a];
      o.bmax[a] = objs[k].bbox_max[a];
    }
    o.channels = objs[k].albedo_channels;
    o.length_scale = objs[k].length_scale;
    o.ndf = objs[k].ndf;
    o.nodes = (size_t)o.n[0] * o.n[1] * o.n[2];
    max_nodes = std::max(max_nodes, o.nodes);
    if ((e = cudaMalloc(&o.mv, o.nodes * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&o.albedo, o.nodes * o.channels * sizeof(float))) != cudaSuccess) {
      free_scene(s);
      return cuda_fail(e, "grid allocation");
    }
    if ((st = set_kernel(o, objs[k])) != GPSS_OK) {
      free_scene(s);
      return st;
    }
  }
  if ((e = cudaMalloc(&s->counters, 16 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&s->tmp_planes, 2 * max_nodes * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->flags, kSceneFlagWords * sizeof(int))) != cudaSuccess) {
    free_scene(s);
    return cuda_fail(e, "scratch allocation");
  }
  s->tmp_capacity = 2 * max_nodes;
  if (light) {
    s->light.kind = light->type;
    double n = std::sqrt((double)light->dir[0] * light->dir[0] + (double)light->dir[1] * light->dir[1] +
                         (double)light->dir[2] * light->dir[2]);
    for (int a = 0; a < 3; ++a) {
      s->light.dir[a] = n > 0 ? (float)(light->dir[a] / n) : (a == 2 ? 1.0f : 0.0f);
      s->light.radiance[a] = light->radiance[a];
    }
  } else {
    s->light.kind = kLightDirectional;
    s->light.dir[0] = 0.0f; s->light.dir[1] = 0.0f; s->light.dir[2] = 1.0f;
    s->light.radiance[0] = s->light.radiance[1] = s->light.radiance[2] = 1.0f;
  }
  if ((st = setup_majorant(s)) != GPSS_OK) { free_scene(s); return st; }
  cudaStream_t cs = (cudaStream_t)stream;
  if ((st = scene_upload(s, objs, n_objs, cs)) != GPSS_OK) { free_scene(s); return st; }
  if ((st = build_majorant(s, cs)) != GPSS_OK) { free_scene(s); return st; }
  *out = s;
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_update(gpss_scene s, const gpss_object_desc* objs, int n_objs, gpss_stream stream) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  gpss_status st = check_objects(objs, n_objs);
  if (st != GPSS_OK) return st;
  if (n_objs != s->n_objs) { set_error("object count differs from the scene's"); return GPSS_ERR_INVALID_ARG; }
  for (int k = 0; k < n_objs; ++k) {
    const ObjectHost& o = s->obj[k];
    if (objs[k].nx != o.n[0] || objs[k].ny != o.n[1] || objs[k].nz != o.n[2] || objs[k].albedo_channels != o.channels) {
      set_error("object %d: sizes differ from the scene's", k);
      return GPSS_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
      if (objs[k].bbox_min[a] != o.bmin[a] || objs[k].bbox_max[a] != o.bmax[a]) {
        set_error("object %d: box differs from the scene's", k);
        return GPSS_ERR_INVALID_ARG;
      }
    s->obj[k].ndf = objs[k].ndf;
    if ((st = set_kernel(s->obj[k], objs[k])) != GPSS_OK) return st;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  if ((st = scene_upload(s, objs, n_objs, cs)) != GPSS_OK) return st;
  s->path_tag = 0;
  ++s->version;
  return build_majorant(s, cs);
}

extern "C" gpss_status gpss_scene_set_traversal(gpss_scene s, int skip_levels, float kappa, gpss_stream stream) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  if (skip_levels < 0 || skip_levels > 6) { set_error("skip_levels must be in [0, 6]"); return GPSS_ERR_INVALID_ARG; }
  if (!(kappa >= 0.0f) || !std::isfinite(kappa)) { set_error("kappa must be finite and >= 0"); return GPSS_ERR_INVALID_ARG; }
  s->skip_levels = skip_levels;
  s->kappa = kappa;
  return build_skip(s, (cudaStream_t)stream);
}

extern "C" gpss_status gpss_scene_set_schedule(gpss_scene s, int shade_min) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  if (shade_min < 1 || shade_min > 32) { set_error("shade_min must be in [1, 32]"); return GPSS_ERR_INVALID_ARG; }
  s->shade_min = shade_min;
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_set_surface_flight(gpss_scene s, int enable) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  if (enable != 0 && enable != 1) { set_error("enable must be 0 or 1"); return GPSS_ERR_INVALID_ARG; }
  s->lin_flight = enable != 0;
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_set_object_grids(gpss_scene s, int enable) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  if (enable != 0 && enable != 1) { set_error("enable must be 0 or 1"); return GPSS_ERR_INVALID_ARG; }
  s->object_grids = enable != 0;
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_set_local_majorant(gpss_scene s, float hot) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  if (!(hot >= 0.0f) || !std::isfinite(hot)) { set_error("hot must be finite and >= 0"); return GPSS_ERR_INVALID_ARG; }
  s->hot = hot;
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_destroy(gpss_scene s) {
  if (!s) { set_error("null scene"); return GPSS_ERR_INVALID_ARG; }
  free_scene(s);
  return GPSS_OK;
}

extern "C" gpss_status gpss_scene_majorant(gpss_scene s, int dims[3], float* values, gpss_stream stream) {
  if (!s || !dims) { set_error("null argument"); return GPSS_ERR_INVALID_ARG; }
  for (int a = 0; a < 3; ++a) dims[a] = s->mg.dims[a];
  if (values) {
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    cudaError_t e = cudaMemcpyAsync(values, s->maj, n * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "majorant copy");
  }
  return GPSS_OK;
}

bool gpss::is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gpss_status gpss::check_path_total(long long npx, long long spp, const char* what) {
  if (npx > 0 && spp > (1LL << 46) / npx) {
    set_error("too many paths (%s above 2^46)", what);
    return GPSS_ERR_INVALID_ARG;
  }
  return GPSS_OK;
}

static gpss_status ensure(float** buf, size_t* cap, size_t n, const char* what) {
  if (*cap >= n) return GPSS_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(buf, n * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, what);
  *cap = n;
  return GPSS_OK;
}

extern "C" gpss_status gpss_render(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts, float* image,
                                   float* sqsum, gpss_stats* stats, gpss_stream stream) {
  if (!s || !image) { set_error("null scene or image"); return GPSS_ERR_INVALID_ARG; }
  gpss_status st = check_opts(opts);
  if (st != GPSS_OK) return st;
  CameraDev C;
  if (!camera_dev(cam, &C)) return GPSS_ERR_INVALID_ARG;
  const size_t npx = (size_t)C.width * C.height;
  const long long total = (long long)npx * opts->spp;
  if ((st = check_path_total((long long)npx, opts->spp, "W*H*spp")) != GPSS_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e;
  const bool host_img = !is_device_ptr(image);
  const bool host_sq = sqsum && !is_device_ptr(sqsum);
  float* dimg = image;
  float* dsq = sqsum;
  if (host_img || host_sq) {
    if ((st = ensure(&s->film, &s->film_capacity, 6 * npx, "film allocation")) != GPSS_OK) return st;
    if (host_img) dimg = s->film;
    if (host_sq) dsq = s->film + 3 * npx;
  }
  float* path_rad = nullptr;
  if (opts->flags & GPSS_FLAG_KEEP_PATH_RADIANCE) {
    if ((st = ensure(&s->path_radiance, &s->path_capacity, 3 * (size_t)total, "path radiance allocation")) != GPSS_OK)
      return st;
    path_rad = s->path_radiance;
  }
  if ((e = cudaMemsetAsync(dimg, 0, 3 * npx * sizeof(float), cs)) != cudaSuccess) return cuda_fail(e, "clear image");
  if (dsq && (e = cudaMemsetAsync(dsq, 0, 3 * npx * sizeof(float), cs)) != cudaSuccess) return cuda_fail(e, "clear sqsum");
  if ((e = cudaMemsetAsync(s->counters, 0, 16 * sizeof(unsigned long long), cs)) != cudaSuccess)
    return cuda_fail(e, "clear counters");
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (stats) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, cs);
  }
  const int block = render_block_size();
  const int grid = render_grid_size(s->device, block);
  e = launch_render(scene_dev(s), C, *opts, dimg, dsq, path_rad, s->counters, grid, block, s->shade_min, cs);
  if (e != cudaSuccess) return cuda_fail(e, "render launch");
  if (stats) cudaEventRecord(ev1, cs);
  if (host_img && (e = cudaMemcpyAsync(image, dimg, 3 * npx * sizeof(float), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
    return cuda_fail(e, "image copy");
  if (host_sq && (e = cudaMemcpyAsync(sqsum, dsq, 3 * npx * sizeof(float), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
    return cuda_fail(e, "sqsum copy");
  if (path_rad) s->path_tag = path_fingerprint(cam, opts, s->version);
  if (stats || host_img || host_sq) {
    unsigned long long c[16];
    if (stats && (e = cudaMemcpyAsync(c, s->counters, sizeof(c), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
      return cuda_fail(e, "stats copy");
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "render");
    if (stats) {
      fill_stats(stats, c, 0.0f);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      stats->ms = ms;
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
    }
  }
  return GPSS_OK;
}
