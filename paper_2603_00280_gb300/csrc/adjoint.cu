// adjoint.cu -- gradients of a rendered image with respect to the scene's grids
// (mean, variance, albedo) and the kernel length scale: the adjoint instance of
// the persistent path kernel (see path_kernel.cuh for the estimator).
#include <algorithm>
#include <cstring>

#include "path_kernel.cuh"

namespace gpss {

// Fingerprint of (camera, options without flags, scene contents): identifies the
// render whose per-path radiance the scene keeps.
uint64_t path_fingerprint(const gpss_camera* cam, const gpss_render_opts* o, uint64_t scene_version) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  gpss_render_opts oo = *o;
  oo.flags &= ~GPSS_FLAG_KEEP_PATH_RADIANCE;
  mix(cam, sizeof(*cam));
  mix(&oo.spp, sizeof(oo.spp));
  mix(&oo.max_bounces, sizeof(oo.max_bounces));
  mix(&oo.seed, sizeof(oo.seed));
  mix(&oo.mix_R, sizeof(oo.mix_R));
  mix(&oo.flags, sizeof(oo.flags));
  mix(&scene_version, sizeof(scene_version));
  return h | 1ull;
}

gpss_status check_opts(const gpss_render_opts* o);

// Adds the interleaved accumulation buffer into the caller's gradient grids.
__global__ void k_split_grad(const float2* __restrict__ mv, float* __restrict__ d_mean, float* __restrict__ d_var,
                             size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 g = mv[i];
    if (d_mean) d_mean[i] += g.x;
    if (d_var) d_var[i] += g.y;
  }
}

// The adjoint instance of the path kernel for the scene (its traversal, as the forward
// render's, so the replay takes the same tentative collisions; the general one where an
// object has a correlation-scale grid, the only general feature the adjoint accepts) on
// a grid of the SMs times its resident blocks.  A.record = 1 runs it as the recording
// forward pass (film image/sqsum, per-path radiance path_radiance).
cudaError_t launch_adjoint_kernel(const SceneDev& S, const CameraDev& C, const PathArgs& P, float* image, float* sqsum,
                                  float* path_radiance, unsigned long long* counters, const AdjOut& A, int device,
                                  cudaStream_t cs) {
  int trav = trav_of(S);
  if (trav != kTravGrid && trav != kTravLocal && trav != kTravMulti && trav != kTravSplit) trav = kTravSplitLocal;
  const bool gen = scene_general(S);
  const int slot = trav == kTravGrid ? 0 : trav == kTravLocal ? 1 : trav == kTravMulti ? 2 : trav == kTravSplit ? 3 : 4;
  const void* fns[2][5] = {{(const void*)k_path<true, kTravGrid, false>, (const void*)k_path<true, kTravLocal, false>,
                            (const void*)k_path<true, kTravMulti, false>, (const void*)k_path<true, kTravSplit, false>,
                            (const void*)k_path<true, kTravSplitLocal, false>},
                           {(const void*)k_path<true, kTravGrid, true>, (const void*)k_path<true, kTravLocal, true>,
                            (const void*)k_path<true, kTravMulti, true>, (const void*)k_path<true, kTravSplit, true>,
                            (const void*)k_path<true, kTravSplitLocal, true>}};
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[gen ? 1 : 0][slot], kPathBlock, 0);
  const int g = sms * (per_sm > 0 ? per_sm : 1);
  float *im = image, *sq = sqsum, *pr = path_radiance;
  unsigned long long* ct = counters;
  if (gen) {
    if (trav == kTravSplitLocal) k_path<true, kTravSplitLocal, true><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravSplit) k_path<true, kTravSplit, true><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravMulti) k_path<true, kTravMulti, true><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravLocal) k_path<true, kTravLocal, true><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else k_path<true, kTravGrid, true><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
  } else {
    if (trav == kTravSplitLocal) k_path<true, kTravSplitLocal, false><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravSplit) k_path<true, kTravSplit, false><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravMulti) k_path<true, kTravMulti, false><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else if (trav == kTravLocal) k_path<true, kTravLocal, false><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
    else k_path<true, kTravGrid, false><<<g, kPathBlock, 0, cs>>>(S, C, P, im, sq, pr, ct, A);
  }
  return cudaGetLastError();
}

}  // namespace gpss

using namespace gpss;

extern "C" gpss_status gpss_render_adjoint(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts,
                                           const float* d_image, float* d_mean, float* d_variance, float* d_albedo,
                                           float* d_length_scale, float* d_correlation_scale, gpss_stats* stats,
                                           gpss_stream stream) {
  if (!s || !d_image) { set_error("null scene or d_image"); return GPSS_ERR_INVALID_ARG; }
  gpss_status st = check_opts(opts);
  if (st != GPSS_OK) return st;
  bool any_cs = false;
  for (int k = 0; k < s->n_objs; ++k) {
    if (s->obj[k].ndf != GPSS_NDF_GPSS) {
      set_error("the adjoint supports the GPSS NDF only (not the height-field macrofacets)");
      return GPSS_ERR_UNSUPPORTED;
    }
    if (s->obj[k].anisotropic()) {
      set_error("the adjoint supports isotropic kernels only (l_b = l_n = l_t, no tangent field)");
      return GPSS_ERR_UNSUPPORTED;
    }
    any_cs = any_cs || s->obj[k].cscale;
  }
  if (d_correlation_scale && !any_cs) {
    set_error("d_correlation_scale given for a scene without a correlation-scale grid");
    return GPSS_ERR_INVALID_ARG;
  }
  CameraDev C;
  if (!camera_dev(cam, &C)) return GPSS_ERR_INVALID_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t npx = (size_t)C.width * C.height;
  const long long total = (long long)npx * opts->spp;
  const uint64_t fp = path_fingerprint(cam, opts, s->version);
  cudaError_t e;
  const int block = render_block_size();
  const int grid = render_grid_size(s->device, block);
  if (s->path_tag != fp) {
    // no kept radiance of this render: run the forward pass first (paths only)
    if (s->path_capacity < 3 * (size_t)total) {
      cudaFree(s->path_radiance);
      s->path_radiance = nullptr;
      s->path_capacity = 0;
      if ((e = cudaMalloc(&s->path_radiance, 3 * (size_t)total * sizeof(float))) != cudaSuccess)
        return cuda_fail(e, "path radiance allocation");
      s->path_capacity = 3 * (size_t)total;
    }
    if (s->film_capacity < 6 * npx) {
      cudaFree(s->film);
      s->film = nullptr;
      s->film_capacity = 0;
      if ((e = cudaMalloc(&s->film, 6 * npx * sizeof(float))) != cudaSuccess) return cuda_fail(e, "film allocation");
      s->film_capacity = 6 * npx;
    }
    if ((e = cudaMemsetAsync(s->film, 0, 3 * npx * sizeof(float), cs)) != cudaSuccess) return cuda_fail(e, "clear film");
    if ((e = cudaMemsetAsync(s->counters, 0, 16 * sizeof(unsigned long long), cs)) != cudaSuccess)
      return cuda_fail(e, "clear counters");
    e = launch_render(scene_dev(s), C, *opts, s->film, nullptr, s->path_radiance, s->counters, grid, block,
                      s->shade_min, cs);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    s->path_tag = fp;
  }
  if ((e = cudaMemsetAsync(s->counters, 0, 16 * sizeof(unsigned long long), cs)) != cudaSuccess)
    return cuda_fail(e, "clear counters");
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (stats) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, cs);
  }
  PathArgs P;
  P.spp = opts->spp;
  P.max_bounces = opts->max_bounces;
  P.seed = opts->seed;
  P.mix_R = opts->mix_R;
  P.npix = (int)npx;
  P.total = total;
  P.inv_spp = 1.0f / (float)opts->spp;
  P.shade_min = s->shade_min;
  P.exact_vndf = (opts->flags & GPSS_FLAG_EXACT_VNDF) ? 1 : 0;
  AdjOut A{};
  A.d_image = d_image;
  A.L_path = s->path_radiance;
  // gradient grids of the objects one after another (object order); albedo: each
  // object's channel planes
  size_t nodes = 0, alb = 0;
  for (int k = 0; k < kMaxObjects; ++k) {
    A.node_off[k] = (long long)nodes;
    A.alb_off[k] = (long long)alb;
    if (k < s->n_objs) {
      nodes += s->obj[k].nodes;
      alb += s->obj[k].nodes * (size_t)s->obj[k].channels;
    }
  }
  A.d_mv = nullptr;
  if (d_mean || d_variance) {
    if (s->grad_capacity < nodes) {
      cudaFree(s->grad_mv);
      s->grad_mv = nullptr;
      s->grad_capacity = 0;
      if ((e = cudaMalloc(&s->grad_mv, nodes * sizeof(float2))) != cudaSuccess) return cuda_fail(e, "gradient buffer");
      s->grad_capacity = nodes;
    }
    if ((e = cudaMemsetAsync(s->grad_mv, 0, nodes * sizeof(float2), cs)) != cudaSuccess)
      return cuda_fail(e, "clear gradient buffer");
    A.d_mv = s->grad_mv;
  }
  A.d_alb = d_albedo;
  A.d_l = d_length_scale;
  A.d_cs = d_correlation_scale;
  e = launch_adjoint_kernel(scene_dev(s), C, P, nullptr, nullptr, nullptr, s->counters, A, s->device, cs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  if (A.d_mv) {
    const int eb = (int)std::min<size_t>((nodes + 255) / 256, 4096);
    k_split_grad<<<eb, 256, 0, cs>>>(A.d_mv, d_mean, d_variance, nodes);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gradient epilogue");
  }
  if (stats) {
    cudaEventRecord(ev1, cs);
    unsigned long long c[16];
    if ((e = cudaMemcpyAsync(c, s->counters, sizeof(c), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
      return cuda_fail(e, "stats copy");
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "adjoint");
    fill_stats(stats, c, 0.0f);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    stats->ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  return GPSS_OK;
}
