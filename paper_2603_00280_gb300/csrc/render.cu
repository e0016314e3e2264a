// render.cu -- forward path tracing of the GPSS medium: the forward instance of
// the persistent path kernel (path_kernel.cuh) and its launch.
#include "path_kernel.cuh"

namespace gpss {

int render_block_size() { return kPathBlock; }

int render_grid_size(int device, int block) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_path<false, kTravGrid, false>, block, 0);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

cudaError_t launch_render(const SceneDev& S, const CameraDev& C, const gpss_render_opts& o, float* image,
                          float* sqsum, float* path_radiance, unsigned long long* counters, int grid,
                          int block, int shade_min, cudaStream_t st) {
  PathArgs P;
  P.spp = o.spp;
  P.max_bounces = o.max_bounces;
  P.seed = o.seed;
  P.mix_R = o.mix_R;
  P.npix = C.width * C.height;
  P.total = (long long)P.npix * o.spp;
  P.inv_spp = 1.0f / (float)o.spp;
  P.shade_min = shade_min;
  P.exact_vndf = (o.flags & GPSS_FLAG_EXACT_VNDF) ? 1 : 0;
  AdjOut A{};
  if (path_radiance) {
    // kept for an adjoint: recorded by the adjoint's own kernel (bit-identical replay)
    A.record = 1;
    int device = 0;
    cudaGetDevice(&device);
    return launch_adjoint_kernel(S, C, P, image, sqsum, path_radiance, counters, A, device, st);
  }
  int trav = trav_of(S);
  if (trav != kTravGrid && trav != kTravLocal && trav != kTravMulti && trav != kTravSplit) trav = kTravSplitLocal;
  if (scene_general(S)) {
    if (trav == kTravSplitLocal)
      k_path<false, kTravSplitLocal, true><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravSplit)
      k_path<false, kTravSplit, true><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravMulti)
      k_path<false, kTravMulti, true><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravLocal)
      k_path<false, kTravLocal, true><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else
      k_path<false, kTravGrid, true><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
  } else {
    if (trav == kTravSplitLocal)
      k_path<false, kTravSplitLocal, false><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravSplit)
      k_path<false, kTravSplit, false><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravMulti)
      k_path<false, kTravMulti, false><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else if (trav == kTravLocal)
      k_path<false, kTravLocal, false><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
    else
      k_path<false, kTravGrid, false><<<grid, block, 0, st>>>(S, C, P, image, sqsum, path_radiance, counters, A);
  }
  return cudaGetLastError();
}

}  // namespace gpss
