// gpss_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gpss.h"
#include "gpss_device.cuh"

namespace gpss {

// Per-call work counters, accumulated on the device (u64 each).
enum Counter : int {
  kCntPaths = 0,
  kCntVertices,
  kCntNull,
  kCntShadow,
  kCntCells,
  kCntTruncated,
  kCntAborted,
  kCntMaxEvents,   // max over paths (atomicMax)
  kCntNonFinite,   // adjoint: gradient contributions skipped as not finite
  kCntNum
};
static_assert(kCntNum + 1 <= 16, "counters + cursor must fit the 16-word counter area");

struct ObjectHost {
  int n[3];
  float bmin[3], bmax[3];
  int channels;
  float length_scale;
  float2* mv = nullptr;      // device (mean, variance)
  float* albedo = nullptr;   // device planes
  size_t nodes = 0;
  float sigma_min = 0.0f;    // smallest standard deviation over the nodes
  int ndf = 0;               // gpss_ndf
  float length_scale_b = 0.0f, length_scale_n = 0.0f;  // resolved (l_t where unset)
  float* cscale = nullptr;   // device correlation-scale factors (nodes), or null
  float* tangent = nullptr;  // device tangent field (3 planes of nodes), or null
  bool thin = false;         // sigma_min below the grid spacing (local majorants pay)
  // the object's own majorant grid (scenes of several objects): geometry, majorants, skip
  MajorantDev og{};
  float* omaj = nullptr;
  float2* oskip = nullptr;
  bool anisotropic() const {
    return length_scale_b != length_scale || length_scale_n != length_scale || tangent != nullptr;
  }
};

constexpr int kSceneFlagWords = 1 + kMaxObjects;  // validation bits + per-object min variance

}  // namespace gpss

struct gpss_scene_s {
  int device = 0;
  int n_objs = 0;
  gpss::ObjectHost obj[gpss::kMaxObjects];
  gpss::LightDev light{};
  gpss::MajorantDev mg{};
  float* maj = nullptr;            // device majorant grid (fine level)
  float2* skip = nullptr;          // device skip grid (M_r, r) per majorant cell
  float* skip_tmp = nullptr;       // 3 x cells scratch for the skip build (largest grid)
  int skip_levels = 5;             // radii 1, 2, ..., 2^(levels-1)
  float kappa = 0.5f;              // expected majorant depth allowed per skip
  int shade_min = 24;              // lanes a warp gathers before shading real vertices
  float hot = 4.0f;                // local-majorant threshold (0 = off; single-object scenes)
  bool lin_flight = false;         // surface-limit analytic flight in local pieces (opt-in)
  bool thin = false;               // some object's sigma_min < its grid spacing (local majorants pay)
  bool object_grids = false;       // several objects: per-object traversal on their own grids (opt-in)
  int brick = 1;                   // majorant cell = brick x finest field cell
  // scratch owned by the scene
  unsigned long long* counters = nullptr;   // kCntNum u64 + work cursor
  float* tmp_planes = nullptr;     // staging for uploads (2 x max nodes)
  size_t tmp_capacity = 0;
  int* flags = nullptr;            // validation / error flags (device)
  float* film = nullptr;           // film used when the caller's image is host memory
  size_t film_capacity = 0;
  float* path_radiance = nullptr;  // per-path radiance kept for the adjoint (optional)
  size_t path_capacity = 0;
  uint64_t path_tag = 0;           // fingerprint of the render that filled path_radiance
  float2* grad_mv = nullptr;       // adjoint: interleaved (d mean, d variance) accumulation
  size_t grad_capacity = 0;
  uint64_t version = 1;            // incremented whenever the grids change
};

namespace gpss {

void set_error(const char* fmt, ...);
// Fills *st from the kCntNum device counters copied to the host.
void fill_stats(gpss_stats* st, const unsigned long long* c, float ms);
gpss_status cuda_fail(cudaError_t e, const char* what);
// Whether p is device (or managed) memory; host memory, pinned or pageable, gives false.
bool is_device_ptr(const void* p);
// INVALID_ARG (with the message set) when a render of npx pixels at spp samples has
// more than 2^46 paths: every render entry point (single, allocation-free, batched)
// enforces this one limit.
gpss_status check_path_total(long long npx, long long spp, const char* what);

gpss_status scene_upload(gpss_scene s, const gpss_object_desc* objs, int n, cudaStream_t st);
gpss_status build_majorant(gpss_scene s, cudaStream_t st);
gpss_status build_skip(gpss_scene s, cudaStream_t st);
SceneDev scene_dev(const gpss_scene_s* s);
bool camera_dev(const gpss_camera* c, CameraDev* out);

// kernels (launch wrappers)
uint64_t path_fingerprint(const gpss_camera* cam, const gpss_render_opts* o, uint64_t scene_version);
// Forward render; with path_radiance (the per-path radiance an adjoint replays) it runs
// the adjoint's kernel in its recording mode instead of the forward kernel.
cudaError_t launch_render(const SceneDev& S, const CameraDev& C, const gpss_render_opts& o, float* image,
                          float* sqsum, float* path_radiance, unsigned long long* counters, int grid,
                          int block, int shade_min, cudaStream_t st);
struct PathArgs;
struct AdjOut;
cudaError_t launch_adjoint_kernel(const SceneDev& S, const CameraDev& C, const PathArgs& P, float* image, float* sqsum,
                                  float* path_radiance, unsigned long long* counters, const AdjOut& A, int device,
                                  cudaStream_t cs);
int render_block_size();
int render_grid_size(int device, int block);

}  // namespace gpss
