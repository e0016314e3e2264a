// noalloc.cu -- gpss_render_noalloc: the forward render without any device
// memory allocation during the call.
//
// Who needs it: callers that may not allocate device memory at render time, e.g.
// a host application that accounts for every device byte itself and forbids
// hidden allocations, or code that renders from a real-time loop where an
// allocation's latency or a failure to allocate is unacceptable.  gpss_render itself allocates nothing for device outputs, but it
// keeps its work counters in the scene and allocates a staging film the first
// time it is given a host image; this variant uses the file-scope array below
// instead, for every call.
//
// The scratch array is static device memory: every GPU that loads the library
// holds it (about 0.8 MB) until the process exits, and every call uses the same
// array.  Its first kNoAllocCounterWords words hold the work cursor and the
// counters of the render kernel; the rest is a film of at most kNoAllocMaxPixels
// pixels x 3 channels.  Each call clears both before the kernel runs, so nothing
// from a previous call leaks into the next one -- but two calls that overlap on
// the GPU (different streams, or different host threads) race on the array.
#include <cstring>
#include <mutex>

#include "gpss_internal.h"

namespace gpss {

constexpr int kNoAllocCounterWords = 32;            // >= kCntNum + 1 (cursor)
constexpr int kNoAllocMaxPixels = 256 * 256;        // film capacity (pixels)
constexpr size_t kNoAllocBytes = kNoAllocCounterWords * sizeof(unsigned long long) +
                                 (size_t)kNoAllocMaxPixels * 3 * sizeof(float);
static_assert(kNoAllocCounterWords >= kCntNum + 1, "counter area too small");

// In host code this name is only a stand-in for the device array: its device
// address comes from cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up on the
// first call made with that device current.
static gpss_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range for the no-allocation render", dev);
    return GPSS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GPSS_OK;
}

gpss_status check_opts(const gpss_render_opts* o);

}  // namespace gpss

using namespace gpss;

extern "C" gpss_status gpss_render_noalloc(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts,
                                           float* image, gpss_stats* stats, gpss_stream stream) {
  if (!s || !image) { set_error("null scene or image"); return GPSS_ERR_INVALID_ARG; }
  gpss_status st = check_opts(opts);
  if (st != GPSS_OK) return st;
  if (opts->flags & GPSS_FLAG_KEEP_PATH_RADIANCE) {
    set_error("gpss_render_noalloc does not keep per-path radiance");
    return GPSS_ERR_INVALID_ARG;
  }
  CameraDev C;
  if (!camera_dev(cam, &C)) return GPSS_ERR_INVALID_ARG;
  const size_t npx = (size_t)C.width * C.height;
  if (npx > (size_t)kNoAllocMaxPixels) {
    set_error("gpss_render_noalloc renders at most %d pixels (got %d x %d); use gpss_render", kNoAllocMaxPixels,
              C.width, C.height);
    return GPSS_ERR_INVALID_ARG;
  }
  if ((st = check_path_total((long long)npx, opts->spp, "W*H*spp")) != GPSS_OK) return st;
  const bool host_img = !is_device_ptr(image);
  void* base = nullptr;
  if ((st = noalloc_scratch(&base)) != GPSS_OK) return st;
  unsigned long long* counters = (unsigned long long*)base;
  float* film = (float*)((unsigned char*)base + kNoAllocCounterWords * sizeof(unsigned long long));
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(counters, 0, kNoAllocCounterWords * sizeof(unsigned long long), cs)) != cudaSuccess)
    return cuda_fail(e, "clear counters");
  if ((e = cudaMemsetAsync(film, 0, 3 * npx * sizeof(float), cs)) != cudaSuccess) return cuda_fail(e, "clear film");
  const int block = render_block_size();
  const int grid = render_grid_size(s->device, block);
  e = launch_render(scene_dev(s), C, *opts, film, nullptr, nullptr, counters, grid, block, s->shade_min, cs);
  if (e != cudaSuccess) return cuda_fail(e, "render launch");
  if ((e = cudaMemcpyAsync(image, film, 3 * npx * sizeof(float), cudaMemcpyDefault, cs)) != cudaSuccess)
    return cuda_fail(e, "image copy");
  // a host image (pinned or pageable) or host stats are complete when the call returns,
  // as with gpss_render: the stream is synchronised whenever either is on the host
  unsigned long long c[kNoAllocCounterWords];
  if (stats && (e = cudaMemcpyAsync(c, counters, sizeof(c), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
    return cuda_fail(e, "stats copy");
  if (stats || host_img) {
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "render");
  }
  if (stats) {
    fill_stats(stats, c, 0.0f);
    stats->ms = 0.0f;
  }
  return GPSS_OK;
}
