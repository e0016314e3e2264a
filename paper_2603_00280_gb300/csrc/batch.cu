// batch.cu -- many scenes in one persistent launch, replayed from a CUDA graph,
// with the launch shape chosen by an autotuner that times the batch itself.
//
// Work distribution.  The paths of all jobs (scene, camera, options) form one
// index space: job j owns [begin_j, begin_j + npix_j * spp_j), and inside a job a
// path's index is gpss_render's (path_of: pixel tiles, samples within a tile).  Resident warps take
// chunks of consecutive indices from one atomic cursor (warp_take), so a chunk mostly
// lies in one job.
// A lane looks its job up when a new path's index leaves its current job's range
// (binary search over the begin offsets) and reads the job's scene, camera and
// options by reference from the device table: lanes of one warp mostly share a
// job, so those loads are uniform and stay in L1.
//
// Graph.  One capture holds: the counter/cursor clear, a kernel that zeroes every
// job's film through the pointers in the table (so new film buffers only need a
// table rewrite), and the persistent kernel.  The table is rewritten (one
// host-to-device copy, ordered on the render's stream before the graph launch)
// only when a film pointer or a scene's device description changed.
//
// Autotuner.  Candidates: block size (64/128/256 threads; grid = SMs x resident
// blocks), shading threshold (lanes a warp gathers before shading real vertices)
// and chunk (paths per cursor fetch).  Coordinate descent from (128, 24, 256),
// one axis after the other: each candidate is timed (CUDA events) on a copy of
// the batch whose spp is reduced so that one launch traces about kTunePaths
// paths, within a total budget of kTuneBudgetMs.  A candidate replaces the
// incumbent only when it is kTuneMargin faster: the reduced copy floors every
// scene at 1 spp, which over-weights low-spp scenes, so small differences there
// do not carry over to the full batch (on the 64-scene uneven batch a 2% win of
// (shade 8, chunk 64) on the copy was a 15% loss on the batch).
#include <algorithm>
#include <cstring>
#include <vector>

#include "path_kernel.cuh"

namespace gpss {

struct JobDev {
  SceneDev S;
  CameraDev C;
  PathArgs P;
  float* image;
  float* sqsum;
};

constexpr int kBatchMaxJobs = 4096;
constexpr long long kTunePaths = 1ll << 24;     // paths per tuning launch (at most, roughly)
constexpr float kTuneMargin = 0.97f;             // a candidate must take < 97% of the incumbent's time
constexpr float kTuneBudgetMs = 5000.0f;         // tuning stops once its launches took this long
constexpr int kBatchDefaultShade = 24;
constexpr int kBatchDefaultChunk = 256;

// largest j with begins[j] <= g (begins ascending, begins[0] = 0)
__device__ __forceinline__ int find_job(const long long* __restrict__ begins, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begins[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Work source of a batch: indices of the flattened job space; a lane looks its job up
// when a new index leaves its current job's range, and a path's scene, options and
// film are its job's.
struct BatchSource {
  const JobDev* __restrict__ jobs;
  const long long* __restrict__ begins;
  int n_jobs;
  long long total;
  int chunk;
  unsigned long long* cursor;
  AdjOut A;
  WarpCursor wc;
  __device__ __forceinline__ void take(Lane& s, unsigned need, int lane) {
    const long long g = warp_take(wc, !s.active, need, lane, cursor, total, chunk);
    if (!s.active && g >= 0 && g < total) {
      if (g < begins[s.job] || g >= begins[s.job + 1]) s.job = find_job(begins, n_jobs, g);
      const JobDev& J = jobs[s.job];
      lane_start<false>(s, J.C, J.P, A, g - begins[s.job]);
    }
  }
  __device__ __forceinline__ bool exhausted() const { return wc.exhausted || wc.next >= total; }
  __device__ __forceinline__ const SceneDev& scene(const Lane& s) const { return jobs[s.job].S; }
  __device__ __forceinline__ const MajorantDev* grids(const Lane& s) const { return jobs[s.job].S.og; }
  __device__ __forceinline__ const PathArgs& args(const Lane& s) const { return jobs[s.job].P; }
  __device__ __forceinline__ const AdjOut& adj() const { return A; }
  __device__ __forceinline__ void finish(Lane& s, LaneCounters& c) {
    const JobDev& J = jobs[s.job];
    lane_finish<false>(s, J.P, J.image, J.sqsum, nullptr, false, c);
  }
};

// The persistent kernel over all jobs: k_path's loop over the batch's work source.  Register cap 96 for every block size, so that 640 lanes per
// SM stay resident.
template <int BLOCK, int TRAV, bool GEN>
__global__ void __maxnreg__(96) k_batch(const JobDev* __restrict__ jobs, const long long* __restrict__ begins,
                                        int n_jobs, long long total, int chunk, int shade_min,
                                        unsigned long long* __restrict__ counters) {
  __shared__ LaneCold s_cold[BLOCK];
  BatchSource src{jobs, begins, n_jobs, total, chunk, counters + kCntNum, AdjOut{}, WarpCursor{0, 0, false}};
  LaneCounters c{0, 0, 0, 0, 0, 0, 0, 0, {0.0f, 0.0f, 0.0f, 0.0f}, 0};
  path_loop<false, TRAV, GEN>(src, shade_min, s_cold, c);
  flush_counters(c, counters, nullptr, 0);
}

// Zeroes every job's film (and sqsum film when present); blockIdx.y = job.
__global__ void k_zero_films(const JobDev* __restrict__ jobs) {
  const JobDev& J = jobs[blockIdx.y];
  const size_t n = 3 * (size_t)J.P.npix;
  float* img = J.image;
  float* sq = J.sqsum;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    img[i] = 0.0f;
    if (sq) sq[i] = 0.0f;
  }
}

template <int BLOCK, int TRAV, bool GEN>
static int batch_grid(int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<BLOCK, TRAV, GEN>, BLOCK, 0);
  return sms * std::max(per_sm, 1);
}

template <int TRAV, bool GEN>
static int grid_for_t(int block, int device) {
  switch (block) {
    case 64: return batch_grid<64, TRAV, GEN>(device);
    case 256: return batch_grid<256, TRAV, GEN>(device);
    default: return batch_grid<128, TRAV, GEN>(device);
  }
}

// The batch instances: the grid walk, local majorants, and per-object intervals with
// local majorants and several objects (which serves every scene).
template <bool GEN>
static int grid_for_g(int block, int trav, int device) {
  if (trav & kTravSplit) return grid_for_t<kTravSplitLocal, GEN>(block, device);  // split or several objects
  if (trav == kTravLocal) return grid_for_t<kTravLocal, GEN>(block, device);
  return grid_for_t<kTravGrid, GEN>(block, device);
}

static int grid_for(int block, int trav, bool gen, int device) {
  return gen ? grid_for_g<true>(block, trav, device) : grid_for_g<false>(block, trav, device);
}

template <int TRAV, bool GEN>
static void launch_batch_t(int block, int grid, const JobDev* jobs, const long long* begins, int n, long long total,
                           int chunk, int shade_min, unsigned long long* counters, cudaStream_t st) {
  switch (block) {
    case 64: k_batch<64, TRAV, GEN><<<grid, 64, 0, st>>>(jobs, begins, n, total, chunk, shade_min, counters); break;
    case 256: k_batch<256, TRAV, GEN><<<grid, 256, 0, st>>>(jobs, begins, n, total, chunk, shade_min, counters); break;
    default: k_batch<128, TRAV, GEN><<<grid, 128, 0, st>>>(jobs, begins, n, total, chunk, shade_min, counters); break;
  }
}

template <bool GEN>
static void launch_batch_g(int block, int trav, int grid, const JobDev* jobs, const long long* begins, int n,
                           long long total, int chunk, int shade_min, unsigned long long* counters, cudaStream_t st) {
  if (trav & kTravSplit)
    launch_batch_t<kTravSplitLocal, GEN>(block, grid, jobs, begins, n, total, chunk, shade_min, counters, st);
  else if (trav == kTravLocal)
    launch_batch_t<kTravLocal, GEN>(block, grid, jobs, begins, n, total, chunk, shade_min, counters, st);
  else
    launch_batch_t<kTravGrid, GEN>(block, grid, jobs, begins, n, total, chunk, shade_min, counters, st);
}

static cudaError_t launch_batch(int block, int trav, bool gen, int grid, const JobDev* jobs, const long long* begins,
                                int n, long long total, int chunk, int shade_min, unsigned long long* counters,
                                cudaStream_t st) {
  if (gen) launch_batch_g<true>(block, trav, grid, jobs, begins, n, total, chunk, shade_min, counters, st);
  else launch_batch_g<false>(block, trav, grid, jobs, begins, n, total, chunk, shade_min, counters, st);
  return cudaGetLastError();
}

gpss_status check_opts(const gpss_render_opts* o);

}  // namespace gpss

using namespace gpss;

struct gpss_batch_s {
  int device = 0;
  int n = 0;
  std::vector<gpss_scene> scenes;
  std::vector<CameraDev> cams;
  std::vector<PathArgs> args;
  std::vector<long long> begins;   // n + 1 path offsets
  long long total = 0;
  JobDev* table_host = nullptr;    // pinned: the table as last uploaded
  JobDev* table_dev = nullptr;
  long long* begins_dev = nullptr;
  unsigned long long* counters = nullptr;  // kCntNum counters + cursor
  cudaEvent_t uploaded = nullptr;  // the last table copy has left table_host
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool table_valid = false;
  int trav = kTravGrid;            // the union of the jobs' traversal kinds (trav_of bits)
  bool gen = false;                // some job's scene needs the general kernel instances
  int block = 128, shade_min = kBatchDefaultShade, chunk = kBatchDefaultChunk, grid = 0;
};

static void free_batch(gpss_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->uploaded) cudaEventDestroy(b->uploaded);
  cudaFreeHost(b->table_host);
  cudaFree(b->table_dev);
  cudaFree(b->begins_dev);
  cudaFree(b->counters);
  delete b;
}

// Fills `out` (n jobs) with the batch's jobs, films as given.
static void fill_table(const gpss_batch_s* b, JobDev* out, float* const* images, float* const* sqsums) {
  for (int i = 0; i < b->n; ++i) {
    JobDev j;
    std::memset(&j, 0, sizeof(j));  // padding too: tables are compared bytewise
    j.S = scene_dev(b->scenes[i]);
    j.C = b->cams[i];
    j.P = b->args[i];
    j.image = images ? images[i] : nullptr;
    j.sqsum = sqsums ? sqsums[i] : nullptr;
    out[i] = j;
  }
}

// Times one launch shape on a tuning table: one launch (the paths and their random
// numbers are fixed, so repeats differ only by scheduling noise), preceded by an
// untimed one the first time a block size runs (module load).  Returns the time
// in ms, or -1 with *err set.
static float time_shape(gpss_batch b, int block, int shade_min, int chunk, const JobDev* jobs, const long long* begins,
                        long long total, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, bool warm,
                        cudaError_t* err) {
  const int grid = grid_for(block, b->trav, b->gen, b->device);
  float ms = 0.0f;
  for (int rep = warm ? 0 : 1; rep < 2; ++rep) {
    cudaMemsetAsync(b->counters, 0, 16 * sizeof(unsigned long long), st);
    cudaEventRecord(e0, st);
    if ((*err = launch_batch(block, b->trav, b->gen, grid, jobs, begins, b->n, total, chunk, shade_min, b->counters, st)) != cudaSuccess)
      return -1.0f;
    cudaEventRecord(e1, st);
    if ((*err = cudaEventSynchronize(e1)) != cudaSuccess) return -1.0f;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  return ms;
}

// Coordinate descent over (block, shade_min, chunk) on a reduced-spp copy of the
// batch; stops early (keeping the best shape so far) once the timed launches
// have taken kTuneBudgetMs.
static gpss_status autotune(gpss_batch b, cudaStream_t st) {
  int div = (int)std::min<long long>((b->total + kTunePaths - 1) / kTunePaths, 1 << 20);
  if (div < 1) div = 1;
  std::vector<PathArgs> targs(b->args);
  std::vector<long long> tbeg(b->n + 1, 0);
  size_t film = 0;
  for (int i = 0; i < b->n; ++i) {
    PathArgs& P = targs[i];
    P.spp = std::max(1, P.spp / div);
    P.total = (long long)P.npix * P.spp;
    P.inv_spp = 1.0f / (float)P.spp;
    tbeg[i + 1] = tbeg[i] + P.total;
    film = std::max(film, 3 * (size_t)P.npix);
  }
  float* scratch = nullptr;
  JobDev* tjobs = nullptr;
  long long* tbegins = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gpss_status status = GPSS_OK;
  cudaError_t e;
  std::vector<JobDev> host(b->n);
  // one film shared by all jobs of the tuning copy: its contents are never read
  if ((e = cudaMalloc(&scratch, film * sizeof(float))) != cudaSuccess) { status = cuda_fail(e, "tuning film"); goto done; }
  if ((e = cudaMalloc(&tjobs, b->n * sizeof(JobDev))) != cudaSuccess) { status = cuda_fail(e, "tuning table"); goto done; }
  if ((e = cudaMalloc(&tbegins, (b->n + 1) * sizeof(long long))) != cudaSuccess) {
    status = cuda_fail(e, "tuning offsets");
    goto done;
  }
  for (int i = 0; i < b->n; ++i) {
    std::memset(&host[i], 0, sizeof(JobDev));
    host[i].S = scene_dev(b->scenes[i]);
    host[i].C = b->cams[i];
    host[i].P = targs[i];
    host[i].image = scratch;
  }
  cudaMemcpyAsync(tjobs, host.data(), b->n * sizeof(JobDev), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(tbegins, tbeg.data(), (b->n + 1) * sizeof(long long), cudaMemcpyHostToDevice, st);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  {
    const long long ttotal = tbeg[b->n];
    struct Cand { int block, shade, chunk; };
    const Cand start{128, kBatchDefaultShade, kBatchDefaultChunk};
    Cand best = start;
    bool warmed[3] = {false, false, false};  // block 64 / 128 / 256
    auto slot = [](int blk) { return blk == 64 ? 0 : blk == 128 ? 1 : 2; };
    float spent = 0.0f;
    float best_ms = time_shape(b, best.block, best.shade, best.chunk, tjobs, tbegins, ttotal, st, e0, e1, true, &e);
    if (best_ms < 0.0f) { status = cuda_fail(e, "tuning launch"); goto done; }
    warmed[1] = true;
    spent += best_ms;
    const int blocks[] = {64, 256};
    const int shades[] = {8, 16, 32};
    const int chunks[] = {64, 128, 512, 1024};
    for (int axis = 0; axis < 3; ++axis) {
      const int* vals = axis == 0 ? blocks : axis == 1 ? shades : chunks;
      const int nv = axis == 0 ? 2 : axis == 1 ? 3 : 4;
      const Cand base = best;
      for (int v = 0; v < nv && spent < kTuneBudgetMs; ++v) {
        Cand c = base;
        if (axis == 0) c.block = vals[v];
        else if (axis == 1) c.shade = vals[v];
        else c.chunk = vals[v];
        const bool warm = !warmed[slot(c.block)];
        const float t = time_shape(b, c.block, c.shade, c.chunk, tjobs, tbegins, ttotal, st, e0, e1, warm, &e);
        if (t < 0.0f) { status = cuda_fail(e, "tuning launch"); goto done; }
        warmed[slot(c.block)] = true;
        spent += warm ? 2.0f * t : t;
        if (t < kTuneMargin * best_ms) {
          best_ms = t;
          best = c;
        }
      }
    }
    b->block = best.block;
    b->shade_min = best.shade;
    b->chunk = best.chunk;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(scratch);
  cudaFree(tjobs);
  cudaFree(tbegins);
  return status;
}

static gpss_status capture_graph(gpss_batch b) {
  cudaError_t e;
  if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(e, "begin capture");
  cudaMemsetAsync(b->counters, 0, 16 * sizeof(unsigned long long), b->capture);
  k_zero_films<<<dim3(64, b->n), 256, 0, b->capture>>>(b->table_dev);
  cudaError_t le = launch_batch(b->block, b->trav, b->gen, b->grid, b->table_dev, b->begins_dev, b->n, b->total, b->chunk,
                                b->shade_min, b->counters, b->capture);
  e = cudaStreamEndCapture(b->capture, &b->graph);
  if (le != cudaSuccess) return cuda_fail(le, "batch launch (capture)");
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
  return GPSS_OK;
}

extern "C" gpss_status gpss_batch_create(const gpss_scene* scenes, const gpss_camera* cams,
                                         const gpss_render_opts* opts, int n, int block_size, gpss_stream stream,
                                         gpss_batch* out) {
  if (!out) { set_error("null output handle"); return GPSS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!scenes || !cams || !opts) { set_error("null scenes, cameras or options"); return GPSS_ERR_INVALID_ARG; }
  if (n < 1 || n > kBatchMaxJobs) { set_error("batch size %d outside 1..%d", n, kBatchMaxJobs); return GPSS_ERR_INVALID_ARG; }
  if (block_size != 0 && block_size != 64 && block_size != 128 && block_size != 256) {
    set_error("block size %d: use 0 (autotune), 64, 128 or 256", block_size);
    return GPSS_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  gpss_batch b = new gpss_batch_s;
  b->device = dev;
  b->n = n;
  b->scenes.assign(scenes, scenes + n);
  b->cams.resize(n);
  b->args.resize(n);
  b->begins.assign(n + 1, 0);
  gpss_status st;
  for (int i = 0; i < n; ++i) {
    if (!scenes[i]) { set_error("scene %d is null", i); free_batch(b); return GPSS_ERR_INVALID_ARG; }
    if (scenes[i]->device != dev) {
      set_error("scene %d lives on device %d, the current device is %d", i, scenes[i]->device, dev);
      free_batch(b);
      return GPSS_ERR_UNSUPPORTED;
    }
    if ((st = check_opts(&opts[i])) != GPSS_OK) { free_batch(b); return st; }
    if (opts[i].flags & ~GPSS_FLAG_EXACT_VNDF) {
      set_error("batch job %d: only GPSS_FLAG_EXACT_VNDF is accepted in a batch", i);
      free_batch(b);
      return GPSS_ERR_INVALID_ARG;
    }
    if (!camera_dev(&cams[i], &b->cams[i])) { free_batch(b); return GPSS_ERR_INVALID_ARG; }
    b->trav |= trav_of(scene_dev(scenes[i]));
    if (scene_general(scene_dev(scenes[i]))) b->gen = true;
    PathArgs& P = b->args[i];
    P.spp = opts[i].spp;
    P.max_bounces = opts[i].max_bounces;
    P.seed = opts[i].seed;
    P.mix_R = opts[i].mix_R;
    P.npix = b->cams[i].width * b->cams[i].height;
    P.total = (long long)P.npix * P.spp;
    P.inv_spp = 1.0f / (float)P.spp;
    P.shade_min = kBatchDefaultShade;
    P.exact_vndf = (opts[i].flags & GPSS_FLAG_EXACT_VNDF) ? 1 : 0;
    b->begins[i + 1] = b->begins[i] + P.total;
  }
  b->total = b->begins[n];
  if (check_path_total(b->total, 1, "paths in the batch") != GPSS_OK) { free_batch(b); return GPSS_ERR_INVALID_ARG; }
  cudaStream_t cs = (cudaStream_t)stream;
  if ((e = cudaMallocHost(&b->table_host, n * sizeof(JobDev))) != cudaSuccess ||
      (e = cudaMalloc(&b->table_dev, n * sizeof(JobDev))) != cudaSuccess ||
      (e = cudaMalloc(&b->begins_dev, (n + 1) * sizeof(long long))) != cudaSuccess ||
      (e = cudaMalloc(&b->counters, 16 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) != cudaSuccess) {
    st = cuda_fail(e, "batch allocation");
    free_batch(b);
    return st;
  }
  if ((e = cudaMemcpyAsync(b->begins_dev, b->begins.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice, cs)) !=
      cudaSuccess) {
    st = cuda_fail(e, "offsets upload");
    free_batch(b);
    return st;
  }
  if (block_size == 0) {
    if ((st = autotune(b, cs)) != GPSS_OK) { free_batch(b); return st; }
  } else {
    b->block = block_size;
  }
  b->grid = grid_for(b->block, b->trav, b->gen, dev);
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) { st = cuda_fail(e, "batch setup"); free_batch(b); return st; }
  if ((st = capture_graph(b)) != GPSS_OK) { free_batch(b); return st; }
  *out = b;
  return GPSS_OK;
}

extern "C" gpss_status gpss_batch_render(gpss_batch b, float* const* images, float* const* sqsums, gpss_stats* stats,
                                         gpss_stream stream) {
  if (!b || !images) { set_error("null batch or images"); return GPSS_ERR_INVALID_ARG; }
  for (int i = 0; i < b->n; ++i)
    if (!images[i]) { set_error("image %d is null", i); return GPSS_ERR_INVALID_ARG; }
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e;
  std::vector<JobDev> want(b->n);
  fill_table(b, want.data(), images, sqsums);
  if (!b->table_valid || std::memcmp(want.data(), b->table_host, b->n * sizeof(JobDev)) != 0) {
    // the previous copy must have left the pinned staging before it is overwritten
    if ((e = cudaEventSynchronize(b->uploaded)) != cudaSuccess) return cuda_fail(e, "table staging");
    std::memcpy(b->table_host, want.data(), b->n * sizeof(JobDev));
    if ((e = cudaMemcpyAsync(b->table_dev, b->table_host, b->n * sizeof(JobDev), cudaMemcpyHostToDevice, cs)) !=
        cudaSuccess)
      return cuda_fail(e, "table upload");
    if ((e = cudaEventRecord(b->uploaded, cs)) != cudaSuccess) return cuda_fail(e, "table event");
    b->table_valid = true;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (stats) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, cs);
  }
  if ((e = cudaGraphLaunch(b->exec, cs)) != cudaSuccess) return cuda_fail(e, "graph launch");
  if (stats) {
    cudaEventRecord(ev1, cs);
    unsigned long long c[16];
    if ((e = cudaMemcpyAsync(c, b->counters, sizeof(c), cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
      return cuda_fail(e, "stats copy");
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "batch render");
    fill_stats(stats, c, 0.0f);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    stats->ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  return GPSS_OK;
}

extern "C" gpss_status gpss_batch_config(gpss_batch b, int* block_size, int* shade_min, int* chunk, int* grid) {
  if (!b) { set_error("null batch"); return GPSS_ERR_INVALID_ARG; }
  if (block_size) *block_size = b->block;
  if (shade_min) *shade_min = b->shade_min;
  if (chunk) *chunk = b->chunk;
  if (grid) *grid = b->grid;
  return GPSS_OK;
}

extern "C" gpss_status gpss_batch_destroy(gpss_batch b) {
  if (!b) return GPSS_OK;
  // graph launches may still run on the caller's streams: wait for the device
  cudaDeviceSynchronize();
  free_batch(b);
  return GPSS_OK;
}
