/*
 * gpss.h -- C-ABI of the GB300 (sm_103a) renderer for Gaussian process
 * statistical surfaces (GPSS), after "Macrofacet Theory for Gaussian Process
 * Statistical Surfaces" (Huang, Cui, Wang, Yan).
 *
 * A GPSS object is a Gaussian process f ~ GP(mu(x), kappa) with the
 * squared-exponential kernel (Eq. se_kernel).  The library renders it as the
 * classic exponential participating medium the paper derives (Sec. 4):
 *   extinction   sigma_t(x,d) = rho(x) sigma(d)          (Eq. generalized_sigma_t)
 *   density      rho = phi(mu;0,sigma^2)/Phi(mu;0,sigma^2)  (Eq. macro_sigma_t)
 *   proj. area   sigma(d) = Lambda(d) cos(theta)           (Eq. generalized_lambda)
 *   NDF          D(m) = int_0^inf t^3 P(t m) dt            (Eq. gdf_to_ndf, macro_ndf)
 *   phase        p(d,d') = F D_d(m) / (4 |d.m|)            (Eq. phase, microfacet_vndf)
 * with per-pixel Monte Carlo path tracing ("null scattering", Sec. 5): delta
 * tracking, ratio-tracking next-event estimation, and the mixture sampler of
 * Sec. 4.2 (Beckmann visible normals with probability R, else uniform).
 *
 * Conventions
 *  - d is the marching direction of a ray (the paper's omega_o for extinction;
 *    for the phase function omega_o = incoming d, omega_i = outgoing d').
 *  - Grids are node-centred over the object's box, x fastest:
 *    index = i + nx*(j + ny*k); fields are interpolated trilinearly and the
 *    normal direction is the gradient of the interpolated mean.
 *  - Unless stated otherwise, pointers to per-element data are DEVICE pointers
 *    and every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream).  The caller owns every buffer it passes.
 *  - Errors: every function returns a gpss_status; no exception crosses the
 *    ABI.  Arguments are validated before any work is queued; a failing call
 *    leaves outputs unspecified.  gpss_last_error() gives a message for the
 *    calling thread.  CUDA faults surface as GPSS_ERR_CUDA on the call that
 *    observes them.
 */
#ifndef GPSS_H
#define GPSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpss_scene_s* gpss_scene;
typedef struct gpss_batch_s* gpss_batch;
typedef void* gpss_stream; /* cudaStream_t */

typedef enum {
  GPSS_OK = 0,
  GPSS_ERR_INVALID_ARG = 1,
  GPSS_ERR_CUDA = 2,
  GPSS_ERR_OOM = 3,
  GPSS_ERR_TIMEOUT = 4,
  GPSS_ERR_UNSUPPORTED = 5
} gpss_status;

/* One GPSS object.  mean/variance/albedo (and tangent, correlation_scale) may be
 * host or device memory (they are copied by gpss_scene_create / gpss_scene_update
 * with cudaMemcpyDefault). */
typedef struct {
  int nx, ny, nz;              /* nodes per axis, each >= 2                        */
  float bbox_min[3], bbox_max[3];
  const float* mean;           /* nx*ny*nz mean mu (a signed distance)             */
  const float* variance;       /* nx*ny*nz variance sigma^2, finite and > 0        */
  const float* albedo;         /* albedo_channels planes of nx*ny*nz, F in [0,1]   */
  int albedo_channels;         /* 1 or 3                                           */
  float length_scale;          /* SE correlation l_t > 0 (Eq. roughness)           */
  int ndf;                     /* gpss_ndf: the macrofacet's NDF                   */
  /* Anisotropic and non-stationary kernels (optional; zero/NULL = the isotropic
   * stationary kernel).  The gradient of the GPSS at x has the covariance
   * sigma^2 diag(1/l_t^2, 1/l_b^2, 1/l_n^2) in the local frame (t, b, n) of Sec. 4.2
   * (the paper's alpha_x, alpha_y, alpha_z = sqrt(2) sigma/l_t, /l_b, /l_n), where
   * n = grad mu/|grad mu| (world z where grad mu = 0), t = the tangent field's
   * component orthogonal to n (any unit vector orthogonal to n where it vanishes)
   * and b = n x t.  Every l is multiplied by the correlation-scale factor s(x) > 0
   * (a spatially varying correlation: with length_scale = 1 the grid is l(x)). */
  float length_scale_b;        /* l_b > 0, or 0 for l_t; l_b != l_t needs tangent   */
  float length_scale_n;        /* l_n > 0, or 0 for l_t                             */
  const float* tangent;        /* NULL or 3 planes (x, y, z) of nx*ny*nz, finite;    */
                               /* trilinearly interpolated                         */
  const float* correlation_scale; /* NULL or nx*ny*nz factors s > 0, trilinear     */
} gpss_object_desc;

/* NDF of an object.  GPSS_NDF_GPSS: the generalized macrofacet of the GPSS
 * (Sec. 4.2, Eq. generalized_sigma_t / macro_ndf).  The height-field macrofacets
 * of Sec. 4.1 keep the density rho and take the projected area Lambda(w)cos(theta)
 * (continued below the horizon by Lambda(-w) = -1 - Lambda(w)) and the phase
 * function of a chosen microfacet NDF about n = grad mu/|grad mu| with roughness
 * alpha = sqrt(2) sigma/l: GPSS_NDF_BECKMANN (the fully anisotropic GPSS with
 * infinite correlation along n) or GPSS_NDF_GGX.  Height-field objects sample their
 * visible normals exactly when the ray arrives from above n (weight F) and the
 * hemisphere uniformly otherwise; mix_R does not apply to them.  The adjoint
 * supports GPSS_NDF_GPSS only.  Height-field objects take the isotropic
 * roughness (l_b = l_n = l_t, no tangent field; a correlation-scale grid is allowed). */
typedef enum { GPSS_NDF_GPSS = 0, GPSS_NDF_BECKMANN = 1, GPSS_NDF_GGX = 2 } gpss_ndf;

typedef enum { GPSS_LIGHT_DIRECTIONAL = 0, GPSS_LIGHT_SKY = 1, GPSS_LIGHT_UNIFORM = 2 } gpss_light_type;

/* Directional: dir = unit vector toward the light, radiance = irradiance (RGB).
 * Sky: for w_z >= 0 lerp((1,1,1), (0.35,0.55,1), w_z), else (0.25,0.22,0.20),
 * times radiance.  Uniform: constant radiance in every direction. */
typedef struct {
  int type;
  float dir[3];
  float radiance[3];
} gpss_light_desc;

typedef enum { GPSS_CAMERA_ORTHO = 0, GPSS_CAMERA_PERSPECTIVE = 1 } gpss_camera_type;

/* forward f = normalize(look_at - eye), right = normalize(f x up),
 * image-up = right x f; pixel (0,0) is the top-left; ndc x = 2(px+jx)/W - 1,
 * y = 1 - 2(py+jy)/H.  Ortho: origin = eye + x ortho_w/2 right + y ortho_h/2 up,
 * direction f.  Perspective: origin eye, direction
 * normalize(f + x tan(fov_y/2) W/H right + y tan(fov_y/2) up). */
typedef struct {
  int type;
  float eye[3], look_at[3], up[3];
  float fov_y_deg, ortho_w, ortho_h;
  int width, height;
} gpss_camera;

/* flags */
#define GPSS_FLAG_KEEP_PATH_RADIANCE 1u /* keep per-path radiance for a later adjoint */
/* Sample the phase function exactly from the GPSS visible-normal distribution
 * max(0,-d.m) D(m)/sigma(d) (slope g ~ max(0,-d.g) N(grad mu, (sigma/l)^2 I),
 * m = g/|g|): weight p/pdf = F exactly, pdf = p/F.  The paper leaves this sampling
 * open (end of Sec. 4.2) and uses the Beckmann/uniform mixture, the default. */
#define GPSS_FLAG_EXACT_VNDF 2u

typedef struct {
  int spp;                 /* samples per pixel, >= 1                               */
  int max_bounces;         /* max real scattering events per path, >= 1 (no RR)     */
  uint64_t seed;           /* Philox key                                            */
  float mix_R;             /* Beckmann share of the sampling mixture, 0 < R < 1     */
  uint32_t flags;
} gpss_render_opts;

typedef struct {
  uint64_t paths, vertices, null_collisions, shadow_steps, majorant_cells, truncated, aborted;
  uint64_t max_path_events;  /* most tentative collisions of one path (flight + shadow) */
  float ms;                /* device time of the render kernel                      */
  uint64_t nonfinite;      /* adjoint: gradient contributions skipped as not finite  */
} gpss_stats;

/* ---------------------------------------------------------------- scenes */

/* Creates a scene: validates the descriptors, copies the grids into the
 * library's layout ((mean, variance) interleaved per node, albedo planes) and
 * builds the majorant grid (an upper bound of sigma_t over all directions per
 * cell of `majorant_brick` x the finest field cell; 0 selects 1).  1 <= n_objs <= 4.
 * light may be NULL (directional light from +z, irradiance 1).  Synchronises
 * `stream` (device-side validation).  INVALID_ARG on bad sizes, non-positive or
 * non-finite variance, albedo outside [0,1], channels not 1/3, l <= 0, a
 * correlation-scale factor <= 0 or non-finite, a non-finite tangent, l_b != l_t
 * without a tangent field, or a height-field object with an anisotropic kernel. */
gpss_status gpss_scene_create(const gpss_object_desc* objs, int n_objs, const gpss_light_desc* light,
                              int majorant_brick, gpss_stream stream, gpss_scene* out);
/* Re-copies the grids (same sizes as at creation) and rebuilds the majorant.  The
 * kernel description may change; an object that gains a tangent field or a
 * correlation-scale grid gets its device copy allocated here. */
gpss_status gpss_scene_update(gpss_scene s, const gpss_object_desc* objs, int n_objs, gpss_stream stream);
/* Empty-space skipping of the majorant traversal: each majorant cell stores the
 * largest radius r in {0, 1, 2, ..., 2^(skip_levels-1)} whose cube of (2r+1)^3
 * cells has a max majorant M_r with M_r * r * h_min <= kappa; a ray crosses such
 * a cube in one step at M_r.  skip_levels in [0, 6] (0 disables skipping),
 * kappa >= 0.  Defaults: 5 and 0.5.  Every choice is unbiased; they trade
 * traversal steps against null collisions (the autotuner's knobs). */
gpss_status gpss_scene_set_traversal(gpss_scene s, int skip_levels, float kappa, gpss_stream stream);
/* Warp scheduling of the render kernel: a warp shades its lanes that reached a
 * real scattering vertex once at least `shade_min` (1..32) of them wait, or no
 * other lane can advance.  Default 24.  Results do not depend on it. */
gpss_status gpss_scene_set_schedule(gpss_scene s, int shade_min);
/* Per-object traversal of scenes of several objects (enable = 1; the default 0
 * walks the union grid everywhere).  The faces of the objects' boxes cut each ray
 * into intervals: an interval inside one box walks that object's own majorant grid
 * (its node spacing, its local majorants when it is thin), an interval inside
 * several boxes walks the union grid (the objects' majorants added), intervals in
 * no box are skipped, and the exponential optical-depth budget carries from one
 * interval to the next.  The union grid alone has the finest spacing over the whole
 * union box, coarsened to stay below 64 Mi cells, which loosens the majorants of
 * objects whose own grids are finer.  Unbiased either way; the grids are built at
 * creation for scenes of several objects.  Measured on the GB300 it takes 44% fewer
 * extinction evaluations on the three-object surface-to-volume scene but 1.7x the
 * time (the walk reads its grid's parameters per step with a per-lane object index),
 * hence off by default; it pays where a thin object shares a scene (its local
 * majorants then apply).  No counterpart in the paper (a traversal
 * structure of this implementation). */
gpss_status gpss_scene_set_object_grids(gpss_scene s, int enable);
/* Local majorants for thin shells (single-object scenes, and each object of a scene
 * of several on its own grid under gpss_scene_set_object_grids): in a
 * majorant cell whose grid majorant times the rest of the ray's segment in the
 * cell exceeds `hot` expected tentative collisions, the traversal bounds sigma_t
 * over shorter pieces computed from the field cell at the piece's start: along
 * the ray the trilinear mean falls at most at a rate B fixed by the cell's edge
 * differences, so sigma_t <= rho_ub(mu(x) - B l) (B + alpha/(2 sqrt(pi))) over a
 * piece of length l (gpss_eval_local_majorant returns these bounds).  This keeps
 * delta/ratio tracking near a surface-like shell (sigma much smaller than the
 * grid spacing) at a few tentative collisions per crossing.  hot >= 0, 0
 * disables; default 4.  Every choice is unbiased. */
gpss_status gpss_scene_set_local_majorant(gpss_scene s, float hot);
/* Surface-limit analytic free flight in the local pieces (enable = 1; the default 0
 * keeps constant pieces, which are as tight and cheaper once the local projected-area
 * bound sigma(d) <= a psi(-B/a) applies).  Where the mean rises along the ray (rays
 * leaving a shell; B < 0 bounds its decrease rate), a piece's majorant follows the
 * linear lower bound mu(t) >= mu0 - B (t - t0) to the cell's exit:
 * sbar(t) = K lambda(u)/sigma_lo, u = (mu0 - B (t - t0))/sigma_u, with sigma_u =
 * sigma_lo while u < 0 and sigma_hi after (lambda the inverse Mills ratio, K the
 * projected-area bound).  Its optical depth, K sigma_u/(sigma_lo B) times a difference
 * of ln Phi (Smith's height form of Sec. 4.1), is inverted in closed form, so the
 * tentative collisions follow the density's decay instead of the start point's
 * density held over the cell (gpss_eval_local_piece returns these pieces).  Unbiased
 * either way. */
gpss_status gpss_scene_set_surface_flight(gpss_scene s, int enable);
/* Frees the scene.  Call after the stream's work on it has completed. */
gpss_status gpss_scene_destroy(gpss_scene s);
/* Majorant grid geometry: dims[3] cells and their values (device copy, may be NULL). */
gpss_status gpss_scene_majorant(gpss_scene s, int dims[3], float* values, gpss_stream stream);

/* ---------------------------------------------------------------- rendering */

/* Forward render (Sec. 5 integrator on the Sec. 4 medium).  image: H*W*3 floats,
 * overwritten with the per-pixel mean radiance; sqsum (nullable): H*W*3 floats,
 * overwritten with the per-pixel sum over samples of the squared path radiance.
 * image/sqsum may be device or host memory (host: rendered into a scene-owned
 * film, then copied back).  stats (host, nullable): filled after the stream is
 * synchronised.  With GPSS_FLAG_KEEP_PATH_RADIANCE the scene keeps each path's
 * radiance for gpss_render_adjoint with the same camera and options; that render runs
 * in the adjoint's own kernel (same estimator, about 1.3x the plain render's time), so
 * that the adjoint's replay repeats its decisions bit for bit.  Path (pixel p,
 * sample j) draws its random numbers from Philox counters keyed by (p, j); the
 * resident threads take paths in 16x16-pixel tiles, all samples of a tile together,
 * which changes only the order of the film's float additions. */
gpss_status gpss_render(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts, float* image,
                        float* sqsum, gpss_stats* stats, gpss_stream stream);

/* Forward render that allocates no device memory during the call (the paper has
 * no counterpart; it is an integration aid).  For callers that may not allocate
 * at render time: applications that account for every device byte themselves
 * (a hidden cudaMalloc would break their budget), and real-time loops where an
 * allocation's latency or failure is unacceptable.  Same result as gpss_render with
 * the same scene, camera and options (image only: no sqsum, no per-path
 * radiance, stats->ms = 0).  The work counters and a film of at most 65536
 * pixels (e.g. 256 x 256) live in a fixed 0.8 MB static device array that every
 * GPU loading the library keeps until the process exits; larger images are
 * rejected with GPSS_ERR_INVALID_ARG, and so are renders of more than 2^46 paths
 * (W*H*spp), as in gpss_render.  image: W*H*3 floats, host or device; a host
 * image (pinned or pageable) and stats are complete when the call returns (the
 * stream is synchronised), a device image is written asynchronously on `stream`.
 * The first call on a device looks up the array's device address (make that
 * first call before any stream capture).  All calls share the array and clear
 * it before use: calls that overlap on the GPU race and must be serialised by
 * the caller. */
gpss_status gpss_render_noalloc(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts, float* image,
                                gpss_stats* stats, gpss_stream stream);

/* Path-replay adjoint (gradients of the image's expectation).  d_image: H*W*3
 * (dLoss/dimage, device).  Gradients are ACCUMULATED (+=) into d_mean, d_variance
 * and d_correlation_scale (the nodes of every object, one object's grid after the
 * other in object order), d_albedo (each object's channel planes, objects in order)
 * and d_length_scale (one float per object: its l_t); any output may be NULL.
 * d_correlation_scale needs some object with a correlation-scale grid (the others'
 * parts stay untouched), INVALID_ARG otherwise.  Objects with the GPSS NDF and an
 * isotropic kernel only (UNSUPPORTED otherwise; the correlation-scale grid is
 * supported).  The paths are those of gpss_render with equal camera and options:
 * if the scene kept their per-path radiance (GPSS_FLAG_KEEP_PATH_RADIANCE on that
 * render, 12 bytes per path, no scene update since) it is reused, else the forward
 * paths are traced first.  Nothing else is kept: each shadow ray is replayed from
 * its random numbers, first for its final transmittance, then for its gradient.
 * stats->aborted counts replayed paths that did not reproduce their forward
 * radiance (expected 0); stats->nonfinite the gradient contributions skipped
 * because their coefficients were not finite (expected ~0).  Method: path replay
 * backpropagation (Vicini et al. 2021) of the Sec. 5 estimator on the Sec. 4
 * medium; the partials of Eq. generalized_sigma_t, Eq. macro_ndf and Eq. phase. */
gpss_status gpss_render_adjoint(gpss_scene s, const gpss_camera* cam, const gpss_render_opts* opts,
                                const float* d_image, float* d_mean, float* d_variance, float* d_albedo,
                                float* d_length_scale, float* d_correlation_scale, gpss_stats* stats,
                                gpss_stream stream);

/* ---------------------------------------------------------------- batches */

/* A batch renders n scenes, each with its own camera and options, in ONE launch
 * of the persistent path kernel, replayed from a captured CUDA graph.  The paths
 * of all scenes form one index space (scene i's paths follow scene i-1's, each
 * scene in gpss_render's order: 16x16-pixel tiles, all samples of a tile
 * together) that the resident threads consume in chunks through one atomic
 * cursor; each path carries the index of its scene in a device table of (scene,
 * camera, options, film pointers).  Scene i's path indices and random numbers are
 * those of gpss_render(scenes[i], cams[i], opts[i]), so the batch estimates each
 * image with the separate render's per-pixel error; the two kernels are separate
 * compilations and may round a rare decision differently (approximate FP32
 * division), so the images agree up to the film's summation order except in a few
 * pixels.  Repeated batch launches agree exactly.  No counterpart in the paper (an
 * execution-model feature).
 *
 *   scenes, cams, opts: n entries each (copied; the scenes must stay alive and
 *     unchanged in layout while the batch exists, and live on the current device;
 *     a scene may appear several times).  opts[i].flags: 0 or GPSS_FLAG_EXACT_VNDF.
 *   n: 1..4096.
 *   block_size: 0 = autotune: block size (64/128/256 threads) x shading threshold
 *     x chunk size, each candidate timed on this batch with its spp reduced so
 *     that one launch traces at most ~8M paths (takes up to a few seconds; the
 *     scratch films are freed before return).  64, 128 or 256: that block size
 *     with the default threshold (24) and chunk (256), no tuning.
 *   stream: the stream tuning runs on (the graph is captured on a private one).
 * INVALID_ARG on a bad argument, UNSUPPORTED for scenes on another device. */
gpss_status gpss_batch_create(const gpss_scene* scenes, const gpss_camera* cams, const gpss_render_opts* opts,
                              int n, int block_size, gpss_stream stream, gpss_batch* out);
/* Renders the batch on `stream` (one graph launch: counter clear, film clear, the
 * persistent kernel).  images[i]: device buffer of H_i*W_i*3 floats, overwritten
 * with the mean radiance.  sqsums: NULL, or n entries each NULL or a device buffer
 * of H_i*W_i*3 floats receiving the per-pixel sum of squared path radiance.  The
 * film pointers are written into the device table (one small host-to-device copy)
 * only when they differ from the previous call's.  stats (host, nullable): sums
 * over all scenes; stats->ms = device time of the graph launch (synchronises). */
gpss_status gpss_batch_render(gpss_batch b, float* const* images, float* const* sqsums, gpss_stats* stats,
                              gpss_stream stream);
/* The launch shape in use: threads per block, shading threshold (lanes a warp
 * gathers before shading), chunk (paths per cursor fetch) and grid (blocks).  Any
 * output may be NULL. */
gpss_status gpss_batch_config(gpss_batch b, int* block_size, int* shade_min, int* chunk, int* grid);
/* Waits for the device to finish (graph launches may still be running on the
 * caller's streams), then frees the batch.  NULL is a no-op. */
gpss_status gpss_batch_destroy(gpss_batch b);

/* ---------------------------------------------------------------- deterministic evaluators
 * Per-query kernels used by the parity tests; all arrays are device memory. */

/* The local majorant that the traversal uses on a ray piece starting at
 * org + t0 dir (object 0; see gpss_scene_set_local_majorant): t_end[i] (piece end,
 * at most t_max[i]; t_end <= t0 when the start is outside the object's box) and
 * sbar[i], an upper bound of sigma_t on [t0, t_end].  All arrays device, n
 * entries (org3, dir3: n*3; dir unit length). */
gpss_status gpss_eval_local_majorant(gpss_scene s, int n, const float* org3, const float* dir3, const float* t0,
                                     const float* t_max, float* t_end, float* sbar, gpss_stream stream);
/* The local piece the traversal takes at org + t0 dir with surface-limit flight on
 * (see gpss_scene_set_surface_flight; no cap from the grid majorant): t_end[i], lin[i]
 * (1: linear-exponential majorant, 0: constant), depth[i] = the majorant's optical
 * depth over [t0, t_end], and for the optical depth tau[i] < depth[i] the tentative
 * collision t_hit[i] and the majorant there sbar_hit[i] (t_hit = t_end, sbar_hit = the
 * majorant at t_end otherwise).  All arrays device, n entries (org3, dir3: n*3). */
gpss_status gpss_eval_local_piece(gpss_scene s, int n, const float* org3, const float* dir3, const float* t0,
                                  const float* t_max, const float* tau, float* t_end, int* lin, float* depth,
                                  float* t_hit, float* sbar_hit, gpss_stream stream);
/* Exact visible-normal sample of object k's phase function at x (see
 * GPSS_FLAG_EXACT_VNDF): uniforms u3 (n*3) -> d_out3 (n*3), w3_out = F per channel
 * (n*3; zero where no sample), pdf_out = p/F over d_out (n). */
gpss_status gpss_sample_phase_vndf(gpss_scene s, int object, int n, const float* pos3, const float* d_in3,
                                   const float* u3, float* d_out3, float* w3_out, float* pdf_out, gpss_stream stream);
/* sigma_t(x, d) summed over objects (Eq. generalized_sigma_t); pos3, dir3: n*3. */
gpss_status gpss_eval_sigma_t(gpss_scene s, int n, const float* pos3, const float* dir3, float* out,
                              gpss_stream stream);
/* Phase function of object k at x (Eq. phase): p3_out n*3 (includes F per channel),
 * pdf_out n (density of the sampling mixture over d_out). */
gpss_status gpss_eval_phase(gpss_scene s, int object, int n, const float* pos3, const float* d_in3,
                            const float* d_out3, float mix_R, float* p3_out, float* pdf_out, gpss_stream stream);
/* Samples the mixture with the given uniforms u3 (n*3): d_out3, weight p/pdf (n*3; pdf the
 * density the sample was drawn from), pdf (n): the mixture pdf evaluated from d_out as
 * gpss_eval_phase evaluates it (the value the renderer's MIS weights use; 0 where the
 * half vector re-derived from d_out, nearly equal to d_in, no longer faces -d_in). */
gpss_status gpss_sample_phase(gpss_scene s, int object, int n, const float* pos3, const float* d_in3,
                              const float* u3, float mix_R, float* d_out3, float* w3_out, float* pdf_out,
                              gpss_stream stream);
/* NDF in the paper's local frame, mean gradient (0,0,G), roughness ax, ay, az (Eq. macro_ndf). */
gpss_status gpss_eval_ndf(int n, const float* m3, float G, float ax, float ay, float az, float* out,
                          gpss_stream stream);
/* Projected area sigma(w) in the same frame (Eq. generalized_lambda times cos). */
gpss_status gpss_eval_projected_area(int n, const float* w3, float G, float ax, float ay, float az, float* out,
                                     gpss_stream stream);
/* Transmittance exp(-int_0^tmax sigma_t) by per-cell Gauss-Legendre quadrature (Eq. sm2tr). */
gpss_status gpss_eval_transmittance(gpss_scene s, int n, const float* org3, const float* dir3, const float* tmax,
                                    float* out, gpss_stream stream);
/* Ratio-tracking estimate of the same transmittance (mean of `samples` estimates),
 * using the renderer's majorant traversal. */
gpss_status gpss_estimate_transmittance(gpss_scene s, int n, const float* org3, const float* dir3,
                                        const float* tmax, int samples, uint64_t seed, float* mean_out,
                                        gpss_stream stream);
/* Delta-tracking free-flight distances along each ray (INFINITY = no collision),
 * `samples` per ray: out n*samples. */
gpss_status gpss_sample_free_flight(gpss_scene s, int n, const float* org3, const float* dir3, int samples,
                                    uint64_t seed, float* out, gpss_stream stream);
/* Philox4x32-10 (Salmon et al. 2011): ctr4 n*4, key2 n*2, out4 n*4 (uint32). */
gpss_status gpss_philox4x32_10(int n, const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4,
                               gpss_stream stream);

/* Message of the last failing call on this thread ("" if none). */
const char* gpss_last_error(void);
/* Library version, (major << 16) | minor. */
int gpss_version(void);

#ifdef __cplusplus
}
#endif
#endif
