/*
 * raygs.h -- C ABI of the GB300 (sm_103a) renderer for ray-based Gaussian splatting.
 *
 * The library renders the RayGS image of Sec. 3.2 (Eq. Q_ray, Eq. rend_opacity,
 * Eq. rendering) of "Hardware-Rasterized Ray-Based Gaussian Splatting" (arXiv 2503.18682),
 * with the paper's per-primitive vertex stage (Sec. 4.1: the smallest enclosing 3D quad,
 * Eq. V_ray) used to bin primitives into screen tiles, its fragment formula (Sec. 4.2,
 * App. A.4) evaluated per pixel, and the approximate anti-aliasing of Sec. 5 (Eq. mip).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Ownership: the caller allocates every buffer.  Device buffers (marked "device") are
 *    read or written by kernels; the library never calls cudaMalloc/cudaFree.  Host-side
 *    plan objects are the only thing the library allocates (plain malloc/new).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work is enqueued on it asynchronously; no entry point synchronises unless
 *    its comment says so.
 *  - Errors: every entry point returns a raygs_status and never aborts or throws.
 *    RAYGS_ERR_INVALID_ARG is returned before any work is enqueued.  RAYGS_ERR_CUDA means a
 *    CUDA call failed; raygs_last_cuda_error() returns its cudaError_t.  Conditions found
 *    on the device (instance capacity exceeded, non-finite attributes) are recorded in
 *    device counters and reported by raygs_read_counters().
 *  - Camera model: pinhole (Sec. 3.1), OpenCV axes (x right, y down, z forward),
 *    x_cam = R x_world + t; pixel (i, j) is the ray ((i+0.5-cx)/fx, (j+0.5-cy)/fy, 1).
 *  - Primitive parameters (Sec. 3, "Scene representation"): mean, rotation quaternion
 *    (w, x, y, z; normalised internally), log of the diagonal scale, opacity logit
 *    (o = sigmoid), colour as spherical-harmonic coefficients whose first coefficient is
 *    the base RGB colour (rgb = max(0, k_0 + sum_{l>=1} Y_lm(d) k_lm), real SH without the
 *    Condon-Shortley phase, d = unit vector from the camera centre to the mean, world frame).
 *  - Image outputs are float32, views concatenated in order; view v starts at pixel
 *    raygs_plan_pixel_offset(plan, v) and is row-major [H][W].
 */
#ifndef RAYGS_H
#define RAYGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RAYGS_MAX_VIEWS 64

typedef enum {
  RAYGS_OK = 0,
  RAYGS_ERR_INVALID_ARG = 1, /* null pointer, bad size or dtype, misaligned buffer, ... */
  RAYGS_ERR_CAPACITY = 2,    /* workspace too small for the plan */
  RAYGS_ERR_CUDA = 3,        /* a CUDA runtime call failed (see raygs_last_cuda_error) */
  RAYGS_ERR_STATE = 4        /* call out of order (e.g. render before bin_sort) */
} raygs_status;

typedef enum { RAYGS_F32 = 0, RAYGS_F16 = 1, RAYGS_BF16 = 2 } raygs_dtype;

/* Primitive set S of Sec. 3 ("Scene representation"), structure of arrays, device memory.
 * Every pointer must be 16-byte aligned. */
typedef struct {
  int64_t n;                  /* number of primitives, 0 <= n < 2^31 */
  const float *means;         /* [n][3] float32, world frame */
  const void *log_scales;     /* [n][3] in scale_dtype */
  const float *quats;         /* [n][4] float32 (w, x, y, z), any nonzero norm */
  const void *opacity_logits; /* [n] in opacity_dtype */
  const void *sh;             /* [n][K][3] in sh_dtype, K = (sh_degree + 1)^2 */
  int32_t sh_degree;          /* 0..3 */
  int32_t scale_dtype;        /* raygs_dtype: F32, F16 or BF16 */
  int32_t opacity_dtype;      /* raygs_dtype: F32 or F16 */
  int32_t sh_dtype;           /* raygs_dtype: F32, F16 or BF16 */
} raygs_scene;

/* Anti-aliasing of a view (Sec. 5).
 *   RAYGS_MIP_OFF:    none.
 *   RAYGS_MIP_APPROX: Eq. mip, the pixel-invariant Sigma^ = Sigma + lambda I with
 *                     lambda = mip_sigma2 |mu|^2 / (fx fy) and the opacity modulated by
 *                     sqrt(|Sigma| c^2 / (|Sigma^| c^^2)).
 *   RAYGS_MIP_EXACT:  the pixel-dependent form that Eq. mip approximates: per pixel ray x,
 *                     Sigma^_x = Sigma + sigma_x^2 tau(x)^2 I with sigma_x^2 = mip_sigma2
 *                     cos^3(theta_x) / (fx fy) and tau(x) the ray's maximum-density depth;
 *                     omega = o m(x) exp(-D_ray(x; mu, Sigma^_x) / 2) with
 *                     m(x) = sqrt(|Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x)).
 *                     A plan's views are either all EXACT or none; no backward. */
typedef enum { RAYGS_MIP_OFF = 0, RAYGS_MIP_APPROX = 1, RAYGS_MIP_EXACT = 2 } raygs_mip;

/* One pinhole view (Sec. 3.1). */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height; /* 1 .. 32768 each */
  float R[9];            /* world -> camera rotation, row-major */
  float t[3];
  float near_z;          /* primitives whose centre depth is <= near_z are culled (Sec. 4.1) */
  int32_t mip;           /* raygs_mip */
} raygs_camera;

/* The divergence D that weighs a primitive at a pixel, omega = o exp(-D/2).
 *   RAYGS_DIV_RAY: D_ray of Sec. 3.2 (Eq. Q_ray), the Mahalanobis distance of the density
 *                  maximum along the pixel ray, with the camera-inside skip of Eq. c.
 *   RAYGS_DIV_GS:  D_gs of Sec. 3.1, the Mahalanobis distance of the pixel centre from the
 *                  projected mean under Sigma_pi = J Sigma J^T (EWA splatting, J the
 *                  Jacobian of the pinhole projection at the mean); no Eq. c skip. */
typedef enum { RAYGS_DIV_RAY = 0, RAYGS_DIV_GS = 1 } raygs_divergence;

/* Renderer settings.  raygs_config_default() fills the documented defaults. */
typedef struct {
  float p_min;            /* support cut-off of Eq. support (default 1/255) */
  float t_stop;           /* compositing stops before T would drop below this (1e-4) */
  float alpha_max;        /* rendered opacity clamp (0.99) */
  float mip_sigma2;       /* sigma^2 of Sec. 5 in pixel^2 at unit distance (0.1) */
  int32_t tile_w, tile_h; /* screen tile in pixels: 16x16 (default), 16x8, 32x16 or 8x8 */
  int32_t fp64_degenerate; /* FP64 vertex stage for near-degenerate primitives (scale
                              ratio max/min > degenerate_ratio): 0 never; 1 (default) in
                              the views where the float32 solve is ill-conditioned (seen
                              nearly edge-on); 2 in every view where they are visible.
                              Whatever the setting, a pair whose skip decision (opacity at
                              the cut-off, camera inside, Sec. 3.2 Eq. c) lies within the
                              float32 rounding of its threshold is decided in FP64 */
  float degenerate_ratio; /* 1e3 */
  int32_t enable_backward; /* 1: reserve workspace for raygs_render_backward (default 0) */
  int32_t batch_records;  /* records the rasteriser stages in shared memory per thread and
                             batch: 1 (default) or 2 */
  int32_t divergence;     /* raygs_divergence: RAYGS_DIV_RAY (default) or RAYGS_DIV_GS.  GS
                             refuses enable_backward and cameras with mip != 0 (INVALID_ARG) */
} raygs_config;

/* Device-side counters of the last preprocess / bin_sort / render sequence. */
typedef struct {
  int64_t n_visible;    /* (primitive, view) pairs that survived culling */
  int64_t n_instances;  /* (primitive, tile) instances emitted (may exceed capacity) */
  int64_t capacity;     /* instance capacity of the plan */
  int64_t n_nonfinite;  /* primitives culled because an attribute was NaN/Inf */
  int32_t overflow;     /* 1 when n_instances > capacity: the image is incomplete */
  int32_t pad;
  int64_t n_rows;       /* (pair, tile row) support rows, including empty ones */
  int64_t n_rows_kept;  /* support rows that hold at least one tile */
} raygs_counters;

/* Reference-gradient outputs of raygs_render_backward: float32 device buffers laid out
 * like the matching scene attributes.  Any pointer may be NULL to skip that gradient. */
typedef struct {
  float *d_means;          /* [n][3] */
  float *d_log_scales;     /* [n][3] */
  float *d_quats;          /* [n][4]  (gradient w.r.t. the un-normalised quaternion) */
  float *d_opacity_logits; /* [n] */
  float *d_sh;             /* [n][K][3] */
} raygs_grads;

typedef struct raygs_plan raygs_plan;

/* ---------------------------------------------------------------- configuration */

/* Fill *cfg with the defaults listed in raygs_config. */
void raygs_config_default(raygs_config *cfg);

/* Human-readable name of a status code (static string). */
const char *raygs_status_string(raygs_status s);

/* cudaError_t of the last failed CUDA call in this thread (0 if none). */
int raygs_last_cuda_error(void);

/* ---------------------------------------------------------------- plan / workspace */

/*
 * Create a plan for rendering `n_views` cameras (1..RAYGS_MAX_VIEWS) of a scene with
 * `n_gaussians` primitives, with room for `max_instances` (primitive, tile) pairs.
 * Host-side only; the cameras are copied.  Returns INVALID_ARG for bad sizes/config.
 */
raygs_status raygs_plan_create(const raygs_camera *cams, int32_t n_views, int64_t n_gaussians,
                               int64_t max_instances, const raygs_config *cfg,
                               raygs_plan **out);

/* Release a plan (host memory only; the caller frees its workspace). NULL is a no-op. */
void raygs_plan_destroy(raygs_plan *plan);

/* Bytes of device workspace the plan needs (256-byte aligned start required). */
size_t raygs_plan_workspace_bytes(const raygs_plan *plan);

/* Attach a caller-owned device workspace of at least raygs_plan_workspace_bytes() bytes
 * and upload the cameras (synchronous H2D copy on the default stream; not for the hot path).
 * Returns CAPACITY if `bytes` is too small, INVALID_ARG if misaligned. */
raygs_status raygs_plan_bind(raygs_plan *plan, void *workspace, size_t bytes);

/* Replace the camera poses (R, t) of all views; sizes and intrinsics must not change.
 * Enqueued as an async H2D copy on `stream` from host memory the library owns. */
raygs_status raygs_plan_set_poses(raygs_plan *plan, const raygs_camera *cams, void *stream);

int64_t raygs_plan_num_pixels(const raygs_plan *plan);          /* sum of W*H over views */
int64_t raygs_plan_pixel_offset(const raygs_plan *plan, int32_t view);
int64_t raygs_plan_num_tiles(const raygs_plan *plan);           /* screen tiles, all views */

/* ---------------------------------------------------------------- hot path */

/*
 * Per-primitive vertex stage for every view (Sec. 3 activation; Sec. 3.2 Eq. c skip;
 * Sec. 5 Eq. mip; Sec. 4.1 and App. A.1-A.3 quad V_ray -> screen tile rectangle; the
 * per-pixel factors of the fragment formula of Sec. 4.2 / App. A.4; colour from SH).
 * With RAYGS_DIV_GS the records instead hold Sigma_pi^-1 of Sec. 3.1 and the tile
 * rectangle bounds the screen ellipse of the EWA support.  With RAYGS_MIP_EXACT views the
 * record is 128 bytes (the per-pixel forms of the exact anti-aliasing) and the rectangle
 * bounds the support of the primitive inflated by a bound of the per-ray smoothing.
 * Reads the scene, writes per-(primitive, view) depth keys, tile rectangles, support
 * ellipses and pixel records into the workspace.  Requires a bound plan and
 * scene->n == n_gaussians.
 */
raygs_status raygs_preprocess(raygs_plan *plan, const raygs_scene *scene, void *stream);

/*
 * Binning for Eq. rendering's depth order: stable on-device radix sort of the visible
 * (primitive, view) pairs by float32 centre depth (ties keep primitive order); per pair and
 * tile row of its rectangle, the run of tiles whose pixel centres can meet its support;
 * stable radix sort of those rows by global tile row; per tile row, the expansion of its
 * rows into per-tile instance lists in depth order and the per-tile [start, end) ranges.
 * The instance total and an overflow flag go to device counters.  Requires
 * raygs_preprocess on the same stream first.
 */
raygs_status raygs_bin_sort(raygs_plan *plan, void *stream);

/*
 * Per-tile rasterisation: for every pixel, the ray-maximum divergence D_ray in closed form
 * (Sec. 4.2 fragment formula with the quad coordinate obtained from the pixel ray; D_gs of
 * Sec. 3.1 with RAYGS_DIV_GS; the exact anti-aliased form of Sec. 5 for RAYGS_MIP_EXACT
 * views), omega = min(alpha_max, o exp(-D/2)) when D <= kappa (Eq. rend_opacity, Eq.
 * support), and front-to-back compositing (Eq. rendering) stopping before T < t_stop.
 *   rgb       [num_pixels][3] float32 device, required
 *   T_final   [num_pixels]    float32 device, optional (NULL): final transmittance
 *   n_contrib [num_pixels]    int32 device, optional (NULL): 1 + position of the last
 *             composited instance in the pixel's tile list (0 if none); needed by backward
 */
raygs_status raygs_render(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib,
                          void *stream);

/*
 * Supersampled anti-aliasing (a box-filter counterpart of the paper's MSAA comparison,
 * Sec. 6; not part of its method): the plan's views were rendered at `factor` times the
 * resolution (each camera's width, height, fx, fy, cx and cy multiplied by factor, so that a
 * pixel's factor x factor block holds its sub-pixel rays).  Writes, per view in plan order,
 * the mean of every block: rgb_lo [sum of (W/factor)(H/factor)][3] and, when both T
 * pointers are non-NULL, T_lo likewise.  All buffers are caller-owned device memory.
 * RAYGS_ERR_INVALID_ARG when a view's width or height is not a multiple of factor or
 * factor is outside 1..16.
 */
raygs_status raygs_resolve_supersampled(const raygs_plan *plan, int32_t factor, const float *rgb_hi,
                                        const float *T_hi, float *rgb_lo, float *T_lo, void *stream);

/*
 * Gradients of a scalar loss L through raygs_render back to the scene parameters
 * (not in the paper, whose renderer is not differentiable; reverse mode of Eq. rendering,
 * Eq. rend_opacity and Eq. Q_ray).  Uses the workspace of the preceding forward pass (same
 * plan, scene unchanged, no instance overflow).  dL_drgb [num_pixels][3] device required;
 * dL_dT [num_pixels] optional.  T_final and n_contrib are the forward outputs.  Gradient
 * buffers are overwritten (not accumulated); gradients of views are summed.  Requires
 * cfg.enable_backward (else RAYGS_ERR_STATE); views with the MIP filter are not
 * differentiated (RAYGS_ERR_INVALID_ARG).
 */
raygs_status raygs_render_backward(raygs_plan *plan, const raygs_scene *scene,
                                   const float *T_final, const int32_t *n_contrib,
                                   const float *dL_drgb, const float *dL_dT,
                                   const raygs_grads *grads, void *stream);

/* Synchronise `stream` and read the device counters of the last sequence. */
raygs_status raygs_read_counters(raygs_plan *plan, raygs_counters *out, void *stream);

/* ---------------------------------------------------------------- batching */

/*
 * Capture raygs_preprocess + raygs_bin_sort + raygs_render for this plan, scene and
 * outputs into a CUDA graph held by the plan (replaces a previous one).  The scene and
 * output pointers are baked in; their contents may change between launches.
 */
raygs_status raygs_graph_capture(raygs_plan *plan, const raygs_scene *scene, float *rgb,
                                 float *T_final, int32_t *n_contrib, void *stream);

/* Launch the captured graph on `stream`. */
raygs_status raygs_graph_launch(raygs_plan *plan, void *stream);

/*
 * Autotuner for the batched launch: for every compiled tile shape (16x16, 16x8, 32x16,
 * 8x8 pixels) and shared-memory batch (1 or 2 records per rasteriser thread), in that
 * order (shape-major), build a plan over `workspace` (caller-owned, at least
 * raygs_autotune_workspace_bytes() bytes), run one untimed pass, skip the candidate if its
 * instances overflow `max_instances`, then time `iters` passes of preprocess + bin_sort +
 * render with CUDA events on `stream`.  Writes the fastest candidate into
 * cfg_inout->tile_w/tile_h/batch_records and, if ms_out is non-NULL, the mean time per pass
 * of each candidate into ms_out[0..7] (-1 when skipped).  Synchronises `stream`.
 * Returns RAYGS_ERR_CAPACITY when no candidate fits.  (Not in the paper.)
 */
raygs_status raygs_autotune(const raygs_camera *cams, int32_t n_views, const raygs_scene *scene,
                            int64_t max_instances, raygs_config *cfg_inout, void *workspace, size_t bytes,
                            float *rgb, float *T_final, int32_t *n_contrib, int32_t iters, void *stream,
                            float *ms_out);

/* Workspace bytes raygs_autotune needs: the largest plan over the candidate shapes. */
size_t raygs_autotune_workspace_bytes(const raygs_camera *cams, int32_t n_views, int64_t n_gaussians,
                                      int64_t max_instances, const raygs_config *cfg);

/* ---------------------------------------------------------------- allocation-free variant */

/* Bytes of the device array raygs_render_noalloc works in (32 MiB). */
#define RAYGS_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/*
 * The same forward render as raygs_preprocess + raygs_bin_sort + raygs_render, for callers
 * that may not allocate device memory: a plugin or engine integration running inside a
 * host application that owns the whole device heap and only hands out its own buffers, or
 * code under a memory budget enforced by an outer allocator.  This entry point allocates
 * nothing (no cudaMalloc/cudaFree, no host heap): all intermediate buffers live in one
 * file-scope device array of RAYGS_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * keeps reserved until the process exits.  The paper has no counterpart; it is a
 * deployment variant of the hot path.
 *
 *  - Inputs/outputs as in raygs_preprocess and raygs_render (caller-owned device buffers);
 *    cams is a host array of n_views cameras; cfg may be NULL for the defaults.  Views with
 *    RAYGS_MIP_EXACT are refused (INVALID_ARG).
 *  - Size limit: the per-(primitive, view) buffers (about 140 bytes each), the tile ranges
 *    and a sort histogram must fit in the array, and the remaining space bounds the
 *    (primitive, tile) instances.  A problem that does not fit is rejected with
 *    RAYGS_ERR_CAPACITY before any work is enqueued; one whose instances overflow the
 *    remaining space returns RAYGS_ERR_CAPACITY after the render (image incomplete).
 *  - Set-up: every call, with the caller's device current, looks up the array's device
 *    address in that device's context; the first call on a device also loads the module
 *    there, so make that first call before any stream capture on that device.
 *  - The call reads a device counter at the end and therefore synchronises `stream`.
 *  - Every call shares the one array, which keeps the last call's contents (the call
 *    clears what must start at zero).  Calls that overlap on the GPU (different streams or
 *    host threads without ordering between them) race on it.
 */
raygs_status raygs_render_noalloc(const raygs_camera *cams, int32_t n_views, const raygs_scene *scene,
                                  const raygs_config *cfg, float *rgb, float *T_final,
                                  int32_t *n_contrib, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RAYGS_H */
