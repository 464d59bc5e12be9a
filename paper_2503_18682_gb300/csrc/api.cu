// C ABI of the RayGS library (declared in include/raygs.h): plans over a caller-owned
// workspace, the hot-path entry points, counters and CUDA-graph batching.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "raygs_internal.cuh"

using namespace raygs;

namespace {
thread_local int g_last_cuda_error = 0;

raygs_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = int(e);
  return RAYGS_ERR_CUDA;
}
}  // namespace

void raygs::note_cuda_error(cudaError_t e) { g_last_cuda_error = int(e); }

struct raygs_plan {
  std::vector<raygs_camera> cams;
  std::vector<DevCam> dcams;
  int64_t total_pixels = 0;
  Work w;
  int stage = 0;  // 0 idle, 1 preprocessed, 2 binned
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

void raygs_config_default(raygs_config *cfg) {
  if (!cfg) return;
  cfg->p_min = 1.0f / 255.0f;
  cfg->t_stop = 1e-4f;
  cfg->alpha_max = 0.99f;
  cfg->mip_sigma2 = 0.1f;
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->fp64_degenerate = 1;
  cfg->degenerate_ratio = 1e3f;
  cfg->enable_backward = 0;
  cfg->divergence = RAYGS_DIV_RAY;
  cfg->batch_records = 1;
}

const char *raygs_status_string(raygs_status s) {
  switch (s) {
    case RAYGS_OK: return "ok";
    case RAYGS_ERR_INVALID_ARG: return "invalid argument";
    case RAYGS_ERR_CAPACITY: return "workspace too small";
    case RAYGS_ERR_CUDA: return "CUDA error";
    case RAYGS_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

int raygs_last_cuda_error(void) { return g_last_cuda_error; }

raygs_status raygs_plan_create(const raygs_camera *cams, int32_t n_views, int64_t n_gaussians,
                               int64_t max_instances, const raygs_config *cfg_in, raygs_plan **out) {
  if (!out) return RAYGS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cams || n_views < 1 || n_views > RAYGS_MAX_VIEWS) return RAYGS_ERR_INVALID_ARG;
  if (n_gaussians < 0 || n_gaussians >= (int64_t(1) << 31)) return RAYGS_ERR_INVALID_ARG;
  if (int64_t(n_views) * n_gaussians >= (int64_t(1) << 32) - 1) return RAYGS_ERR_INVALID_ARG;
  if (max_instances < 0 || max_instances >= (int64_t(1) << 32) - 4 * kEmitTile) return RAYGS_ERR_INVALID_ARG;
  raygs_config cfg;
  if (cfg_in) cfg = *cfg_in; else raygs_config_default(&cfg);
  if (!config_valid(cfg)) return RAYGS_ERR_INVALID_ARG;
  for (int v = 0; v < n_views; ++v)
    if (!camera_valid(cams[v])) return RAYGS_ERR_INVALID_ARG;
  raygs_plan *p = new (std::nothrow) raygs_plan();
  if (!p) return RAYGS_ERR_INVALID_ARG;
  p->cams.assign(cams, cams + n_views);
  p->dcams.resize(n_views);
  int64_t tb = 0, trows = 0, pb = 0;
  int max_tx = 0;
  if (!plan_views(cams, n_views, cfg, p->dcams.data(), tb, trows, pb, max_tx)) {
    delete p;
    return RAYGS_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  cudaGetLastError();  // clear a "no device" error of the probe on GPU-less hosts
  Work &w = p->w;
  w.n_views = n_views;
  w.n = n_gaussians;
  w.tiles = tb;
  w.trows = trows;
  w.max_tiles_x = max_tx;
  w.cap = max_instances;
  w.num_sms = sms;
  w.G = sort_grid(sms);
  w.cfg = cfg;
  w.L = make_layout(n_views, n_gaussians, tb, trows, max_instances, w.G, max_tx, cfg.enable_backward != 0,
                    cams[0].mip == RAYGS_MIP_EXACT);
  p->total_pixels = pb;
  *out = p;
  return RAYGS_OK;
}

void raygs_plan_destroy(raygs_plan *plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  delete plan;
}

size_t raygs_plan_workspace_bytes(const raygs_plan *plan) { return plan ? plan->w.L.total : 0; }

raygs_status raygs_plan_bind(raygs_plan *plan, void *workspace, size_t bytes) {
  if (!plan || !workspace) return RAYGS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return RAYGS_ERR_INVALID_ARG;
  if (bytes < plan->w.L.total) return RAYGS_ERR_CAPACITY;
  plan->w.base = static_cast<char *>(workspace);
  cudaError_t e = cudaMemcpy(plan->w.base + plan->w.L.cams, plan->dcams.data(),
                             sizeof(DevCam) * plan->w.n_views, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemset(plan->w.base + plan->w.L.counters, 0, sizeof(Counters));
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 0;
  return RAYGS_OK;
}

raygs_status raygs_plan_set_poses(raygs_plan *plan, const raygs_camera *cams, void *stream) {
  if (!plan || !cams || !plan->w.base) return RAYGS_ERR_INVALID_ARG;
  for (int v = 0; v < plan->w.n_views; ++v) {
    const raygs_camera &c = cams[v], &o = plan->cams[v];
    if (c.width != o.width || c.height != o.height || c.fx != o.fx || c.fy != o.fy || c.cx != o.cx ||
        c.cy != o.cy || c.mip != o.mip || c.near_z != o.near_z)
      return RAYGS_ERR_INVALID_ARG;
  }
  for (int v = 0; v < plan->w.n_views; ++v) {
    DevCam d;
    fill_devcam(cams[v], plan->w.cfg, d);
    d.tile_base = plan->dcams[v].tile_base;
    d.trow_base = plan->dcams[v].trow_base;
    d.pix_base = plan->dcams[v].pix_base;
    plan->dcams[v] = d;
    plan->cams[v] = cams[v];
  }
  cudaError_t e = cudaMemcpyAsync(plan->w.base + plan->w.L.cams, plan->dcams.data(),
                                  sizeof(DevCam) * plan->w.n_views, cudaMemcpyHostToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

int64_t raygs_plan_num_pixels(const raygs_plan *plan) { return plan ? plan->total_pixels : 0; }
int64_t raygs_plan_num_tiles(const raygs_plan *plan) { return plan ? plan->w.tiles : 0; }
raygs_status raygs_resolve_supersampled(const raygs_plan *plan, int32_t factor, const float *rgb_hi,
                                        const float *T_hi, float *rgb_lo, float *T_lo, void *stream) {
  if (!plan || !rgb_hi || !rgb_lo || factor < 1 || factor > 16) return RAYGS_ERR_INVALID_ARG;
  long long base_lo = 0;
  for (int v = 0; v < plan->w.n_views; ++v) {
    const raygs_camera &c = plan->cams[v];
    if (c.width % factor != 0 || c.height % factor != 0) return RAYGS_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int v = 0; v < plan->w.n_views; ++v) {
    const raygs_camera &c = plan->cams[v];
    const int w_lo = c.width / factor, h_lo = c.height / factor;
    cudaError_t e = launch_resolve(rgb_hi, T_hi, rgb_lo, T_lo, w_lo, h_lo, factor, plan->dcams[v].pix_base, base_lo, st);
    if (e != cudaSuccess) return cuda_fail(e);
    base_lo += (long long)w_lo * h_lo;
  }
  return RAYGS_OK;
}

int64_t raygs_plan_pixel_offset(const raygs_plan *plan, int32_t view) {
  if (!plan || view < 0 || view >= plan->w.n_views) return -1;
  return plan->dcams[view].pix_base;
}

raygs_status raygs_preprocess(raygs_plan *plan, const raygs_scene *scene, void *stream) {
  if (!plan || !plan->w.base) return RAYGS_ERR_INVALID_ARG;
  raygs_status s = scene_valid(scene, plan->w.n);
  if (s != RAYGS_OK) return s;
  cudaError_t e = run_preprocess(plan->w, *scene, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 1;
  return RAYGS_OK;
}

raygs_status raygs_bin_sort(raygs_plan *plan, void *stream) {
  if (!plan || !plan->w.base) return RAYGS_ERR_INVALID_ARG;
  if (plan->stage < 1) return RAYGS_ERR_STATE;
  cudaError_t e = run_bin_sort(plan->w, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 2;
  return RAYGS_OK;
}

static raygs_status render_impl(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib, bool count,
                                void *stream) {
  if (!plan || !plan->w.base || !rgb) return RAYGS_ERR_INVALID_ARG;
  if (plan->stage < 2) return RAYGS_ERR_STATE;
  cudaError_t e = run_render(plan->w, rgb, T_final, n_contrib, count, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

raygs_status raygs_render(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib, void *stream) {
  return render_impl(plan, rgb, T_final, n_contrib, false, stream);
}

raygs_status raygs_read_counters(raygs_plan *plan, raygs_counters *out, void *stream) {
  if (!plan || !plan->w.base || !out) return RAYGS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Counters h;
  cudaError_t e =
      cudaMemcpyAsync(&h, plan->w.base + plan->w.L.counters, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  out->n_visible = h.n_visible;
  // when the tile rows overflowed, the instance total is incomplete: report the larger need
  const unsigned long long cap = (unsigned long long)plan->w.cap;
  out->n_instances = int64_t(h.n_rows > cap && h.n_rows > h.n_instances ? h.n_rows : h.n_instances);
  out->capacity = plan->w.cap;
  out->n_nonfinite = int64_t(h.n_nonfinite);
  out->overflow = int32_t(h.overflow);
  out->pad = 0;
  out->n_rows = int64_t(h.n_rows);
  out->n_rows_kept = int64_t(h.n_rows_kept);
  return RAYGS_OK;
}

raygs_status raygs_graph_capture(raygs_plan *plan, const raygs_scene *scene, float *rgb, float *T_final,
                                 int32_t *n_contrib, void *stream) {
  if (!plan || !plan->w.base || !rgb) return RAYGS_ERR_INVALID_ARG;
  raygs_status s = scene_valid(scene, plan->w.n);
  if (s != RAYGS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (st == nullptr) return RAYGS_ERR_INVALID_ARG;  // capture needs a non-default stream
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  raygs_status r1 = raygs_preprocess(plan, scene, stream);
  raygs_status r2 = r1 == RAYGS_OK ? raygs_bin_sort(plan, stream) : r1;
  raygs_status r3 = r2 == RAYGS_OK ? raygs_render(plan, rgb, T_final, n_contrib, stream) : r2;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  if (r3 != RAYGS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r3;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  plan->exec = exec;
  return RAYGS_OK;
}

raygs_status raygs_graph_launch(raygs_plan *plan, void *stream) {
  if (!plan || !plan->exec) return RAYGS_ERR_STATE;
  cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

raygs_status raygs_render_backward(raygs_plan *plan, const raygs_scene *scene, const float *T_final,
                                   const int32_t *n_contrib, const float *dL_drgb, const float *dL_dT,
                                   const raygs_grads *grads, void *stream) {
  if (!plan || !plan->w.base || !T_final || !n_contrib || !dL_drgb || !grads) return RAYGS_ERR_INVALID_ARG;
  if (!plan->w.cfg.enable_backward) return RAYGS_ERR_STATE;
  if (plan->stage < 2) return RAYGS_ERR_STATE;
  for (const raygs_camera &c : plan->cams)
    if (c.mip) return RAYGS_ERR_INVALID_ARG;  // no derivative of the anti-aliasing term
  raygs_status s = scene_valid(scene, plan->w.n);
  if (s != RAYGS_OK) return s;
  cudaError_t e = run_backward(plan->w, *scene, T_final, n_contrib, dL_drgb, dL_dT, *grads,
                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

/* ------------------------------------------------------------------ diagnostics
 * Not part of the documented ABI: an instrumented render that also counts, into
 * host_counts[0..3], evaluated and composited (pixel, primitive) pairs, the list entries the
 * rasteriser staged before its tiles stopped (consumed instances) and its (thread, record)
 * iterations; and raw access to the binning buffers for tests. */
raygs_status raygs_debug_render_counted(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib,
                                        unsigned long long *host_counts, void *stream) {
  raygs_status s = render_impl(plan, rgb, T_final, n_contrib, true, stream);
  if (s != RAYGS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(host_counts, plan->w.base + plan->w.L.evals, 4 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

/* Device pointers of internal buffers (valid after bin_sort):
 * which: 0 depth keys [V*N], 1 rects [V*N] (uint2), 2 records [V*N] (64 B),
 *        3 sorted pair ids [n_visible], 4 support rows sorted by tile row [n_rows_kept]
 *        (uint2: sorted pair position, first tile column | run length << 16),
 *        5 instance lists (sorted pair positions, tile by tile), 6 tile ranges [tiles] (uint2),
 *        7 support ellipses [V*N] (32 B), 8 raw counters, 9 per-tile stop positions of the
 *        last instrumented render [tiles] (kCulled: the list ran out first) */
void *raygs_debug_buffer(raygs_plan *plan, int which) {
  if (!plan || !plan->w.base) return nullptr;
  const Work &w = plan->w;
  switch (which) {
    case 0: return w.base + w.L.depth;
    case 1: return w.base + w.L.rect;
    case 2: return w.base + w.L.rec;
    case 3: return w.base + w.L.s1v[w.s1_final];
    case 4: return w.base + w.L.rv[w.s2_rows];
    case 5: return w.base + w.L.inst;
    case 6: return w.base + w.L.ranges;
    case 7: return w.base + w.L.ell;
    case 8: return w.base + w.L.counters;
    case 9: return w.base + w.L.tstop;
  }
  return nullptr;
}

}  // extern "C"
