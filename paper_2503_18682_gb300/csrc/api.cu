// C ABI of the RayGS library (declared in include/raygs.h): plans, caller-owned workspace
// carving, the hot-path entry points and CUDA-graph batching.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "raygs_internal.cuh"

using namespace raygs;

namespace raygs {
void note_cuda_error(cudaError_t e);
}

namespace {
thread_local int g_last_cuda_error = 0;


raygs_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = int(e);
  return RAYGS_ERR_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

void raygs::note_cuda_error(cudaError_t e) { g_last_cuda_error = int(e); }

namespace {
int bits_for(uint64_t n) {  // bits needed to represent values < n
  int b = 0;
  while (b < 32 && (uint64_t(1) << b) < n) ++b;
  return b;
}
}  // namespace

struct raygs_plan {
  int n_views = 0;
  int64_t n = 0;
  int64_t capacity = 0;
  raygs_config cfg{};
  std::vector<raygs_camera> cams;
  std::vector<DevCam> dcams;
  int64_t total_tiles = 0, total_pixels = 0;
  int num_sms = 0, G = 0;
  // workspace layout (byte offsets)
  size_t ws_bytes = 0;
  size_t o_cams = 0, o_counters = 0, o_evals = 0, o_depth = 0, o_rect = 0, o_rec = 0;
  size_t o_s1k[2] = {0, 0}, o_s1v[2] = {0, 0}, o_cnt = 0, o_off = 0, o_partial = 0, o_tstart = 0;
  size_t o_ik[2] = {0, 0}, o_iv[2] = {0, 0}, o_hist = 0, o_ranges = 0, o_deg = 0, o_degc = 0;
  uint32_t tstart_len = 0;
  char *ws = nullptr;
  // results of the last bin_sort
  int s1_final = 0, s2_final = 0, s2_passes = 0;
  int stage = 0;  // 0 idle, 1 preprocessed, 2 binned
  // graph
  cudaGraphExec_t exec = nullptr;
  Counters host_counters{};
  std::vector<DevCam> staging;

  template <typename T>
  T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
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

static bool valid_tile(int w, int h) {
  return (w == 16 && h == 16) || (w == 16 && h == 8) || (w == 32 && h == 16) || (w == 8 && h == 8);
}

static void fill_devcam(const raygs_camera &c, const raygs_config &cfg, DevCam &d) {
  std::memset(&d, 0, sizeof(d));
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
  d.ifx = float(1.0 / double(c.fx));
  d.ify = float(1.0 / double(c.fy));
  d.W = c.width; d.H = c.height;
  for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
  d.near_z = c.near_z;
  d.mip = c.mip ? 1 : 0;
  for (int k = 0; k < 3; ++k)
    d.C[k] = float(-(double(c.R[k]) * c.t[0] + double(c.R[3 + k]) * c.t[1] + double(c.R[6 + k]) * c.t[2]));
  d.xmin = float((0.5 - double(c.cx)) / double(c.fx));
  d.xmax = float((double(c.width) - 0.5 - double(c.cx)) / double(c.fx));
  d.ymin = float((0.5 - double(c.cy)) / double(c.fy));
  d.ymax = float((double(c.height) - 0.5 - double(c.cy)) / double(c.fy));
  d.tiles_x = (c.width + cfg.tile_w - 1) / cfg.tile_w;
  d.tiles_y = (c.height + cfg.tile_h - 1) / cfg.tile_h;
}

raygs_status raygs_plan_create(const raygs_camera *cams, int32_t n_views, int64_t n_gaussians,
                               int64_t max_instances, const raygs_config *cfg_in, raygs_plan **out) {
  if (!out) return RAYGS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cams || n_views < 1 || n_views > RAYGS_MAX_VIEWS) return RAYGS_ERR_INVALID_ARG;
  if (n_gaussians < 0 || n_gaussians >= (int64_t(1) << 31)) return RAYGS_ERR_INVALID_ARG;
  if (int64_t(n_views) * n_gaussians >= (int64_t(1) << 32) - 1) return RAYGS_ERR_INVALID_ARG;
  if (max_instances < 0 || max_instances >= (int64_t(1) << 32) - kEmitTile) return RAYGS_ERR_INVALID_ARG;
  raygs_config cfg;
  if (cfg_in) cfg = *cfg_in; else raygs_config_default(&cfg);
  if (!valid_tile(cfg.tile_w, cfg.tile_h)) return RAYGS_ERR_INVALID_ARG;
  if (!(cfg.p_min > 0.f && cfg.p_min < 1.f) || !(cfg.t_stop >= 0.f && cfg.t_stop < 1.f) ||
      !(cfg.alpha_max > 0.f && cfg.alpha_max < 1.f) || !(cfg.mip_sigma2 >= 0.f) ||
      !(cfg.degenerate_ratio > 1.f))
    return RAYGS_ERR_INVALID_ARG;
  for (int v = 0; v < n_views; ++v) {
    const raygs_camera &c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768) return RAYGS_ERR_INVALID_ARG;
    if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy) || !(c.near_z > 0.f))
      return RAYGS_ERR_INVALID_ARG;
  }
  raygs_plan *p = new (std::nothrow) raygs_plan();
  if (!p) return RAYGS_ERR_INVALID_ARG;
  p->n_views = n_views;
  p->n = n_gaussians;
  p->capacity = max_instances;
  p->cfg = cfg;
  p->cams.assign(cams, cams + n_views);
  p->dcams.resize(n_views);
  int64_t tb = 0, pb = 0;
  for (int v = 0; v < n_views; ++v) {
    fill_devcam(cams[v], cfg, p->dcams[v]);
    p->dcams[v].tile_base = int(tb);
    p->dcams[v].pix_base = pb;
    tb += int64_t(p->dcams[v].tiles_x) * p->dcams[v].tiles_y;
    pb += int64_t(cams[v].width) * cams[v].height;
  }
  if (tb >= (int64_t(1) << 31)) { delete p; return RAYGS_ERR_INVALID_ARG; }
  p->total_tiles = tb;
  p->total_pixels = pb;

  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  p->num_sms = sms;
  p->G = 4 * sms;
  if (p->G > 1024) p->G = 1024;

  // workspace layout
  const size_t A = 256;
  const size_t VN = size_t(n_views) * size_t(n_gaussians);
  const size_t cap = size_t(max_instances);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, A); return r; };
  p->o_cams = take(sizeof(DevCam) * n_views);
  p->o_counters = take(sizeof(Counters));
  p->o_evals = take(2 * sizeof(unsigned long long));
  p->o_depth = take(4 * VN);
  p->o_rect = take(8 * VN);
  p->o_rec = take(sizeof(Rec) * VN);
  for (int i = 0; i < 2; ++i) { p->o_s1k[i] = take(4 * VN); p->o_s1v[i] = take(4 * VN); }
  p->o_cnt = take(4 * VN);
  p->o_off = take(4 * VN);
  p->o_partial = take(4 * size_t(p->G));
  p->tstart_len = uint32_t(cap / kEmitTile + 2);
  p->o_tstart = take(4 * size_t(p->tstart_len));
  for (int i = 0; i < 2; ++i) { p->o_ik[i] = take(4 * cap + 16); p->o_iv[i] = take(4 * cap + 16); }
  p->o_hist = take(4 * 256 * size_t(p->G));
  p->o_ranges = take(8 * size_t(tb));
  p->o_deg = take(4 * size_t(n_gaussians));
  p->o_degc = take(4);
  p->ws_bytes = o;
  p->s2_passes = (bits_for(uint64_t(tb)) + 7) / 8;
  *out = p;
  return RAYGS_OK;
}

void raygs_plan_destroy(raygs_plan *plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  delete plan;
}

size_t raygs_plan_workspace_bytes(const raygs_plan *plan) { return plan ? plan->ws_bytes : 0; }

raygs_status raygs_plan_bind(raygs_plan *plan, void *workspace, size_t bytes) {
  if (!plan || !workspace) return RAYGS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return RAYGS_ERR_INVALID_ARG;
  if (bytes < plan->ws_bytes) return RAYGS_ERR_CAPACITY;
  plan->ws = static_cast<char *>(workspace);
  cudaError_t e = cudaMemcpy(plan->ws + plan->o_cams, plan->dcams.data(), sizeof(DevCam) * plan->n_views,
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemset(plan->ws + plan->o_counters, 0, sizeof(Counters));
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 0;
  return RAYGS_OK;
}

raygs_status raygs_plan_set_poses(raygs_plan *plan, const raygs_camera *cams, void *stream) {
  if (!plan || !cams || !plan->ws) return RAYGS_ERR_INVALID_ARG;
  for (int v = 0; v < plan->n_views; ++v) {
    const raygs_camera &c = cams[v], &o = plan->cams[v];
    if (c.width != o.width || c.height != o.height || c.fx != o.fx || c.fy != o.fy || c.cx != o.cx ||
        c.cy != o.cy || c.mip != o.mip || c.near_z != o.near_z)
      return RAYGS_ERR_INVALID_ARG;
  }
  plan->staging = plan->dcams;
  for (int v = 0; v < plan->n_views; ++v) {
    DevCam d;
    fill_devcam(cams[v], plan->cfg, d);
    d.tile_base = plan->dcams[v].tile_base;
    d.pix_base = plan->dcams[v].pix_base;
    plan->staging[v] = d;
    plan->cams[v] = cams[v];
  }
  plan->dcams = plan->staging;
  cudaError_t e = cudaMemcpyAsync(plan->ws + plan->o_cams, plan->dcams.data(), sizeof(DevCam) * plan->n_views,
                                  cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

int64_t raygs_plan_num_pixels(const raygs_plan *plan) { return plan ? plan->total_pixels : 0; }
int64_t raygs_plan_num_tiles(const raygs_plan *plan) { return plan ? plan->total_tiles : 0; }
int64_t raygs_plan_pixel_offset(const raygs_plan *plan, int32_t view) {
  if (!plan || view < 0 || view >= plan->n_views) return -1;
  return plan->dcams[view].pix_base;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static raygs_status check_scene(const raygs_plan *plan, const raygs_scene *s) {
  if (!s || s->n != plan->n) return RAYGS_ERR_INVALID_ARG;
  if (s->sh_degree < 0 || s->sh_degree > 3) return RAYGS_ERR_INVALID_ARG;
  auto dt_ok = [](int d, bool allow_bf16) { return d == RAYGS_F32 || d == RAYGS_F16 || (allow_bf16 && d == RAYGS_BF16); };
  if (!dt_ok(s->scale_dtype, true) || !dt_ok(s->opacity_dtype, false) || !dt_ok(s->sh_dtype, true))
    return RAYGS_ERR_INVALID_ARG;
  if (s->n > 0) {
    if (!s->means || !s->log_scales || !s->quats || !s->opacity_logits || !s->sh) return RAYGS_ERR_INVALID_ARG;
    if (!aligned16(s->means) || !aligned16(s->log_scales) || !aligned16(s->quats) ||
        !aligned16(s->opacity_logits) || !aligned16(s->sh))
      return RAYGS_ERR_INVALID_ARG;
  }
  return RAYGS_OK;
}

raygs_status raygs_preprocess(raygs_plan *plan, const raygs_scene *scene, void *stream) {
  if (!plan || !plan->ws) return RAYGS_ERR_INVALID_ARG;
  raygs_status s = check_scene(plan, scene);
  if (s != RAYGS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(plan->ws + plan->o_counters, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return cuda_fail(e);
  PrepParams P;
  P.means = scene->means;
  P.log_scales = scene->log_scales;
  P.quats = scene->quats;
  P.logits = scene->opacity_logits;
  P.sh = scene->sh;
  P.sh_degree = scene->sh_degree;
  P.scale_dtype = scene->scale_dtype;
  P.opacity_dtype = scene->opacity_dtype;
  P.sh_dtype = scene->sh_dtype;
  P.n = int(plan->n);
  P.n_views = plan->n_views;
  P.cams = plan->at<DevCam>(plan->o_cams);
  P.p_min = plan->cfg.p_min;
  P.mip_sigma2 = plan->cfg.mip_sigma2;
  P.degenerate_ratio = plan->cfg.degenerate_ratio;
  P.fp64_degenerate = plan->cfg.fp64_degenerate;
  P.tile_w = plan->cfg.tile_w;
  P.tile_h = plan->cfg.tile_h;
  P.depth_key = plan->at<uint32_t>(plan->o_depth);
  P.rect = plan->at<uint2>(plan->o_rect);
  P.rec = plan->at<Rec>(plan->o_rec);
  P.counters = plan->at<Counters>(plan->o_counters);
  P.deg_list = plan->at<uint32_t>(plan->o_deg);
  P.deg_count = plan->at<uint32_t>(plan->o_degc);
  e = launch_preprocess(P, plan->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 1;
  return RAYGS_OK;
}

raygs_status raygs_bin_sort(raygs_plan *plan, void *stream) {
  if (!plan || !plan->ws) return RAYGS_ERR_INVALID_ARG;
  if (plan->stage < 1) return RAYGS_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Counters *ctr = plan->at<Counters>(plan->o_counters);
  const uint32_t VN = uint32_t(size_t(plan->n_views) * size_t(plan->n));
  uint32_t *hist = plan->at<uint32_t>(plan->o_hist);
  cudaError_t e;
  // 1. depth sort of the visible pairs: 4 passes of 8 bits over the float32 key
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    SortPass sp;
    sp.keys_in = pass == 0 ? plan->at<uint32_t>(plan->o_depth) : plan->at<uint32_t>(plan->o_s1k[cur]);
    sp.vals_in = pass == 0 ? nullptr : plan->at<uint32_t>(plan->o_s1v[cur]);
    int dst = pass == 0 ? 0 : 1 - cur;
    sp.keys_out = plan->at<uint32_t>(plan->o_s1k[dst]);
    sp.vals_out = plan->at<uint32_t>(plan->o_s1v[dst]);
    sp.d_count = pass == 0 ? nullptr : &ctr->n_visible;
    sp.count_max = VN;
    sp.shift = 8 * pass;
    sp.filter = pass == 0 ? 1 : 0;
    sp.hist = hist;
    sp.G = plan->G;
    sp.d_total = pass == 0 ? &ctr->n_visible : nullptr;
    e = launch_sort_pass(sp, st);
    if (e != cudaSuccess) return cuda_fail(e);
    cur = dst;
  }
  plan->s1_final = cur;
  const uint32_t *pairs = plan->at<uint32_t>(plan->o_s1v[cur]);
  // 2. per-pair tile counts and offsets
  ScanParams S;
  S.pairs = pairs;
  S.rect = plan->at<uint2>(plan->o_rect);
  S.cnt = plan->at<uint32_t>(plan->o_cnt);
  S.off = plan->at<uint32_t>(plan->o_off);
  S.partial = plan->at<uint32_t>(plan->o_partial);
  S.tile_start = plan->at<uint32_t>(plan->o_tstart);
  S.counters = ctr;
  S.capacity = uint32_t(plan->capacity);
  S.tile_start_len = plan->tstart_len;
  e = launch_count_scan(S, plan->G, st);
  if (e != cudaSuccess) return cuda_fail(e);
  // 3. emission in depth order
  EmitParams E;
  E.pairs = pairs;
  E.rect = S.rect;
  E.off = S.off;
  E.tile_start = S.tile_start;
  E.cams = plan->at<DevCam>(plan->o_cams);
  E.counters = ctr;
  E.n = int(plan->n);
  E.keys = plan->at<uint32_t>(plan->o_ik[0]);
  E.vals = plan->at<uint32_t>(plan->o_iv[0]);
  e = launch_emit(E, plan->G, st);
  if (e != cudaSuccess) return cuda_fail(e);
  // 4. stable sort of instances by tile id
  cur = 0;
  for (int pass = 0; pass < plan->s2_passes; ++pass) {
    SortPass sp;
    sp.keys_in = plan->at<uint32_t>(plan->o_ik[cur]);
    sp.vals_in = plan->at<uint32_t>(plan->o_iv[cur]);
    sp.keys_out = plan->at<uint32_t>(plan->o_ik[1 - cur]);
    sp.vals_out = plan->at<uint32_t>(plan->o_iv[1 - cur]);
    sp.d_count = &ctr->n_inst_clamped;
    sp.count_max = uint32_t(plan->capacity);
    sp.shift = 8 * pass;
    sp.filter = 0;
    sp.hist = hist;
    sp.G = plan->G;
    sp.d_total = nullptr;
    e = launch_sort_pass(sp, st);
    if (e != cudaSuccess) return cuda_fail(e);
    cur = 1 - cur;
  }
  plan->s2_final = cur;
  // 5. tile ranges
  uint2 *ranges = plan->at<uint2>(plan->o_ranges);
  e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * size_t(plan->total_tiles), st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_ranges(plan->at<uint32_t>(plan->o_ik[cur]), ctr, ranges, plan->G, st);
  if (e != cudaSuccess) return cuda_fail(e);
  plan->stage = 2;
  return RAYGS_OK;
}

static raygs_status render_impl(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib, bool count,
                                void *stream) {
  if (!plan || !plan->ws || !rgb) return RAYGS_ERR_INVALID_ARG;
  if (plan->stage < 2) return RAYGS_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RenderParams P;
  P.cams = plan->at<DevCam>(plan->o_cams);
  P.n_views = plan->n_views;
  P.ranges = plan->at<uint2>(plan->o_ranges);
  P.inst_vals = plan->at<uint32_t>(plan->o_iv[plan->s2_final]);
  P.pairs = plan->at<uint32_t>(plan->o_s1v[plan->s1_final]);
  P.rec = plan->at<Rec>(plan->o_rec);
  P.t_stop = plan->cfg.t_stop;
  P.alpha_max = plan->cfg.alpha_max;
  P.rgb = rgb;
  P.Tf = T_final;
  P.ncontrib = n_contrib;
  P.eval_counts = plan->at<unsigned long long>(plan->o_evals);
  cudaError_t e;
  if (count) {
    e = cudaMemsetAsync(P.eval_counts, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = launch_render(P, plan->cfg.tile_w, plan->cfg.tile_h, plan->total_tiles, count, st);
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

raygs_status raygs_render(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib, void *stream) {
  return render_impl(plan, rgb, T_final, n_contrib, false, stream);
}

raygs_status raygs_read_counters(raygs_plan *plan, raygs_counters *out, void *stream) {
  if (!plan || !plan->ws || !out) return RAYGS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Counters h;
  cudaError_t e = cudaMemcpyAsync(&h, plan->ws + plan->o_counters, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  out->n_visible = h.n_visible;
  out->n_instances = int64_t(h.n_instances);
  out->capacity = plan->capacity;
  out->n_nonfinite = int64_t(h.n_nonfinite);
  out->overflow = int32_t(h.overflow);
  return RAYGS_OK;
}

raygs_status raygs_graph_capture(raygs_plan *plan, const raygs_scene *scene, float *rgb, float *T_final,
                                 int32_t *n_contrib, void *stream) {
  if (!plan || !plan->ws || !rgb) return RAYGS_ERR_INVALID_ARG;
  raygs_status s = check_scene(plan, scene);
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
  (void)plan; (void)scene; (void)T_final; (void)n_contrib; (void)dL_drgb; (void)dL_dT; (void)grads;
  (void)stream;
  return RAYGS_ERR_STATE;
}

/* ------------------------------------------------------------------ diagnostics
 * Not part of the documented ABI: instrumented render that also counts evaluated and
 * composited (pixel, primitive) pairs, and raw access to the binning buffers for tests. */
raygs_status raygs_debug_render_counted(raygs_plan *plan, float *rgb, float *T_final, int32_t *n_contrib,
                                        unsigned long long *host_counts, void *stream) {
  raygs_status s = render_impl(plan, rgb, T_final, n_contrib, true, stream);
  if (s != RAYGS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(host_counts, plan->ws + plan->o_evals, 2 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  return RAYGS_OK;
}

/* Device pointers of internal buffers (valid after bin_sort):
 * which: 0 depth keys [V*N], 1 rects [V*N] (uint2), 2 records [V*N] (64 B),
 *        3 sorted pair ids [n_visible], 4 instance tile ids [n_instances] (sorted),
 *        5 instance sorted-pair positions, 6 tile ranges [tiles] (uint2),
 *        7 per-pair offsets [n_visible], 8 per-pair tile counts [n_visible] */
void *raygs_debug_buffer(raygs_plan *plan, int which) {
  if (!plan || !plan->ws) return nullptr;
  switch (which) {
    case 0: return plan->ws + plan->o_depth;
    case 1: return plan->ws + plan->o_rect;
    case 2: return plan->ws + plan->o_rec;
    case 3: return plan->ws + plan->o_s1v[plan->s1_final];
    case 4: return plan->ws + plan->o_ik[plan->s2_final];
    case 5: return plan->ws + plan->o_iv[plan->s2_final];
    case 6: return plan->ws + plan->o_ranges;
    case 7: return plan->ws + plan->o_off;
    case 8: return plan->ws + plan->o_cnt;
  }
  return nullptr;
}

}  // extern "C"
