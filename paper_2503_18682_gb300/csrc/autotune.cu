// Launch-configuration autotuner: times the whole hot path (vertex stage, binning,
// rasteriser) for every compiled tile shape and rasteriser batch on the caller's own scene
// and views, in one caller-owned workspace, and keeps the fastest.  Host-side plans only;
// no device memory is allocated.
#include <vector>

#include "raygs_internal.cuh"

using namespace raygs;

namespace {

struct Candidate {
  int tw, th, nb;
};
constexpr Candidate kCandidates[] = {{16, 16, 1}, {16, 16, 2}, {16, 8, 1}, {16, 8, 2},
                                     {32, 16, 1}, {32, 16, 2}, {8, 8, 1},  {8, 8, 2}};
constexpr int kNumCandidates = int(sizeof(kCandidates) / sizeof(kCandidates[0]));

}  // namespace

extern "C" {

size_t raygs_autotune_workspace_bytes(const raygs_camera *cams, int32_t n_views, int64_t n_gaussians,
                                      int64_t max_instances, const raygs_config *cfg_in) {
  raygs_config cfg;
  if (cfg_in) cfg = *cfg_in; else raygs_config_default(&cfg);
  size_t best = 0;
  for (int c = 0; c < kNumCandidates; ++c) {
    cfg.tile_w = kCandidates[c].tw;
    cfg.tile_h = kCandidates[c].th;
    cfg.batch_records = kCandidates[c].nb;
    raygs_plan *p = nullptr;
    if (raygs_plan_create(cams, n_views, n_gaussians, max_instances, &cfg, &p) != RAYGS_OK) return 0;
    size_t b = raygs_plan_workspace_bytes(p);
    raygs_plan_destroy(p);
    if (b > best) best = b;
  }
  return best;
}

raygs_status raygs_autotune(const raygs_camera *cams, int32_t n_views, const raygs_scene *scene,
                            int64_t max_instances, raygs_config *cfg_inout, void *workspace, size_t bytes,
                            float *rgb, float *T_final, int32_t *n_contrib, int32_t iters, void *stream,
                            float *ms_out) {
  if (!cams || !scene || !cfg_inout || !workspace || !rgb || iters < 1) return RAYGS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  raygs_config cfg = *cfg_inout;
  float best_ms = -1.f;
  int best = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    note_cuda_error(e);
    return RAYGS_ERR_CUDA;
  }
  raygs_status result = RAYGS_OK;
  for (int c = 0; c < kNumCandidates && result == RAYGS_OK; ++c) {
    if (ms_out) ms_out[c] = -1.f;
    cfg.tile_w = kCandidates[c].tw;
    cfg.tile_h = kCandidates[c].th;
    cfg.batch_records = kCandidates[c].nb;
    raygs_plan *p = nullptr;
    raygs_status s = raygs_plan_create(cams, n_views, scene->n, max_instances, &cfg, &p);
    if (s != RAYGS_OK) { result = s; break; }
    if (raygs_plan_workspace_bytes(p) > bytes) { raygs_plan_destroy(p); continue; }
    s = raygs_plan_bind(p, workspace, bytes);
    // one untimed pass, then check that the instances fit this candidate's tiles
    if (s == RAYGS_OK) s = raygs_preprocess(p, scene, stream);
    if (s == RAYGS_OK) s = raygs_bin_sort(p, stream);
    if (s == RAYGS_OK) s = raygs_render(p, rgb, T_final, n_contrib, stream);
    raygs_counters ctr;
    if (s == RAYGS_OK) s = raygs_read_counters(p, &ctr, stream);
    if (s != RAYGS_OK) { raygs_plan_destroy(p); result = s; break; }
    if (ctr.overflow) { raygs_plan_destroy(p); continue; }
    cudaEventRecord(e0, st);
    for (int i = 0; i < iters && s == RAYGS_OK; ++i) {
      s = raygs_preprocess(p, scene, stream);
      if (s == RAYGS_OK) s = raygs_bin_sort(p, stream);
      if (s == RAYGS_OK) s = raygs_render(p, rgb, T_final, n_contrib, stream);
    }
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { note_cuda_error(e); s = RAYGS_ERR_CUDA; }
    float ms = 0.f;
    if (s == RAYGS_OK) cudaEventElapsedTime(&ms, e0, e1);
    raygs_plan_destroy(p);
    if (s != RAYGS_OK) { result = s; break; }
    ms /= float(iters);
    if (ms_out) ms_out[c] = ms;
    if (best < 0 || ms < best_ms) { best = c; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != RAYGS_OK) return result;
  if (best < 0) return RAYGS_ERR_CAPACITY;
  cfg_inout->tile_w = kCandidates[best].tw;
  cfg_inout->tile_h = kCandidates[best].th;
  cfg_inout->batch_records = kCandidates[best].nb;
  return RAYGS_OK;
}

}  // extern "C"
