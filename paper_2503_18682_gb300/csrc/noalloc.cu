// Allocation-free forward render.
//
// Some callers cannot allocate device memory: a plugin or engine integration that runs
// inside a host application which owns the whole device heap and only hands it buffers,
// or code under a memory budget enforced by an outer allocator, where a cudaMalloc from a
// library is forbidden.  For them raygs_render_noalloc renders a small scene with every
// intermediate buffer (per-view records, sort keys, instance lists, tile ranges, counters)
// carved from one file-scope device array of fixed size: the library allocates nothing,
// neither device memory (no cudaMalloc/cudaFree) nor host heap.
//
// The array is a module-scope __device__ variable: every GPU that loads this library keeps
// kNoAllocScratchBytes of device memory reserved for it until the process exits.
#include "raygs_internal.cuh"

namespace raygs {

constexpr size_t kNoAllocScratchBytes = RAYGS_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace raygs

using namespace raygs;

namespace {

// Device address of the scratch array in the current device's context.  Host code cannot
// use the symbol itself (it names a host-side shadow).  The lookup is made on every call:
// it is cheap once the module is loaded, and it stays right if the context was destroyed
// and created again (cudaDeviceReset), where the array may sit at a new address.  The
// first call on a device loads the module there.
raygs_status scratch_for_current_device(void **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    note_cuda_error(e);
    return RAYGS_ERR_CUDA;
  }
  *out = p;
  return RAYGS_OK;
}

}  // namespace

extern "C" raygs_status raygs_render_noalloc(const raygs_camera *cams, int32_t n_views, const raygs_scene *scene,
                                             const raygs_config *cfg_in, float *rgb, float *T_final,
                                             int32_t *n_contrib, void *stream) {
  if (!cams || !scene || !rgb || n_views < 1 || n_views > RAYGS_MAX_VIEWS) return RAYGS_ERR_INVALID_ARG;
  raygs_config cfg;
  if (cfg_in) cfg = *cfg_in; else raygs_config_default(&cfg);
  cfg.enable_backward = 0;
  if (!config_valid(cfg)) return RAYGS_ERR_INVALID_ARG;
  const int64_t n = scene->n;
  if (n < 0 || n >= (int64_t(1) << 31)) return RAYGS_ERR_INVALID_ARG;
  raygs_status s = scene_valid(scene, n);
  if (s != RAYGS_OK) return s;

  // Per-view constants, on the stack (no heap).
  DevCam dc[RAYGS_MAX_VIEWS];
  int64_t tiles = 0, trows = 0, pixels = 0;
  int max_tx = 0;
  if (!plan_views(cams, n_views, cfg, dc, tiles, trows, pixels, max_tx)) return RAYGS_ERR_INVALID_ARG;
  if (cams[0].mip == RAYGS_MIP_EXACT) return RAYGS_ERR_INVALID_ARG;  // needs the second record buffer

  void *scratch = nullptr;
  s = scratch_for_current_device(&scratch);
  if (s != RAYGS_OK) return s;
  int dev = 0, sms = 0;
  cudaError_t ae = cudaGetDevice(&dev);
  if (ae == cudaSuccess) ae = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ae != cudaSuccess || sms <= 0) {
    note_cuda_error(ae);
    return RAYGS_ERR_CUDA;
  }

  // Size check: the fixed part must fit; the rest of the array bounds the tile rows and
  // instances (kBytesPerCapacity bytes per unit of capacity).
  Work w;
  w.n_views = n_views;
  w.n = n;
  w.tiles = tiles;
  w.trows = trows;
  w.max_tiles_x = max_tx;
  w.num_sms = sms;
  w.G = sort_grid(sms);
  w.cfg = cfg;
  const Layout L0 = make_layout(n_views, n, tiles, trows, 0, w.G, max_tx, false, false);
  if (L0.total + 8192 > kNoAllocScratchBytes) return RAYGS_ERR_CAPACITY;
  int64_t cap = int64_t((kNoAllocScratchBytes - L0.total - 8192) / (kBytesPerCapacity + 1));
  w.L = make_layout(n_views, n, tiles, trows, cap, w.G, max_tx, false, false);
  while (w.L.total > kNoAllocScratchBytes && cap > 0) {
    cap -= 4096;
    w.L = make_layout(n_views, n, tiles, trows, cap, w.G, max_tx, false, false);
  }
  if (cap <= 0 || w.L.total > kNoAllocScratchBytes) return RAYGS_ERR_CAPACITY;
  w.cap = cap;
  w.base = static_cast<char *>(scratch);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto fail = [](cudaError_t e) { note_cuda_error(e); return RAYGS_ERR_CUDA; };
  cudaError_t e = cudaMemcpyAsync(w.base + w.L.cams, dc, sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(e);
  // run_preprocess clears the counters, the only state that must start at zero (the array
  // keeps the previous call's contents)
  if ((e = run_preprocess(w, *scene, st)) != cudaSuccess) return fail(e);
  if ((e = run_bin_sort(w, st)) != cudaSuccess) return fail(e);
  if ((e = run_render(w, rgb, T_final, n_contrib, false, st)) != cudaSuccess) return fail(e);

  // Report an overflow of the tile rows or instances (the image would be incomplete).
  const Counters *ctr = w.at<Counters>(w.L.counters);
  uint32_t overflow = 0;
  if ((e = cudaMemcpyAsync(&overflow, &ctr->overflow, sizeof(overflow), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
  return overflow ? RAYGS_ERR_CAPACITY : RAYGS_OK;
}
