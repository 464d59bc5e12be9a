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
#include <cmath>
#include <cstring>
#include <mutex>

#include "raygs_internal.cuh"

namespace raygs {

constexpr size_t kNoAllocScratchBytes = RAYGS_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace raygs

using namespace raygs;

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device.  Host code cannot use the
// symbol itself (it names a host-side shadow); the address is looked up once per device
// with that device current, which also loads the module on that device.
raygs_status scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { note_cuda_error(e); return RAYGS_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) return RAYGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) { note_cuda_error(e); return RAYGS_ERR_CUDA; }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RAYGS_OK;
}

struct Layout {
  size_t cams, counters, depth, rect, rec, s1k[2], s1v[2], cnt, off, partial, tstart, ik[2], iv[2],
      hist, ranges, deg, degc, total;
  uint32_t tstart_len;
};

Layout layout_for(int n_views, int64_t n, int64_t tiles, int64_t cap, int G) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o = up256(o + b); return r; };
  const size_t VN = size_t(n_views) * size_t(n);
  L.cams = take(sizeof(DevCam) * n_views);
  L.counters = take(sizeof(Counters));
  L.depth = take(4 * VN);
  L.rect = take(8 * VN);
  L.rec = take(sizeof(Rec) * VN);
  for (int i = 0; i < 2; ++i) { L.s1k[i] = take(4 * VN); L.s1v[i] = take(4 * VN); }
  L.cnt = take(4 * VN);
  L.off = take(4 * VN);
  L.partial = take(4 * size_t(G));
  L.tstart_len = uint32_t(size_t(cap) / kEmitTile + 2);
  L.tstart = take(4 * size_t(L.tstart_len));
  for (int i = 0; i < 2; ++i) { L.ik[i] = take(4 * size_t(cap) + 16); L.iv[i] = take(4 * size_t(cap) + 16); }
  L.hist = take(4 * 256 * size_t(G));
  L.ranges = take(8 * size_t(tiles));
  L.deg = take(4 * size_t(n));
  L.degc = take(4);
  L.total = o;
  return L;
}

}  // namespace

extern "C" raygs_status raygs_render_noalloc(const raygs_camera *cams, int32_t n_views, const raygs_scene *scene,
                                             const raygs_config *cfg_in, float *rgb, float *T_final,
                                             int32_t *n_contrib, void *stream) {
  if (!cams || !scene || !rgb || n_views < 1 || n_views > RAYGS_MAX_VIEWS) return RAYGS_ERR_INVALID_ARG;
  raygs_config cfg;
  if (cfg_in) cfg = *cfg_in; else raygs_config_default(&cfg);
  const bool tile_ok = (cfg.tile_w == 16 && cfg.tile_h == 16) || (cfg.tile_w == 16 && cfg.tile_h == 8) ||
                       (cfg.tile_w == 32 && cfg.tile_h == 16) || (cfg.tile_w == 8 && cfg.tile_h == 8);
  if (!tile_ok || !(cfg.p_min > 0.f && cfg.p_min < 1.f) || !(cfg.t_stop >= 0.f && cfg.t_stop < 1.f) ||
      !(cfg.alpha_max > 0.f && cfg.alpha_max < 1.f) || !(cfg.mip_sigma2 >= 0.f) || !(cfg.degenerate_ratio > 1.f))
    return RAYGS_ERR_INVALID_ARG;
  const int64_t n = scene->n;
  if (n < 0 || n >= (int64_t(1) << 31) || scene->sh_degree < 0 || scene->sh_degree > 3) return RAYGS_ERR_INVALID_ARG;
  auto dt_ok = [](int d, bool bf) { return d == RAYGS_F32 || d == RAYGS_F16 || (bf && d == RAYGS_BF16); };
  if (!dt_ok(scene->scale_dtype, true) || !dt_ok(scene->opacity_dtype, false) || !dt_ok(scene->sh_dtype, true))
    return RAYGS_ERR_INVALID_ARG;
  auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (n > 0 && (!scene->means || !scene->log_scales || !scene->quats || !scene->opacity_logits || !scene->sh ||
                !a16(scene->means) || !a16(scene->log_scales) || !a16(scene->quats) ||
                !a16(scene->opacity_logits) || !a16(scene->sh)))
    return RAYGS_ERR_INVALID_ARG;

  // Per-view constants, on the stack (no heap).
  DevCam dc[RAYGS_MAX_VIEWS];
  int64_t tiles = 0, pixels = 0;
  for (int v = 0; v < n_views; ++v) {
    const raygs_camera &c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768 || !(c.fx > 0.f) || !(c.fy > 0.f) ||
        !std::isfinite(c.cx) || !std::isfinite(c.cy) || !(c.near_z > 0.f))
      return RAYGS_ERR_INVALID_ARG;
    DevCam &d = dc[v];
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
    d.tile_base = int(tiles);
    d.pix_base = pixels;
    tiles += int64_t(d.tiles_x) * d.tiles_y;
    pixels += int64_t(c.width) * c.height;
  }

  void *scratch = nullptr;
  raygs_status s = scratch_for_current_device(&scratch);
  if (s != RAYGS_OK) return s;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  const int G = sms * 4 > 1024 ? 1024 : sms * 4;

  // Size check: the fixed part must fit; the rest of the array holds the instance lists.
  Layout L0 = layout_for(n_views, n, tiles, 0, G);
  if (L0.total + 4096 > kNoAllocScratchBytes) return RAYGS_ERR_CAPACITY;
  int64_t cap = int64_t((kNoAllocScratchBytes - L0.total - 4096) / 17);
  Layout L = layout_for(n_views, n, tiles, cap, G);
  while (L.total > kNoAllocScratchBytes && cap > 0) {
    cap -= 4096;
    L = layout_for(n_views, n, tiles, cap, G);
  }
  if (cap <= 0 || L.total > kNoAllocScratchBytes) return RAYGS_ERR_CAPACITY;

  char *ws = static_cast<char *>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto fail = [](cudaError_t e) { note_cuda_error(e); return RAYGS_ERR_CUDA; };
  cudaError_t e = cudaMemcpyAsync(ws + L.cams, dc, sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(e);
  // everything that must start at zero: the counters (the array keeps the last call's data)
  e = cudaMemsetAsync(ws + L.counters, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return fail(e);

  Counters *ctr = reinterpret_cast<Counters *>(ws + L.counters);
  PrepParams P;
  P.means = scene->means; P.log_scales = scene->log_scales; P.quats = scene->quats;
  P.logits = scene->opacity_logits; P.sh = scene->sh;
  P.sh_degree = scene->sh_degree; P.scale_dtype = scene->scale_dtype;
  P.opacity_dtype = scene->opacity_dtype; P.sh_dtype = scene->sh_dtype;
  P.n = int(n); P.n_views = n_views;
  P.cams = reinterpret_cast<const DevCam *>(ws + L.cams);
  P.p_min = cfg.p_min; P.mip_sigma2 = cfg.mip_sigma2; P.degenerate_ratio = cfg.degenerate_ratio;
  P.fp64_degenerate = cfg.fp64_degenerate; P.tile_w = cfg.tile_w; P.tile_h = cfg.tile_h;
  P.depth_key = reinterpret_cast<uint32_t *>(ws + L.depth);
  P.rect = reinterpret_cast<uint2 *>(ws + L.rect);
  P.rec = reinterpret_cast<Rec *>(ws + L.rec);
  P.counters = ctr;
  P.deg_list = reinterpret_cast<uint32_t *>(ws + L.deg);
  P.deg_count = reinterpret_cast<uint32_t *>(ws + L.degc);
  if ((e = launch_preprocess(P, sms, st)) != cudaSuccess) return fail(e);

  const uint32_t VN = uint32_t(size_t(n_views) * size_t(n));
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    SortPass sp;
    sp.keys_in = reinterpret_cast<const uint32_t *>(ws + (pass == 0 ? L.depth : L.s1k[cur]));
    sp.vals_in = pass == 0 ? nullptr : reinterpret_cast<const uint32_t *>(ws + L.s1v[cur]);
    const int dst = pass == 0 ? 0 : 1 - cur;
    sp.keys_out = reinterpret_cast<uint32_t *>(ws + L.s1k[dst]);
    sp.vals_out = reinterpret_cast<uint32_t *>(ws + L.s1v[dst]);
    sp.d_count = pass == 0 ? nullptr : &ctr->n_visible;
    sp.count_max = VN;
    sp.shift = 8 * pass;
    sp.filter = pass == 0 ? 1 : 0;
    sp.hist = hist;
    sp.G = G;
    sp.d_total = pass == 0 ? &ctr->n_visible : nullptr;
    if ((e = launch_sort_pass(sp, st)) != cudaSuccess) return fail(e);
    cur = dst;
  }
  const uint32_t *pairs = reinterpret_cast<const uint32_t *>(ws + L.s1v[cur]);
  ScanParams S;
  S.pairs = pairs;
  S.rect = reinterpret_cast<const uint2 *>(ws + L.rect);
  S.cnt = reinterpret_cast<uint32_t *>(ws + L.cnt);
  S.off = reinterpret_cast<uint32_t *>(ws + L.off);
  S.partial = reinterpret_cast<uint32_t *>(ws + L.partial);
  S.tile_start = reinterpret_cast<uint32_t *>(ws + L.tstart);
  S.counters = ctr;
  S.capacity = uint32_t(cap);
  S.tile_start_len = L.tstart_len;
  if ((e = launch_count_scan(S, G, st)) != cudaSuccess) return fail(e);
  EmitParams E;
  E.pairs = pairs; E.rect = S.rect; E.off = S.off; E.tile_start = S.tile_start;
  E.cams = P.cams; E.counters = ctr; E.n = int(n);
  E.keys = reinterpret_cast<uint32_t *>(ws + L.ik[0]);
  E.vals = reinterpret_cast<uint32_t *>(ws + L.iv[0]);
  if ((e = launch_emit(E, G, st)) != cudaSuccess) return fail(e);
  int bits = 0;
  while (bits < 32 && (uint64_t(1) << bits) < uint64_t(tiles)) ++bits;
  const int passes = (bits + 7) / 8;
  cur = 0;
  for (int pass = 0; pass < passes; ++pass) {
    SortPass sp;
    sp.keys_in = reinterpret_cast<const uint32_t *>(ws + L.ik[cur]);
    sp.vals_in = reinterpret_cast<const uint32_t *>(ws + L.iv[cur]);
    sp.keys_out = reinterpret_cast<uint32_t *>(ws + L.ik[1 - cur]);
    sp.vals_out = reinterpret_cast<uint32_t *>(ws + L.iv[1 - cur]);
    sp.d_count = &ctr->n_inst_clamped;
    sp.count_max = uint32_t(cap);
    sp.shift = 8 * pass;
    sp.filter = 0;
    sp.hist = hist;
    sp.G = G;
    sp.d_total = nullptr;
    if ((e = launch_sort_pass(sp, st)) != cudaSuccess) return fail(e);
    cur = 1 - cur;
  }
  uint2 *ranges = reinterpret_cast<uint2 *>(ws + L.ranges);
  if ((e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * size_t(tiles), st)) != cudaSuccess) return fail(e);
  if ((e = launch_ranges(reinterpret_cast<const uint32_t *>(ws + L.ik[cur]), ctr, ranges, G, st)) != cudaSuccess)
    return fail(e);
  RenderParams R;
  R.cams = P.cams; R.n_views = n_views; R.ranges = ranges;
  R.inst_vals = reinterpret_cast<const uint32_t *>(ws + L.iv[cur]);
  R.pairs = pairs; R.rec = P.rec;
  R.t_stop = cfg.t_stop; R.alpha_max = cfg.alpha_max;
  R.rgb = rgb; R.Tf = T_final; R.ncontrib = n_contrib; R.eval_counts = nullptr;
  if ((e = launch_render(R, cfg.tile_w, cfg.tile_h, tiles, false, st)) != cudaSuccess) return fail(e);

  // Report an instance overflow (the image would be incomplete): read the counter.
  uint32_t overflow = 0;
  if ((e = cudaMemcpyAsync(&overflow, &ctr->overflow, sizeof(overflow), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
  return overflow ? RAYGS_ERR_CAPACITY : RAYGS_OK;
}
