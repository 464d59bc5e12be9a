// Workspace layout and the order of kernel launches of the three hot-path stages, shared
// by the plan API (caller-owned workspace) and the allocation-free entry point.
#include <cmath>

#include <algorithm>

#include "raygs_internal.cuh"

namespace raygs {

namespace {
size_t up256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

void fill_devcam(const raygs_camera &c, const raygs_config &cfg, DevCam &d) {
  d = DevCam{};
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
  d.ifx = float(1.0 / double(c.fx));
  d.ify = float(1.0 / double(c.fy));
  d.W = c.width; d.H = c.height;
  for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
  d.near_z = c.near_z;
  d.mip = c.mip;
  for (int k = 0; k < 3; ++k)
    d.C[k] = float(-(double(c.R[k]) * c.t[0] + double(c.R[3 + k]) * c.t[1] + double(c.R[6 + k]) * c.t[2]));
  d.xmin = float((0.5 - double(c.cx)) / double(c.fx));
  d.xmax = float((double(c.width) - 0.5 - double(c.cx)) / double(c.fx));
  d.ymin = float((0.5 - double(c.cy)) / double(c.fy));
  d.ymax = float((double(c.height) - 0.5 - double(c.cy)) / double(c.fy));
  const float sl[4] = {d.xmin, d.xmax, d.ymin, d.ymax};
  for (int k = 0; k < 4; ++k) d.fn[k] = float(std::sqrt(1.0 + double(sl[k]) * double(sl[k])));
  d.tiles_x = (c.width + cfg.tile_w - 1) / cfg.tile_w;
  d.tiles_y = (c.height + cfg.tile_h - 1) / cfg.tile_h;
}

bool config_valid(const raygs_config &cfg) {
  const bool tile_ok = (cfg.tile_w == 16 && cfg.tile_h == 16) || (cfg.tile_w == 16 && cfg.tile_h == 8) ||
                       (cfg.tile_w == 32 && cfg.tile_h == 16) || (cfg.tile_w == 8 && cfg.tile_h == 8);
  return tile_ok && cfg.p_min > 0.f && cfg.p_min < 1.f && cfg.t_stop >= 0.f && cfg.t_stop < 1.f &&
         cfg.alpha_max > 0.f && cfg.alpha_max < 1.f && cfg.mip_sigma2 >= 0.f && cfg.degenerate_ratio > 1.f &&
         cfg.fp64_degenerate >= 0 && cfg.fp64_degenerate <= 2 && (cfg.enable_backward == 0 || cfg.enable_backward == 1) &&
         (cfg.batch_records == 1 || cfg.batch_records == 2) && (cfg.divergence == 0 || cfg.divergence == 1) &&
         !(cfg.divergence == 1 && cfg.enable_backward);
}

bool camera_valid(const raygs_camera &c) {
  return c.width >= 1 && c.height >= 1 && c.width <= 32768 && c.height <= 32768 && c.fx > 0.f && c.fy > 0.f &&
         std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy) &&
         c.near_z > 0.f && c.mip >= RAYGS_MIP_OFF && c.mip <= RAYGS_MIP_EXACT;
}

raygs_status scene_valid(const raygs_scene *s, int64_t n) {
  if (!s || s->n != n) return RAYGS_ERR_INVALID_ARG;
  if (s->sh_degree < 0 || s->sh_degree > 3) return RAYGS_ERR_INVALID_ARG;
  auto dt_ok = [](int d, bool allow_bf16) {
    return d == RAYGS_F32 || d == RAYGS_F16 || (allow_bf16 && d == RAYGS_BF16);
  };
  if (!dt_ok(s->scale_dtype, true) || !dt_ok(s->opacity_dtype, false) || !dt_ok(s->sh_dtype, true))
    return RAYGS_ERR_INVALID_ARG;
  auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (s->n > 0) {
    if (!s->means || !s->log_scales || !s->quats || !s->opacity_logits || !s->sh) return RAYGS_ERR_INVALID_ARG;
    if (!a16(s->means) || !a16(s->log_scales) || !a16(s->quats) || !a16(s->opacity_logits) || !a16(s->sh))
      return RAYGS_ERR_INVALID_ARG;
  }
  return RAYGS_OK;
}

int sort_grid(int num_sms) {
  int g = 4 * num_sms;
  return g > 1024 ? 1024 : (g < 1 ? 1 : g);
}

int tile_sort_bits(int64_t tiles) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) < tiles) ++b;
  return b;
}

Layout make_layout(int n_views, int64_t n, int64_t tiles, int64_t trows, int64_t cap, int G, int max_tiles_x,
                   bool backward, bool mip_exact) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = up256(o + bytes); return r; };
  const size_t VN = size_t(n_views) * size_t(n);
  const size_t C = size_t(cap);
  L.cams = take(sizeof(DevCam) * size_t(n_views));
  L.counters = take(sizeof(Counters));
  L.evals = take(4 * sizeof(unsigned long long));
  L.tilectr = take(16);
  L.tscan = take(2 * sizeof(unsigned long long));
  L.depth = take(4 * VN);
  L.rect = take(8 * VN);
  L.tcnt = take(VN);
  L.ell = take(sizeof(Ell) * VN);
  L.rec = take(sizeof(Rec) * VN);
  L.recx = mip_exact ? take(sizeof(Rec) * VN) : 0;
  for (int i = 0; i < 2; ++i) { L.s1k[i] = take(4 * VN); L.s1v[i] = take(4 * VN); }
  L.off = take(4 * VN);
  L.partial = take(4 * size_t(G));
  L.rtstart_len = uint32_t(C / kEmitTile + 2);
  L.rtstart = take(4 * size_t(L.rtstart_len));
  // per unit of capacity: kBytesPerCapacity bytes
  L.seg = take(8 * C + 16);
  L.seg_len = take(4 * C + 16);
  L.seg_off = take(4 * C + 16);
  for (int i = 0; i < 2; ++i) { L.rk[i] = take(4 * C + 16); L.rv[i] = take(8 * C + 16); }
  L.inst = take(4 * C + 16);
  L.trange = take(8 * size_t(trows) + 16);
  L.trinst = take(8 * size_t(trows) + 16);
  const int chunk_rows = expand_chunk_rows(cap, max_tiles_x);
  const int64_t max_chunks = expand_max_chunks(trows, cap, chunk_rows);
  L.cbase = take(4 * size_t(trows + 1) + 16);
  L.ccnt = take(4 * size_t(max_chunks) * size_t(max_tiles_x > 0 ? max_tiles_x : 1) + 16);
  L.hist = take(4 * 512 * size_t(G) + 4 * (512 * size_t(G) / 2048 + 1));
  L.ranges = take(8 * size_t(tiles));
  L.tstop = take(4 * size_t(tiles) + 16);
  L.deg = take(4 * VN);
  L.degc = take(4);
  L.partials = backward ? take(4 * kGradW * C + 16) : 0;
  L.pg = backward ? take(4 * kGradW * VN + 16) : 0;
  L.total = o;
  return L;
}

bool plan_views(const raygs_camera *cams, int n_views, const raygs_config &cfg, DevCam *dc, int64_t &tiles,
                int64_t &trows, int64_t &pixels, int &max_tiles_x) {
  tiles = 0; trows = 0; pixels = 0; max_tiles_x = 0;
  for (int v = 0; v < n_views; ++v) {
    if (!camera_valid(cams[v])) return false;
    if (cfg.divergence == 1 && cams[v].mip) return false;  // Eq. mip is a RayGS term
    // the exact anti-aliasing uses its own record and rasteriser for the whole batch
    if ((cams[v].mip == RAYGS_MIP_EXACT) != (cams[0].mip == RAYGS_MIP_EXACT)) return false;
    fill_devcam(cams[v], cfg, dc[v]);
    if (dc[v].tiles_x > kMaxTilesX) return false;
    dc[v].tile_base = int(tiles);
    dc[v].trow_base = int(trows);
    dc[v].pix_base = pixels;
    tiles += int64_t(dc[v].tiles_x) * dc[v].tiles_y;
    trows += dc[v].tiles_y;
    pixels += int64_t(cams[v].width) * cams[v].height;
    if (dc[v].tiles_x > max_tiles_x) max_tiles_x = dc[v].tiles_x;
    if (tiles >= (int64_t(1) << 31)) return false;
  }
  return true;
}

cudaError_t run_preprocess(Work &w, const raygs_scene &scene, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w.base + w.L.counters, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return e;
  PrepParams P{};
  P.means = scene.means;
  P.log_scales = scene.log_scales;
  P.quats = scene.quats;
  P.logits = scene.opacity_logits;
  P.sh = scene.sh;
  P.sh_degree = scene.sh_degree;
  P.scale_dtype = scene.scale_dtype;
  P.opacity_dtype = scene.opacity_dtype;
  P.sh_dtype = scene.sh_dtype;
  P.n = int(w.n);
  P.n_views = w.n_views;
  P.cams = w.at<DevCam>(w.L.cams);
  P.p_min = w.cfg.p_min;
  P.mip_sigma2 = w.cfg.mip_sigma2;
  P.degenerate_ratio = w.cfg.degenerate_ratio;
  P.fp64_degenerate = w.cfg.fp64_degenerate;
  P.divergence = w.cfg.divergence;
  P.tile_w = w.cfg.tile_w;
  P.tile_h = w.cfg.tile_h;
  P.depth_key = w.at<uint32_t>(w.L.depth);
  P.rect = w.at<uint2>(w.L.rect);
  P.trow_cnt = w.at<uint8_t>(w.L.tcnt);
  P.ell = w.at<Ell>(w.L.ell);
  P.rec = w.at<Rec>(w.L.rec);
  P.recx = w.L.recx ? w.at<Rec>(w.L.recx) : nullptr;
  P.counters = w.at<Counters>(w.L.counters);
  P.deg_list = w.at<uint32_t>(w.L.deg);
  P.deg_count = w.at<uint32_t>(w.L.degc);
  return launch_preprocess(P, w.num_sms, st);
}

cudaError_t run_bin_sort(Work &w, cudaStream_t st) {
  Counters *ctr = w.at<Counters>(w.L.counters);
  const uint32_t VN = uint32_t(size_t(w.n_views) * size_t(w.n));
  const uint32_t cap = uint32_t(w.cap);
  uint32_t *hist = w.at<uint32_t>(w.L.hist);
  cudaError_t e;
  // 1. depth sort of the visible pairs: 4 passes of 8 bits over the float32 key; the values
  // carry each pair's tile-row count above its id (bits of the largest id)
  int id_bits = 1;
  while (id_bits < 32 && (uint64_t(1) << id_bits) < uint64_t(VN)) ++id_bits;
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    SortPass sp{};
    sp.keys_in = w.at<uint32_t>(pass == 0 ? w.L.depth : w.L.s1k[cur]);
    sp.vals_in = pass == 0 ? nullptr : w.at<uint32_t>(w.L.s1v[cur]);
    const int dst = pass == 0 ? 0 : 1 - cur;
    sp.keys_out = w.at<uint32_t>(w.L.s1k[dst]);
    sp.vals_out = w.at<uint32_t>(w.L.s1v[dst]);
    sp.d_count = pass == 0 ? nullptr : &ctr->n_visible;
    sp.count_max = VN;
    sp.shift = 8 * pass;
    sp.bits = 8;
    sp.filter = pass == 0 ? 1 : 0;
    sp.hist = hist;
    sp.G = w.G;
    sp.d_total = pass == 0 ? &ctr->n_visible : nullptr;
    sp.row_cnt8 = pass == 0 ? w.at<uint8_t>(w.L.tcnt) : nullptr;
    sp.id_bits = id_bits;
    sp.row_rect = pass == 3 ? w.at<uint2>(w.L.rect) : nullptr;
    if ((e = launch_sort_pass(sp, st)) != cudaSuccess) return e;
    cur = dst;
  }
  w.s1_final = cur;
  const uint32_t *pairs = w.at<uint32_t>(w.L.s1v[cur]);
  // 2a. pairs -> tile rows
  ScanJob J{};
  J.cnt = w.at<uint32_t>(w.L.s1k[cur]);  // the last depth pass left each pair's row count here
  J.off = w.at<uint32_t>(w.L.off);
  J.d_n = &ctr->n_visible;
  J.partial = w.at<uint32_t>(w.L.partial);
  J.tile_start = w.at<uint32_t>(w.L.rtstart);
  J.tstart_len = w.L.rtstart_len;
  J.d_total = &ctr->n_rows;
  J.d_total_clamped = &ctr->n_rows_clamped;
  J.cap = cap;
  J.d_overflow = &ctr->overflow;
  if ((e = launch_scan(J, w.G, st)) != cudaSuccess) return e;
  // 2b. rows -> tile spans inside the support ellipse
  RowsParams R{};
  R.pairs = pairs;
  R.rect = w.at<uint2>(w.L.rect);
  R.ell = w.at<Ell>(w.L.ell);
  R.rec = w.at<Rec>(w.L.rec);
  R.row_off = J.off;
  R.row_tstart = J.tile_start;
  R.cams = w.at<DevCam>(w.L.cams);
  R.counters = ctr;
  R.n = int(w.n);
  R.tile_w = w.cfg.tile_w;
  R.tile_h = w.cfg.tile_h;
  R.seg = w.at<uint2>(w.L.seg);
  R.seg_len = w.cfg.enable_backward ? w.at<uint32_t>(w.L.seg_len) : nullptr;
  R.row_key = w.at<uint32_t>(w.L.rk[0]);
  R.trow_inst = w.at<unsigned long long>(w.L.trinst);
  R.trows = int(w.trows);
  R.trow_ranges = w.at<uint2>(w.L.trange);
  if ((e = cudaMemsetAsync(R.trow_inst, 0, sizeof(unsigned long long) * size_t(w.trows), st)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(R.trow_ranges, 0, sizeof(uint2) * size_t(w.trows), st)) != cudaSuccess) return e;
  if ((e = launch_rows(R, w.G, st)) != cudaSuccess) return e;
  ScanJob J2{};
  J2.cnt = R.seg_len;
  J2.off = w.at<uint32_t>(w.L.seg_off);
  J2.d_n = &ctr->n_rows_clamped;
  J2.partial = w.at<uint32_t>(w.L.partial);
  J2.tile_start = nullptr;
  J2.tstart_len = 0;
  J2.d_total = &ctr->n_instances;
  J2.d_total_clamped = &ctr->n_inst_clamped;
  J2.cap = cap;
  J2.d_overflow = &ctr->overflow;
  // the emission offsets only index the backward's partials
  const bool emission = w.cfg.enable_backward != 0;
  if (emission && (e = launch_scan(J2, w.G, st)) != cudaSuccess) return e;
  // first instance of every tile row, the instance total and the capacity check
  if ((e = launch_trow_scan(R.trow_inst, R.trow_ranges, int(w.trows), ctr, cap, st)) != cudaSuccess) return e;
  // 3. stable sort of the non-empty rows by global tile row (at most 8-bit digits); the first
  // pass drops the empty rows and reads each row's payload as the row pass wrote it
  const int rbits = tile_sort_bits(w.trows);
  const int rpasses = (rbits + 7) / 8;
  // digits of equal width (at least 4 bits): the first pass scatters into fewer buckets
  // (64 instead of 256 for 12-bit tile rows), so its output runs are longer
  const int rdigit = std::max(4, (rbits + rpasses - 1) / rpasses);
  cur = 0;
  for (int pass = 0; pass < rpasses; ++pass) {
    SortPass sp{};
    sp.keys_in = w.at<uint32_t>(w.L.rk[pass == 0 ? 0 : cur]);
    sp.vals_in = nullptr;
    const int dst = pass == 0 ? 1 : 1 - cur;
    // (the sorted keys themselves are not read after the last pass)
    sp.keys_out = pass + 1 < rpasses ? w.at<uint32_t>(w.L.rk[dst]) : nullptr;
    sp.vals_out = nullptr;
    sp.d_count = pass == 0 ? &ctr->n_rows_clamped : &ctr->n_rows_kept;
    sp.count_max = cap;
    sp.shift = rdigit * pass;
    sp.bits = rdigit;
    sp.filter = pass == 0 ? 1 : 0;
    sp.hist = hist;
    sp.G = w.G;
    sp.d_total = pass == 0 ? &ctr->n_rows_kept : nullptr;
    sp.wide = 1;
    sp.wvals_in = pass == 0 ? R.seg : w.at<uint2>(w.L.rv[cur]);
    sp.wvals_out = w.at<uint2>(w.L.rv[dst]);
    if ((e = launch_sort_pass(sp, st)) != cudaSuccess) return e;
    cur = dst;
  }
  w.s2_rows = cur;
  // 4. tile-row ranges of the sorted rows, instances per tile, tile offsets, lists
  // (each tile row's range of sorted rows came from the tile-row scan above)
  uint2 *trange = R.trow_ranges;
  ExpandParams X{};
  X.cams = R.cams;
  X.n_views = w.n_views;
  X.trow_ranges = trange;
  X.rows = w.at<uint2>(w.L.rv[cur]);
  X.trow_base = R.trow_inst;
  X.ranges = w.at<uint2>(w.L.ranges);
  X.inst = w.at<uint32_t>(w.L.inst);
  X.cap = cap;
  X.chunk_base = w.at<uint32_t>(w.L.cbase);
  X.chunk_cnt = w.at<uint32_t>(w.L.ccnt);
  X.chunk_rows = expand_chunk_rows(w.cap, w.max_tiles_x);
  X.trows = int(w.trows);
  X.max_tiles_x = w.max_tiles_x;
  X.max_chunks = int(expand_max_chunks(w.trows, w.cap, X.chunk_rows));
  return launch_expand(X, st);
}

cudaError_t run_render(const Work &w, float *rgb, float *T_final, int32_t *n_contrib, bool count,
                       cudaStream_t st) {
  RenderParams P{};
  P.cams = w.at<DevCam>(w.L.cams);
  P.n_views = w.n_views;
  P.ranges = w.at<uint2>(w.L.ranges);
  P.inst_vals = w.at<uint32_t>(w.L.inst);
  P.pairs = w.at<uint32_t>(w.L.s1v[w.s1_final]);
  P.rec = w.at<Rec>(w.L.rec);
  P.t_stop = w.cfg.t_stop;
  P.alpha_max = w.cfg.alpha_max;
  P.qmix = w.cfg.divergence == 1 ? 0.f : 1.f;
  P.recx = w.L.recx ? w.at<Rec>(w.L.recx) : nullptr;
  P.p_min = w.cfg.p_min;
  P.rgb = rgb;
  P.Tf = T_final;
  P.ncontrib = n_contrib;
  P.eval_counts = w.at<unsigned long long>(w.L.evals);
  P.tile_stop = count ? w.at<uint32_t>(w.L.tstop) : nullptr;
  if (count) {
    cudaError_t e = cudaMemsetAsync(P.eval_counts, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (P.recx) return launch_render_mipx(P, w.cfg.tile_w, w.cfg.tile_h, w.tiles, count, st);
  if (w.tiles == 0) return cudaSuccess;
  P.tile_counter = w.at<unsigned int>(w.L.tilectr);
  P.n_tiles = int(w.tiles);
  cudaError_t e = cudaMemsetAsync(P.tile_counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  return launch_render(P, w.cfg.tile_w, w.cfg.tile_h, w.cfg.batch_records, w.num_sms, count, st);
}

cudaError_t run_backward(const Work &w, const raygs_scene &scene, const float *T_final, const int32_t *n_contrib,
                         const float *dL_drgb, const float *dL_dT, const raygs_grads &grads, cudaStream_t st) {
  BackParams B{};
  B.cams = w.at<DevCam>(w.L.cams);
  B.n_views = w.n_views;
  B.ranges = w.at<uint2>(w.L.ranges);
  B.inst_vals = w.at<uint32_t>(w.L.inst);
  B.pairs = w.at<uint32_t>(w.L.s1v[w.s1_final]);
  B.rec = w.at<Rec>(w.L.rec);
  B.rect = w.at<uint2>(w.L.rect);
  B.row_off = w.at<uint32_t>(w.L.off);
  B.seg = w.at<uint2>(w.L.seg);
  B.seg_off = w.at<uint32_t>(w.L.seg_off);
  B.t_stop = w.cfg.t_stop;
  B.alpha_max = w.cfg.alpha_max;
  B.Tf = T_final;
  B.ncontrib = n_contrib;
  B.dL_drgb = dL_drgb;
  B.dL_dT = dL_dT;
  B.partials = w.at<float>(w.L.partials);
  cudaError_t e = launch_render_backward(B, w.cfg.tile_w, w.cfg.tile_h, w.tiles, st);
  if (e != cudaSuccess) return e;
  PairGradParams Q{};
  Q.pairs = B.pairs;
  Q.row_off = B.row_off;
  Q.seg_off = B.seg_off;
  Q.counters = w.at<Counters>(w.L.counters);
  Q.partials = B.partials;
  Q.pg = w.at<float>(w.L.pg);
  if ((e = launch_pair_grads(Q, w.G, st)) != cudaSuccess) return e;
  ParamGradParams R{};
  R.means = scene.means;
  R.log_scales = scene.log_scales;
  R.quats = scene.quats;
  R.logits = scene.opacity_logits;
  R.sh = scene.sh;
  R.sh_degree = scene.sh_degree;
  R.scale_dtype = scene.scale_dtype;
  R.opacity_dtype = scene.opacity_dtype;
  R.sh_dtype = scene.sh_dtype;
  R.n = int(w.n);
  R.n_views = w.n_views;
  R.cams = B.cams;
  R.p_min = w.cfg.p_min;
  R.degenerate_ratio = w.cfg.degenerate_ratio;
  R.fp64_degenerate = w.cfg.fp64_degenerate;
  R.depth_key = w.at<uint32_t>(w.L.depth);
  R.pg = Q.pg;
  R.d_means = grads.d_means;
  R.d_log_scales = grads.d_log_scales;
  R.d_quats = grads.d_quats;
  R.d_logits = grads.d_opacity_logits;
  R.d_sh = grads.d_sh;
  R.num_sms = w.num_sms;
  R.fp64_list = w.at<uint32_t>(w.L.deg);
  R.fp64_count = w.at<uint32_t>(w.L.degc);
  if ((e = cudaMemsetAsync(R.fp64_count, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  return launch_param_grads(R, st);
}

}  // namespace raygs
