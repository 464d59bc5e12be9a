// Internal declarations shared by the CUDA translation units of the RayGS library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "raygs.h"

namespace raygs {

constexpr uint32_t kCulled = 0xFFFFFFFFu;  // depth-key marker of a culled (primitive, view)
constexpr float kLog2e = 1.4426950408889634f;

// Per-view constants as the kernels see them (device copy built by the plan).
struct DevCam {
  float fx, fy, cx, cy;
  float ifx, ify;              // 1/fx, 1/fy
  int W, H;
  float R[9];                  // world -> camera, row-major
  float t[3];
  float near_z;
  int mip;
  float C[3];                  // camera centre in the world frame
  float xmin, xmax, ymin, ymax;  // slopes of the outermost pixel-centre rays
  float fn[4];                 // sqrt(1 + slope^2) of each: norms of the side-plane normals
  int tiles_x, tiles_y;
  int tile_base;               // first global tile id of the view
  int trow_base;               // first global tile row of the view
  long long pix_base;          // first output pixel of the view
};

// 64-byte per-(primitive, view) pixel record consumed by the rasteriser.
//   a = (u_hi, v_hi, u_lo, v_lo)   projected centre in pixels, double-float
//   b = (G00, G01, G10, G11)       y01' = G (px - u) = sqrt(kp) y01, with y01 scaled so that
//                                  y2(centre) = 1; q' = |y01'|^2 = kp |y01|^2
//   c = (h0, h1, kp, c2h)          y2 = 1 + h . (px - u); kp = (c^2-kappa)/kappa;
//                                  c2h = c^2 log2(e) / 2; the support is q' <= y2^2, y2 > 0
//   d = (lo2o, r, g, b)            log2 of the (modulated) opacity; colour
struct __align__(16) Rec {
  float4 a, b, c, d;
};

// Device-side counters (one per workspace).
struct Counters {
  uint32_t n_visible;       // valid (primitive, view) pairs after culling
  uint32_t n_rows_clamped;  // min(tile rows, capacity)
  uint32_t n_inst_clamped;  // min(instances, capacity)
  uint32_t overflow;        // rows or instances exceeded the capacity
  unsigned long long n_rows;
  unsigned long long n_instances;
  unsigned long long n_nonfinite;
  uint32_t n_fp64;          // (primitive, view) pairs recomputed in FP64
  uint32_t n_rows_kept;     // support rows with at least one tile
};

// Screen-space support of a (primitive, view), one 32-byte sector for the tile-row pass:
// its tile rectangle (as in the rect array) and the ellipse of pixel centres p with
// (p - c)^T [[a, b], [b, d]] (p - c) <= 1 that holds exactly the rays with D <= kappa (up to
// rounding), det = ad - b^2.  a < 0 marks a support that is not a bounded ellipse in the
// image (or is too ill-conditioned in float32): binning then bounds it tile by tile from
// the pair's record; a = -2 keeps every tile of the rectangle (the exact anti-aliasing
// records hold no conic).
struct __align__(32) Ell {
  uint32_t r0, r1;  // tx0 | ty0 << 16, tx1 | ty1 << 16
  float cx, cy, a, b, d, det;
};

struct RasterCfg {
  float t_stop;
  float alpha_max;
};

// Packed inclusive tile rectangle: x = tx0 | ty0 << 16, y = tx1 | ty1 << 16.
__host__ __device__ inline uint32_t rect_count(uint2 r) {
  uint32_t tx0 = r.x & 0xFFFF, ty0 = r.x >> 16, tx1 = r.y & 0xFFFF, ty1 = r.y >> 16;
  return (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
}

// ---------------------------------------------------------------- double-float helpers
// Error-free transforms (Knuth two-sum, FMA two-product) written with explicitly rounded
// intrinsics so that the compiler cannot contract or reassociate them.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  float e = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, e);
}

// a / b for double-float a, b (one Newton correction; ~44 significant bits).
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  // r = a - q1 * b
  df p = two_prod(q1, b.hi);
  float r = __fsub_rn(a.hi, p.hi);
  r = __fsub_rn(r, p.lo);
  r = __fadd_rn(r, a.lo);
  r = __fsub_rn(r, __fmul_rn(q1, b.lo));
  float q2 = __fdiv_rn(r, b.hi);
  return quick_two_sum(q1, q2);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------- attribute loads
__device__ __forceinline__ float load_attr(const void *base, int64_t idx, int dtype) {
  if (dtype == RAYGS_F16) return __half2float(reinterpret_cast<const __half *>(base)[idx]);
  if (dtype == RAYGS_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[idx]);
  return reinterpret_cast<const float *>(base)[idx];
}

inline int dtype_bytes(int dtype) { return dtype == RAYGS_F32 ? 4 : 2; }

// ---------------------------------------------------------------- kernel parameters
struct PrepParams {
  const float *means;
  const void *log_scales;
  const float *quats;
  const void *logits;
  const void *sh;
  int sh_degree, scale_dtype, opacity_dtype, sh_dtype;
  int n;
  int n_views;
  const DevCam *cams;
  float p_min, mip_sigma2, degenerate_ratio;
  int fp64_degenerate;
  int divergence;  // 0: D_ray (Eq. Q_ray); 1: D_gs (Sec. 3.1)
  int tile_w, tile_h;
  uint32_t *depth_key;
  uint2 *rect;
  uint8_t *trow_cnt;    // tile rows of each pair's rectangle, saturated at 255
  Ell *ell;
  Rec *rec;
  Rec *recx;            // second half of the exact anti-aliasing record (views with mip = 2)
  Counters *counters;
  uint32_t *deg_list;   // (view, primitive) pairs left to the FP64 kernel
  uint32_t *deg_count;
};

struct SortPass {
  const uint32_t *keys_in;
  const uint32_t *vals_in;
  uint32_t *keys_out;       // nullable: the pass writes only the values
  uint32_t *vals_out;
  const uint32_t *d_count;  // device item count (nullable: count_max is used)
  uint32_t count_max;
  int shift;
  int bits;                 // digit width of this pass (8 for item ids, 4-8 for support rows)
  int filter;               // drop kCulled keys; value = item index
  uint32_t *hist;           // [512][G]
  int G;
  uint32_t *d_total;        // receives the number of items kept (nullable)
  // wide mode (tile-row sort of the support rows): 8-byte values (sorted pair position,
  // first tile column | run length << 16), as the row pass writes them
  int wide;
  const uint2 *wvals_in;
  uint2 *wvals_out;
  // The depth sort carries each pair's tile-row count above its id: the first pass packs
  // min(count, field) into the bits above id_bits (row_cnt8: the dense per-pair count,
  // saturated at 255; a full field means "not known"), and the last pass (row_rect set)
  // writes the count in place of the key (the keys are not needed after it) and the bare id
  // as the value, taking the count from the pair's rectangle when the field was full.
  // id_bits = 32 leaves no field: every count comes from the rectangle.
  const uint8_t *row_cnt8;
  int id_bits;
  const uint2 *row_rect;
};

// Exclusive scan of per-unit output counts, with the unit that holds the first output of
// every block of kEmitTile outputs (load-balanced expansion).
struct ScanJob {
  const uint32_t *cnt;
  uint32_t *off;
  const uint32_t *d_n;      // number of units (device; nullable: n_static is used)
  uint32_t n_static;
  uint32_t *partial;        // [G]
  uint32_t *tile_start;
  uint32_t tstart_len;
  unsigned long long *d_total;
  uint32_t *d_total_clamped;
  uint32_t cap;
  uint32_t *d_overflow;
};

struct RowsParams {
  const uint32_t *pairs;    // sorted pair ids
  const uint2 *rect;
  const Ell *ell;
  const Rec *rec;
  const uint32_t *row_off;
  const uint32_t *row_tstart;
  const DevCam *cams;
  const Counters *counters;
  int n;                    // primitives per view
  int tile_w, tile_h;
  uint2 *seg;               // per row: (sorted pair position, txa | len << 16), len the tiles
                            // of the row inside the support (the tile-row sort's payload)
  uint32_t *seg_len;        // per row: len again, for the emission-offset scan (backward
                            // plans only; nullable)
  uint32_t *row_key;        // per row: global tile row, or kCulled when the run is empty
  unsigned long long *trow_inst;  // [tile rows] instances of each tile row (accumulated)
  uint2 *trow_ranges;             // [tile rows] .y: non-empty rows of each tile row (accumulated)
  int trows;
};
constexpr int kTrowsShared = 2048;  // tile rows whose totals a CTA keeps in shared memory

// Per-tile-row passes over the support rows sorted by tile row (stable, so each tile row
// lists its rows in depth order): per-tile instance counts, then the instance lists.
struct ExpandParams {
  const DevCam *cams;
  int n_views;
  const uint2 *trow_ranges;  // [tile rows] range of the tile row in the sorted rows
  const uint2 *rows;         // sorted rows: (sorted pair position, txa | len << 16)
  const unsigned long long *trow_base;  // [tile rows] first instance of each tile row
  uint2 *ranges;             // [tiles] instance range of every tile (clamped to cap)
  uint32_t *inst;            // [cap] sorted pair position of every instance
  uint32_t cap;
  // Each tile row's sorted rows are cut into chunks of chunk_rows rows (at least one chunk
  // per tile row), one CTA each: chunk_base[t] is tile row t's first chunk (chunk_base[trows]
  // the number of chunks), chunk_cnt[chunk][x] the chunk's instances in tile column x.
  uint32_t *chunk_base;
  uint32_t *chunk_cnt;
  int chunk_rows, trows, max_tiles_x, max_chunks;
};

struct RenderParams {
  const DevCam *cams;
  int n_views;
  const uint2 *ranges;
  const uint32_t *inst_vals;
  const uint32_t *pairs;
  const Rec *rec;
  float t_stop, alpha_max;
  float qmix;  // 1: D_ray fragment formula, D ~ q / (q + r); 0: D_gs, D ~ q (records with h = 0)
  unsigned int *tile_counter;  // next unclaimed tile of the persistent rasteriser (zeroed per launch)
  int n_tiles;
  const Rec *recx;  // exact anti-aliasing: second half of each record (then rec holds the first)
  float p_min;
  float *rgb;
  float *Tf;
  int *ncontrib;
  // [4]: evaluated and composited (pixel, primitive) pairs, list entries the CTAs staged
  // (consumed instances), (thread, record) iterations with a live pixel
  unsigned long long *eval_counts;
  uint32_t *tile_stop;  // instrumented variant: per tile, list entries staged before every pixel
                        // stopped, or kCulled when the list ran out first (nullable)
};

constexpr int kEmitTile = 2048;
constexpr int kMaxTilesX = 4096;  // tiles in one tile row (32768-pixel views at 8-pixel tiles)
constexpr int kGradW = 13;  // per-instance / per-pair gradient partials (see backward.cu)

struct BackParams {
  const DevCam *cams;
  int n_views;
  const uint2 *ranges;
  const uint32_t *inst_vals;
  const uint32_t *pairs;
  const Rec *rec;
  const uint2 *rect;
  const uint32_t *row_off;
  const uint2 *seg;
  const uint32_t *seg_off;
  float t_stop, alpha_max;
  const float *Tf;
  const int *ncontrib;
  const float *dL_drgb;
  const float *dL_dT;   // nullable
  float *partials;      // [capacity][kGradW] by emission index
};

struct PairGradParams {
  const uint32_t *pairs;
  const uint32_t *row_off;
  const uint32_t *seg_off;
  const Counters *counters;
  const float *partials;
  float *pg;            // [V*N][kGradW] by pair id
};

struct ParamGradParams {
  const float *means;
  const void *log_scales;
  const float *quats;
  const void *logits;
  const void *sh;
  int sh_degree, scale_dtype, opacity_dtype, sh_dtype;
  int n, n_views;
  const DevCam *cams;
  float p_min, degenerate_ratio;
  int fp64_degenerate;
  const uint32_t *depth_key;
  const float *pg;
  float *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh;
  int num_sms;
  uint32_t *fp64_list;   // primitives left to the FP64 kernel (the forward's FP64 pair list,
  uint32_t *fp64_count;  // free by the time of the backward) and their count (zeroed first)
};

// Records e as the thread's last CUDA error (read back by raygs_last_cuda_error).
void note_cuda_error(cudaError_t e);

cudaError_t launch_preprocess(const PrepParams &P, int num_sms, cudaStream_t st);
cudaError_t launch_sort_pass(const SortPass &p, cudaStream_t st);
cudaError_t launch_scan(const ScanJob &J, int G, cudaStream_t st);
cudaError_t launch_rows(const RowsParams &R, int G, cudaStream_t st);
cudaError_t launch_trow_scan(unsigned long long *trow_inst, uint2 *trow_ranges, int trows, Counters *c, uint32_t cap,
                             cudaStream_t st);
cudaError_t launch_expand(const ExpandParams &E, cudaStream_t st);
int expand_chunk_rows(int64_t cap, int max_tiles_x);
int64_t expand_max_chunks(int64_t trows, int64_t cap, int chunk_rows);
cudaError_t launch_render(const RenderParams &P, int tile_w, int tile_h, int batch_records, int num_sms,
                          bool count, cudaStream_t st);
cudaError_t launch_render_mipx(const RenderParams &P, int tile_w, int tile_h, int64_t n_tiles, bool count,
                               cudaStream_t st);
cudaError_t launch_render_backward(const BackParams &P, int tile_w, int tile_h, int64_t n_tiles, cudaStream_t st);
cudaError_t launch_pair_grads(const PairGradParams &P, int G, cudaStream_t st);
cudaError_t launch_param_grads(const ParamGradParams &P, cudaStream_t st);
cudaError_t launch_resolve(const float *rgb_hi, const float *T_hi, float *rgb_lo, float *T_lo, int w_lo, int h_lo,
                           int factor, long long base_hi, long long base_lo, cudaStream_t st);

// ---------------------------------------------------------------- workspace
// Byte offsets of every buffer inside one caller-owned (or library-static) workspace.
struct Layout {
  size_t tilectr, cams, counters, evals, tstop, tscan, depth, rect, tcnt, ell, rec, recx, s1k[2], s1v[2], off, partial, rtstart,
      seg, seg_len, seg_off, rk[2], rv[2], trange, trinst, cbase, ccnt, inst, hist, ranges, deg, degc, partials, pg, total;
  uint32_t rtstart_len;
};

Layout make_layout(int n_views, int64_t n, int64_t tiles, int64_t trows, int64_t cap, int G, int max_tiles_x,
                   bool backward, bool mip_exact);

// Workspace bytes per unit of instance capacity (tile rows and instances share it).
constexpr size_t kBytesPerCapacity = 8 + 4 + 4 + 2 * 4 + 2 * 8 + 4;

// A bound workspace and the sizes it was laid out for.
struct Work {
  char *base = nullptr;
  Layout L{};
  int n_views = 0;
  int64_t n = 0, tiles = 0, trows = 0, cap = 0;
  int max_tiles_x = 0;
  int G = 0, num_sms = 0;
  raygs_config cfg{};
  int s1_final = 0, s2_rows = 0;  // which ping-pong buffers hold the sorted results
  template <typename T>
  T *at(size_t off) const { return reinterpret_cast<T *>(base + off); }
};

// Host-side helpers shared by the entry points.
void fill_devcam(const raygs_camera &c, const raygs_config &cfg, DevCam &d);
// Per-view constants and the global tile, tile-row and pixel numbering of a batch of views;
// false when a view is invalid or the batch is too large to number in 31 bits.
bool plan_views(const raygs_camera *cams, int n_views, const raygs_config &cfg, DevCam *dc, int64_t &tiles,
                int64_t &trows, int64_t &pixels, int &max_tiles_x);
bool config_valid(const raygs_config &cfg);
bool camera_valid(const raygs_camera &c);
raygs_status scene_valid(const raygs_scene *s, int64_t n);

int sort_grid(int num_sms);
int tile_sort_bits(int64_t tiles);
cudaError_t run_preprocess(Work &w, const raygs_scene &scene, cudaStream_t st);
cudaError_t run_bin_sort(Work &w, cudaStream_t st);
cudaError_t run_render(const Work &w, float *rgb, float *T_final, int32_t *n_contrib, bool count,
                       cudaStream_t st);
cudaError_t run_backward(const Work &w, const raygs_scene &scene, const float *T_final, const int32_t *n_contrib,
                         const float *dL_drgb, const float *dL_dT, const raygs_grads &grads, cudaStream_t st);

}  // namespace raygs
