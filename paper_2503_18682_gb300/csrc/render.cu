// Per-tile rasterisation and front-to-back compositing (Sec. 3 Eq. rendering and
// Eq. rend_opacity; Sec. 4.2 fragment formula).
//
// One CTA per screen tile of any view; one thread per pixel.  The tile's instance list
// (depth order) is consumed in batches: each thread stages one 64-byte record in shared
// memory, converting the projected centre to a tile-relative offset in double-float so
// that per-pixel offsets stay exact to float32 rounding of the offset itself.  Per pixel:
//   y01 = G (px - u), y2 = 1 + h . (px - u), q = |y01|^2, r = y2^2
//   contributes iff y2 > 0 and kp q <= r           (D <= kappa, Eq. support)
//   D log2(e)/2 = c2h q / (q + r)                   (fragment formula)
//   omega = min(alpha_max, 2^(log2 o - D log2(e)/2))
// Compositing stops before a primitive that would take T below t_stop; a CTA leaves the
// list as soon as every pixel has stopped.
#include "raygs_internal.cuh"

namespace raygs {


template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(TW *TH) render_kernel(RenderParams P) {
  constexpr int NT = TW * TH;
  __shared__ float4 s_A[NT], s_B[NT], s_C[NT], s_D[NT];
  __shared__ int s_view;
  const int tile = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int v = 0;
    while (v + 1 < P.n_views && P.cams[v + 1].tile_base <= tile) ++v;
    s_view = v;
  }
  __syncthreads();
  const DevCam &cam = P.cams[s_view];
  const int local = tile - cam.tile_base;
  const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
  const int px0 = tx * TW, py0 = ty * TH;
  const int lx = tid % TW, ly = tid / TW;
  const int px = px0 + lx, py = py0 + ly;
  const bool inside = px < cam.W && py < cam.H;
  const uint2 rg = P.ranges[tile];
  const float ox_tile = float(px0) + 0.5f, oy_tile = float(py0) + 0.5f;
  const float fl_x = float(lx), fl_y = float(ly);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !inside;
  unsigned long long n_eval = 0, n_comp = 0;

  for (uint32_t start = rg.x; start < rg.y; start += NT) {
    if (__syncthreads_and(done)) break;
    const uint32_t i = start + tid;
    if (i < rg.y) {
      const uint32_t pos = P.inst_vals[i];
      const Rec r = P.rec[P.pairs[pos]];
      df ox = two_sum(ox_tile, -r.a.x);
      df oy = two_sum(oy_tile, -r.a.y);
      s_A[tid] = make_float4(__fadd_rn(ox.hi, __fsub_rn(ox.lo, r.a.z)),
                             __fadd_rn(oy.hi, __fsub_rn(oy.lo, r.a.w)), r.b.x, r.b.y);
      s_B[tid] = make_float4(r.b.z, r.b.w, r.c.x, r.c.y);
      s_C[tid] = make_float4(r.c.z, r.c.w, r.d.x, 0.f);
      s_D[tid] = make_float4(r.d.y, r.d.z, r.d.w, 0.f);
    }
    __syncthreads();
    const int nb = min(NT, int(rg.y - start));
    if (!done) {
      int j = 0;
      for (; j < nb; ++j) {
        const float4 A = s_A[j], B = s_B[j];
        const float dx = A.x + fl_x, dy = A.y + fl_y;
        const float y0 = fmaf(A.z, dx, A.w * dy);
        const float y1 = fmaf(B.x, dx, B.y * dy);
        const float y2 = fmaf(B.z, dx, fmaf(B.w, dy, 1.f));
        const float q = fmaf(y0, y0, y1 * y1);
        const float rr = y2 * y2;
        const float4 Cc = s_C[j];
        if (y2 > 0.f && Cc.x * q <= rr) {
          const float E = Cc.y * __fdividef(q, q + rr);
          const float al = fminf(P.alpha_max, ex2_approx(Cc.z - E));
          const float Tn = T * (1.f - al);
          if (Tn < P.t_stop) {
            done = true;
            break;
          }
          const float4 Dd = s_D[j];
          const float w = al * T;
          C0 = fmaf(w, Dd.x, C0);
          C1 = fmaf(w, Dd.y, C1);
          C2 = fmaf(w, Dd.z, C2);
          T = Tn;
          last = int(start - rg.x) + j + 1;
          if (COUNT) ++n_comp;
        }
      }
      if (COUNT) n_eval += (j < nb) ? j + 1 : nb;
    }
  }
  if (inside) {
    const long long pix = cam.pix_base + (long long)py * cam.W + px;
    P.rgb[3 * pix] = C0;
    P.rgb[3 * pix + 1] = C1;
    P.rgb[3 * pix + 2] = C2;
    if (P.Tf) P.Tf[pix] = T;
    if (P.ncontrib) P.ncontrib[pix] = last;
  }
  if (COUNT) {
    // warp reduce, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_eval += __shfl_down_sync(0xffffffffu, n_eval, o);
      n_comp += __shfl_down_sync(0xffffffffu, n_comp, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(&P.eval_counts[0], n_eval);
      atomicAdd(&P.eval_counts[1], n_comp);
    }
  }
}

cudaError_t launch_render(const RenderParams &P, int tile_w, int tile_h, int64_t n_tiles, bool count,
                          cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  const unsigned grid = unsigned(n_tiles);
#define RAYGS_RENDER_CASE(TW, TH)                                                      \
  if (tile_w == TW && tile_h == TH) {                                                  \
    if (count) render_kernel<TW, TH, true><<<grid, TW * TH, 0, st>>>(P);               \
    else render_kernel<TW, TH, false><<<grid, TW * TH, 0, st>>>(P);                    \
    return cudaGetLastError();                                                         \
  }
  RAYGS_RENDER_CASE(16, 16)
  RAYGS_RENDER_CASE(16, 8)
  RAYGS_RENDER_CASE(32, 16)
  RAYGS_RENDER_CASE(8, 8)
#undef RAYGS_RENDER_CASE
  return cudaErrorInvalidValue;
}

}  // namespace raygs
