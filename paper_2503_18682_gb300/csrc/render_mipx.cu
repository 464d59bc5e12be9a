// Per-tile rasterisation with the exact, pixel-dependent anti-aliasing of Sec. 5: the
// pixel-invariant Sigma^ of Eq. mip replaced by Sigma^_x = Sigma + sigma_x^2 tau(x)^2 I and
// the modulation sqrt(|Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x)) evaluated for
// every pixel ray.  Work distribution, record pipeline, compositing and termination are
// those of the plain rasteriser (render.cu); the record is two 64-byte halves (rec, recx)
// whose fields are described with MipxOut in preprocess.cu.  Per pixel, with delta the
// offset from the projected centre:
//   y_k = b_k + g_k . delta, e_k = A_k . delta, t = m . y / |y|^2   (tau under Sigma, ray
//   x = (X, Y, 1)), l = t^2 / |x|, u_k = 1 + l w_k
//   Num = sum u_k e_k^2, Den = sum y_k^2 prod_{j != k} u_j
//   contributes iff t > 0, sum m_k y_k prod_{j != k} u_j > 0 (tau^ > 0) and
//   omega = o sqrt(|y|^2 / Den) exp(-Num / (2 Den)) >= p_min; the test Num <= kappa Den
//   (the modulation never exceeds 1) rejects first without a division.
#include "raygs_internal.cuh"
#include "raster_math.cuh"

namespace raygs {

template <int TW, int TH, int PX, bool COUNT>
__global__ void __launch_bounds__(TW *TH / PX, 8) render_mipx_kernel(RenderParams P) {
  constexpr int NT = TW * TH / PX;  // threads; one record per thread and batch
  constexpr int QX = TW / PX;       // threads per tile row
  __shared__ float4 s_S[7][NT];
  __shared__ Rec s_raw[2][NT];
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
  const int lx = tid % QX, ly = tid / QX;
  const int px = px0 + lx, py = py0 + ly;
  const uint2 rg = P.ranges[tile];
  const float ox_tile = float(px0) + 0.5f, oy_tile = float(py0) + 0.5f;
  const float fl_x = float(lx), fl_y = float(ly), step = float(QX);
  const float c2h = 0.5f * kLog2e;

  float T[PX], C0[PX], C1[PX], C2[PX], ixn[PX];
  int last[PX];
  uint32_t alive = 0;
  const float Yr = (float(py) + 0.5f - cam.cy) * cam.ify;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    T[k] = 1.f; C0[k] = 0.f; C1[k] = 0.f; C2[k] = 0.f; last[k] = 0;
    if (py < cam.H && px + k * QX < cam.W) alive |= 1u << k;
    const float Xr = (float(px + k * QX) + 0.5f - cam.cx) * cam.ifx;
    ixn[k] = rsqrtf(fmaf(Xr, Xr, fmaf(Yr, Yr, 1.f)));  // 1 / |x|
  }
  const uint32_t inside = alive;
  unsigned long long n_eval = 0, n_comp = 0;

  // two-stage pipeline as in render.cu: raw halves of the next batch in flight (cp.async),
  // pair indices of the batch after that in a register
  uint32_t nxt;
  {
    const uint32_t i = rg.x + tid;
    if (i < rg.y) {
      const uint32_t pr = P.pairs[P.inst_vals[i]];
      cp_async_rec(&s_raw[0][tid], &P.rec[pr]);
      cp_async_rec(&s_raw[1][tid], &P.recx[pr]);
    }
    cp_async_commit();
    const uint32_t i2 = rg.x + NT + tid;
    nxt = i2 < rg.y ? P.pairs[P.inst_vals[i2]] : 0u;
  }

  for (uint32_t start = rg.x; start < rg.y; start += NT) {
    if (__syncthreads_and(alive == 0)) break;
    cp_async_wait_all();
    if (start + tid < rg.y) {
      const Rec &r = s_raw[0][tid], &q = s_raw[1][tid];
      const df ox = two_sum(ox_tile, -r.a.x);
      const df oy = two_sum(oy_tile, -r.a.y);
      s_S[0][tid] = make_float4(__fadd_rn(ox.hi, __fsub_rn(ox.lo, r.a.z)),
                                __fadd_rn(oy.hi, __fsub_rn(oy.lo, r.a.w)), r.b.x, r.b.y);
      s_S[1][tid] = make_float4(r.b.z, r.b.w, r.c.x, r.c.y);
      s_S[2][tid] = make_float4(r.c.z, r.c.w, r.d.x, r.d.y);
      s_S[3][tid] = make_float4(r.d.z, r.d.w, q.a.x, q.a.y);
      s_S[4][tid] = make_float4(q.a.z, q.b.x, q.b.y, q.b.z);
      s_S[5][tid] = make_float4(q.c.x, q.c.y, q.c.z, q.a.w);
      s_S[6][tid] = make_float4(q.b.w, q.d.x, q.d.y, q.d.z);
    }
    __syncthreads();
    {
      const uint32_t i = start + NT + tid;
      if (i < rg.y) {
        cp_async_rec(&s_raw[0][tid], &P.rec[nxt]);
        cp_async_rec(&s_raw[1][tid], &P.recx[nxt]);
      }
      cp_async_commit();
      const uint32_t i2 = start + 2 * NT + tid;
      nxt = i2 < rg.y ? P.pairs[P.inst_vals[i2]] : 0u;
    }
    const int nb = min(NT, int(rg.y - start));
    for (int j = 0; j < nb && alive; ++j) {
      const float4 S0 = s_S[0][j], S1 = s_S[1][j], S2 = s_S[2][j], S3 = s_S[3][j];
      const float4 S4 = s_S[4][j], S5 = s_S[5][j];
      if (COUNT) n_eval += __popc(alive);
      const float dy = S0.y + fl_y;
      const float dx0 = S0.x + fl_x;
      // row terms of the affine forms
      const float e0r = S0.w * dy, e1r = S1.y * dy, e2r = S1.w * dy;
      const float y0r = fmaf(S2.y, dy, S3.z), y1r = fmaf(S2.w, dy, S3.w), y2r = fmaf(S3.y, dy, S4.x);
      float om[PX];
      uint32_t hit = 0;
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        const float dx = dx0 + float(k) * step;
        const float e0 = fmaf(S0.z, dx, e0r), e1 = fmaf(S1.x, dx, e1r), e2 = fmaf(S1.z, dx, e2r);
        const float y0 = fmaf(S2.x, dx, y0r), y1 = fmaf(S2.z, dx, y1r), y2 = fmaf(S3.x, dx, y2r);
        const float my0 = S4.y * y0, my1 = S4.z * y1, my2 = S4.w * y2;
        const float tn = my0 + my1 + my2;
        const float yy = fmaf(y0, y0, fmaf(y1, y1, y2 * y2));
        const float t = __fdividef(tn, yy);
        const float l = t * t * ixn[k];
        const float u0 = fmaf(l, S5.x, 1.f), u1 = fmaf(l, S5.y, 1.f), u2 = fmaf(l, S5.z, 1.f);
        const float u12 = u1 * u2, u02 = u0 * u2, u01 = u0 * u1;
        const float num = fmaf(u0 * e0, e0, fmaf(u1 * e1, e1, u2 * e2 * e2));
        const float den = fmaf(y0 * y0, u12, fmaf(y1 * y1, u02, y2 * y2 * u01));
        const float sg = fmaf(my0, u12, fmaf(my1, u02, my2 * u01));
        om[k] = 0.f;
        if (tn > 0.f && sg > 0.f && num <= s_S[6][j].x * den) {
          const float iden = __fdividef(1.f, den);
          const float lg = __log2f(yy * iden);
          const float w = ex2_approx(fmaf(0.5f, lg, S5.w) - c2h * num * iden);
          om[k] = w;
          if (w >= P.p_min) hit |= 1u << k;
        }
      }
      hit &= alive;
      if (hit) {
        const float4 S6 = s_S[6][j];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          if (hit & (1u << k)) {
            const float al = fminf(P.alpha_max, om[k]);
            const float w = al * T[k];
            const float Tn = T[k] - w;
            if (Tn < P.t_stop) {
              alive &= ~(1u << k);
            } else {
              C0[k] = fmaf(w, S6.y, C0[k]);
              C1[k] = fmaf(w, S6.z, C1[k]);
              C2[k] = fmaf(w, S6.w, C2[k]);
              T[k] = Tn;
              last[k] = int(start - rg.x) + j + 1;
              if (COUNT) ++n_comp;
            }
          }
        }
      }
    }
  }
  cp_async_wait_all();  // no copy may outlive the block
  if (inside) {
    const long long pix = cam.pix_base + (long long)py * cam.W + px;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      if (inside & (1u << k)) {
        const long long o = pix + k * QX;
        P.rgb[3 * o] = C0[k];
        P.rgb[3 * o + 1] = C1[k];
        P.rgb[3 * o + 2] = C2[k];
        if (P.Tf) P.Tf[o] = T[k];
        if (P.ncontrib) P.ncontrib[o] = last[k];
      }
    }
  }
  if (COUNT) {
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

cudaError_t launch_render_mipx(const RenderParams &P, int tile_w, int tile_h, int64_t n_tiles, bool count,
                               cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  const unsigned grid = unsigned(n_tiles);
#define RAYGS_MIPX_CASE(TW, TH, PX)                                                        \
  if (tile_w == TW && tile_h == TH) {                                                      \
    if (count) render_mipx_kernel<TW, TH, PX, true><<<grid, TW * TH / PX, 0, st>>>(P);     \
    else render_mipx_kernel<TW, TH, PX, false><<<grid, TW * TH / PX, 0, st>>>(P);          \
    return cudaGetLastError();                                                             \
  }
  RAYGS_MIPX_CASE(16, 16, 4)
  RAYGS_MIPX_CASE(16, 8, 4)
  RAYGS_MIPX_CASE(32, 16, 8)
  RAYGS_MIPX_CASE(8, 8, 2)
#undef RAYGS_MIPX_CASE
  return cudaErrorInvalidValue;
}

}  // namespace raygs
