// Per-tile rasterisation and front-to-back compositing (Sec. 3 Eq. rendering and
// Eq. rend_opacity; Sec. 4.2 fragment formula).
//
// Persistent CTAs (one per resident slot) claim the screen tiles of all views from a
// counter, one at a time; each thread shades PX pixels of a tile row.  A tile's instance list (depth order) is consumed in batches: each thread
// stages records in shared memory, converting the projected centre to a tile-relative
// offset in double-float so that per-pixel offsets stay exact to the float32 rounding of
// the offset itself.  Per pixel, with delta = pixel centre - projected centre:
//   y01 = G delta, y2 = 1 + h . delta, q = |y01|^2, r = y2^2
//   contributes iff y2 > 0 and kp q - r <= 0          (D <= kappa, Eq. support)
//   D log2(e)/2 = c2h q / (q + r)                     (fragment formula)
//   omega = min(alpha_max, 2^(log2 o - D log2(e)/2))
// With the GS divergence of Sec. 3.1 the records carry h = 0 and G with G^T G = Sigma_pi^-1,
// so that r = 1, the test reads q <= kappa and D log2(e)/2 = c2h q (DIV = 1 below).  The
// records' G carries sqrt(kp), so that the support test is the single compare q' <= r.
// A thread's PX pixels lie on one tile row, interleaved with the other threads of that
// row (columns lx, lx + QX, lx + 2 QX, ...), so that a footprint covering a range of
// columns hits the same pixel slots k in every lane of the row and the per-slot
// compositing stays convergent.  The PX pixels share the row term of y and step the
// column term by QX pixels (y += QX G[:,0]).  Compositing of a pixel stops before a primitive that would take T
// below t_stop; a thread skips records once its pixels have all stopped, and the CTA
// leaves the list once every thread has.
#include "raygs_internal.cuh"
#include "raster_math.cuh"

namespace raygs {

template <int TW, int TH, int PX, int NBF, bool COUNT, int DIV>
__global__ void __launch_bounds__(TW *TH / PX, 16) render_kernel(RenderParams P) {
  constexpr int NT = TW * TH / PX;  // threads
  constexpr int NB = NBF * NT;      // records per batch
  constexpr int QX = TW / PX;       // threads per tile row
  __shared__ float4 s_A[NB], s_B[NB], s_C[NB], s_D[NB];
  __shared__ Rec s_raw[NB];
  __shared__ int s_view, s_tile;
  const int tid = threadIdx.x;
  // persistent CTAs: each claims the next tile until none is left
  for (;;) {
  if (tid == 0) s_tile = int(atomicAdd(P.tile_counter, 1u));
  __syncthreads();
  const int tile = s_tile;
  if (tile >= P.n_tiles) break;
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

  float T[PX], C0[PX], C1[PX], C2[PX];
  int last[PX];
  uint32_t alive = 0;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    T[k] = 1.f; C0[k] = 0.f; C1[k] = 0.f; C2[k] = 0.f; last[k] = 0;
    if (py < cam.H && px + k * QX < cam.W) alive |= 1u << k;
  }
  const uint32_t inside = alive;
  unsigned long long n_eval = 0, n_comp = 0, n_iter = 0;
  uint32_t stop_at = rg.y;  // first list entry the CTA did not stage

  // Records move through a two-stage pipeline: while a batch is composited, the raw
  // records of the next batch are in flight to shared memory (cp.async) and the record
  // indices of the batch after that are being loaded into registers.
  constexpr int PER = NB / NT;
  uint32_t nxt[PER];
#pragma unroll
  for (int rr = 0; rr < PER; ++rr) {
    const uint32_t i = rg.x + tid + rr * NT;
    if (i < rg.y) cp_async_rec(&s_raw[tid + rr * NT], &P.rec[P.pairs[P.inst_vals[i]]]);
  }
  cp_async_commit();
#pragma unroll
  for (int rr = 0; rr < PER; ++rr) {
    const uint32_t i = rg.x + NB + tid + rr * NT;
    nxt[rr] = i < rg.y ? P.pairs[P.inst_vals[i]] : 0u;
  }

  for (uint32_t start = rg.x; start < rg.y; start += NB) {
    if (__syncthreads_and(alive == 0)) {
      stop_at = start;
      break;
    }
    cp_async_wait_all();  // this thread's raw slots of the batch have landed
#pragma unroll
    for (int rr = 0; rr < PER; ++rr) {
      const int slot = tid + rr * NT;
      if (start + slot < rg.y)
        stage_record<DIV>(s_raw[slot], ox_tile, oy_tile, s_A[slot], s_B[slot], s_C[slot], s_D[slot]);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < PER; ++rr) {
      const uint32_t i = start + NB + tid + rr * NT;
      if (i < rg.y) cp_async_rec(&s_raw[tid + rr * NT], &P.rec[nxt[rr]]);
    }
    cp_async_commit();
#pragma unroll
    for (int rr = 0; rr < PER; ++rr) {
      const uint32_t i = start + 2 * NB + tid + rr * NT;
      nxt[rr] = i < rg.y ? P.pairs[P.inst_vals[i]] : 0u;
    }
    const int nb = min(NB, int(rg.y - start));
    // two records per iteration give the scheduler independent work (8 pixels per thread
    // would spill)
#pragma unroll(PX >= 8 ? 1 : 2)
    for (int j = 0; j < nb && alive; ++j) {
      const float4 A = s_A[j], B = s_B[j];
      const float4 Cc = s_C[j];
      if (COUNT) { n_eval += __popc(alive); ++n_iter; }
      // with 8 pixels per thread a conservative segment test pays for itself (fewer
      // pixels per thread are cheaper to test directly); the instrumented variant tests
      // every pixel, so its image checks the filter
      if (PX >= 8 && !COUNT && !row_may_hit<PX>(A, B, Cc, s_D[j].w, fl_x, fl_y, step)) continue;
      float q[PX], r[PX], y0[PX], y1[PX], y2[PX];
      uint32_t hit = eval_pixels<PX>(A, B, fl_x, fl_y, step, q, r, y0, y1, y2);
      hit &= alive;
      if (hit) {
        const float4 Dd = s_D[j];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          if (hit & (1u << k)) {
            const float al = fminf(P.alpha_max, pixel_opacity<DIV>(Cc, q[k], r[k]));
            const float w = al * T[k];
            const float Tn = T[k] - w;
            if (Tn < P.t_stop) {
              alive &= ~(1u << k);
            } else {
              C0[k] = fmaf(w, Dd.x, C0[k]);
              C1[k] = fmaf(w, Dd.y, C1[k]);
              C2[k] = fmaf(w, Dd.z, C2[k]);
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
  const bool alive_any = COUNT ? __syncthreads_or(alive != 0) : false;
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
      n_iter += __shfl_down_sync(0xffffffffu, n_iter, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(&P.eval_counts[0], n_eval);
      atomicAdd(&P.eval_counts[1], n_comp);
      atomicAdd(&P.eval_counts[3], n_iter);
    }
    if (tid == 0) {
      atomicAdd(&P.eval_counts[2], (unsigned long long)(stop_at - rg.x));
      if (P.tile_stop) P.tile_stop[tile] = alive_any ? kCulled : stop_at - rg.x;
    }
  }
  __syncthreads();  // shared state and s_tile are free before the next claim
  }
}

// One CTA per resident slot (occupancy of the instantiation x SMs), at most one per tile.
template <typename K>
static unsigned persistent_grid(K kernel, int threads, int num_sms, int n_tiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long g = (long long)per_sm * (long long)(num_sms > 0 ? num_sms : 1);
  return unsigned(g < n_tiles ? g : n_tiles);
}

cudaError_t launch_render(const RenderParams &P, int tile_w, int tile_h, int batch_records, int num_sms,
                          bool count, cudaStream_t st) {
  if (P.n_tiles <= 0) return cudaSuccess;
  const bool gs = P.qmix == 0.f;  // D_gs records (Sec. 3.1)
#define RAYGS_RENDER_LAUNCH(TW, TH, PX, NBF, C, D)                                                   \
  {                                                                                                   \
    auto k = render_kernel<TW, TH, PX, NBF, C, D>;                                                    \
    k<<<persistent_grid(k, TW * TH / PX, num_sms, P.n_tiles), TW * TH / PX, 0, st>>>(P);              \
  }
#define RAYGS_RENDER_CASE(TW, TH, PX, NBF)                                                             \
  if (tile_w == TW && tile_h == TH && batch_records == NBF) {                                         \
    if (gs) {                                                                                         \
      if (count) RAYGS_RENDER_LAUNCH(TW, TH, PX, NBF, true, 1)                                        \
      else RAYGS_RENDER_LAUNCH(TW, TH, PX, NBF, false, 1)                                             \
    } else {                                                                                          \
      if (count) RAYGS_RENDER_LAUNCH(TW, TH, PX, NBF, true, 0)                                        \
      else RAYGS_RENDER_LAUNCH(TW, TH, PX, NBF, false, 0)                                             \
    }                                                                                                 \
    return cudaGetLastError();                                                                        \
  }
  RAYGS_RENDER_CASE(16, 16, 4, 1)
  RAYGS_RENDER_CASE(16, 8, 4, 1)
  RAYGS_RENDER_CASE(32, 16, 8, 1)
  RAYGS_RENDER_CASE(8, 8, 2, 1)
  RAYGS_RENDER_CASE(16, 16, 4, 2)
  RAYGS_RENDER_CASE(16, 8, 4, 2)
  RAYGS_RENDER_CASE(32, 16, 8, 2)
  RAYGS_RENDER_CASE(8, 8, 2, 2)
#undef RAYGS_RENDER_CASE
#undef RAYGS_RENDER_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace raygs
