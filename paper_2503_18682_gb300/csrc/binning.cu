// Binning for the depth order of Eq. rendering.
//
//   1. Stable LSD radix sort of the visible (primitive, view) pairs by float32 centre
//      depth.  The first pass reads the dense per-(view, primitive) key array, drops
//      culled entries and materialises the pair index as the value, so ties keep the
//      primitive order within a view.
//   2. Two-level, load-balanced expansion in that order: each pair -> the tile rows of its
//      screen rectangle; each row -> the tiles of the row whose pixel centres can meet the
//      pair's support ellipse (an exact conic test, so tiles the support misses get no
//      instance); each tile -> one instance (global tile id, sorted pair position).
//   3. Stable LSD radix sort of the instances by tile id -> per tile, depth order.
//   4. Per-tile [start, end) ranges.
//
// The radix sort is reduce-then-scan (upsweep histogram, one-CTA scan, downsweep
// scatter) with persistent CTAs that own contiguous tile ranges: no CTA ever waits on
// another.  The upsweep counts runs of equal digits per thread; ranking inside a tile is
// stable (warp match + per-warp counters) and the scatter goes through shared memory so
// that global writes are coalesced runs.
#include "raygs_internal.cuh"

namespace raygs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;  // 2048 items

__device__ __forceinline__ void cta_tiles(uint32_t count, uint32_t &lo, uint32_t &hi) {
  uint32_t ntiles = (count + kSortTile - 1) / kSortTile;
  uint32_t t0 = uint32_t((uint64_t(ntiles) * blockIdx.x) / gridDim.x);
  uint32_t t1 = uint32_t((uint64_t(ntiles) * (blockIdx.x + 1)) / gridDim.x);
  lo = t0 * kSortTile;
  hi = min(t1 * uint32_t(kSortTile), count);
  if (lo > hi) lo = hi;
}

__device__ __forceinline__ uint32_t pass_count(const SortPass &p) {
  return p.d_count ? min(*p.d_count, p.count_max) : p.count_max;
}

// Digit histogram of the CTA's items.  Each thread counts 16 consecutive keys as runs of
// equal digits (the tile-id passes see long runs: instances come in depth order, tile rows
// in order) and adds each run once to its warp's shared histogram.
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) sort_upsweep(SortPass p) {
  constexpr int R = 1 << BITS;
  constexpr int KPT = 16;  // keys per thread per step
  __shared__ uint32_t h[kSortWarps][R];
  for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  uint32_t lo, hi;
  cta_tiles(pass_count(p), lo, hi);
  const int warp = threadIdx.x >> 5;
  for (uint32_t base = lo; base < hi; base += kSortThreads * KPT) {
    const uint32_t i0 = base + threadIdx.x * KPT;
    uint32_t k[KPT];
    if (i0 + KPT <= hi) {
#pragma unroll
      for (int q = 0; q < KPT / 4; ++q) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p.keys_in + i0 + 4 * q);
        k[4 * q] = v.x; k[4 * q + 1] = v.y; k[4 * q + 2] = v.z; k[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < KPT; ++j) k[j] = i0 + j < hi ? p.keys_in[i0 + j] : kCulled;
    }
    uint32_t cur = 0xFFFFFFFFu, cnt = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const bool valid = i0 + j < hi && !(p.filter && k[j] == kCulled);
      if (!valid) continue;
      const uint32_t d = (k[j] >> p.shift) & (R - 1);
      if (d == cur) {
        ++cnt;
      } else {
        if (cnt) atomicAdd(&h[warp][cur], cnt);
        cur = d;
        cnt = 1;
      }
    }
    if (cnt) atomicAdd(&h[warp][cur], cnt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < R; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
    p.hist[size_t(d) * p.G + blockIdx.x] = s;
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan (blockDim.x multiple of 32, <= 1024).  Returns the exclusive
// prefix; *total receives the block total.  Uses `ws` (>= 33 words of shared memory).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *ws, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_incl_scan(x);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? ws[lane] : 0u;
    uint32_t vi = warp_incl_scan(v);
    if (lane < nw) ws[lane] = vi - v;
    if (lane == nw - 1) ws[32] = vi;
  }
  __syncthreads();
  uint32_t r = inc - x + ws[warp];
  *total = ws[32];
  __syncthreads();
  return r;
}

// Exclusive scan of `n` entries in place with one CTA of 1024 threads; the total goes to
// *d_total when non-null.
__global__ void __launch_bounds__(1024) scan_single_cta(uint32_t *data, int n, uint32_t *d_total) {
  __shared__ uint32_t ws[33];
  const int seg = (n + 1023) / 1024;
  const int b = threadIdx.x * seg, e = min(b + seg, n);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += data[i];
  uint32_t tot;
  uint32_t run = block_excl_scan(s, ws, &tot);
  for (int i = b; i < e; ++i) {
    uint32_t v = data[i];
    data[i] = run;
    run += v;
  }
  if (d_total && threadIdx.x == 0) *d_total = tot;
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads, 4) sort_downsweep(SortPass p) {
  constexpr int R = 1 << BITS;
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_cnt[kSortWarps][R];
  __shared__ uint32_t s_base[R];
  __shared__ uint32_t s_tpre[R];
  __shared__ uint32_t s_tot[R];
  __shared__ uint32_t s_ws[33];

  uint32_t lo, hi;
  cta_tiles(pass_count(p), lo, hi);
  for (int d = threadIdx.x; d < R; d += kSortThreads) s_base[d] = p.hist[size_t(d) * p.G + blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;

  // keys and values of the next tile are loaded while the current one is ranked
  uint32_t nkey[kSortIPT], nval[kSortIPT];
  auto load_tile = [&](uint32_t base) {
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      const bool ok = idx < hi;
      nkey[r] = ok ? p.keys_in[idx] : 0u;
      nval[r] = ok ? (p.filter ? idx : p.vals_in[idx]) : 0u;
    }
  };
  if (lo < hi) load_tile(lo);
  for (uint32_t base = lo; base < hi; base += kSortTile) {
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    uint32_t key[kSortIPT], val[kSortIPT], off[kSortIPT];
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) { key[r] = nkey[r]; val[r] = nval[r]; }
    if (base + kSortTile < hi) load_tile(base + kSortTile);
    __syncthreads();
    uint32_t vmask = 0;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      const bool ok = idx < hi;
      const uint32_t k = key[r];
      const uint32_t v = val[r];
      const bool valid = ok && !(p.filter && k == kCulled);
      uint32_t d = (k >> p.shift) & (R - 1);
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : uint32_t(R + lane));
      uint32_t c = valid ? s_cnt[warp][d] : 0u;
      __syncwarp();
      if (valid && lane == 31 - __clz(peers)) s_cnt[warp][d] = c + __popc(peers);
      __syncwarp();
      off[r] = c + __popc(peers & lt);
      vmask |= valid ? (1u << r) : 0u;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t c = s_cnt[w][d];
        s_cnt[w][d] = run;
        run += c;
      }
      s_tot[d] = run;
    }
    __syncthreads();
    {
      constexpr int PER = (R + kSortThreads - 1) / kSortThreads;
      uint32_t loc[PER];
      uint32_t s = 0;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        int d = threadIdx.x * PER + j;
        loc[j] = d < R ? s_tot[d] : 0u;
        s += loc[j];
      }
      uint32_t tot;
      uint32_t run = block_excl_scan(s, s_ws, &tot);
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        int d = threadIdx.x * PER + j;
        if (d < R) s_tpre[d] = run;
        run += loc[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      if (vmask & (1u << r)) {
        uint32_t d = (key[r] >> p.shift) & (R - 1);
        uint32_t pos = s_tpre[d] + s_cnt[warp][d] + off[r];
        s_keys[pos] = key[r];
        s_vals[pos] = val[r];
      }
    }
    __syncthreads();
    const uint32_t nvalid = s_tpre[R - 1] + s_tot[R - 1];
    for (uint32_t j = threadIdx.x; j < nvalid; j += kSortThreads) {
      uint32_t k = s_keys[j];
      uint32_t d = (k >> p.shift) & (R - 1);
      uint32_t dst = s_base[d] + j - s_tpre[d];
      p.keys_out[dst] = k;
      p.vals_out[dst] = s_vals[j];
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) s_base[d] += s_tot[d];
    __syncthreads();
  }
}

// Exclusive scan of the digit-major histogram [R][G] in place, in three steps: per-block
// sums (one block per 2048 entries), a scan of the block sums, and the block-local scans.
constexpr int kHistBlock = 2048;

__global__ void __launch_bounds__(256) hist_reduce_kernel(const uint32_t *hist, int n, uint32_t *bsum) {
  __shared__ uint32_t ws[33];
  const int b0 = blockIdx.x * kHistBlock;
  uint32_t s = 0;
  for (int i = b0 + threadIdx.x; i < min(b0 + kHistBlock, n); i += blockDim.x) s += hist[i];
  uint32_t tot;
  block_excl_scan(s, ws, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) hist_bsum_kernel(uint32_t *bsum, int nb, uint32_t *d_total) {
  __shared__ uint32_t ws[33];
  const int per = (nb + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(b + per, nb);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += bsum[i];
  uint32_t tot;
  uint32_t run = block_excl_scan(s, ws, &tot);
  for (int i = b; i < e; ++i) {
    const uint32_t v = bsum[i];
    bsum[i] = run;
    run += v;
  }
  if (d_total && threadIdx.x == 0) *d_total = tot;
}

__global__ void __launch_bounds__(256) hist_offsets_kernel(uint32_t *hist, int n, const uint32_t *bsum) {
  __shared__ uint32_t ws[33];
  const int b0 = blockIdx.x * kHistBlock;
  constexpr int PER = kHistBlock / 256;
  uint32_t v[PER], s = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = b0 + threadIdx.x * PER + j;
    v[j] = i < n ? hist[i] : 0u;
    s += v[j];
  }
  uint32_t tot;
  uint32_t run = bsum[blockIdx.x] + block_excl_scan(s, ws, &tot);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = b0 + threadIdx.x * PER + j;
    if (i < n) hist[i] = run;
    run += v[j];
  }
}

cudaError_t launch_sort_pass(const SortPass &p, cudaStream_t st) {
  const int n = (p.bits == 9 ? 512 : 256) * p.G;
  const int nb = (n + kHistBlock - 1) / kHistBlock;
  uint32_t *bsum = p.hist + n;  // scratch after the histogram (the layout reserves 512*G + G)
  if (p.bits == 9) sort_upsweep<9><<<p.G, kSortThreads, 0, st>>>(p);
  else sort_upsweep<8><<<p.G, kSortThreads, 0, st>>>(p);
  hist_reduce_kernel<<<nb, 256, 0, st>>>(p.hist, n, bsum);
  hist_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nb, p.d_total);
  hist_offsets_kernel<<<nb, 256, 0, st>>>(p.hist, n, bsum);
  if (p.bits == 9) sort_downsweep<9><<<p.G, kSortThreads, 0, st>>>(p);
  else sort_downsweep<8><<<p.G, kSortThreads, 0, st>>>(p);
  return cudaGetLastError();
}

// --------------------------------------------------------------- generic unit scan
__device__ __forceinline__ void cta_range_units(uint32_t count, uint32_t &lo, uint32_t &hi) {
  constexpr uint32_t U = 1024;
  uint32_t nu = (count + U - 1) / U;
  uint32_t t0 = uint32_t((uint64_t(nu) * blockIdx.x) / gridDim.x);
  uint32_t t1 = uint32_t((uint64_t(nu) * (blockIdx.x + 1)) / gridDim.x);
  lo = min(t0 * U, count);
  hi = min(t1 * U, count);
}

__global__ void __launch_bounds__(256) scan_reduce_kernel(ScanJob J) {
  __shared__ uint32_t ws[33];
  uint32_t lo, hi;
  cta_range_units(*J.d_n, lo, hi);
  uint32_t s = 0;
  for (uint32_t p = lo + threadIdx.x; p < hi; p += blockDim.x) s += J.cnt[p];
  uint32_t tot;
  block_excl_scan(s, ws, &tot);
  if (threadIdx.x == 0) J.partial[blockIdx.x] = tot;
}

// Exclusive scan of the G <= 1024 per-CTA partial sums (64-bit running total); writes the
// total, the capacity-clamped total and the overflow flag.
__global__ void __launch_bounds__(32) scan_partials_kernel(ScanJob J, int G) {
  if (threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int i = 0; i < G; ++i) {
    uint32_t v = J.partial[i];
    J.partial[i] = uint32_t(min(run, 0xFFFFFFFFull));
    run += v;
  }
  *J.d_total = run;
  *J.d_total_clamped = run > J.cap ? J.cap : uint32_t(run);
  if (run > J.cap) *J.d_overflow = 1u;
}

__global__ void __launch_bounds__(256) scan_offsets_kernel(ScanJob J) {
  __shared__ uint32_t ws[33];
  uint32_t lo, hi;
  cta_range_units(*J.d_n, lo, hi);
  uint32_t carry = J.partial[blockIdx.x];
  for (uint32_t base = lo; base < hi; base += 256 * 4) {
    uint32_t c[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t p = base + threadIdx.x * 4 + j;
      c[j] = p < hi ? J.cnt[p] : 0u;
      s += c[j];
    }
    uint32_t tot;
    uint32_t run = carry + block_excl_scan(s, ws, &tot);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t p = base + threadIdx.x * 4 + j;
      if (p < hi) {
        J.off[p] = run;
        // every output block whose first output falls in [run, run + c) starts at unit p
        uint32_t t = (run + kEmitTile - 1) / kEmitTile;
        for (; uint64_t(t) * kEmitTile < uint64_t(run) + c[j] && t < J.tstart_len; ++t) J.tile_start[t] = p;
      }
      run += c[j];
    }
    carry += tot;
  }
}

cudaError_t launch_scan(const ScanJob &J, int G, cudaStream_t st) {
  scan_reduce_kernel<<<G, 256, 0, st>>>(J);
  scan_partials_kernel<<<1, 32, 0, st>>>(J, G);
  scan_offsets_kernel<<<G, 256, 0, st>>>(J);
  return cudaGetLastError();
}

// ------------------------------------------------------------ pair -> tile rows
__global__ void __launch_bounds__(256) count_rows_kernel(const uint32_t *pairs, const uint2 *rect, uint32_t *cnt,
                                                         const Counters *c) {
  const uint32_t n = c->n_visible;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    uint2 r = rect[pairs[p]];
    cnt[p] = (r.y >> 16) - (r.x >> 16) + 1;
  }
}

cudaError_t launch_count_rows(const uint32_t *pairs, const uint2 *rect, uint32_t *cnt, const Counters *c, int G,
                              cudaStream_t st) {
  count_rows_kernel<<<G, 256, 0, st>>>(pairs, rect, cnt, c);
  return cudaGetLastError();
}

// Pixel-centre columns of the band ya <= y <= yb (pixel-centre rows) inside the ellipse.
// The right boundary x_r(y) is concave with its maximum at the rightmost point of the
// ellipse, the left one convex: clamping that point's y into the band gives the extremes.
__device__ __forceinline__ bool ellipse_band(const Ell &e, float ya, float yb, float &xa, float &xb) {
  const float rho = e.rho * 1.001f + 1e-6f;
  const float hy = sqrtf(rho * e.a / e.det);
  const float lo = fmaxf(ya - e.cy, -hy), hi = fminf(yb - e.cy, hy);
  if (lo > hi) return false;
  const float hx = sqrtf(rho * e.d / e.det);
  const float ydx = -e.b * hx / e.d;  // y offset of the rightmost point
  const float yr = fminf(fmaxf(ydx, lo), hi), yl = fminf(fmaxf(-ydx, lo), hi);
  const float xr = (-e.b * yr + sqrtf(fmaxf(e.a * rho - e.det * yr * yr, 0.f))) / e.a;
  const float xl = (-e.b * yl - sqrtf(fmaxf(e.a * rho - e.det * yl * yl, 0.f))) / e.a;
  xa = e.cx + xl;
  xb = e.cx + xr;
  return true;
}

// Supports that are not a bounded ellipse (the primitive's cone of rays reaches the
// camera plane, or the ellipse is too ill-conditioned in float32) are still convex: the
// image of one nappe of an elliptic cone cut by the plane z = 1.  Within a band of pixel
// rows their pixels therefore occupy one contiguous run of tiles, found by testing tile
// rectangles from both ends of the row.

// Does the segment delta(t) = P + t E, t in [0, 1] (pixel offsets from the projected
// centre) meet the support kp |G delta|^2 <= y2^2, y2 = 1 + h.delta > 0?  Along the
// segment y01 = a + t b and y2 = al + t be, so f = kp |y01|^2 - y2^2 is a quadratic in t;
// its minimum over the part where y2 > 0 is compared with a margin of 1e-4 of the
// magnitude of its terms, far above float32 rounding: the answer errs only towards yes.
__device__ __forceinline__ bool segment_meets_support(const Rec &r, float Px, float Py, float Ex, float Ey) {
  const float kp = r.c.z;
  const float a0 = fmaf(r.b.x, Px, r.b.y * Py), a1 = fmaf(r.b.z, Px, r.b.w * Py);
  const float b0 = fmaf(r.b.x, Ex, r.b.y * Ey), b1 = fmaf(r.b.z, Ex, r.b.w * Ey);
  const float al = fmaf(r.c.x, Px, fmaf(r.c.y, Py, 1.f)), be = fmaf(r.c.x, Ex, r.c.y * Ey);
  const float slack = 1e-5f * (fabsf(al) + fabsf(be)) + 1e-6f;
  float t0 = 0.f, t1 = 1.f;
  if (be > 0.f) t0 = fmaxf(t0, (-slack - al) / be);
  else if (be < 0.f) t1 = fminf(t1, (-slack - al) / be);
  else if (al < -slack) return false;
  if (!(t0 <= t1)) return false;
  const float qa = fmaf(a0, a0, a1 * a1), qb = fmaf(b0, b0, b1 * b1), qab = fmaf(a0, b0, a1 * b1);
  const float A = fmaf(kp, qb, -be * be);
  const float Bh = fmaf(kp, qab, -al * be);
  const float Cc = fmaf(kp, qa, -al * al);
  const float margin = 1e-4f * (2.f * fmaf(kp, qa, al * al) + 2.f * fmaf(kp, qb, be * be)) + 1e-6f;
  float m = fminf(fmaf(fmaf(A, t0, 2.f * Bh), t0, Cc), fmaf(fmaf(A, t1, 2.f * Bh), t1, Cc));
  if (A > 0.f) {
    const float tv = -Bh / A;
    if (tv > t0 && tv < t1) m = fminf(m, fmaf(Bh, tv, Cc));
  }
  return m <= margin;
}

// First (from_left) or last tile column in [tx0, tx1] whose pixel centres in rows
// [ya, yb] can meet the support; -1 if none.
__device__ int support_tile_end(const Rec &r, const DevCam &cam, int tile_w, float ya, float yb, int tx0, int tx1,
                                bool from_left) {
  const float ux = r.a.x, uy = r.a.y, lx = r.a.z, ly = r.a.w;
  const float dya = (ya - uy) - ly, dyb = (yb - uy) - ly;
  const int n = tx1 - tx0 + 1;
  for (int i = 0; i < n; ++i) {
    const int tx = from_left ? tx0 + i : tx1 - i;
    const float xa = float(tx * tile_w) + 0.5f;
    const float xb = float(min((tx + 1) * tile_w, cam.W)) - 0.5f;
    const float dxa = (xa - ux) - lx, dxb = (xb - ux) - lx;
    if ((dxa <= 0.f && dxb >= 0.f && dya <= 0.f && dyb >= 0.f) ||      // the centre itself
        segment_meets_support(r, dxa, dya, 0.f, dyb - dya) ||
        segment_meets_support(r, dxb, dya, 0.f, dyb - dya) ||
        segment_meets_support(r, dxa, dya, dxb - dxa, 0.f) ||
        segment_meets_support(r, dxa, dyb, dxb - dxa, 0.f))
      return tx;
  }
  return -1;
}

__global__ void __launch_bounds__(256) rows_kernel(RowsParams R) {
  __shared__ uint32_t s_off[kEmitTile + 1];
  __shared__ uint32_t s_pair[kEmitTile + 1];
  const uint32_t total = R.counters->n_rows_clamped;
  const unsigned long long total_all = R.counters->n_rows;
  const uint32_t nvis = R.counters->n_visible;
  const uint32_t ntile = (total + kEmitTile - 1) / kEmitTile;
  const unsigned long long ntile_all = (total_all + kEmitTile - 1) / kEmitTile;
  for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const uint32_t e0 = t * kEmitTile, e1 = min(e0 + uint32_t(kEmitTile), total);
    const uint32_t p_lo = R.row_tstart[t];
    const uint32_t p_hi = (uint64_t(t) + 1 < ntile_all) ? R.row_tstart[t + 1] : nvis - 1;
    const int np = int(p_hi - p_lo) + 1;  // <= kEmitTile + 1: every pair has >= 1 row
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
      s_off[j] = R.row_off[p_lo + j];
      s_pair[j] = R.pairs[p_lo + j];
    }
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int a = 0, b = np - 1;
      while (a < b) {
        int m = (a + b + 1) >> 1;
        if (s_off[m] <= e) a = m; else b = m - 1;
      }
      const uint32_t pair = s_pair[a];
      const uint2 r = R.rect[pair];
      const uint32_t tx0 = r.x & 0xFFFF, ty0 = r.x >> 16, tx1 = r.y & 0xFFFF;
      const uint32_t ty = ty0 + (e - s_off[a]);
      uint32_t xa_t = tx0, xb_t = tx1;
      const Ell el = R.ell[pair];
      bool empty = false;
      const DevCam &cam = R.cams[pair / uint32_t(R.n)];
      const float ya = float(ty * R.tile_h) + 0.5f;
      const float yb = float(min((ty + 1) * uint32_t(R.tile_h), uint32_t(cam.H))) - 0.5f;
      if (el.rho < 0.f) {
        const Rec rc = R.rec[pair];
        const int a0 = support_tile_end(rc, cam, R.tile_w, ya, yb, int(tx0), int(tx1), true);
        if (a0 < 0) {
          empty = true;
        } else {
          xa_t = uint32_t(a0);
          xb_t = uint32_t(support_tile_end(rc, cam, R.tile_w, ya, yb, a0, int(tx1), false));
        }
      } else {
        float xa, xb;
        if (!ellipse_band(el, ya - 0.02f, yb + 0.02f, xa, xb)) {
          empty = true;
        } else {
          // pixel centres i + 0.5 in [xa, xb] (with a margin), as tile columns
          const float fa = ceilf(fminf(fmaxf(xa - 0.52f, -1.f), 65536.f * R.tile_w));
          const float fb = floorf(fminf(fmaxf(xb - 0.48f, -1.f), 65536.f * R.tile_w));
          if (fa > fb || fb < 0.f) {
            empty = true;
          } else {
            const uint32_t ia = uint32_t(fmaxf(fa, 0.f)), ib = uint32_t(fb);
            xa_t = max(tx0, ia / uint32_t(R.tile_w));
            xb_t = min(tx1, ib / uint32_t(R.tile_w));
            if (xa_t > xb_t) empty = true;
          }
        }
      }
      R.seg[e] = make_uint2(p_lo + uint32_t(a), ty | (xa_t << 16));
      R.seg_len[e] = empty ? 0u : xb_t - xa_t + 1;
    }
    __syncthreads();
  }
}

cudaError_t launch_rows(const RowsParams &R, int G, cudaStream_t st) {
  rows_kernel<<<G, 256, 0, st>>>(R);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- emission
__global__ void __launch_bounds__(256) emit_kernel(EmitParams E) {
  __shared__ uint32_t s_off[kEmitTile + 1];
  __shared__ uint2 s_seg[kEmitTile + 1];
  const uint32_t total = E.counters->n_inst_clamped;
  const unsigned long long total_all = E.counters->n_instances;
  const uint32_t nrows = E.counters->n_rows_clamped;
  const uint32_t ntile = (total + kEmitTile - 1) / kEmitTile;
  const unsigned long long ntile_all = (total_all + kEmitTile - 1) / kEmitTile;
  for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const uint32_t e0 = t * kEmitTile, e1 = min(e0 + uint32_t(kEmitTile), total);
    const uint32_t r_lo = E.tile_start[t];
    const uint32_t r_hi = (uint64_t(t) + 1 < ntile_all) ? E.tile_start[t + 1] : nrows - 1;
    const int nr = int(r_hi - r_lo) + 1;
    const bool in_smem = nr <= kEmitTile + 1;  // rows of zero length can make it larger
    if (in_smem) {
      for (int j = threadIdx.x; j < nr; j += blockDim.x) {
        s_off[j] = E.seg_off[r_lo + j];
        s_seg[j] = E.seg[r_lo + j];
      }
    }
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int a = 0, b = nr - 1;  // largest row with offset <= e (a row of length 0 never wins)
      while (a < b) {
        int m = (a + b + 1) >> 1;
        uint32_t om = in_smem ? s_off[m] : E.seg_off[r_lo + m];
        if (om <= e) a = m; else b = m - 1;
      }
      const uint2 sg = in_smem ? s_seg[a] : E.seg[r_lo + a];
      const uint32_t off = in_smem ? s_off[a] : E.seg_off[r_lo + a];
      const uint32_t pos = sg.x;
      const uint32_t ty = sg.y & 0xFFFF, tx = (sg.y >> 16) + (e - off);
      const DevCam &cam = E.cams[E.pairs[pos] / uint32_t(E.n)];
      E.keys[e] = uint32_t(cam.tile_base) + ty * uint32_t(cam.tiles_x) + tx;
      E.vals[e] = pos;
    }
    __syncthreads();
  }
}

cudaError_t launch_emit(const EmitParams &E, int G, cudaStream_t st) {
  emit_kernel<<<G, 256, 0, st>>>(E);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- tile ranges
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t *keys, const Counters *c, uint2 *ranges) {
  const uint32_t n = c->n_inst_clamped;
  const uint32_t nq = (n + 3) / 4;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t i0 = 4 * q;
    uint32_t k[4];
    if (i0 + 3 < n) {
      uint4 v = *reinterpret_cast<const uint4 *>(keys + i0);
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : 0xFFFFFFFFu;
    }
    uint32_t prev = i0 == 0 ? 0xFFFFFFFFu : keys[i0 - 1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = i0 + j;
      if (i >= n) break;
      if (i == 0 || prev != k[j]) {
        ranges[k[j]].x = i;
        if (i > 0) ranges[prev].y = i;
      }
      if (i == n - 1) ranges[k[j]].y = n;
      prev = k[j];
    }
  }
}

cudaError_t launch_ranges(const uint32_t *keys, const Counters *c, uint2 *ranges, int G, cudaStream_t st) {
  ranges_kernel<<<G, 256, 0, st>>>(keys, c, ranges);
  return cudaGetLastError();
}

}  // namespace raygs
