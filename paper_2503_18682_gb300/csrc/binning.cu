// Binning for the depth order of Eq. rendering.
//
//   1. Stable LSD radix sort of the visible (primitive, view) pairs by float32 centre
//      depth.  The first pass reads the dense per-(view, primitive) key array, drops
//      culled entries and materialises the pair index as the value, so ties keep the
//      primitive order within a view; the last pass leaves each pair's tile-row count in
//      place of its key.
//   2. Support rows: each pair -> the tile rows of its screen rectangle; each row -> the
//      run of tiles whose pixel centres can meet the pair's support (the band of a bounded
//      ellipse, or an exact conic test tile by tile), with per-tile-row instance totals.
//   3. Stable LSD radix sort of the non-empty rows by global tile row (depth order kept
//      inside a tile row).
//   4. Per tile row, in chunks of rows: the rows expanded into per-tile instance lists in
//      depth order, and the per-tile [start, end) ranges.
//
// The radix sort is reduce-then-scan (upsweep histogram, one-CTA scan, downsweep
// scatter) with persistent CTAs that own contiguous tile ranges: no CTA ever waits on
// another.  The upsweep counts runs of equal digits per thread; ranking inside a tile is
// stable (warp multi-split by digit-bit ballots + per-warp counters) and the scatter goes
// through shared memory so that global writes are coalesced runs.
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

// Values are 4-byte item ids, or (WIDE) the 8-byte payload of a support row.
template <bool WIDE>
struct SortVal {
  using T = uint32_t;
  // the first pass materialises the item id, with the pair's tile-row count packed above it
  static __device__ __forceinline__ T load(const SortPass &p, uint32_t idx) {
    if (!p.filter) return p.vals_in[idx];
    if (!p.row_cnt8 || p.id_bits >= 32) return idx;
    const uint32_t field = 0xFFFFFFFFu >> p.id_bits;
    const uint32_t c = p.row_cnt8[idx];
    return idx | ((c < 255u && c < field ? c : field) << p.id_bits);
  }
  static __device__ __forceinline__ void store(const SortPass &p, uint32_t dst, T v) { p.vals_out[dst] = v; }
};
template <>
struct SortVal<true> {
  using T = uint2;
  static __device__ __forceinline__ T load(const SortPass &p, uint32_t idx) { return p.wvals_in[idx]; }
  static __device__ __forceinline__ void store(const SortPass &p, uint32_t dst, T v) { p.wvals_out[dst] = v; }
};

template <int BITS, bool WIDE>
__global__ void __launch_bounds__(kSortThreads, 4) sort_downsweep(SortPass p) {
  constexpr int R = 1 << BITS;
  using VT = typename SortVal<WIDE>::T;
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ VT s_vals[kSortTile];
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

  // The keys of the next tile are loaded while the current one is ranked, and so are its
  // 4-byte values; 8-byte values would not leave registers for that, so they are loaded
  // at the start of their own tile (they are first needed after the ranking).
  uint32_t nkey[kSortIPT];
  VT nval[kSortIPT];
  auto load_keys = [&](uint32_t base) {
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      nkey[r] = idx < hi ? p.keys_in[idx] : 0u;
    }
  };
  auto load_vals = [&](uint32_t base, VT *dst) {
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      dst[r] = idx < hi ? SortVal<WIDE>::load(p, idx) : VT{};
    }
  };
  if (lo < hi) {
    load_keys(lo);
    if (!WIDE) load_vals(lo, nval);
  }
  for (uint32_t base = lo; base < hi; base += kSortTile) {
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    uint32_t key[kSortIPT], off[kSortIPT];
    VT val[kSortIPT];
    if (WIDE) load_vals(base, val);
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      key[r] = nkey[r];
      if (!WIDE) val[r] = nval[r];
    }
    if (base + kSortTile < hi) {
      load_keys(base + kSortTile);
      if (!WIDE) load_vals(base + kSortTile, nval);
    }
    __syncthreads();
    uint32_t vmask = 0;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      const bool ok = idx < hi;
      const uint32_t k = key[r];
      const bool valid = ok && !(p.filter && k == kCulled);
      uint32_t d = (k >> p.shift) & (R - 1);
      // lanes holding the same digit: one ballot per digit bit (warp-level multi-split)
      uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int bit = 0; bit < BITS; ++bit) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
        peers &= ((d >> bit) & 1u) ? bal : ~bal;
      }
      if (!valid) peers = 1u << lane;
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
      uint32_t kout = k;
      VT vout = s_vals[j];
      if constexpr (!WIDE) {
        if (p.row_rect) {  // the last depth pass: the tile-row count as key, the bare id
          const bool packed = p.id_bits < 32;
          const uint32_t field = packed ? 0xFFFFFFFFu >> p.id_bits : 0u;
          const uint32_t f = packed ? vout >> p.id_bits : 0u;
          const uint32_t id = packed ? vout & ((1u << p.id_bits) - 1u) : vout;
          if (f < field) {
            kout = f;
          } else {
            const uint2 r = p.row_rect[id];
            kout = (r.y >> 16) - (r.x >> 16) + 1;
          }
          vout = id;
        }
      }
      if (p.keys_out) p.keys_out[dst] = kout;
      SortVal<WIDE>::store(p, dst, vout);
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

// One LSD pass: 8-bit digits over item ids (the depth sort), 4 to 8 bits over support
// rows (the tile-row sort).
template <int BITS, bool WIDE>
static void sort_pass(const SortPass &p, cudaStream_t st) {
  const int n = (1 << BITS) * p.G;
  const int nb = (n + kHistBlock - 1) / kHistBlock;
  uint32_t *bsum = p.hist + n;  // scratch after the histogram (the layout reserves 512*G + G)
  sort_upsweep<BITS><<<p.G, kSortThreads, 0, st>>>(p);
  hist_reduce_kernel<<<nb, 256, 0, st>>>(p.hist, n, bsum);
  hist_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nb, p.d_total);
  hist_offsets_kernel<<<nb, 256, 0, st>>>(p.hist, n, bsum);
  sort_downsweep<BITS, WIDE><<<p.G, kSortThreads, 0, st>>>(p);
}

cudaError_t launch_sort_pass(const SortPass &p, cudaStream_t st) {
  if (!p.wide) {
    if (p.bits != 8) return cudaErrorInvalidValue;
    sort_pass<8, false>(p, st);
  } else {
    switch (p.bits) {
      case 4: sort_pass<4, true>(p, st); break;
      case 5: sort_pass<5, true>(p, st); break;
      case 6: sort_pass<6, true>(p, st); break;
      case 7: sort_pass<7, true>(p, st); break;
      case 8: sort_pass<8, true>(p, st); break;
      default: return cudaErrorInvalidValue;
    }
  }
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
  cta_range_units(J.d_n ? *J.d_n : J.n_static, lo, hi);
  uint32_t s = 0;
  for (uint32_t p = lo + threadIdx.x; p < hi; p += blockDim.x) s += J.cnt[p];
  uint32_t tot;
  block_excl_scan(s, ws, &tot);
  if (threadIdx.x == 0) J.partial[blockIdx.x] = tot;
}

// Exclusive scan of the G <= 1024 per-CTA partial sums (one thread each, 64-bit running
// sums); writes the total, the capacity-clamped total and the overflow flag.
__global__ void __launch_bounds__(1024) scan_partials_kernel(ScanJob J, int G) {
  __shared__ unsigned long long ws[32];
  const int t = int(threadIdx.x), lane = t & 31, warp = t >> 5;
  const unsigned long long v = t < G ? J.partial[t] : 0ull;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = ws[lane];
    unsigned long long z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    ws[lane] = z - w;  // warps before this one
  }
  __syncthreads();
  const unsigned long long excl = ws[warp] + x - v;
  if (t < G) J.partial[t] = uint32_t(min(excl, 0xFFFFFFFFull));
  if (t == 1023) {
    const unsigned long long run = excl + v;  // every partial (threads >= G add 0)
    *J.d_total = run;
    *J.d_total_clamped = run > J.cap ? J.cap : uint32_t(run);
    if (run > J.cap) *J.d_overflow = 1u;
  }
}

__global__ void __launch_bounds__(256) scan_offsets_kernel(ScanJob J) {
  __shared__ uint32_t ws[33];
  uint32_t lo, hi;
  cta_range_units(J.d_n ? *J.d_n : J.n_static, lo, hi);
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
  scan_partials_kernel<<<1, 1024, 0, st>>>(J, G);
  scan_offsets_kernel<<<G, 256, 0, st>>>(J);
  return cudaGetLastError();
}

// ------------------------------------------------------------ pair -> tile rows

// Pixel-centre columns of the band ya <= y <= yb (pixel-centre rows) inside the ellipse.
// The right boundary x_r(y) is concave with its maximum at the rightmost point of the
// ellipse, the left one convex: clamping that point's y into the band gives the extremes.
__device__ __forceinline__ bool ellipse_band(const Ell &e, float ya, float yb, float &xa, float &xb) {
  const float rho = 1.001f;
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
// rows their pixels therefore occupy one contiguous run of tiles, whose ends are found by
// bisection with a vertical-line test.

// Does the segment delta(t) = P + t E, t in [0, 1] (pixel offsets from the projected
// centre) meet the support |G delta|^2 <= y2^2, y2 = 1 + h.delta > 0 (the record's G carries
// sqrt(kp))?  Along the segment y01' = a + t b and y2 = al + t be, so f = |y01'|^2 - y2^2 is a
// quadratic in t;
// its minimum over the part where y2 > 0 is compared with a margin of 1e-4 of the
// magnitude of its terms, far above float32 rounding: the answer errs only towards yes.
// t_at receives the parameter of that minimum.
__device__ __forceinline__ bool segment_meets_support(const Rec &r, float Px, float Py, float Ex, float Ey,
                                                      float *t_at = nullptr) {
  const float kp = 1.f;
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
  const float f0 = fmaf(fmaf(A, t0, 2.f * Bh), t0, Cc), f1 = fmaf(fmaf(A, t1, 2.f * Bh), t1, Cc);
  float m = f0, tm = t0;
  if (f1 < m) { m = f1; tm = t1; }
  if (A > 0.f) {
    const float tv = -Bh / A;
    if (tv > t0 && tv < t1) {
      const float fv = fmaf(Bh, tv, Cc);
      if (fv < m) { m = fv; tm = tv; }
    }
  }
  if (t_at) *t_at = tm;
  return m <= margin;
}

// Can the pixel centres of the rectangle [dxa, dxb] x [dya, dyb] (offsets from the projected
// centre) meet the support?  For a convex support: the rectangle holds the projected centre,
// or one of its edges meets the support.
__device__ __forceinline__ bool tile_meets_support(const Rec &r, float dxa, float dxb, float dya, float dyb) {
  return (dxa <= 0.f && dxb >= 0.f && dya <= 0.f && dyb >= 0.f) ||
         segment_meets_support(r, dxa, dya, 0.f, dyb - dya) || segment_meets_support(r, dxb, dya, 0.f, dyb - dya) ||
         segment_meets_support(r, dxa, dya, dxb - dxa, 0.f) || segment_meets_support(r, dxa, dyb, dxb - dxa, 0.f);
}

// First and last tile column in [tx0, tx1] whose pixel centres in rows [ya, yb] can meet
// the support; false if none.  A point of the support inside the band is found on the
// band's boundary or is the projected centre itself (a convex set that meets a rectangle
// but not its boundary lies inside it).  Left of that point, tile t meets the support
// exactly when the vertical line through its last pixel-centre column does (the support's
// columns within the band form an interval), and symmetrically on the right.
__device__ bool support_tile_span(const Rec &r, const DevCam &cam, int tile_w, float ya, float yb, int tx0, int tx1,
                                  int &first, int &last) {
  const float ux = r.a.x, uy = r.a.y, lx = r.a.z, ly = r.a.w;
  const float dya = (ya - uy) - ly, dyb = (yb - uy) - ly;
  auto col_dx = [&](int px_centre_times2) {  // pixel-centre column (2x, exact) as an offset
    return (0.5f * float(px_centre_times2) - ux) - lx;
  };
  auto left_col = [&](int tx) { return col_dx(2 * tx * tile_w + 1); };
  auto right_col = [&](int tx) { return col_dx(2 * min((tx + 1) * tile_w, cam.W) - 1); };
  auto vert = [&](float dx) { return segment_meets_support(r, dx, dya, 0.f, dyb - dya); };
  const float dxL = left_col(tx0), dxR = right_col(tx1);
  // a tile that holds a point of the support (any tile at least as wide as that point's
  // pixel column is a conservative choice)
  int tstar = -1;
  float t;
  if (vert(dxL)) {
    tstar = tx0;
  } else if (vert(dxR)) {
    tstar = tx1;
  } else {
    float cx = 0.f;
    bool inside = dya <= 0.f && dyb >= 0.f && dxL <= 0.f && dxR >= 0.f;
    if (!inside && segment_meets_support(r, dxL, dya, dxR - dxL, 0.f, &t)) { inside = true; cx = fmaf(t, dxR - dxL, dxL); }
    if (!inside && segment_meets_support(r, dxL, dyb, dxR - dxL, 0.f, &t)) { inside = true; cx = fmaf(t, dxR - dxL, dxL); }
    if (!inside) return false;
    // the minimum along a long horizontal segment carries a wide margin: confirm the point
    // with the (short) vertical test, else scan the row tile by tile
    if (!vert(cx)) {
      for (first = tx0; first <= tx1; ++first)
        if (tile_meets_support(r, left_col(first), right_col(first), dya, dyb)) break;
      if (first > tx1) return false;
      for (last = tx1; last > first; --last)
        if (tile_meets_support(r, left_col(last), right_col(last), dya, dyb)) break;
      return true;
    }
    const float px = (cx + lx) + ux;  // pixel x of the point
    tstar = min(max(int(floorf(px / float(tile_w))), tx0), tx1);
  }
  int lo = tx0, hi = tstar;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (vert(right_col(mid))) hi = mid; else lo = mid + 1;
  }
  first = lo;
  lo = tstar; hi = tx1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (vert(left_col(mid))) lo = mid; else hi = mid - 1;
  }
  last = lo;
  return true;
}

__global__ void __launch_bounds__(256) rows_kernel(RowsParams R) {
  __shared__ uint32_t s_off[kEmitTile + 1];
  __shared__ uint32_t s_pair[kEmitTile + 1];
  __shared__ uint16_t s_owner[kEmitTile];     // the tile's pair (local index) of each row
  // this CTA's instances (low 40 bits) and non-empty rows (high 24 bits) per tile row
  __shared__ unsigned long long s_trow[kTrowsShared];
  const uint32_t total = R.counters->n_rows_clamped;
  const unsigned long long total_all = R.counters->n_rows;
  const uint32_t nvis = R.counters->n_visible;
  const uint32_t ntile = (total + kEmitTile - 1) / kEmitTile;
  // shared totals while this CTA's rows fit the 24-bit row field (then a tile row's
  // instances, at most 65,535 per row, fit the 40-bit field)
  const bool shared_trows = R.trows <= kTrowsShared &&
                            uint64_t((ntile + gridDim.x - 1) / gridDim.x) * kEmitTile < (1ull << 24);
  if (shared_trows)
    for (int i = threadIdx.x; i < R.trows; i += blockDim.x) s_trow[i] = 0ull;
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
    // each pair marks its rows in this tile with its local index
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
      const uint32_t first = max(s_off[j], e0), next = j + 1 < np ? min(s_off[j + 1], e1) : e1;
      for (uint32_t e = first; e < next; ++e) s_owner[e - e0] = uint16_t(j);
    }
    __syncthreads();
    // two rows per thread at a time: both loads are issued before either row's arithmetic
    for (uint32_t e_base = e0; e_base < e1; e_base += 2 * blockDim.x) {
      uint32_t ee[2];
      int aa[2];
      Ell el2[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        ee[u] = e_base + u * blockDim.x + threadIdx.x;
        const int a = s_owner[min(ee[u], e1 - 1) - e0];
        aa[u] = a;
        const uint32_t pair = s_pair[a];
        el2[u] = R.ell[pair];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t e = ee[u];
        if (e >= e1) break;
        const int a = aa[u];
        const uint32_t pair = s_pair[a];
        const Ell &el = el2[u];
        const uint32_t tx0 = el.r0 & 0xFFFF, ty0 = el.r0 >> 16, tx1 = el.r1 & 0xFFFF;
        const uint32_t ty = ty0 + (e - s_off[a]);
        uint32_t xa_t = tx0, xb_t = tx1;
        bool empty = false;
        const DevCam &cam = R.cams[pair / uint32_t(R.n)];
        const float ya = float(ty * R.tile_h) + 0.5f;
        const float yb = float(min((ty + 1) * uint32_t(R.tile_h), uint32_t(cam.H))) - 0.5f;
        if (el.a == -2.f) {
          // the whole rectangle row (a bound without a conic of its own)
        } else if (!(el.a > 0.f)) {
          const Rec rc = R.rec[pair];
          int a0, b0;
          if (!support_tile_span(rc, cam, R.tile_w, ya, yb, int(tx0), int(tx1), a0, b0)) {
            empty = true;
          } else {
            xa_t = uint32_t(a0);
            xb_t = uint32_t(b0);
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
        const uint32_t len = empty ? 0u : xb_t - xa_t + 1;
        R.seg[e] = make_uint2(p_lo + uint32_t(a), xa_t | (len << 16));  // the sort's payload as is
        if (R.seg_len) R.seg_len[e] = len;
        R.row_key[e] = empty ? kCulled : uint32_t(cam.trow_base) + ty;
        if (!empty) {
          const uint32_t grow = uint32_t(cam.trow_base) + ty, len = xb_t - xa_t + 1;
          if (shared_trows) {
            atomicAdd(&s_trow[grow], (unsigned long long)len + (1ull << 40));
          } else {
            atomicAdd(&R.trow_inst[grow], (unsigned long long)len);
            atomicAdd(&R.trow_ranges[grow].y, 1u);
          }
        }
      }
    }
    __syncthreads();
  }
  if (shared_trows)
    for (int i = threadIdx.x; i < R.trows; i += blockDim.x)
      if (s_trow[i]) {
        atomicAdd(&R.trow_inst[i], s_trow[i] & ((1ull << 40) - 1ull));
        atomicAdd(&R.trow_ranges[i].y, uint32_t(s_trow[i] >> 40));
      }
}

cudaError_t launch_rows(const RowsParams &R, int G, cudaStream_t st) {
  rows_kernel<<<G, 256, 0, st>>>(R);
  return cudaGetLastError();
}

// ------------------------------------------------- tile rows -> per-tile instance lists
__device__ __forceinline__ const DevCam &view_of_trow(const ExpandParams &E, int grow, int &v_out) {
  int v = 0;
  while (v + 1 < E.n_views && E.cams[v + 1].trow_base <= grow) ++v;
  v_out = v;
  return E.cams[v];
}

// Exclusive scans of the per-tile-row totals (one block): the instance totals in place
// (64-bit running sums: each tile row's first instance, the instance total, its capacity
// clamp and the overflow flag), and the non-empty row counts into each tile row's range of
// rows in the tile-row sort's output (rows of a tile row are contiguous there, the sort
// being stable by tile row).
__global__ void __launch_bounds__(1024) trow_scan_kernel(unsigned long long *v, uint2 *ranges, int n, Counters *c,
                                                         uint32_t cap) {
  __shared__ unsigned long long ws[32];
  __shared__ uint32_t rws[33];
  const int per = (n + 1023) / 1024;
  const int b = min(n, int(threadIdx.x) * per), e = min(n, b + per);
  {
    uint32_t rs = 0;
    for (int i = b; i < e; ++i) rs += ranges[i].y;
    uint32_t rtot;
    uint32_t rrun = block_excl_scan(rs, rws, &rtot);
    for (int i = b; i < e; ++i) {
      const uint32_t k = ranges[i].y;
      ranges[i] = make_uint2(rrun, rrun + k);
      rrun += k;
    }
  }
  unsigned long long s = 0;
  for (int i = b; i < e; ++i) s += v[i];
  // block exclusive scan of s (warp scans of 64-bit values, then of the warp totals)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long t = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  unsigned long long run = (warp ? ws[warp - 1] : 0ull) + x - s;
  for (int i = b; i < e; ++i) {
    const unsigned long long t = v[i];
    v[i] = run;
    run += t;
  }
  if (threadIdx.x == 1023) {
    const unsigned long long total = ws[31];
    c->n_instances = total;
    c->n_inst_clamped = total > cap ? cap : uint32_t(total);
    if (total > cap) c->overflow = 1u;
  }
}

cudaError_t launch_trow_scan(unsigned long long *trow_inst, uint2 *trow_ranges, int trows, Counters *c, uint32_t cap,
                             cudaStream_t st) {
  trow_scan_kernel<<<1, 1024, 0, st>>>(trow_inst, trow_ranges, trows, c, cap);
  return cudaGetLastError();
}

// Instance lists of one tile row.  Rows are taken in sorted (depth) order, NT * KR at a
// time, in 32-row groups (KR * NT / 32 groups: row q of the step is lane q % 32 of group
// q / 32); every lane marks the tiles of its row in its group's bit mask per tile, and the
// rank of (row, tile) is the tile's running cursor plus the rows of lower groups and lower
// lanes that cover the same tile.  Each tile's list keeps depth order.  The masks are
// double-buffered (the buffer of the next step is cleared while this one is read) and the
// rows of the next step are loaded during this one.
// The chunk of rows a CTA owns: tile row t (largest t with chunk_base[t] <= chunk) and its
// rows [first, last).
__device__ __forceinline__ bool chunk_of(const ExpandParams &E, uint32_t chunk, int &t, int &c, uint2 &rows) {
  if (chunk >= E.chunk_base[E.trows]) return false;
  int lo = 0, hi = E.trows - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (E.chunk_base[m] <= chunk) lo = m; else hi = m - 1;
  }
  t = lo;
  c = int(chunk - E.chunk_base[t]);
  const uint2 rr = E.trow_ranges[t];
  const uint32_t first = rr.x + uint32_t(c) * uint32_t(E.chunk_rows);
  rows = make_uint2(min(first, rr.y), min(first + uint32_t(E.chunk_rows), rr.y));
  return true;
}

// Chunks per tile row (at least one) and their exclusive scan (one block).
__global__ void __launch_bounds__(1024) chunk_scan_kernel(ExpandParams E) {
  __shared__ uint32_t ws[33];
  const int per = (E.trows + 1023) / 1024;
  const int b = min(E.trows, int(threadIdx.x) * per), e = min(E.trows, b + per);
  auto nchunks = [&](int t) {
    const uint2 rr = E.trow_ranges[t];
    const uint32_t n = rr.y - rr.x;
    return n == 0 ? 1u : (n + uint32_t(E.chunk_rows) - 1) / uint32_t(E.chunk_rows);
  };
  uint32_t s = 0;
  for (int t = b; t < e; ++t) s += nchunks(t);
  uint32_t tot;
  uint32_t run = block_excl_scan(s, ws, &tot);
  for (int t = b; t < e; ++t) {
    E.chunk_base[t] = run;
    run += nchunks(t);
  }
  if (threadIdx.x == 0) E.chunk_base[E.trows] = min(tot, uint32_t(E.max_chunks));
}

// Instances per tile column of one chunk: each row covers the tile columns
// [txa, txa + len); a difference array over the columns and its prefix sum count them.
__global__ void __launch_bounds__(256) chunk_count_kernel(ExpandParams E) {
  extern __shared__ uint32_t s_diff[];  // [max_tiles_x + 1]
  __shared__ uint32_t s_ws[33];
  int t, c;
  uint2 rows;
  if (!chunk_of(E, blockIdx.x, t, c, rows)) return;
  int v;
  const DevCam &cam = view_of_trow(E, t, v);
  const int TX = cam.tiles_x;
  for (int x = threadIdx.x; x <= TX; x += blockDim.x) s_diff[x] = 0u;
  __syncthreads();
  // four rows per thread at a time, their loads issued before any of their atomics
  for (uint32_t i0 = rows.x + threadIdx.x; i0 < rows.y; i0 += 4 * blockDim.x) {
    uint32_t pk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t i = i0 + k * blockDim.x;
      pk[k] = i < rows.y ? E.rows[i].y : 0u;  // 0: no tiles
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (pk[k] >> 16) {
        atomicAdd(&s_diff[pk[k] & 0xFFFFu], 1u);
        atomicSub(&s_diff[(pk[k] & 0xFFFFu) + (pk[k] >> 16)], 1u);
      }
    }
  }
  __syncthreads();
  const int per = (TX + int(blockDim.x) - 1) / int(blockDim.x);
  const int x0 = min(TX, int(threadIdx.x) * per), x1 = min(TX, x0 + per);
  uint32_t dsum = 0;
  for (int x = x0; x < x1; ++x) dsum += s_diff[x];
  uint32_t dtot;
  uint32_t run = block_excl_scan(dsum, s_ws, &dtot);
  uint32_t *out = E.chunk_cnt + size_t(blockIdx.x) * size_t(E.max_tiles_x);
  for (int x = x0; x < x1; ++x) {
    run += s_diff[x];
    out[x] = run;
  }
}

// Instance lists of one chunk of a tile row.  Its cursor in tile column x starts after the
// tile row's earlier tiles (all chunks) and after the earlier chunks' instances in x; chunk 0
// also writes the tile row's ranges.  Rows are then taken in sorted (depth) order, NT * KR
// at a time, in 32-row groups (KR * NT / 32 groups: row q of the step is lane q % 32 of group
// q / 32); every lane marks the tiles of its row in its group's bit mask per tile, and the
// rank of (row, tile) is the tile's running cursor plus the rows of lower groups and lower
// lanes that cover the same tile.  Each tile's list keeps depth order.  The masks are
// double-buffered (the buffer of the next step is cleared while this one is read) and the
// rows of the next step are loaded during this one.
template <int NT, int KR>
__global__ void __launch_bounds__(NT) expand_kernel(ExpandParams E) {
  constexpr int VW = NT / 32 * KR;  // row groups per step
  extern __shared__ uint32_t s_mem[];
  int grow, chunk_c;
  uint2 rr;
  if (!chunk_of(E, blockIdx.x, grow, chunk_c, rr)) return;
  int v;
  const DevCam &cam = view_of_trow(E, grow, v);
  const int TX = cam.tiles_x;
  const int TP = TX | 1;                     // odd row stride: no bank conflicts down a column
  uint32_t *s_cur = s_mem;                   // [TX] next free slot of each tile
  uint32_t *s_pre = s_cur + TX;              // [VW][TP] first slot of each group
  uint32_t *s_mask = s_pre + VW * TP;        // [2][VW][TP]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t tile0 = uint32_t(cam.tile_base) + uint32_t(grow - cam.trow_base) * uint32_t(TX);
  {
    // per tile column: instances of the whole tile row and of the earlier chunks
    const uint32_t cb = E.chunk_base[grow], nch = E.chunk_base[grow + 1] - cb;
    uint32_t *s_tot = s_pre, *s_bef = s_pre + TX;  // 2 TX words of the group-prefix buffer
    for (int x = threadIdx.x; x < TX; x += NT) {
      uint32_t tot = 0, bef = 0;
      for (uint32_t k = 0; k < nch; ++k) {
        const uint32_t n = E.chunk_cnt[size_t(cb + k) * size_t(E.max_tiles_x) + x];
        tot += n;
        bef += k < uint32_t(chunk_c) ? n : 0u;
      }
      s_tot[x] = tot;
      s_bef[x] = bef;
    }
    __syncthreads();
    __shared__ uint32_t s_ws[33];
    const int per = (TX + NT - 1) / NT;
    const int x0 = min(TX, int(threadIdx.x) * per), x1 = min(TX, x0 + per);
    uint32_t csum = 0;
    for (int x = x0; x < x1; ++x) csum += s_tot[x];
    uint32_t ctot;
    const uint32_t cpre = block_excl_scan(csum, s_ws, &ctot);  // instances before the column chunk
    const unsigned long long base = E.trow_base[grow];
    uint32_t o = uint32_t(min(base, (unsigned long long)E.cap)) + cpre;
    for (int x = x0; x < x1; ++x) {
      const uint32_t n = s_tot[x];
      s_cur[x] = o + s_bef[x];
      if (chunk_c == 0) E.ranges[tile0 + x] = make_uint2(min(o, E.cap), min(o + n, E.cap));
      o += n;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * VW * TP; j += NT) s_mask[j] = 0u;
  constexpr uint32_t STEP = uint32_t(NT) * KR;
  uint2 nxt[KR];
  auto load_rows = [&](uint32_t base) {
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const uint32_t i = base + uint32_t(k * NT) + threadIdx.x;
      nxt[k] = i < rr.y ? E.rows[i] : make_uint2(0u, 0u);
    }
  };
  if (rr.x < rr.y) load_rows(rr.x);
  int buf = 0;
  for (uint32_t base = rr.x; base < rr.y; base += STEP) {
    uint2 cur[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) cur[k] = nxt[k];
    if (base + STEP < rr.y) load_rows(base + STEP);
    uint32_t *mask = s_mask + buf * VW * TP;
    __syncthreads();  // masks of this buffer cleared; the previous step's reads are done
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int g = k * (NT / 32) + warp;
      const uint32_t xa = cur[k].y & 0xFFFFu, len = cur[k].y >> 16;
      for (uint32_t t = 0; t < len; ++t) atomicOr(&mask[g * TP + int(xa + t)], 1u << lane);
    }
    __syncthreads();
    // per tile (one thread each), the group counts in group order
    uint32_t *other = s_mask + (1 - buf) * VW * TP;
    for (int x = threadIdx.x; x < TX; x += NT) {
      uint32_t run = s_cur[x];
#pragma unroll 8
      for (int g = 0; g < VW; ++g) {
        s_pre[g * TP + x] = run;
        run += __popc(mask[g * TP + x]);
        other[g * TP + x] = 0u;
      }
      s_cur[x] = run;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int g = k * (NT / 32) + warp;
      const uint32_t xa = cur[k].y & 0xFFFFu, len = cur[k].y >> 16;
      for (uint32_t t = 0; t < len; ++t) {
        const int x = int(xa + t);
        const uint32_t dst = s_pre[g * TP + x] + __popc(mask[g * TP + x] & lt);
        if (dst < E.cap) E.inst[dst] = cur[k].x;
      }
    }
    buf = 1 - buf;
  }
}

template <int NT, int KR>
size_t expand_smem(int max_tiles_x) {
  return sizeof(uint32_t) * size_t(max_tiles_x + 1) * size_t(1 + 3 * (NT / 32) * KR);
}


int expand_chunk_rows(int64_t cap, int max_tiles_x) {
  // 8192 rows per chunk, more when the per-chunk column counts would pass 32 M entries
  int64_t ch = 8192;
  const int64_t need = (cap * int64_t(max_tiles_x > 0 ? max_tiles_x : 1)) / (int64_t(32) << 20) + 1;
  if (need > ch) ch = need;
  return int(ch > (int64_t(1) << 30) ? (int64_t(1) << 30) : ch);
}

int64_t expand_max_chunks(int64_t trows, int64_t cap, int chunk_rows) {
  return trows + cap / chunk_rows + 1;
}

cudaError_t launch_expand(const ExpandParams &E, cudaStream_t st) {
  if (E.trows == 0) return cudaSuccess;
  chunk_scan_kernel<<<1, 1024, 0, st>>>(E);
  chunk_count_kernel<<<E.max_chunks, 256, sizeof(uint32_t) * size_t(E.max_tiles_x + 1), st>>>(E);
  constexpr size_t kBudget = 200 * 1024;
  auto run = [&](auto kernel, int nt, size_t smem) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    kernel<<<E.max_chunks, nt, smem, st>>>(E);
    return cudaGetLastError();
  };
  const int mtx = E.max_tiles_x;
  if (expand_smem<256, 4>(mtx) <= kBudget) return run(expand_kernel<256, 4>, 256, expand_smem<256, 4>(mtx));
  if (expand_smem<256, 1>(mtx) <= kBudget) return run(expand_kernel<256, 1>, 256, expand_smem<256, 1>(mtx));
  return run(expand_kernel<128, 1>, 128, expand_smem<128, 1>(mtx));
}

}  // namespace raygs
