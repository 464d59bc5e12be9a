// Binning for the depth order of Eq. rendering.
//
//   1. Stable LSD radix sort of the visible (primitive, view) pairs by float32 centre
//      depth.  The first pass reads the dense per-(view, primitive) key array, drops
//      culled entries and materialises the pair index as the value, so ties keep the
//      primitive order within a view.
//   2. Per sorted pair: number of covered tiles, exclusive scan -> instance offsets.
//   3. Load-balanced emission: one thread per instance writes (global tile id, sorted
//      position); instances come out in depth order.
//   4. Stable LSD radix sort of the instances by tile id -> per tile, depth order.
//   5. Per-tile [start, end) ranges.
//
// The radix sort is reduce-then-scan (upsweep histogram, one-CTA scan, downsweep
// scatter) with persistent CTAs that own contiguous tile ranges: no CTA ever waits on
// another.  Ranking inside a tile is stable (warp match + per-warp counters) and the
// scatter goes through shared memory so that global writes are coalesced runs.
#include "raygs_internal.cuh"

namespace raygs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortIPT = 16;
constexpr int kSortTile = kSortThreads * kSortIPT;  // 4096 items


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

template <int BITS>
__global__ void __launch_bounds__(kSortThreads) sort_upsweep(SortPass p) {
  constexpr int R = 1 << BITS;
  __shared__ uint32_t h[kSortWarps][R];
  for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  uint32_t lo, hi;
  cta_tiles(pass_count(p), lo, hi);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t base = lo; base < hi; base += kSortThreads * 4) {
    uint32_t i = base + threadIdx.x * 4;
    uint32_t k[4];
    bool ok[4];
    if (i + 3 < hi) {
      uint4 v = *reinterpret_cast<const uint4 *>(p.keys_in + i);
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
      ok[0] = ok[1] = ok[2] = ok[3] = true;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ok[j] = i + j < hi;
        k[j] = ok[j] ? p.keys_in[i + j] : 0u;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      bool valid = ok[j] && !(p.filter && k[j] == kCulled);
      uint32_t d = (k[j] >> p.shift) & (R - 1);
      uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : uint32_t(R + lane));
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[warp][d], uint32_t(__popc(peers)));
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < R; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
    p.hist[size_t(d) * p.G + blockIdx.x] = s;
  }
}

// Exclusive scan of `n` entries in place with one CTA of 1024 threads; the total is
// written to *d_total when non-null.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan (blockDim.x multiple of 32, <= 1024). Returns the exclusive
// prefix; *total receives the block total.  Uses `ws` (>= 32 words of shared memory).
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
__global__ void __launch_bounds__(kSortThreads) sort_downsweep(SortPass p) {
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

  for (uint32_t base = lo; base < hi; base += kSortTile) {
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t key[kSortIPT], val[kSortIPT], off[kSortIPT];
    uint32_t vmask = 0;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      uint32_t idx = base + warp * (32 * kSortIPT) + r * 32 + lane;
      bool ok = idx < hi;
      uint32_t k = ok ? p.keys_in[idx] : 0u;
      uint32_t v = ok ? (p.filter ? idx : p.vals_in[idx]) : 0u;
      bool valid = ok && !(p.filter && k == kCulled);
      uint32_t d = (k >> p.shift) & (R - 1);
      uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : uint32_t(R + lane));
      uint32_t c = valid ? s_cnt[warp][d] : 0u;
      __syncwarp();
      if (valid && lane == 31 - __clz(peers)) s_cnt[warp][d] = c + __popc(peers);
      __syncwarp();
      off[r] = c + __popc(peers & lt);
      key[r] = k;
      val[r] = v;
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
    // exclusive scan of the tile's digit counts
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

cudaError_t launch_sort_pass(const SortPass &p, cudaStream_t st) {
  sort_upsweep<8><<<p.G, kSortThreads, 0, st>>>(p);
  scan_single_cta<<<1, 1024, 0, st>>>(p.hist, 256 * p.G, p.d_total);
  sort_downsweep<8><<<p.G, kSortThreads, 0, st>>>(p);
  return cudaGetLastError();
}

// ------------------------------------------------------------- tile counts and scan

__device__ __forceinline__ void cta_range_items(uint32_t count, uint32_t &lo, uint32_t &hi) {
  constexpr uint32_t U = 1024;
  uint32_t nu = (count + U - 1) / U;
  uint32_t t0 = uint32_t((uint64_t(nu) * blockIdx.x) / gridDim.x);
  uint32_t t1 = uint32_t((uint64_t(nu) * (blockIdx.x + 1)) / gridDim.x);
  lo = min(t0 * U, count);
  hi = min(t1 * U, count);
}

__global__ void __launch_bounds__(256) count_tiles_kernel(ScanParams S) {
  __shared__ uint32_t ws[33];
  uint32_t lo, hi;
  cta_range_items(S.counters->n_visible, lo, hi);
  uint32_t s = 0;
  for (uint32_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    uint32_t c = rect_count(S.rect[S.pairs[p]]);
    S.cnt[p] = c;
    s += c;
  }
  uint32_t tot;
  block_excl_scan(s, ws, &tot);
  if (threadIdx.x == 0) S.partial[blockIdx.x] = tot;
}

// Exclusive scan of the G <= 1024 per-CTA partial sums (64-bit running total), and the
// instance totals: n_instances, the capacity-clamped count and the overflow flag.
__global__ void __launch_bounds__(32) scan_partials_kernel(ScanParams S, int G) {
  if (threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int i = 0; i < G; ++i) {
    uint32_t v = S.partial[i];
    S.partial[i] = uint32_t(min(run, 0xFFFFFFFFull));
    run += v;
  }
  S.counters->n_instances = run;
  S.counters->n_inst_clamped = run > S.capacity ? S.capacity : uint32_t(run);
  S.counters->overflow = run > S.capacity ? 1u : 0u;
}

__global__ void __launch_bounds__(256) offsets_kernel(ScanParams S) {
  __shared__ uint32_t ws[33];
  uint32_t lo, hi;
  cta_range_items(S.counters->n_visible, lo, hi);
  uint32_t carry = S.partial[blockIdx.x];
  for (uint32_t base = lo; base < hi; base += 256 * 4) {
    uint32_t c[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t p = base + threadIdx.x * 4 + j;
      c[j] = p < hi ? S.cnt[p] : 0u;
      s += c[j];
    }
    uint32_t tot;
    uint32_t run = carry + block_excl_scan(s, ws, &tot);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t p = base + threadIdx.x * 4 + j;
      if (p < hi) {
        S.off[p] = run;
        // every emit tile whose first instance falls in [run, run + c) starts at p
        uint32_t t = (run + kEmitTile - 1) / kEmitTile;
        for (; uint64_t(t) * kEmitTile < uint64_t(run) + c[j] && t < S.tile_start_len; ++t)
          S.tile_start[t] = p;
      }
      run += c[j];
    }
    carry += tot;
  }
}

// ------------------------------------------------------------------- emission

__global__ void __launch_bounds__(256) emit_kernel(EmitParams E) {
  __shared__ uint32_t s_off[kEmitTile + 1];
  __shared__ uint32_t s_pair[kEmitTile + 1];
  __shared__ uint2 s_rect[kEmitTile + 1];
  const uint32_t total = E.counters->n_inst_clamped;
  const unsigned long long total_all = E.counters->n_instances;
  const uint32_t nvis = E.counters->n_visible;
  const uint32_t ntile = (total + kEmitTile - 1) / kEmitTile;
  const unsigned long long ntile_all = (total_all + kEmitTile - 1) / kEmitTile;
  for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const uint32_t e0 = t * kEmitTile, e1 = min(e0 + uint32_t(kEmitTile), total);
    const uint32_t p_lo = E.tile_start[t];
    const uint32_t p_hi = (uint64_t(t) + 1 < ntile_all) ? E.tile_start[t + 1] : nvis - 1;
    const int np = int(p_hi - p_lo) + 1;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
      uint32_t pr = E.pairs[p_lo + j];
      s_off[j] = E.off[p_lo + j];
      s_pair[j] = pr;
      s_rect[j] = E.rect[pr];
    }
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int a = 0, b = np - 1;  // largest j with s_off[j] <= e
      while (a < b) {
        int m = (a + b + 1) >> 1;
        if (s_off[m] <= e) a = m; else b = m - 1;
      }
      uint32_t k = e - s_off[a];
      uint2 r = s_rect[a];
      uint32_t tx0 = r.x & 0xFFFF, ty0 = r.x >> 16, tx1 = r.y & 0xFFFF;
      uint32_t rw = tx1 - tx0 + 1;
      uint32_t ty = ty0 + k / rw, tx = tx0 + k % rw;
      uint32_t v = s_pair[a] / uint32_t(E.n);
      const DevCam &cam = E.cams[v];
      E.keys[e] = uint32_t(cam.tile_base) + ty * uint32_t(cam.tiles_x) + tx;
      E.vals[e] = p_lo + uint32_t(a);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t *keys, const Counters *c, uint2 *ranges) {
  const uint32_t n = c->n_inst_clamped;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
    if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
  }
}

cudaError_t launch_count_scan(const ScanParams &S, int G, cudaStream_t st) {
  count_tiles_kernel<<<G, 256, 0, st>>>(S);
  scan_partials_kernel<<<1, 32, 0, st>>>(S, G);
  offsets_kernel<<<G, 256, 0, st>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_emit(const EmitParams &E, int G, cudaStream_t st) {
  emit_kernel<<<G, 256, 0, st>>>(E);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t *keys, const Counters *c, uint2 *ranges, int G, cudaStream_t st) {
  ranges_kernel<<<G, 256, 0, st>>>(keys, c, ranges);
  return cudaGetLastError();
}

}  // namespace raygs
