// Gradients of an image loss through the rasteriser back to the primitive parameters.
// The paper's renderer is not differentiable; this is the reverse-mode derivative of the
// same image (Eq. rendering, Eq. rend_opacity, Eq. Q_ray), without the MIP term.
//
// Reverse replay (render_backward_kernel): per tile, per pixel, from the last composited
// instance back to the first, with T_i = T_{i+1} / (1 - omega_i), S the colour composited
// behind instance i and g = dL/dC, gT = dL/dT_final:
//   dL/domega_i = T_i g.rgb_i - (g.S + gT T_final) / (1 - omega_i)
//   dL/drgb_i   = g omega_i T_i
// With y = K x a whitening of the primitive (K Sigma K^T = I, K mu = c e3), the ray maximum
// lies at tau y, rho = tau y - c e3 = c (y2 y01, -q) / (q + r), and by the envelope theorem
//   dD/dmu = -2 K^T rho,   dD/dSigma^-1 = (Q rho)(Q rho)^T,  Q = K^-1 = Sigma K^T.
// Each pixel adds dL/dD rho (3), dL/dD rho rho^T (6), dL/domega omega (1, -> log opacity)
// and dL/drgb (3): 13 partial sums per (instance), reduced over the tile's pixels in
// registers, warp shuffles and shared memory, and written once per instance at its
// emission index (no global atomics).  Emission order groups the instances of a
// (primitive, view) pair, so pair_grads_kernel sums contiguous runs, and
// param_grads_kernel applies K, Q and the chain rule to the parameters, one thread per
// primitive looping over views.
#include "raygs_internal.cuh"
#include "raster_math.cuh"
#include "stage_math.cuh"

namespace raygs {

__device__ __forceinline__ uint32_t emission_index(const BackParams &P, uint32_t pos, uint32_t ty, uint32_t tx) {
  const uint32_t pair = P.pairs[pos];
  const uint2 rc = P.rect[pair];
  const uint32_t rs = P.row_off[pos] + (ty - (rc.x >> 16));
  const uint32_t txa = P.seg[rs].y & 0xFFFFu;
  return P.seg_off[rs] + (tx - txa);
}

// Sum 16 per-lane values over the warp by recursive halving: at each step a lane keeps half
// of its values and adds its partner's copy of them (16 shuffles in all, against 80 for 16
// separate butterflies).  Afterwards lane L holds the warp total of component
// 8 b4 + 4 b3 + 2 b2 + b1 (b_i the bits of L); lanes L and L ^ 1 hold the same one.
__device__ __forceinline__ float warp_sum16(float v[16], int lane) {
#pragma unroll
  for (int half = 8, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool upper = lane & o;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[i + half];
      const float keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ int warp_sum16_component(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

template <int TW, int TH, int PX>
__global__ void __launch_bounds__(TW *TH / PX, (PX >= 8 ? 512 : 896) / (TW * TH / PX)) render_backward_kernel(BackParams P) {
  constexpr int NT = TW * TH / PX;
  constexpr int NB = NT;
  constexpr int QX = TW / PX;
  constexpr int NW = NT / 32;
  __shared__ float4 s_A[NB], s_B[NB], s_C[NB], s_D[NB];
  __shared__ float s_isk[NB];  // 1 / sqrt(kp) of each staged record
  __shared__ uint32_t s_e[NB];
  __shared__ float s_acc[NB][kGradW];
  // per pixel slot (thread-major): final T and the loss gradients, read on every hit
  __shared__ float4 s_g[PX][NT];
  __shared__ float s_tfin[PX][NT];
  __shared__ int s_view, s_lmax;
  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    int v = 0;
    while (v + 1 < P.n_views && P.cams[v + 1].tile_base <= tile) ++v;
    s_view = v;
    s_lmax = 0;
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

  float Tk[PX], S0[PX], S1[PX], S2[PX];
  int last[PX];
  int lmax = 0;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    const bool in = py < cam.H && px + k * QX < cam.W;
    const long long pix = cam.pix_base + (long long)py * cam.W + px + k * QX;
    const float tf = in ? P.Tf[pix] : 1.f;
    s_tfin[k][tid] = tf;
    Tk[k] = tf;
    last[k] = in ? P.ncontrib[pix] : 0;
    s_g[k][tid] = make_float4(in ? P.dL_drgb[3 * pix] : 0.f, in ? P.dL_drgb[3 * pix + 1] : 0.f,
                              in ? P.dL_drgb[3 * pix + 2] : 0.f, (in && P.dL_dT) ? P.dL_dT[pix] : 0.f);
    S0[k] = S1[k] = S2[k] = 0.f;
    lmax = max(lmax, last[k]);
  }
  atomicMax(&s_lmax, lmax);
  __syncthreads();
  const int L = s_lmax;
  const int len = int(rg.y - rg.x);
  // instances past the last composited one of every pixel get zero partials
  for (int i = L + tid; i < len; i += NT) {
    const uint32_t e = emission_index(P, P.inst_vals[rg.x + i], ty, tx);
#pragma unroll
    for (int c = 0; c < kGradW; ++c) P.partials[size_t(e) * kGradW + c] = 0.f;
  }

  for (int end = L; end > 0; end -= NB) {
    const int start = max(0, end - NB);
    const int nb = end - start;
    __syncthreads();
    for (int slot = tid; slot < nb; slot += NT) {
      const uint32_t pos = P.inst_vals[rg.x + start + slot];
      const Rec r = P.rec[P.pairs[pos]];
      stage_record<0>(r, ox_tile, oy_tile, s_A[slot], s_B[slot], s_C[slot], s_D[slot]);
      s_isk[slot] = rsqrtf(r.c.z);
      s_e[slot] = emission_index(P, pos, ty, tx);
    }
    for (int i = tid; i < nb * kGradW; i += NT) (&s_acc[0][0])[i] = 0.f;
    __syncthreads();
    for (int j = nb - 1; j >= 0; --j) {
      const int pos = start + j;
      const float4 A = s_A[j], B = s_B[j];
      float q[PX], r[PX], y0[PX], y1[PX], y2[PX];
      const float4 Cs = s_C[j];
      // as in the forward pass, the segment filter pays only at 8 pixels per thread
      const uint32_t hit = (PX < 8 || row_may_hit<PX>(A, B, Cs, s_D[j].w, fl_x, fl_y, step))
                               ? eval_pixels<PX>(A, B, fl_x, fl_y, step, q, r, y0, y1, y2)
                               : 0u;
      float acc[kGradW];
#pragma unroll
      for (int c = 0; c < kGradW; ++c) acc[c] = 0.f;
      bool any = false;
      // the staged G carries sqrt(kp): y01 = y01' / sqrt(kp), q = q' / kp
      const float isk = s_isk[j], ikp = isk * isk;
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        if ((hit & (1u << k)) && pos < last[k]) {
          any = true;
          const float4 gg = s_g[k][tid];
          const float g0 = gg.x, g1 = gg.y, g2 = gg.z, gT = gg.w, Tfin = s_tfin[k][tid];
          const float4 Cc = s_C[j], Dd = s_D[j];
          const float raw = pixel_opacity<0>(Cc, q[k], r[k]);
          const bool clamped = raw > P.alpha_max;
          const float om = clamped ? P.alpha_max : raw;
          const float onem = 1.f - om;
          const float Ti = Tk[k] / onem;
          const float gc = g0 * Dd.x + g1 * Dd.y + g2 * Dd.z;
          const float gS = g0 * S0[k] + g1 * S1[k] + g2 * S2[k];
          const float dLdw = Ti * gc - (gS + gT * Tfin) / onem;
          const float wT = om * Ti;
          acc[10] += g0 * wT;
          acc[11] += g1 * wT;
          acc[12] += g2 * wT;
          S0[k] = fmaf(Dd.x, wT, S0[k]);
          S1[k] = fmaf(Dd.y, wT, S1[k]);
          S2[k] = fmaf(Dd.z, wT, S2[k]);
          Tk[k] = Ti;
          if (!clamped) {
            const float dLdD = -0.5f * om * dLdw;
            acc[9] += dLdw * om;
            const float qu = q[k] * ikp;
            const float inv = sqrtf(Cc.y * (2.f / kLog2e)) / (qu + r[k]);
            const float rho0 = y2[k] * (y0[k] * isk) * inv, rho1 = y2[k] * (y1[k] * isk) * inv, rho2 = -qu * inv;
            acc[0] += dLdD * rho0;
            acc[1] += dLdD * rho1;
            acc[2] += dLdD * rho2;
            acc[3] += dLdD * rho0 * rho0;
            acc[4] += dLdD * rho0 * rho1;
            acc[5] += dLdD * rho0 * rho2;
            acc[6] += dLdD * rho1 * rho1;
            acc[7] += dLdD * rho1 * rho2;
            acc[8] += dLdD * rho2 * rho2;
          }
        }
      }
      if (__any_sync(0xffffffffu, any)) {
        float v16[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v16[c] = c < kGradW ? acc[c] : 0.f;
        const float tot = warp_sum16(v16, lane);
        const int c = warp_sum16_component(lane);
        if ((lane & 1) == 0 && c < kGradW) {
          if (NW == 1) s_acc[j][c] += tot;
          else atomicAdd(&s_acc[j][c], tot);
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < nb * kGradW; i += NT) {
      const int slot = i / kGradW, c = i - slot * kGradW;
      P.partials[size_t(s_e[slot]) * kGradW + c] = s_acc[slot][c];
    }
  }
}

cudaError_t launch_render_backward(const BackParams &P, int tile_w, int tile_h, int64_t n_tiles, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  const unsigned grid = unsigned(n_tiles);
#define RAYGS_BWD_CASE(TW, TH, PX)                                                     \
  if (tile_w == TW && tile_h == TH) {                                                  \
    render_backward_kernel<TW, TH, PX><<<grid, TW * TH / PX, 0, st>>>(P);              \
    return cudaGetLastError();                                                         \
  }
  RAYGS_BWD_CASE(16, 16, 4)
  RAYGS_BWD_CASE(16, 8, 4)
  RAYGS_BWD_CASE(32, 16, 8)
  RAYGS_BWD_CASE(8, 8, 2)
#undef RAYGS_BWD_CASE
  return cudaErrorInvalidValue;
}

// Sum of the partials of each (primitive, view) pair over the contiguous run of its
// instances in emission order: eight lanes per sorted pair (four pairs per warp; a pair has
// about six instances on the 720p workload), then an xor reduction inside each group of
// eight lanes, whose lanes write the 13 totals.
__global__ void __launch_bounds__(256) pair_grads_kernel(PairGradParams P) {
  constexpr int GL = 8;  // lanes per pair
  const uint32_t nvis = P.counters->n_visible;
  const uint32_t ninst = P.counters->n_inst_clamped;
  const int lane = threadIdx.x & 31, sl = lane & (GL - 1);
  const uint32_t groups = (gridDim.x * blockDim.x) / GL;
  const uint32_t g0 = (blockIdx.x * blockDim.x + threadIdx.x) / GL;
  // every lane of a warp runs the same number of iterations (full-warp shuffles)
  const uint32_t iters = (nvis + groups - 1) / groups;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint32_t p = g0 + it * groups;
    float acc[kGradW];
#pragma unroll
    for (int c = 0; c < kGradW; ++c) acc[c] = 0.f;
    if (p < nvis) {
      const uint32_t e0 = P.seg_off[P.row_off[p]];
      const uint32_t e1 = p + 1 < nvis ? P.seg_off[P.row_off[p + 1]] : ninst;
      for (uint32_t e = e0 + sl; e < e1; e += GL) {
#pragma unroll
        for (int c = 0; c < kGradW; ++c) acc[c] += P.partials[size_t(e) * kGradW + c];
      }
    }
#pragma unroll
    for (int o = GL / 2; o >= 1; o >>= 1) {
#pragma unroll
      for (int c = 0; c < kGradW; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
    if (p < nvis) {
      float *dst = P.pg + size_t(P.pairs[p]) * kGradW;
#pragma unroll
      for (int c = 0; c < kGradW; ++c)
        if (c % GL == sl) dst[c] = acc[c];
    }
  }
}

cudaError_t launch_pair_grads(const PairGradParams &P, int G, cudaStream_t st) {
  pair_grads_kernel<<<G, 256, 0, st>>>(P);
  return cudaGetLastError();
}

// The whitening rows of a (primitive, view) exactly as the vertex stage built them (same
// precision choice), plus Sigma and c.
template <typename T>
__device__ void view_whitening(const float muf[3], const df muc[3], const T Rp[9], const T s[3], const DevCam &cam,
                               float K[3][3], float Sig[3][3], float Rc_out[9]) {
  T mu[3];
  if (sizeof(T) == 8) {
    for (int i = 0; i < 3; ++i) mu[i] = T(double(muc[i].hi) + double(muc[i].lo));
  } else {
    for (int i = 0; i < 3; ++i) mu[i] = T(muf[i]);
  }
  T Rc[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rc[3 * i + j] = T(cam.R[3 * i]) * Rp[j] + T(cam.R[3 * i + 1]) * Rp[3 + j] + T(cam.R[3 * i + 2]) * Rp[6 + j];
  T m[3], c2 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m[k] = (Rc[k] * mu[0] + Rc[3 + k] * mu[1] + Rc[6 + k] * mu[2]) / s[k];
    c2 += m[k] * m[k];
  }
  const T c = t_sqrt(c2);
  T k0[3], k1[3];
  plane_whitening<T>(mu, Rc, s, k0, k1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T w = Rc[3 * i] * m[0] / s[0] + Rc[3 * i + 1] * m[1] / s[1] + Rc[3 * i + 2] * m[2] / s[2];
    K[0][i] = float(k0[i]);
    K[1][i] = float(k1[i]);
    K[2][i] = float(w / c);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T v = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) v += Rc[3 * i + k] * s[k] * s[k] * Rc[3 * j + k];
      Sig[i][j] = float(v);
    }
#pragma unroll
  for (int i = 0; i < 9; ++i) Rc_out[i] = float(Rc[i]);
}

constexpr int kParamThreads = 64;

// Chain rule of one primitive over the views where it is visible; SH gradients are
// accumulated into dsh (this thread's row of shared memory), the other parameter
// gradients written directly.
// FP64 = false handles the primitives that need no FP64 whitening in any view and returns
// false for the others without writing anything; FP64 = true handles exactly those (the
// near-degenerate ones), so that the FP64 code holds no registers in the common kernel.
template <int DEG, bool FP64>
__device__ __forceinline__ bool param_grads_one(const ParamGradParams &P, int g, const float *coef, float *dsh,
                                                int dsh_stride = 1) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const float mx = P.means[3 * int64_t(g)], my = P.means[3 * int64_t(g) + 1], mz = P.means[3 * int64_t(g) + 2];
  float ls[3], q4[4];
  for (int k = 0; k < 3; ++k) ls[k] = load_attr(P.log_scales, 3 * int64_t(g) + k, P.scale_dtype);
  for (int k = 0; k < 4; ++k) q4[k] = P.quats[4 * int64_t(g) + k];
  const float logit = load_attr(P.logits, g, P.opacity_dtype);
  float Rp[9];
  quat_rot<float>(q4[0], q4[1], q4[2], q4[3], Rp);
  const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
  const float o = 1.f / (1.f + expf(-logit));
  bool degenerate = false;
  if (P.fp64_degenerate) {
    const float lmax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]), lmin = fminf(fminf(ls[0], ls[1]), ls[2]);
    degenerate = (lmax - lmin) > logf(P.degenerate_ratio);
  }
  if (degenerate != FP64) return false;

  float dmu[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dRp[9], dlogit = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) dRp[i] = 0.f;

  for (int v = 0; v < P.n_views; ++v) {
    const int64_t idx = int64_t(v) * P.n + g;
    if (P.depth_key[idx] == kCulled) continue;
    const DevCam &cam = P.cams[v];
    const float *pg = P.pg + size_t(idx) * kGradW;
    float a[3] = {pg[0], pg[1], pg[2]};
    const float b00 = pg[3], b01 = pg[4], b02 = pg[5], b11 = pg[6], b12 = pg[7], b22 = pg[8];
    const float lo = pg[9];
    const float col[3] = {pg[10], pg[11], pg[12]};
    df muc[3];
    mean_cam_df(cam, mx, my, mz, muc);
    const float muf[3] = {muc[0].hi, muc[1].hi, muc[2].hi};
    float Km[3][3], Sig[3][3], Rc[9];
    bool use_fp64 = false;
    if (degenerate) {
      // same precision choice as the vertex stage
      float k0[3], k1[3], Rcf[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          Rcf[3 * i + j] = cam.R[3 * i] * Rp[j] + cam.R[3 * i + 1] * Rp[3 + j] + cam.R[3 * i + 2] * Rp[6 + j];
      const bool ok = plane_whitening<float>(muf, Rcf, s, k0, k1);
      use_fp64 = P.fp64_degenerate == 2 || !ok;
    }
    if (FP64 && use_fp64) {
      double Rpd[9], sd[3];
      quat_rot<double>(double(q4[0]), double(q4[1]), double(q4[2]), double(q4[3]), Rpd);
      for (int k = 0; k < 3; ++k) sd[k] = exp(double(ls[k]));
      view_whitening<double>(muf, muc, Rpd, sd, cam, Km, Sig, Rc);
    } else {
      view_whitening<float>(muf, muc, Rp, s, cam, Km, Sig, Rc);
    }
    // dL/dmu_c = -2 K^T a
    float dmuc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dmuc[i] = -2.f * (a[0] * Km[0][i] + a[1] * Km[1][i] + a[2] * Km[2][i]);
    // dL/dSigma^-1 (camera) = Sigma (K^T B K) Sigma
    const float Bm[3][3] = {{b00, b01, b02}, {b01, b11, b12}, {b02, b12, b22}};
    float KB[3][3], M1[3][3], T1[3][3], Gc[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) KB[i][j] = Km[0][i] * Bm[0][j] + Km[1][i] * Bm[1][j] + Km[2][i] * Bm[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M1[i][j] = KB[i][0] * Km[0][j] + KB[i][1] * Km[1][j] + KB[i][2] * Km[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) T1[i][j] = Sig[i][0] * M1[0][j] + Sig[i][1] * M1[1][j] + Sig[i][2] * M1[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Gc[i][j] = T1[i][0] * Sig[0][j] + T1[i][1] * Sig[1][j] + T1[i][2] * Sig[2][j];
    // world frame: Sigma_c^-1 = R Sigma_w^-1 R^T, mu_c = R mu_w + t
    float Gw[3][3], tmp[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tmp[i][j] = cam.R[i] * Gc[0][j] + cam.R[3 + i] * Gc[1][j] + cam.R[6 + i] * Gc[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Gw[i][j] = tmp[i][0] * cam.R[j] + tmp[i][1] * cam.R[3 + j] + tmp[i][2] * cam.R[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) dmu[i] += cam.R[i] * dmuc[0] + cam.R[3 + i] * dmuc[1] + cam.R[6 + i] * dmuc[2];
    // Sigma_w^-1 = sum_k n_k n_k^T / s_k^2, n_k = column k of R_p
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float n0 = Rp[k], n1 = Rp[3 + k], n2 = Rp[6 + k];
      const float Gn0 = Gw[0][0] * n0 + Gw[0][1] * n1 + Gw[0][2] * n2;
      const float Gn1 = Gw[1][0] * n0 + Gw[1][1] * n1 + Gw[1][2] * n2;
      const float Gn2 = Gw[2][0] * n0 + Gw[2][1] * n1 + Gw[2][2] * n2;
      const float is2 = 1.f / (s[k] * s[k]);
      dls[k] += -2.f * is2 * (n0 * Gn0 + n1 * Gn1 + n2 * Gn2);
      dRp[k] += 2.f * is2 * Gn0;
      dRp[3 + k] += 2.f * is2 * Gn1;
      dRp[6 + k] += 2.f * is2 * Gn2;
    }
    dlogit += lo * (1.f - o);
    // colour: rgb = max(0, k0 + sum_k Y_k(d) k_k), d = (mu - C) / |mu - C|
    const float ex = mx - cam.C[0], ey = my - cam.C[1], ez = mz - cam.C[2];
    const float inv_len = rsqrtf(ex * ex + ey * ey + ez * ez);
    const float dx = ex * inv_len, dy = ey * inv_len, dz = ez * inv_len;
    // the colour before its clamp at 0 (each basis term recomputed where it is used, so that
    // no per-term arrays stay live), then the gradients of the channels above the clamp
    float val[3] = {coef[0], coef[1], coef[2]};
#pragma unroll
    for (int k = 1; k < K; ++k) {
      float Yk, ax, ay, az;
      sh_term(k, dx, dy, dz, Yk, ax, ay, az);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) val[ch] = fmaf(Yk, coef[3 * k + ch], val[ch]);
    }
    const float cl[3] = {val[0] > 0.f ? col[0] : 0.f, val[1] > 0.f ? col[1] : 0.f, val[2] > 0.f ? col[2] : 0.f};
    float gd[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float Yk, ax, ay, az;
      sh_term(k, dx, dy, dz, Yk, ax, ay, az);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) dsh[(3 * k + ch) * dsh_stride] += cl[ch] * Yk;
      const float sk = cl[0] * coef[3 * k] + cl[1] * coef[3 * k + 1] + cl[2] * coef[3 * k + 2];
      gd[0] = fmaf(sk, ax, gd[0]);
      gd[1] = fmaf(sk, ay, gd[1]);
      gd[2] = fmaf(sk, az, gd[2]);
    }
    const float dd = dx * gd[0] + dy * gd[1] + dz * gd[2];
    dmu[0] += (gd[0] - dx * dd) * inv_len;
    dmu[1] += (gd[1] - dy * dd) * inv_len;
    dmu[2] += (gd[2] - dz * dd) * inv_len;
  }
  // quaternion: R(q^) with q^ = q/|q|
  const float qn = rsqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
  const float w = q4[0] * qn, x = q4[1] * qn, y = q4[2] * qn, z = q4[3] * qn;
  const float *G = dRp;
  const float gw = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  const float gx = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] -
                          2.f * x * G[8]);
  const float gy = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] -
                          2.f * y * G[8]);
  const float gz = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] +
                          y * G[7]);
  const float dot = w * gw + x * gx + y * gy + z * gz;
  if (P.d_means) {
    P.d_means[3 * int64_t(g)] = dmu[0];
    P.d_means[3 * int64_t(g) + 1] = dmu[1];
    P.d_means[3 * int64_t(g) + 2] = dmu[2];
  }
  if (P.d_log_scales) {
    for (int k = 0; k < 3; ++k) P.d_log_scales[3 * int64_t(g) + k] = dls[k];
  }
  if (P.d_quats) {
    P.d_quats[4 * int64_t(g)] = (gw - w * dot) * qn;
    P.d_quats[4 * int64_t(g) + 1] = (gx - x * dot) * qn;
    P.d_quats[4 * int64_t(g) + 2] = (gy - y * dot) * qn;
    P.d_quats[4 * int64_t(g) + 3] = (gz - z * dot) * qn;
  }
  if (P.d_logits) P.d_logits[g] = dlogit;
  return true;
}

template <int DEG>
__global__ void __launch_bounds__(kParamThreads, 8) param_grads_kernel(ParamGradParams P) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int K3 = 3 * K, SHP = K3 + 1;  // padded row
  // SH coefficients in and their gradients out go through shared memory with coalesced
  // 16-byte transfers (one row of 3K values per primitive); the gradients accumulate over
  // the views in shared memory too
  __shared__ float s_sh[kParamThreads * SHP];
  __shared__ float s_dsh[kParamThreads * SHP];
  __shared__ uint8_t s_keep[kParamThreads];
  const int g0 = blockIdx.x * blockDim.x;
  const int nb = min(int(blockDim.x), P.n - g0);
  stage_attr(s_sh, P.sh, int64_t(g0) * K3, nb * K3, P.sh_dtype, K3, 1);
  float *dsh = s_dsh + threadIdx.x * SHP;
  for (int i = 0; i < K3; ++i) dsh[i] = 0.f;
  __syncthreads();
  const int g = g0 + threadIdx.x;
  const bool active = g < P.n;
  const float *coef = s_sh + threadIdx.x * SHP;
  // a primitive left to the FP64 kernel keeps its SH gradients out of the coalesced store
  const bool done = active && param_grads_one<DEG, false>(P, g, coef, dsh);
  s_keep[threadIdx.x] = done ? 1 : 0;
  if (active && !done) P.fp64_list[atomicAdd(P.fp64_count, 1u)] = uint32_t(g);
  __syncthreads();
  if (P.d_sh) {
    float *dst = P.d_sh + int64_t(g0) * K3;
    for (int e = threadIdx.x; e < nb * K3; e += blockDim.x)
      if (s_keep[e / K3]) dst[e] = s_dsh[(e / K3) * SHP + e % K3];
  }
}

// The near-degenerate primitives (FP64 whitening in the views where the float32 one is
// ill-conditioned) that param_grads_kernel listed, grid-stride with direct loads: few
// enough that coalescing does not matter.
template <int DEG>
__global__ void __launch_bounds__(128) param_grads_fp64_kernel(ParamGradParams P) {
  constexpr int K3 = 3 * (DEG + 1) * (DEG + 1);
  const uint32_t count = *P.fp64_count;
  for (uint32_t li = blockIdx.x * blockDim.x + threadIdx.x; li < count; li += gridDim.x * blockDim.x) {
    const int g = int(P.fp64_list[li]);
    float coef[K3];
    for (int k = 0; k < K3; ++k) coef[k] = load_attr(P.sh, int64_t(g) * K3 + k, P.sh_dtype);
    float dsh[K3];
    for (int k = 0; k < K3; ++k) dsh[k] = 0.f;
    if (param_grads_one<DEG, true>(P, g, coef, dsh) && P.d_sh)
      for (int k = 0; k < K3; ++k) P.d_sh[int64_t(g) * K3 + k] = dsh[k];
  }
}

cudaError_t launch_param_grads(const ParamGradParams &P, cudaStream_t st) {
  if (P.n == 0) return cudaSuccess;
  const int blocks = (P.n + kParamThreads - 1) / kParamThreads;
  switch (P.sh_degree) {
    case 0: param_grads_kernel<0><<<blocks, kParamThreads, 0, st>>>(P); break;
    case 1: param_grads_kernel<1><<<blocks, kParamThreads, 0, st>>>(P); break;
    case 2: param_grads_kernel<2><<<blocks, kParamThreads, 0, st>>>(P); break;
    default: param_grads_kernel<3><<<blocks, kParamThreads, 0, st>>>(P); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !P.fp64_degenerate) return e;
  const int64_t want = (int64_t(P.n) + 127) / 128, cap = int64_t(P.num_sms > 0 ? P.num_sms : 1) * 2;
  const int gb = int(want < cap ? want : cap);
  switch (P.sh_degree) {
    case 0: param_grads_fp64_kernel<0><<<gb, 128, 0, st>>>(P); break;
    case 1: param_grads_fp64_kernel<1><<<gb, 128, 0, st>>>(P); break;
    case 2: param_grads_fp64_kernel<2><<<gb, 128, 0, st>>>(P); break;
    default: param_grads_fp64_kernel<3><<<gb, 128, 0, st>>>(P); break;
  }
  return cudaGetLastError();
}

}  // namespace raygs
