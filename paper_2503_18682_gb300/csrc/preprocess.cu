// Per-primitive vertex stage (Sec. 3, Sec. 3.2, Sec. 4.1, Sec. 5 of the paper; Sec. 3.1 for
// the GS divergence) for every view of a batch.  One thread per primitive loops over the views; attributes are staged
// once per CTA with 16-byte coalesced loads and converted to float32 in shared memory.
//
// Outputs per (view v, primitive g), index v*N + g:
//   depth_key  float32 bits of the view-space centre depth, or kCulled
//   rect       inclusive screen-tile rectangle that bounds the support (the support
//              ellipse's box, or the projected quad's, Eq. V_ray)
//   ell        32-byte support sector: the rectangle again and the support ellipse
//   rec        64-byte pixel record (see Rec): the factors of the fragment formula of
//              Sec. 4.2 / App. A.4 in a form that is evaluated from the pixel ray
//
// For primitives whose scale ratio exceeds degenerate_ratio, the float32 result of a view
// is replaced by the same stage run in FP64 (preprocess_fp64_kernel) when the float32
// solve is ill-conditioned in that view (the disk is seen nearly edge-on), or for every
// visible view when fp64_degenerate == 2.  Independently of that setting, a pair whose
// float32 skip decision (opacity below the cut-off, Eq. support; camera inside, Eq. c) lies
// within the float32 rounding of its threshold is decided by the FP64 stage.
#include "raygs_internal.cuh"
#include "stage_math.cuh"

namespace raygs {


constexpr int kPrepThreads = 128;

struct StageOut {
  float G[4], h[2], kp, c2h, lo2o;
  int tx0, ty0, tx1, ty1;
  bool illcond;  // the 2x2 projected covariance lost more than 3 digits in its Cholesky
  // support ellipse (p - u - dc)^T M (p - u - dc) <= rho in pixel offsets from the centre
  float dc0, dc1, M00, M01, M11, rho, det;
};

// A sphere of radius rad around mu lies entirely outside one of the four side planes of
// the view's frustum (through the outermost pixel-centre rays).
template <typename T>
__device__ __forceinline__ bool outside_frustum(const T mu[3], T rad, const DevCam &cam) {
  return mu[0] - T(cam.xmin) * mu[2] < -rad * T(cam.fn[0]) || T(cam.xmax) * mu[2] - mu[0] < -rad * T(cam.fn[1]) ||
         mu[1] - T(cam.ymin) * mu[2] < -rad * T(cam.fn[2]) || T(cam.ymax) * mu[2] - mu[1] < -rad * T(cam.fn[3]);
}

// Inclusive tile rectangle of the pixels whose centres lie in the screen box [xmn, xmx] x
// [ymn, ymx] (with a small conservative margin), or of the whole view when `full`.
// Returns false when the box holds no pixel centre of the view.
__device__ __forceinline__ bool tile_rect(bool full, float xmn, float xmx, float ymn, float ymx, const DevCam &cam,
                                          int tile_w, int tile_h, StageOut &out) {
  int i0, i1, j0, j1;
  if (full) {
    i0 = 0; j0 = 0; i1 = cam.W - 1; j1 = cam.H - 1;
  } else {
    if (!(xmn <= xmx) || !(ymn <= ymx)) return false;  // empty or NaN
    const float lim = 1.0e8f;
    float mgx = 1e-3f + 1e-5f * fmaxf(fabsf(xmn), fabsf(xmx));
    float mgy = 1e-3f + 1e-5f * fmaxf(fabsf(ymn), fabsf(ymx));
    // pixel centre i + 0.5 inside [xmn, xmx] (with a small conservative margin)
    float fi0 = ceilf(fminf(fmaxf(xmn - 0.5f - mgx, -lim), lim));
    float fi1 = floorf(fminf(fmaxf(xmx - 0.5f + mgx, -lim), lim));
    float fj0 = ceilf(fminf(fmaxf(ymn - 0.5f - mgy, -lim), lim));
    float fj1 = floorf(fminf(fmaxf(ymx - 0.5f + mgy, -lim), lim));
    fi0 = fmaxf(fi0, 0.f); fj0 = fmaxf(fj0, 0.f);
    fi1 = fminf(fi1, float(cam.W - 1)); fj1 = fminf(fj1, float(cam.H - 1));
    if (fi0 > fi1 || fj0 > fj1) return false;
    i0 = int(fi0); i1 = int(fi1); j0 = int(fj0); j1 = int(fj1);
  }
  out.tx0 = i0 / tile_w; out.tx1 = i1 / tile_w;
  out.ty0 = j0 / tile_h; out.ty1 = j1 / tile_h;
  return true;
}

// Outcome of a vertex stage: the pair is skipped, kept, or (float32 only) one of its two
// skip decisions -- kappa <= 0 (Eq. support) and c^2 <= kappa (Eq. c) -- lies within the
// float32 rounding of its threshold, and the FP64 stage decides.
enum StageResult { kSkip = 0, kKeep = 1, kUndecided = 2 };

// Relative rounding bound of a float32 camera-frame projection R_c^T mu, as a fraction of
// |mu|_1 (the float mean, the float rotation and the three-term dot product), with a
// fourfold margin.
constexpr float kProjErr32 = 2e-6f;

// Sec. 4.1 vertex stage: the smallest enclosing quad V_ray (App. A.1-A.3) of the
// primitive's support in the camera frame and the screen bounding box of its projected
// vertices; full = true when a vertex lies behind the camera plane (the box is then the
// whole view).  m = S^-1 R_c^T mu, c = |m|.
template <typename T>
__device__ __forceinline__ void quad_screen_box(const T mu[3], const T Rc[9], const T s[3], const T m[3], T c, T c2,
                                                T kappa, const DevCam &cam, bool &full, float &xmn, float &xmx,
                                                float &ymn, float &ymx) {
  // mu^ = S^-1 R^T mu / c; R_{mu^<-v} of App. A.1 (columns 0, 1).
  T mh0 = m[0] / c, mh1 = m[1] / c, mh2 = m[2] / c;
  bool up = mh2 >= T(0);
  T a0 = mh0, a1 = mh1, a2 = up ? mh2 + T(1) : mh2 - T(1);
  T inv = T(2) / (a0 * a0 + a1 * a1 + a2 * a2);
  T r0[3] = {inv * a0 * a0 - T(1), inv * a1 * a0, inv * a2 * a0};
  T r1[3] = {inv * a0 * a1, inv * a1 * a1 - T(1), inv * a2 * a1};
  if (!up) { r0[0] = -r0[0]; r0[1] = -r0[1]; r0[2] = -r0[2]; }  // times P = diag(-1,1,-1)
  // Q_{0:2} = R S R_{mu^<-v} restricted to its first two columns (Eq. invPhi).
  T q0[3], q1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q0[i] = Rc[3 * i] * s[0] * r0[0] + Rc[3 * i + 1] * s[1] * r0[1] + Rc[3 * i + 2] * s[2] * r0[2];
    q1[i] = Rc[3 * i] * s[0] * r1[0] + Rc[3 * i + 1] * s[1] * r1[1] + Rc[3 * i + 2] * s[2] * r1[2];
  }
  // Eq. optim2: u1 = top eigenvector of B = Q_{0:2}^T Q_{0:2} (half-angle form).
  T B00 = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
  T B01 = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2];
  T B11 = q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2];
  T dd = B00 - B11, rho = t_sqrt(dd * dd + T(4) * B01 * B01);
  T u1x = T(1), u1y = T(0);
  if (rho > T(1e-12) * (B00 + B11)) {
    if (dd >= T(0)) { u1x = dd + rho; u1y = T(2) * B01; }
    else { u1x = T(2) * B01; u1y = rho - dd; }
    T un = T(1) / t_sqrt(u1x * u1x + u1y * u1y);
    u1x *= un; u1y *= un;
  }
  // u0 = u1 rotated by +90 degrees; Z_ray = (sqrt(kappa)/b) O, b = sqrt(1 - kappa/c^2).
  T zs = t_sqrt(kappa) / t_sqrt(T(1) - kappa / c2);
  T A0[3], A1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    A0[i] = zs * (-u1y * q0[i] + u1x * q1[i]);  // Q_{0:2} u0
    A1[i] = zs * (u1x * q0[i] + u1y * q1[i]);   // Q_{0:2} u1
  }
  // Eq. V_ray: vertices mu + (+-1) A0 + (+-1) A1; screen bounding box of their projections.
  full = false;
  xmn = 3.0e38f; xmx = -3.0e38f; ymn = 3.0e38f; ymx = -3.0e38f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T sa = (k & 2) ? T(1) : T(-1), sb = (k == 1 || k == 2) ? T(1) : T(-1);
    T px = mu[0] + sa * A0[0] + sb * A1[0];
    T py = mu[1] + sa * A0[1] + sb * A1[1];
    T pz = mu[2] + sa * A0[2] + sb * A1[2];
    if (!(pz > T(1e-12))) { full = true; continue; }
    float u = float(T(cam.fx) * px / pz + T(cam.cx));
    float v = float(T(cam.fy) * py / pz + T(cam.cy));
    xmn = fminf(xmn, u); xmx = fmaxf(xmx, u); ymn = fminf(ymn, v); ymx = fmaxf(ymx, v);
  }
}

// The per-(primitive, view) stage in precision T.  mu: camera-frame mean; Rp: world-frame
// rotation; s: scales; o: prior opacity.  Returns kSkip when the primitive is skipped or
// covers no pixel of this view.  With `decide` (float32 only), a skip decision within
// rounding of its threshold returns kUndecided instead.
template <typename T>
__device__ int view_stage(const T mu[3], const T Rp[9], const T s_in[3], T o, const DevCam &cam,
                          float p_min, float mip_sigma2, int tile_w, int tile_h, StageOut &out,
                          bool apply_mip = true, bool decide = true, const float *pre = nullptr) {
  const bool band = decide && sizeof(T) == 4;
  const T mu1 = fabs(mu[0]) + fabs(mu[1]) + fabs(mu[2]);
  T e_o = T(2e-6);  // relative rounding bound of o (the float32 sigmoid; grows with Eq. mip)
  // R_c = R_wc R_p: columns n_k are the primitive's axes in the camera frame.
  T Rc[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rc[3 * i + j] = T(cam.R[3 * i]) * Rp[j] + T(cam.R[3 * i + 1]) * Rp[3 + j] +
                      T(cam.R[3 * i + 2]) * Rp[6 + j];
  T pk[3], s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pk[k] = Rc[k] * mu[0] + Rc[3 + k] * mu[1] + Rc[6 + k] * mu[2];  // n_k . mu
    s[k] = s_in[k];
  }
  if (apply_mip && cam.mip == RAYGS_MIP_APPROX) {
    // Sec. 5, Eq. mip: Sigma^ = Sigma + lam I with lam = sigma^2 |mu|^2 / (fx fy); the
    // opacity is modulated by sqrt(|Sigma| c^2 / (|Sigma^| c^^2)).
    T lam = T(mip_sigma2) * (mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]) /
            (T(cam.fx) * T(cam.fy));
    T c2 = 0, c2h = 0, ratio = 1, e2 = 0, e2h = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T s2 = s[k] * s[k], s2h = s2 + lam;
      c2 += pk[k] * pk[k] / s2;
      c2h += pk[k] * pk[k] / s2h;
      // rounding of c^2 and c^^2 through the projections pk
      e2 += T(2) * fabs(pk[k]) * T(kProjErr32) * mu1 / s2;
      e2h += T(2) * fabs(pk[k]) * T(kProjErr32) * mu1 / s2h;
      ratio *= s2 / s2h;
      s[k] = t_sqrt(s2h);
    }
    o *= t_sqrt(ratio * c2 / c2h);
    e_o += T(0.5) * (e2 / c2 + e2h / c2h) + T(1e-6);
  }
  // Eq. support: kappa = -2 log(p_min / o); skip when kappa <= 0.  Without the MIP term o
  // is the primitive's own, and pre = (kappa, log2 o) holds them, computed once per
  // primitive with the same operations.
  const bool use_pre = pre && !(apply_mip && cam.mip == RAYGS_MIP_APPROX);
  T kappa = use_pre ? T(pre[0]) : T(2) * t_log(o / T(p_min));
  if (band && fabs(kappa) <= T(2) * e_o + T(1e-6)) return kUndecided;
  if (!(kappa > T(0))) return kSkip;

  // Conservative frustum test: every supported ray passes within sqrt(kappa) s_max of mu.
  {
    T smax = fmax(fmax(s[0], s[1]), s[2]);
    T rad = t_sqrt(kappa) * smax * T(1.001) + T(1e-6);
    if (outside_frustum<T>(mu, rad, cam)) return kSkip;
  }

  // Sec. 3.2 Eq. c: c^2 = mu^T Sigma^-1 mu = |S^-1 R^T mu|^2; skip when c^2 <= kappa.
  T m[3], is[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    is[k] = T(1) / s[k];
    m[k] = pk[k] * is[k];
  }
  T c2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
  if (band) {
    // each m_k carries the projection's rounding over s_k (large for thin primitives seen
    // from near their plane), kappa that of log o
    T e_c2 = T(1e-6) * (c2 + kappa) + T(2) * e_o;
#pragma unroll
    for (int k = 0; k < 3; ++k) e_c2 += T(2) * fabs(m[k]) * (T(kProjErr32) * mu1 * is[k] + T(1e-6) * fabs(m[k]));
    if (fabs(c2 - kappa) <= e_c2) return kUndecided;
  }
  if (!(c2 > kappa)) return kSkip;
  T c = t_sqrt(c2);

  bool full = false;
  float xmn = 3.0e38f, xmx = -3.0e38f, ymn = 3.0e38f, ymx = -3.0e38f;

  // ---- Per-pixel factors.  With y = K x, K = Q^-1 (App. A.4 steps g-i),
  // D = c^2 |y01|^2 / |y|^2, which is the fragment formula 1/(c^-2 + |Z a|^-2) with the
  // quad coordinate Z a = c U^T y01 / y2 read off the pixel ray.  The rows of K01 span the
  // Sigma-orthonormal complement of mu, built stably from an orthonormal basis E of the
  // plane orthogonal to mu: K01 = L^-1 E^T with L L^T = E^T Sigma E.  Since K01 mu = 0,
  // y01 only needs the pixel offset from the projected centre.
  T k0[3], k1[3];
  out.illcond = !plane_whitening<T>(mu, Rc, s, k0, k1);
  T scl = mu[2] / c;  // normalise so that y2 = 1 on the centre ray
  // the record's G carries sqrt(kp), so that the rasteriser's support test kp q <= r reads
  // q' <= r with q' = |G delta|^2
  const T gsc = scl * t_sqrt((c2 - kappa) / kappa);
  out.G[0] = float(k0[0] * T(cam.ifx) * gsc);
  out.G[1] = float(k0[1] * T(cam.ify) * gsc);
  out.G[2] = float(k1[0] * T(cam.ifx) * gsc);
  out.G[3] = float(k1[1] * T(cam.ify) * gsc);
  // y2 = mu^T Sigma^-1 x / c; Sigma^-1 mu = sum_k n_k m_k / s_k.
  T w0 = Rc[0] * m[0] * is[0] + Rc[1] * m[1] * is[1] + Rc[2] * m[2] * is[2];
  T w1 = Rc[3] * m[0] * is[0] + Rc[4] * m[1] * is[1] + Rc[5] * m[2] * is[2];
  T sh = mu[2] / c2;
  out.h[0] = float(w0 * T(cam.ifx) * sh);
  out.h[1] = float(w1 * T(cam.ify) * sh);
  out.kp = float((c2 - kappa) / kappa);
  out.c2h = float(c2 * T(0.5 * 1.4426950408889634));
  out.lo2o = use_pre ? pre[1] : float(t_log(o) * T(1.4426950408889634));

  // ---- Screen-space support: with delta = px - u (pixels), D <= kappa and y2 > 0 hold
  // exactly when f(delta) = kp |G delta|^2 - (1 + h.delta)^2 <= 0, a conic
  // delta^T M delta - 2 h.delta - 1 <= 0 with M = kp G^T G - h h^T.  When M is positive
  // definite (and not too ill-conditioned for float32 use) the support is the ellipse
  // (delta - dc)^T M (delta - dc) <= rho with dc = M^-1 h, rho = 1 + h.dc; its bounding box
  // tightens the quad's, and binning tests tile rows against it.
  {
    const T g00 = k0[0] * T(cam.ifx) * scl, g01 = k0[1] * T(cam.ify) * scl;
    const T g10 = k1[0] * T(cam.ifx) * scl, g11 = k1[1] * T(cam.ify) * scl;
    const T hh0 = w0 * T(cam.ifx) * sh, hh1 = w1 * T(cam.ify) * sh;
    const T kpt = (c2 - kappa) / kappa;
    const T M00 = kpt * (g00 * g00 + g10 * g10) - hh0 * hh0;
    const T M01 = kpt * (g00 * g01 + g10 * g11) - hh0 * hh1;
    const T M11 = kpt * (g01 * g01 + g11 * g11) - hh1 * hh1;
    const T det = M00 * M11 - M01 * M01;
    out.rho = -1.f;
    out.M00 = -1.f;  // no bounded ellipse unless set below
    bool bounded = false;
    if (M00 > T(0) && M11 > T(0) && det > T(1e-4) * M00 * M11) {
      const T dc0 = (M11 * hh0 - M01 * hh1) / det, dc1 = (M00 * hh1 - M01 * hh0) / det;
      const T rho = T(1) + hh0 * dc0 + hh1 * dc1;
      if (rho > T(0)) {
        out.dc0 = float(dc0); out.dc1 = float(dc1);
        out.M00 = float(M00 / rho); out.M01 = float(M01 / rho); out.M11 = float(M11 / rho);
        out.rho = float(rho); out.det = float(det / (rho * rho));
        // the bounding box of a bounded support ellipse bounds the pixels (also where the
        // quad reaches behind the camera) and is the tightest box of the support: the quad
        // is not needed then
        const T ucx = T(cam.fx) * mu[0] / mu[2] + T(cam.cx) + dc0;
        const T ucy = T(cam.fy) * mu[1] / mu[2] + T(cam.cy) + dc1;
        const T hx = t_sqrt(rho * T(1.001) * M11 / det), hy = t_sqrt(rho * T(1.001) * M00 / det);
        bounded = true;
        xmn = float(ucx - hx); xmx = float(ucx + hx); ymn = float(ucy - hy); ymx = float(ucy + hy);
      }
    }
    // otherwise the support is bounded by the paper's quad (Sec. 4.1)
    if (!bounded) quad_screen_box<T>(mu, Rc, s, m, c, c2, kappa, cam, full, xmn, xmx, ymn, ymx);
  }
  return tile_rect(full, xmn, xmx, ymn, ymx, cam, tile_w, tile_h, out) ? kKeep : kSkip;
}

// GS vertex stage (Sec. 3.1) in precision T: Sigma_pi = J Sigma J^T with J the Jacobian of
// the projection at the camera-frame mean mu, and records for D_gs = delta^T Sigma_pi^-1
// delta.  With M = J R_c S (2x3, rows m0, m1), Sigma_pi = M M^T and det Sigma_pi =
// |m0 x m1|^2 (Cauchy-Binet).  Since m_i = S R_c^T j_i and j0 x j1 = (fx fy / z^2) mu / z,
// m0 x m1 = (s0 s1 s2 fx fy / z^3) S^-1 R_c^T mu, so det Sigma_pi = (s0 s1 s2 fx fy / z^3)^2 c^2
// with c^2 = mu^T Sigma^-1 mu: a sum of squares, free of the cancellation that the
// 2x2 determinant (or the cross product) suffers for thin disks seen edge-on.  The record holds
// the upper Cholesky factor G of A = Sigma_pi^-1 (G^T G = A, G10 = 0), h = 0,
// kp = 1 / kappa and c2h = log2(e) / 2, so the rasteriser's test reads |G delta|^2 <= kappa
// and its exponent D_gs log2(e) / 2.  The support is the ellipse delta^T A delta <= kappa.
// There is no camera-inside skip (Eq. c) and no Eq. mip term.
template <typename T>
__device__ int gs_view_stage(const T mu[3], const T Rp[9], const T s[3], T o, const DevCam &cam, float p_min,
                             int tile_w, int tile_h, StageOut &out) {
  T kappa = T(2) * t_log(o / T(p_min));
  if (sizeof(T) == 4 && fabs(kappa) <= T(5e-6)) return kUndecided;  // o within rounding of p_min
  if (!(kappa > T(0))) return kSkip;
  T Rc[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rc[3 * i + j] = T(cam.R[3 * i]) * Rp[j] + T(cam.R[3 * i + 1]) * Rp[3 + j] +
                      T(cam.R[3 * i + 2]) * Rp[6 + j];
  // rows of J: (fx / z) (e_0 - (x / z) e_2) and (fy / z) (e_1 - (y / z) e_2)
  const T iz = T(1) / mu[2];
  const T ax = mu[0] * iz, ay = mu[1] * iz;
  const T jx = T(cam.fx) * iz, jy = T(cam.fy) * iz;
  T m0[3], m1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m0[k] = jx * (Rc[k] - ax * Rc[6 + k]) * s[k];
    m1[k] = jy * (Rc[3 + k] - ay * Rc[6 + k]) * s[k];
  }
  const T P00 = m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2];
  const T P01 = m0[0] * m1[0] + m0[1] * m1[1] + m0[2] * m1[2];
  const T P11 = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
  T c2 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T mk = (Rc[k] * mu[0] + Rc[3 + k] * mu[1] + Rc[6 + k] * mu[2]) / s[k];
    c2 += mk * mk;
  }
  const T sd = s[0] * s[1] * s[2] * jx * jy * iz;
  const T det = sd * sd * c2;  // det Sigma_pi
  if (!(det > T(0)) || !(P00 > T(0)) || !(P11 > T(0))) return kSkip;
  // A = Sigma_pi^-1 = [[P11, -P01], [-P01, P00]] / det; G00 = sqrt(A00), G01 = A01 / G00,
  // G11 = sqrt(det A) / G00 with det A = 1 / det Sigma_pi
  const T idet = T(1) / det;
  const T A00 = P11 * idet, A01 = -P01 * idet, A11 = P00 * idet;
  const T g00 = t_sqrt(A00);
  // G scaled by sqrt(kp) = 1 / sqrt(kappa), as for RayGS
  const T isk = T(1) / t_sqrt(kappa);
  out.G[0] = float(g00 * isk);
  out.G[1] = float(A01 / g00 * isk);
  out.G[2] = 0.f;
  out.G[3] = float(T(1) / (t_sqrt(det) * g00) * isk);
  out.h[0] = 0.f;
  out.h[1] = 0.f;
  out.kp = float(T(1) / kappa);
  out.c2h = float(0.5 * 1.4426950408889634);
  out.lo2o = float(t_log(o) * T(1.4426950408889634));
  out.illcond = false;
  // support ellipse, normalised by kappa; its bounding box half-widths sqrt(kappa Sigma_pi)
  const T ik = T(1) / kappa;
  out.dc0 = 0.f; out.dc1 = 0.f;
  out.M00 = float(A00 * ik); out.M01 = float(A01 * ik); out.M11 = float(A11 * ik);
  out.rho = float(kappa);
  out.det = float(idet * ik * ik);
  const T ucx = jx * mu[0] + T(cam.cx), ucy = jy * mu[1] + T(cam.cy);
  const T hx = t_sqrt(kappa * T(1.001) * P00), hy = t_sqrt(kappa * T(1.001) * P11);
  return tile_rect(false, float(ucx - hx), float(ucx + hx), float(ucy - hy), float(ucy + hy), cam, tile_w,
                   tile_h, out)
             ? kKeep
             : kSkip;
}

// Per-pixel constants of the exact anti-aliasing (Sec. 5, pixel-dependent form), in the
// frame of Sigma's axes (camera-frame columns r_k of R_c, scales s_k), for the pixel offset
// delta = p - u from the projected centre and the ray x = (X, Y, 1):
//   y_k = (r_k . x) / s_k = b_k + g_k . delta                  whitened ray (S^-1 R_c^T x)
//   e_k = (m x y)_k = (s_k / s0 s1 s2) r_k . (mu x (x - mu / mu_z)) = A_k . delta
//                                                              (m = S^-1 R_c^T mu), exact
//                                                              in delta, no cancellation
//   tau = m . y / |y|^2 (Sigma), lambda = sigma^2 cos^3(theta) tau_unit^2 / (fx fy)
//       = (sigma^2 / (fx fy)) tau^2 / |x|,   u_k = 1 + lambda / s_k^2 = 1 + (tau^2 / |x|) w_k
// and with Sigma^_x = Sigma + lambda I (Lagrange's identity in the weighted frame)
//   D_ray(x; mu, Sigma^_x) = sum_k u_k e_k^2 / sum_k y_k^2 prod_{j != k} u_j = Num / Den
//   m(x)^2 = |Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x) = |y|^2 / Den
//   tau^_x > 0  <=>  sum_k m_k y_k prod_{j != k} u_j > 0.
struct MipxOut {
  float A[6], g[6], b[3], m[3], w[3], kappa;
};

// The exact anti-aliasing stage.  The binning support is that of the primitive inflated to
// Sigma + Lambda I, Lambda a bound of lambda(x) over the rays the primitive reaches: there
// D^ <= kappa (the modulation is <= 1), so the Sigma^-closest point lies within
// sqrt(kappa (s_max^2 + lambda)) of mu, tau differs from its depth by at most
// s_max sqrt(kappa (1 + lambda / s_min^2)), hence tau <= (|mu| + 2 sqrt(kappa) s_max) / (1 - k)
// with k = sqrt(kappa) sigma_a (1 + s_max / s_min) < 1 (sigma_a^2 = sigma^2 / (fx fy) bounds
// sigma_x^2), and D^(x) >= D(x; Sigma + Lambda I) for lambda(x) <= Lambda.  When k >= 1/2, or
// when the inflated support reaches the camera, the pair covers its whole view.
template <typename T>
__device__ int mipx_view_stage(const T mu[3], const T Rp[9], const T s[3], T o, const DevCam &cam, float p_min,
                               float mip_sigma2, int tile_w, int tile_h, StageOut &out, MipxOut &X) {
  const bool band = sizeof(T) == 4;
  const T kappa = T(2) * t_log(o / T(p_min));
  if (band && fabs(kappa) <= T(5e-6)) return kUndecided;  // o within rounding of p_min
  if (!(kappa > T(0))) return kSkip;
  T Rc[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rc[3 * i + j] = T(cam.R[3 * i]) * Rp[j] + T(cam.R[3 * i + 1]) * Rp[3 + j] +
                      T(cam.R[3 * i + 2]) * Rp[6 + j];
  T pk[3], mt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pk[k] = Rc[k] * mu[0] + Rc[3 + k] * mu[1] + Rc[6 + k] * mu[2];
    mt[k] = pk[k] / s[k];
  }
  const T c2 = mt[0] * mt[0] + mt[1] * mt[1] + mt[2] * mt[2];
  if (band) {  // Eq. c within rounding of its threshold (see view_stage)
    const T mu1 = fabs(mu[0]) + fabs(mu[1]) + fabs(mu[2]);
    T e_c2 = T(1e-6) * (c2 + kappa) + T(5e-6);
#pragma unroll
    for (int k = 0; k < 3; ++k) e_c2 += T(2) * fabs(mt[k]) * (T(kProjErr32) * mu1 / s[k] + T(1e-6) * fabs(mt[k]));
    if (fabs(c2 - kappa) <= e_c2) return kUndecided;
  }
  if (!(c2 > kappa)) return kSkip;  // Eq. c on the plain primitive
  const T smax = fmax(fmax(s[0], s[1]), s[2]), smin = fmin(fmin(s[0], s[1]), s[2]);
  const T sa2 = T(mip_sigma2) / (T(cam.fx) * T(cam.fy));
  const T kk = t_sqrt(kappa) * t_sqrt(sa2) * (T(1) + smax / smin);
  bool full = true;
  out.illcond = true;
  if (kk < T(0.5)) {
    const T mun = t_sqrt(mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]);
    const T taumax = (mun + T(2) * t_sqrt(kappa) * smax) / (T(1) - kk);
    const T Lam = sa2 * taumax * taumax * T(1.001);
    T sI[3], c2I = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sI[k] = t_sqrt(s[k] * s[k] + Lam);
      c2I += pk[k] * pk[k] / (sI[k] * sI[k]);
    }
    if (c2I > kappa * T(1.001)) {
      full = false;
      if (view_stage<T>(mu, Rp, sI, o, cam, p_min, 0.f, tile_w, tile_h, out, false, false) != kKeep) return kSkip;
      if (!(out.M00 > 0.f)) out.M00 = -2.f;  // not a bounded ellipse: whole rectangle rows
    }
  }
  if (full) {
    out.tx0 = 0; out.ty0 = 0;
    out.tx1 = (cam.W - 1) / tile_w; out.ty1 = (cam.H - 1) / tile_h;
    out.M00 = -2.f; out.M01 = 0.f; out.M11 = 0.f; out.det = 0.f; out.dc0 = 0.f; out.dc1 = 0.f;
  }
  const T ps = s[0] * s[1] * s[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T rx = Rc[k], ry = Rc[3 + k], rz = Rc[6 + k];
    const T ck = s[k] / ps;
    X.A[2 * k] = float(ck * (ry * mu[2] - rz * mu[1]) * T(cam.ifx));
    X.A[2 * k + 1] = float(ck * (rz * mu[0] - rx * mu[2]) * T(cam.ify));
    X.g[2 * k] = float(rx * T(cam.ifx) / s[k]);
    X.g[2 * k + 1] = float(ry * T(cam.ify) / s[k]);
    X.b[k] = float(mt[k] / mu[2]);
    X.m[k] = float(mt[k]);
    X.w[k] = float(sa2 / (s[k] * s[k]));
  }
  X.kappa = float(kappa);
  out.lo2o = float(t_log(o) * T(1.4426950408889634));
  return kKeep;
}

__device__ __forceinline__ void write_record_mipx(const PrepParams &P, int64_t idx, const DevCam &cam,
                                                  const df muc[3], const StageOut &so, const MipxOut &X,
                                                  const float rgb[3], float z, bool write_key) {
  df Xc = df_div(muc[0], muc[2]);
  df Yc = df_div(muc[1], muc[2]);
  df u = df_add(df_mul_f(Xc, cam.fx), df{cam.cx, 0.f});
  df v = df_add(df_mul_f(Yc, cam.fy), df{cam.cy, 0.f});
  Rec r, q;
  r.a = make_float4(u.hi, v.hi, u.lo, v.lo);
  r.b = make_float4(X.A[0], X.A[1], X.A[2], X.A[3]);
  r.c = make_float4(X.A[4], X.A[5], X.g[0], X.g[1]);
  r.d = make_float4(X.g[2], X.g[3], X.g[4], X.g[5]);
  q.a = make_float4(X.b[0], X.b[1], X.b[2], so.lo2o);
  q.b = make_float4(X.m[0], X.m[1], X.m[2], X.kappa);
  q.c = make_float4(X.w[0], X.w[1], X.w[2], 0.f);
  q.d = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
  P.rec[idx] = r;
  P.recx[idx] = q;
  Ell e;
  e.r0 = uint32_t(so.tx0) | (uint32_t(so.ty0) << 16);
  e.r1 = uint32_t(so.tx1) | (uint32_t(so.ty1) << 16);
  e.cx = u.hi + so.dc0;
  e.cy = v.hi + so.dc1;
  e.a = so.M00; e.b = so.M01; e.d = so.M11; e.det = so.det;
  P.ell[idx] = e;
  // the rectangle also in its own compact array (the backward gathers it by pair), and its
  // tile-row count in a byte that the first depth-sort pass reads in pair order
  P.rect[idx] = make_uint2(e.r0, e.r1);
  P.trow_cnt[idx] = uint8_t(min(so.ty1 - so.ty0 + 1, 255));
  if (write_key) P.depth_key[idx] = __float_as_uint(z);
}

__device__ __forceinline__ void write_record(const PrepParams &P, int64_t idx, const DevCam &cam,
                                             const df muc[3], const StageOut &so, const float rgb[3],
                                             float z, bool write_key) {
  df X = df_div(muc[0], muc[2]);
  df Yv = df_div(muc[1], muc[2]);
  df u = df_add(df_mul_f(X, cam.fx), df{cam.cx, 0.f});
  df v = df_add(df_mul_f(Yv, cam.fy), df{cam.cy, 0.f});
  Rec r;
  r.a = make_float4(u.hi, v.hi, u.lo, v.lo);
  r.b = make_float4(so.G[0], so.G[1], so.G[2], so.G[3]);
  r.c = make_float4(so.h[0], so.h[1], so.kp, so.c2h);
  r.d = make_float4(so.lo2o, rgb[0], rgb[1], rgb[2]);
  P.rec[idx] = r;
  Ell e;
  e.r0 = uint32_t(so.tx0) | (uint32_t(so.ty0) << 16);
  e.r1 = uint32_t(so.tx1) | (uint32_t(so.ty1) << 16);
  e.cx = u.hi + so.dc0;
  e.cy = v.hi + so.dc1;
  e.a = so.M00; e.b = so.M01; e.d = so.M11; e.det = so.det;
  P.ell[idx] = e;
  // the rectangle also in its own compact array (the backward gathers it by pair), and its
  // tile-row count in a byte that the first depth-sort pass reads in pair order
  P.rect[idx] = make_uint2(e.r0, e.r1);
  P.trow_cnt[idx] = uint8_t(min(so.ty1 - so.ty0 + 1, 255));
  if (write_key) P.depth_key[idx] = __float_as_uint(z);
}

// Two passes per chunk of kViewChunk views, so that the expensive stage runs on dense
// work: a cheap conservative cull of every (primitive, view) pair (near plane, and the
// frustum test with the largest support radius the pair can have), compacting the
// survivors per warp into a shared list in primitive order; then one thread per listed
// pair for the full stage, whose own tests decide.
constexpr int kViewChunk = 16;

// Stage variants, one per plan (compiled apart so that the RayGS stage keeps its registers):
// RayGS with or without Eq. mip per view, the GS divergence, and RayGS with the exact
// pixel-dependent anti-aliasing in every view.
enum StageMode { kStageRay = 0, kStageGS = 1, kStageExact = 2 };

template <int MODE, typename T>
__device__ __forceinline__ int stage_for(const T mu[3], const T Rp[9], const T s[3], T o, const DevCam &cam,
                                          const PrepParams &P, StageOut &so, MipxOut &mx,
                                          const float *pre = nullptr) {
  if (MODE == kStageGS) return gs_view_stage<T>(mu, Rp, s, o, cam, P.p_min, P.tile_w, P.tile_h, so);
  if (MODE == kStageExact)
    return mipx_view_stage<T>(mu, Rp, s, o, cam, P.p_min, P.mip_sigma2, P.tile_w, P.tile_h, so, mx);
  return view_stage<T>(mu, Rp, s, o, cam, P.p_min, P.mip_sigma2, P.tile_w, P.tile_h, so, true, true, pre);
}

template <int DEG, int MODE>
__global__ void __launch_bounds__(kPrepThreads) preprocess_kernel(PrepParams P) {
  constexpr int K3 = 3 * (DEG + 1) * (DEG + 1);
  // padded SH row: whole 16-byte slots, an odd number of them
  constexpr int K4 = (K3 + 3) / 4;
  constexpr int SHP = 4 * (K4 % 2 == 1 ? K4 : K4 + 1);
  __shared__ float s_means[kPrepThreads * 3];
  // log-scales, quaternions and logits are read once, for the per-primitive constants;
  // their space then holds the list of (primitive, view) pairs
  static_assert(kPrepThreads * kViewChunk * sizeof(uint16_t) <= kPrepThreads * 8 * sizeof(float), "list");
  __shared__ __align__(16) float s_scratch[kPrepThreads * 8];
  float *s_ls = s_scratch;
  float *s_q = s_scratch + 3 * kPrepThreads;
  float *s_logit = s_scratch + 7 * kPrepThreads;
  uint16_t *s_list = reinterpret_cast<uint16_t *>(s_scratch);
  __shared__ __align__(16) float s_sh[kPrepThreads * SHP];
  __shared__ float s_R[kPrepThreads * 9];   // rotation of each primitive
  __shared__ float s_s[kPrepThreads * 3];   // scales
  __shared__ float s_o[kPrepThreads];       // prior opacity
  __shared__ float2 s_pre[kPrepThreads];    // kappa and log2 of the prior opacity
  __shared__ float s_rad[kPrepThreads];     // sqrt(kappa) s_max (0: cull in every view)
  __shared__ float s_s2max[kPrepThreads];   // s_max^2
  __shared__ uint8_t s_deg[kPrepThreads];
  __shared__ int s_n;
  extern __shared__ DevCam s_cams[];

  const int g0 = blockIdx.x * kPrepThreads;
  const int nb = min(kPrepThreads, P.n - g0);
  for (int i = threadIdx.x; i < P.n_views * (int)(sizeof(DevCam) / 4); i += blockDim.x)
    reinterpret_cast<float *>(s_cams)[i] = reinterpret_cast<const float *>(P.cams)[i];
  stage_attr(s_means, P.means, int64_t(g0) * 3, nb * 3, RAYGS_F32, 3, 0);
  stage_attr(s_ls, P.log_scales, int64_t(g0) * 3, nb * 3, P.scale_dtype, 3, 0);
  stage_attr(s_q, P.quats, int64_t(g0) * 4, nb * 4, RAYGS_F32, 4, 0);
  stage_attr(s_logit, P.logits, g0, nb, P.opacity_dtype, 1, 0);
  // FP32 SH rows of whole 16-byte slots are copied asynchronously: the copies land while
  // the per-primitive constants and the cull pass run, and are waited for before the full
  // stage, the first reader (the other forms are converted on the way in)
  const bool sh_async = P.sh_dtype == RAYGS_F32 && K3 % 4 == 0 && (reinterpret_cast<uintptr_t>(P.sh) & 15) == 0;
  if (sh_async) {
    const char *src = reinterpret_cast<const char *>(P.sh) + int64_t(g0) * K3 * 4;
    for (int i = threadIdx.x; i < nb * (K3 / 4); i += blockDim.x) {
      const int row = i / (K3 / 4), col = i - row * (K3 / 4);
      const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(&s_sh[row * SHP + 4 * col]));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 16 * int64_t(i)) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  } else {
    stage_attr(s_sh, P.sh, int64_t(g0) * K3, nb * K3, P.sh_dtype, K3, SHP - K3);
  }
  __syncthreads();

  // per-primitive constants
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int g = g0 + t;
  if (t < nb) {
    const float mx = s_means[3 * t], my = s_means[3 * t + 1], mz = s_means[3 * t + 2];
    const float l0 = s_ls[3 * t], l1 = s_ls[3 * t + 1], l2 = s_ls[3 * t + 2];
    const float qw = s_q[4 * t], qx = s_q[4 * t + 1], qy = s_q[4 * t + 2], qz = s_q[4 * t + 3];
    const float logit = s_logit[t];
    const bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(l0) && isfinite(l1) &&
                        isfinite(l2) && isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) &&
                        isfinite(logit) && (qw * qw + qx * qx + qy * qy + qz * qz > 0.f);
    bool degenerate = false;
    if (finite && P.fp64_degenerate) {
      const float lmax = fmaxf(fmaxf(l0, l1), l2), lmin = fminf(fminf(l0, l1), l2);
      degenerate = (lmax - lmin) > logf(P.degenerate_ratio);
    }
    s_deg[t] = degenerate ? 1 : 0;
    s_rad[t] = 0.f;
    if (!finite) {
      atomicAdd(&P.counters->n_nonfinite, 1ull);
    } else {
      quat_rot<float>(qw, qx, qy, qz, &s_R[9 * t]);
      const float s0 = expf(l0), s1 = expf(l1), s2 = expf(l2);
      s_s[3 * t] = s0; s_s[3 * t + 1] = s1; s_s[3 * t + 2] = s2;
      const float o = 1.f / (1.f + expf(-logit));
      s_o[t] = o;
      // kappa of the unmodulated opacity bounds every view's (the MIP factor is <= 1)
      const float kappa0 = 2.f * logf(o / P.p_min);
      s_pre[t] = make_float2(kappa0, logf(o) * 1.4426950408889634f);
      const float smax = fmaxf(fmaxf(s0, s1), s2);
      s_s2max[t] = smax * smax;
      // < 0: culled everywhere; an opacity within rounding of p_min goes on to the full
      // stage, which leaves the decision to the FP64 stage
      s_rad[t] = kappa0 > 0.f ? sqrtf(kappa0) : (kappa0 >= -1e-5f ? 4e-3f : -1.f);
    }
  }

  for (int v0 = 0; v0 < P.n_views; v0 += kViewChunk) {
    const int v1 = min(P.n_views, v0 + kViewChunk);
    if (t == 0) s_n = 0;
    __syncthreads();
    // pass 1: cheap cull, view by view, warp-compacted in primitive order
    for (int v = v0; v < v1; ++v) {
      bool keep = false;
      if (t < nb) {
        const float sk = s_rad[t];
        const int64_t idx = int64_t(v) * P.n + g;
        float z = 0.f;
        if (sk > 0.f) {
          const DevCam &cam = s_cams[v];
          const float mx = s_means[3 * t], my = s_means[3 * t + 1], mz = s_means[3 * t + 2];
          z = depth_f32(cam, mx, my, mz);
          if (z > cam.near_z) {
            // a float32 camera-frame mean: the cull radius below carries its rounding
            // (a few ulp of |R m| + |t|) with a wide margin
            float mu[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
              mu[r] = fmaf(cam.R[3 * r], mx, fmaf(cam.R[3 * r + 1], my, fmaf(cam.R[3 * r + 2], mz, cam.t[r])));
            const float mag = fabsf(mx) + fabsf(my) + fabsf(mz) + fabsf(cam.t[0]) + fabsf(cam.t[1]) + fabsf(cam.t[2]);
            float s2 = s_s2max[t];
            if (cam.mip)
              s2 += P.mip_sigma2 * (mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]) / (cam.fx * cam.fy);
            const float rad = sk * sqrtf(s2) * 1.01f + 1e-5f * (fabsf(mu[0]) + fabsf(mu[1]) + fabsf(mu[2])) +
                              2e-6f * mag + 1e-5f;
            // the GS support is the linearised projection, not bounded by the sphere's
            // cone: its exact screen box decides in the full stage
            keep = MODE != kStageRay || !outside_frustum<float>(mu, rad, cam);
          }
        }
        // every key of the warp's 32 consecutive pairs at once (full sectors): the depth of
        // a kept pair (the full stage writes kCulled over it if it culls the pair), the
        // marker of a culled one
        P.depth_key[idx] = keep ? __float_as_uint(z) : kCulled;
      }
      const uint32_t ball = __ballot_sync(0xffffffffu, keep);
      int base = 0;
      if (lane == 0 && ball) base = atomicAdd(&s_n, __popc(ball));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) s_list[base + __popc(ball & ((1u << lane) - 1u))] = uint16_t(t | ((v - v0) << 8));
    }
    (void)warp;
    if (sh_async) asm volatile("cp.async.wait_all;\n" ::: "memory");  // this thread's SH copies
    __syncthreads();
    // pass 2: the full stage on the listed pairs
    const int n_items = s_n;
    for (int j = t; j < n_items; j += kPrepThreads) {
      const int tt = s_list[j] & 0xFF, v = v0 + (s_list[j] >> 8);
      const int gg = g0 + tt;
      const int64_t idx = int64_t(v) * P.n + gg;
      const DevCam &cam = s_cams[v];
      const float mx = s_means[3 * tt], my = s_means[3 * tt + 1], mz = s_means[3 * tt + 2];
      const float z = depth_f32(cam, mx, my, mz);
      df muc[3];
      mean_cam_df(cam, mx, my, mz, muc);
      const float mu[3] = {muc[0].hi, muc[1].hi, muc[2].hi};
      const float sv[3] = {s_s[3 * tt], s_s[3 * tt + 1], s_s[3 * tt + 2]};
      float Rp[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rp[k] = s_R[9 * tt + k];
      StageOut so;
      MipxOut mxo;
      const float pre[2] = {s_pre[tt].x, s_pre[tt].y};
      const int res = stage_for<MODE, float>(mu, Rp, sv, s_o[tt], cam, P, so, mxo, pre);
      if (res != kKeep) {
        P.depth_key[idx] = kCulled;
        if (res == kUndecided) P.deg_list[atomicAdd(P.deg_count, 1u)] = uint32_t(idx);
        continue;
      }
      const float dx = mx - cam.C[0], dy = my - cam.C[1], dz = mz - cam.C[2];
      const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
      float rgb[3];
      sh_colour<DEG>(s_sh + tt * SHP, dx * dn, dy * dn, dz * dn, rgb);
      // (the cull pass wrote this pair's key)
      if (MODE == kStageExact) write_record_mipx(P, idx, cam, muc, so, mxo, rgb, z, false);
      else write_record(P, idx, cam, muc, so, rgb, z, false);
      if (s_deg[tt] && (P.fp64_degenerate == 2 || so.illcond)) {
        const uint32_t slot = atomicAdd(P.deg_count, 1u);
        P.deg_list[slot] = uint32_t(idx);
      }
    }
    __syncthreads();
  }
  if (sh_async) asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy outlives the block
}

// FP64 vertex stage for the (view, primitive) pairs listed by preprocess_kernel.  The
// float32 record, rectangle and key of each pair are overwritten.  Grid-stride over the
// device-side list.
template <int DEG, int MODE>
__global__ void __launch_bounds__(128) preprocess_fp64_kernel(PrepParams P) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const uint32_t count = *P.deg_count;
  for (uint32_t li = blockIdx.x * blockDim.x + threadIdx.x; li < count; li += gridDim.x * blockDim.x) {
    const int64_t idx = P.deg_list[li];
    const int v = int(idx / P.n);
    const int g = int(idx - int64_t(v) * P.n);
    const float mx = P.means[3 * int64_t(g)], my = P.means[3 * int64_t(g) + 1], mz = P.means[3 * int64_t(g) + 2];
    double ls[3], qd[4];
    for (int k = 0; k < 3; ++k) ls[k] = load_attr(P.log_scales, 3 * int64_t(g) + k, P.scale_dtype);
    for (int k = 0; k < 4; ++k) qd[k] = P.quats[4 * int64_t(g) + k];
    const double logit = load_attr(P.logits, g, P.opacity_dtype);
    double Rp[9];
    quat_rot<double>(qd[0], qd[1], qd[2], qd[3], Rp);
    const double s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
    const double o = 1.0 / (1.0 + exp(-logit));
    const DevCam &cam = P.cams[v];
    const float z = depth_f32(cam, mx, my, mz);
    df muc[3];
    mean_cam_df(cam, mx, my, mz, muc);
    const double mu[3] = {double(muc[0].hi) + double(muc[0].lo), double(muc[1].hi) + double(muc[1].lo),
                          double(muc[2].hi) + double(muc[2].lo)};
    StageOut so;
    MipxOut mxo;
    if (stage_for<MODE, double>(mu, Rp, s, o, cam, P, so, mxo) != kKeep) {
      P.depth_key[idx] = kCulled;
      continue;
    }
    float coef[3 * K];
    for (int k = 0; k < 3 * K; ++k) coef[k] = load_attr(P.sh, int64_t(g) * 3 * K + k, P.sh_dtype);
    float dx = mx - cam.C[0], dy = my - cam.C[1], dz = mz - cam.C[2];
    float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    float rgb[3];
    sh_colour<DEG>(coef, dx * dn, dy * dn, dz * dn, rgb);
    if (MODE == kStageExact) write_record_mipx(P, idx, cam, muc, so, mxo, rgb, z, true);
    else write_record(P, idx, cam, muc, so, rgb, z, true);
  }
}

// ------------------------------------------------------------------------ launcher
cudaError_t launch_preprocess(const PrepParams &P, int num_sms, cudaStream_t st) {
  if (P.n == 0) return cudaSuccess;
  int blocks = (P.n + kPrepThreads - 1) / kPrepThreads;
  size_t dyn = sizeof(DevCam) * P.n_views;
  cudaMemsetAsync(P.deg_count, 0, sizeof(uint32_t), st);
  const int mode = P.divergence == 1 ? kStageGS : P.recx ? kStageExact : kStageRay;
#define RAYGS_PREP(D, M) preprocess_kernel<D, M><<<blocks, kPrepThreads, dyn, st>>>(P)
#define RAYGS_PREP_MODES(D)                 \
  if (mode == kStageGS) RAYGS_PREP(D, 1);         \
  else if (mode == kStageExact) RAYGS_PREP(D, 2); \
  else RAYGS_PREP(D, 0);
  switch (P.sh_degree) {
    case 0: RAYGS_PREP_MODES(0) break;
    case 1: RAYGS_PREP_MODES(1) break;
    case 2: RAYGS_PREP_MODES(2) break;
    default: RAYGS_PREP_MODES(3) break;
  }
#undef RAYGS_PREP_MODES
#undef RAYGS_PREP
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {  // the listed pairs: near-degenerate ones and undecided skip decisions
    int gb = num_sms * 4;
#define RAYGS_FP64(D, M) preprocess_fp64_kernel<D, M><<<gb, 128, 0, st>>>(P)
#define RAYGS_FP64_MODES(D)                 \
  if (mode == kStageGS) RAYGS_FP64(D, 1);         \
  else if (mode == kStageExact) RAYGS_FP64(D, 2); \
  else RAYGS_FP64(D, 0);
    switch (P.sh_degree) {
      case 0: RAYGS_FP64_MODES(0) break;
      case 1: RAYGS_FP64_MODES(1) break;
      case 2: RAYGS_FP64_MODES(2) break;
      default: RAYGS_FP64_MODES(3) break;
    }
#undef RAYGS_FP64_MODES
#undef RAYGS_FP64
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace raygs
