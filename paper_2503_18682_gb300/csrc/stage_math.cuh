// Per-(primitive, view) math shared by the vertex stage (preprocess.cu) and the parameter
// gradients (backward.cu), so that both derive bit-identical quantities.
#pragma once

#include "raygs_internal.cuh"

namespace raygs {

__device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_log(double x) { return log(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }

// Rotation of a quaternion (w, x, y, z) after normalisation, closed-form matrix.
template <typename T>
__device__ __forceinline__ void quat_rot(T w, T x, T y, T z, T R[9]) {
  T inv = T(1) / t_sqrt(w * w + x * x + y * y + z * z);
  w *= inv; x *= inv; y *= inv; z *= inv;
  R[0] = T(1) - T(2) * (y * y + z * z); R[1] = T(2) * (x * y - w * z); R[2] = T(2) * (x * z + w * y);
  R[3] = T(2) * (x * y + w * z); R[4] = T(1) - T(2) * (x * x + z * z); R[5] = T(2) * (y * z - w * x);
  R[6] = T(2) * (x * z - w * y); R[7] = T(2) * (y * z + w * x); R[8] = T(1) - T(2) * (x * x + y * y);
}

// Rows k0, k1 of K01: a Sigma-orthonormal basis of the complement of mu (K01 Sigma
// K01^T = I, K01 mu = 0), built stably from an orthonormal basis E of the plane orthogonal
// to mu and the Cholesky factor L of E^T Sigma E (K01 = L^-1 E^T).  Sigma = Rc S^2 Rc^T
// with Rc row-major and s the scales.  Returns false when the Cholesky lost more than
// three digits (the primitive is seen nearly edge-on).
template <typename T>
__device__ __forceinline__ bool plane_whitening(const T mu[3], const T Rc[9], const T s[3], T k0[3], T k1[3]) {
  T nn = t_sqrt(mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]);
  T n0 = mu[0] / nn, n1 = mu[1] / nn, n2 = mu[2] / nn;
  T sg = n2 >= T(0) ? T(1) : T(-1);
  T ba = T(-1) / (sg + n2);
  T bb = n0 * n1 * ba;
  T e1[3] = {T(1) + sg * n0 * n0 * ba, sg * bb, -sg * n0};
  T e2[3] = {bb, sg + n1 * n1 * ba, -n1};
  T M0[3], M1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    M0[k] = (e1[0] * Rc[k] + e1[1] * Rc[3 + k] + e1[2] * Rc[6 + k]) * s[k];
    M1[k] = (e2[0] * Rc[k] + e2[1] * Rc[3 + k] + e2[2] * Rc[6 + k]) * s[k];
  }
  T a00 = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2];
  T a01 = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
  T a11 = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2];
  T l00 = t_sqrt(a00);
  T l10 = a01 / l00;
  T schur = a11 - l10 * l10;
  const bool ok = schur > T(1e-3) * a11;
  T l11 = t_sqrt(fmax(schur, a11 * T(1e-30)));
  T f10 = l10 / l00;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    k0[i] = e1[i] / l00;
    k1[i] = (e2[i] - f10 * e1[i]) / l11;
  }
  return ok;
}

// Cooperative copy of `count` consecutive attributes starting at element `first` of `src`
// into float32 shared memory, 16-byte vector loads where aligned.  dst element e goes to
// dst[(e / row) * (row + pad) + e % row] (pad breaks shared-memory bank conflicts).
__device__ __forceinline__ void stage_attr(float *dst, const void *src, int64_t first, int count, int dtype,
                           int row, int pad) {
  const int tid = threadIdx.x, nt = blockDim.x;
  auto put = [&](int e, float v) { dst[(e / row) * (row + pad) + e % row] = v; };
  if (dtype == RAYGS_F32) {
    const float *s = reinterpret_cast<const float *>(src) + first;
    int nvec = ((reinterpret_cast<uintptr_t>(s) & 15) == 0) ? count / 4 : 0;
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    for (int i = tid; i < nvec; i += nt) {
      float4 v = __ldg(s4 + i);
      put(4 * i, v.x); put(4 * i + 1, v.y); put(4 * i + 2, v.z); put(4 * i + 3, v.w);
    }
    for (int e = 4 * nvec + tid; e < count; e += nt) put(e, __ldg(s + e));
  } else {
    const uint16_t *s = reinterpret_cast<const uint16_t *>(src) + first;
    int nvec = ((reinterpret_cast<uintptr_t>(s) & 15) == 0) ? count / 8 : 0;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(s);
    auto cvt = [&](uint16_t b) -> float {
      if (dtype == RAYGS_F16) return __half2float(__ushort_as_half(b));
      return __uint_as_float(uint32_t(b) << 16);
    };
    for (int i = tid; i < nvec; i += nt) {
      uint4 v = __ldg(s4 + i);
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        put(8 * i + 2 * j, cvt(uint16_t(w[j] & 0xFFFF)));
        put(8 * i + 2 * j + 1, cvt(uint16_t(w[j] >> 16)));
      }
    }
    for (int e = 8 * nvec + tid; e < count; e += nt) put(e, cvt(__ldg(s + e)));
  }
}

// Camera-frame mean in double-float: R mu + t with error-free products and sums.
__device__ __forceinline__ void mean_cam_df(const DevCam &cam, float mx, float my, float mz, df out[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    df acc = {cam.t[r], 0.f};
    acc = df_add(acc, two_prod(cam.R[3 * r], mx));
    acc = df_add(acc, two_prod(cam.R[3 * r + 1], my));
    acc = df_add(acc, two_prod(cam.R[3 * r + 2], mz));
    out[r] = acc;
  }
}

// Depth key: the fused chain fmaf(R20, x, fmaf(R21, y, fmaf(R22, z, t2))) in float32.
__device__ __forceinline__ float depth_f32(const DevCam &cam, float mx, float my, float mz) {
  return __fmaf_rn(cam.R[6], mx, __fmaf_rn(cam.R[7], my, __fmaf_rn(cam.R[8], mz, cam.t[2])));
}

// Real spherical harmonics (no Condon-Shortley phase) of unit direction (x, y, z) applied
// to coefficients coef[k*3 + ch] (stride-1 floats); the first coefficient is the colour.
template <int DEG>
__device__ __forceinline__ void sh_colour(const float *coef, float x, float y, float z, float rgb[3]) {
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = coef[ch];
  if (DEG >= 1) {
    const float c1 = 0.4886025119029199f;  // sqrt(3/(4 pi))
    float Y[3] = {c1 * y, c1 * z, c1 * x};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(Y[k], coef[3 * (1 + k) + ch], rgb[ch]);
  }
  if (DEG >= 2) {
    const float c2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
    const float c2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
    const float c2c = 0.5462742152960396f;   // sqrt(15/(16 pi))
    float Y[5] = {c2a * x * y, c2a * y * z, c2b * (3.f * z * z - 1.f), c2a * x * z, c2c * (x * x - y * y)};
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(Y[k], coef[3 * (4 + k) + ch], rgb[ch]);
  }
  if (DEG >= 3) {
    const float c3a = 0.5900435899266435f;  // sqrt(35/(32 pi))
    const float c3b = 2.890611442640554f;   // sqrt(105/(4 pi))
    const float c3c = 0.4570457994644658f;  // sqrt(21/(32 pi))
    const float c3d = 0.3731763325901154f;  // sqrt(7/(16 pi))
    const float c3e = 1.445305721320277f;   // sqrt(105/(16 pi))
    float z2 = z * z;
    float Y[7] = {c3a * y * (3.f * x * x - y * y), c3b * x * y * z, c3c * y * (5.f * z2 - 1.f),
                  c3d * z * (5.f * z2 - 3.f), c3c * x * (5.f * z2 - 1.f), c3e * z * (x * x - y * y),
                  c3a * x * (x * x - 3.f * y * y)};
#pragma unroll
    for (int k = 0; k < 7; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(Y[k], coef[3 * (9 + k) + ch], rgb[ch]);
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(rgb[ch], 0.f);
}

// One real SH basis term k (0 .. 15; term 0 is the colour's constant 1) and its gradient
// with respect to the direction components (x, y, z), the same functions as sh_colour.
// Called with a compile-time k inside unrolled loops, so that the switch folds away.
__device__ __forceinline__ void sh_term(int k, float x, float y, float z, float &Y, float &gx, float &gy, float &gz) {
  const float c1 = 0.4886025119029199f;
  const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
  const float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
  const float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
  gx = gy = gz = 0.f;
  switch (k) {
    case 0: Y = 1.f; break;
    case 1: Y = c1 * y; gy = c1; break;
    case 2: Y = c1 * z; gz = c1; break;
    case 3: Y = c1 * x; gx = c1; break;
    case 4: Y = c2a * x * y; gx = c2a * y; gy = c2a * x; break;
    case 5: Y = c2a * y * z; gy = c2a * z; gz = c2a * y; break;
    case 6: Y = c2b * (3.f * z * z - 1.f); gz = 6.f * c2b * z; break;
    case 7: Y = c2a * x * z; gx = c2a * z; gz = c2a * x; break;
    case 8: Y = c2c * (x * x - y * y); gx = 2.f * c2c * x; gy = -2.f * c2c * y; break;
    case 9: Y = c3a * y * (3.f * x * x - y * y); gx = 6.f * c3a * x * y; gy = 3.f * c3a * (x * x - y * y); break;
    case 10: Y = c3b * x * y * z; gx = c3b * y * z; gy = c3b * x * z; gz = c3b * x * y; break;
    case 11: Y = c3c * y * (5.f * z * z - 1.f); gy = c3c * (5.f * z * z - 1.f); gz = 10.f * c3c * y * z; break;
    case 12: Y = c3d * z * (5.f * z * z - 3.f); gz = c3d * (15.f * z * z - 3.f); break;
    case 13: Y = c3c * x * (5.f * z * z - 1.f); gx = c3c * (5.f * z * z - 1.f); gz = 10.f * c3c * x * z; break;
    case 14:
      Y = c3e * z * (x * x - y * y);
      gx = 2.f * c3e * x * z; gy = -2.f * c3e * y * z; gz = c3e * (x * x - y * y);
      break;
    default: Y = c3a * x * (x * x - 3.f * y * y); gx = 3.f * c3a * (x * x - y * y); gy = -6.f * c3a * x * y; break;
  }
}

// Real SH basis values Y[k] (k = 1 .. (DEG+1)^2 - 1; Y[0] is the colour's constant 1) and
// their gradients dY[k] with respect to the (unnormalised) direction components.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float Y[16], float dY[16][3]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) { Y[k] = 0.f; dY[k][0] = dY[k][1] = dY[k][2] = 0.f; }
  Y[0] = 1.f;
  if (DEG >= 1) {
    const float c1 = 0.4886025119029199f;
    Y[1] = c1 * y; dY[1][1] = c1;
    Y[2] = c1 * z; dY[2][2] = c1;
    Y[3] = c1 * x; dY[3][0] = c1;
  }
  if (DEG >= 2) {
    const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    Y[4] = c2a * x * y; dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    Y[5] = c2a * y * z; dY[5][1] = c2a * z; dY[5][2] = c2a * y;
    Y[6] = c2b * (3.f * z * z - 1.f); dY[6][2] = 6.f * c2b * z;
    Y[7] = c2a * x * z; dY[7][0] = c2a * z; dY[7][2] = c2a * x;
    Y[8] = c2c * (x * x - y * y); dY[8][0] = 2.f * c2c * x; dY[8][1] = -2.f * c2c * y;
  }
  if (DEG >= 3) {
    const float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    const float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
    const float z2 = z * z;
    Y[9] = c3a * y * (3.f * x * x - y * y); dY[9][0] = 6.f * c3a * x * y; dY[9][1] = 3.f * c3a * (x * x - y * y);
    Y[10] = c3b * x * y * z; dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    Y[11] = c3c * y * (5.f * z2 - 1.f); dY[11][1] = c3c * (5.f * z2 - 1.f); dY[11][2] = 10.f * c3c * y * z;
    Y[12] = c3d * z * (5.f * z2 - 3.f); dY[12][2] = c3d * (15.f * z2 - 3.f);
    Y[13] = c3c * x * (5.f * z2 - 1.f); dY[13][0] = c3c * (5.f * z2 - 1.f); dY[13][2] = 10.f * c3c * x * z;
    Y[14] = c3e * z * (x * x - y * y); dY[14][0] = 2.f * c3e * x * z; dY[14][1] = -2.f * c3e * y * z;
    dY[14][2] = c3e * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.f * y * y); dY[15][0] = 3.f * c3a * (x * x - y * y); dY[15][1] = -6.f * c3a * x * y;
  }
}

}  // namespace raygs
