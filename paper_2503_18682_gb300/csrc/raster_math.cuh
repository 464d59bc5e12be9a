// Per-pixel evaluation shared by the forward rasteriser and its backward replay, so that
// both take bit-identical support decisions and opacities.
#pragma once

#include "raygs_internal.cuh"

namespace raygs {

// Staged record (shared-memory layout of one 64-byte Rec, tile-relative):
//   A = (ox, oy, G00, G01)   ox, oy: tile origin pixel centre minus projected centre
//   B = (G10, G11, h0, h1)
//   C = (kp, c2h, lo2o, c)   c = sqrt(mu^T Sigma^-1 mu) (backward only)
//   D = (r, g, b, 0)
__device__ __forceinline__ void stage_record(const Rec &r, float ox_tile, float oy_tile, float4 &A, float4 &B,
                                             float4 &C, float4 &D) {
  const df ox = two_sum(ox_tile, -r.a.x);
  const df oy = two_sum(oy_tile, -r.a.y);
  A = make_float4(__fadd_rn(ox.hi, __fsub_rn(ox.lo, r.a.z)), __fadd_rn(oy.hi, __fsub_rn(oy.lo, r.a.w)), r.b.x,
                  r.b.y);
  B = make_float4(r.b.z, r.b.w, r.c.x, r.c.y);
  C = make_float4(r.c.z, r.c.w, r.d.x, sqrtf(r.c.w * (2.0f / kLog2e)));
  // second difference of f = kp q - r along a pixel row (constant: f is quadratic)
  const float a2 = 2.f * fmaf(r.c.z, fmaf(r.b.x, r.b.x, r.b.z * r.b.z), -r.c.x * r.c.x);
  D = make_float4(r.d.y, r.d.z, r.d.w, a2);
}

// Conservative row filter: f = kp q - r (<= 0 exactly on the support, with y2 > 0) at PX
// consecutive pixels by forward differences, f_{k+1} = f_k + d_k, d_{k+1} = d_k + a2.
// Returns false only when every pixel is outside the support by more than the rounding
// error of the recurrence; the exact per-pixel test (eval_pixels) decides otherwise.
template <int PX>
__device__ __forceinline__ bool row_may_hit(const float4 &A, const float4 &B, float kp, float a2, float fl_x,
                                            float fl_y) {
  const float dy = A.y + fl_y;
  const float dx = A.x + fl_x;
  const float y0 = fmaf(A.z, dx, A.w * dy);
  const float y1 = fmaf(B.x, dx, B.y * dy);
  const float y2 = fmaf(B.z, dx, fmaf(B.w, dy, 1.f));
  float f = fmaf(kp, fmaf(y0, y0, y1 * y1), -y2 * y2);
  float d = fmaf(2.f, fmaf(kp, fmaf(y0, A.z, y1 * B.x), -y2 * B.z), 0.5f * a2);
  const float margin = 1e-3f + 1e-5f * (fabsf(f) + float(PX) * fabsf(d) + float(PX * PX) * fabsf(a2));
  float m = f;
#pragma unroll
  for (int k = 1; k < PX; ++k) {
    f += d;
    d += a2;
    m = fminf(m, f);
  }
  return !(m > margin);
}

// Support test of PX consecutive pixels (columns fl_x .. fl_x + PX - 1 of row fl_y,
// relative to the tile origin).  Returns the hit mask; q, r (and y) per pixel.
template <int PX>
__device__ __forceinline__ uint32_t eval_pixels(const float4 &A, const float4 &B, float kp, float fl_x, float fl_y,
                                                float q[PX], float r[PX], float y0s[PX], float y1s[PX],
                                                float y2s[PX]) {
  const float dy = A.y + fl_y;
  const float dx = A.x + fl_x;
  float y0 = fmaf(A.z, dx, A.w * dy);
  float y1 = fmaf(B.x, dx, B.y * dy);
  float y2 = fmaf(B.z, dx, fmaf(B.w, dy, 1.f));
  uint32_t hit = 0;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    if (k) { y0 += A.z; y1 += B.x; y2 += B.z; }
    q[k] = fmaf(y0, y0, y1 * y1);
    r[k] = y2 * y2;
    y0s[k] = y0; y1s[k] = y1; y2s[k] = y2;
    if (y2 > 0.f && fmaf(kp, q[k], -r[k]) <= 0.f) hit |= 1u << k;
  }
  return hit;
}

// Rendered opacity before the clamp (fragment formula + Eq. rend_opacity).
__device__ __forceinline__ float pixel_opacity(const float4 &C, float q, float r) {
  const float E = C.y * __fdividef(q, q + r);
  return ex2_approx(C.z - E);
}

}  // namespace raygs
