// Per-pixel evaluation shared by the forward rasteriser and its backward replay, so that
// both take bit-identical support decisions and opacities.
#pragma once

#include "raygs_internal.cuh"

namespace raygs {

// Asynchronous global -> shared copy of one 64-byte record (four 16-byte cp.async
// transfers, bypassing L1), completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ void cp_async_rec(Rec *dst, const Rec *src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
  for (int c = 0; c < 4; ++c)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16 * c), "l"(g + 16 * c) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Staged record (shared-memory layout of one 64-byte Rec, tile-relative):
//   A = (ox, oy, G00, G01)   ox, oy: tile origin pixel centre minus projected centre
//   B = (G10, G11, h0, h1)   (G carries sqrt(kp): q' = |G delta|^2 = kp q)
//   C = (kp, c2h', lo2o, sc) c2h' = c2h for D_ray, c2h / kp for D_gs (DIV = 1);
//                            sc = G00^2 + G10^2 + h0^2
//   D = (r, g, b, a2)        a2 = 2 (G00^2 + G10^2 - h0^2)
// Along a pixel row, f = q' - r is a quadratic in the column with second derivative a2,
// and q' + r (the magnitude that bounds the rounding of f) grows by at most sc per column
// squared.
template <int DIV>
__device__ __forceinline__ void stage_record(const Rec &r, float ox_tile, float oy_tile, float4 &A, float4 &B,
                                             float4 &C, float4 &D) {
  const df ox = two_sum(ox_tile, -r.a.x);
  const df oy = two_sum(oy_tile, -r.a.y);
  A = make_float4(__fadd_rn(ox.hi, __fsub_rn(ox.lo, r.a.z)), __fadd_rn(oy.hi, __fsub_rn(oy.lo, r.a.w)), r.b.x,
                  r.b.y);
  B = make_float4(r.b.z, r.b.w, r.c.x, r.c.y);
  const float gg = fmaf(r.b.x, r.b.x, r.b.z * r.b.z);
  const float hh = r.c.x * r.c.x;
  C = make_float4(r.c.z, DIV == 1 ? r.c.w / r.c.z : r.c.w, r.d.x, gg + hh);
  D = make_float4(r.d.y, r.d.z, r.d.w, 2.f * (gg - hh));
}

// Conservative segment filter.  A thread's PX pixels lie on one row at columns
// fl_x + k s (k = 0 .. PX-1).  With t = k / (PX-1), f(t) = f0 + G1 t + A2 t^2 / 2 exactly,
// so the minimum of f over the segment is f0, f(1) or, when the vertex lies inside,
// f0 - G1^2 / (2 A2).  Returns false only when that minimum exceeds a margin that bounds
// the float rounding of f at every pixel (each pixel's q' + r is at most
// 2 (q0 + r0) + 2 (s (PX-1))^2 sc); the exact per-pixel test (eval_pixels) decides
// otherwise, so skipping never changes a result.
template <int PX>
__device__ __forceinline__ bool row_may_hit(const float4 &A, const float4 &B, const float4 &C, float a2,
                                            float fl_x, float fl_y, float s) {
  const float dy = A.y + fl_y;
  const float dx = A.x + fl_x;
  const float y0 = fmaf(A.z, dx, A.w * dy);
  const float y1 = fmaf(B.x, dx, B.y * dy);
  const float y2 = fmaf(B.z, dx, fmaf(B.w, dy, 1.f));
  const float q0 = fmaf(y0, y0, y1 * y1);
  const float r0 = y2 * y2;
  const float f0 = q0 - r0;
  constexpr float L = float(PX - 1);
  const float sL = s * L;
  // df/dcolumn at the first pixel, scaled to the whole segment
  const float G1 = 2.f * (fmaf(y0, A.z, y1 * B.x) - y2 * B.z) * sL;
  const float A2 = a2 * (sL * sL);
  const float margin = 1e-3f + 1e-5f * (2.f * (q0 + r0) + 2.f * (sL * sL) * C.w + fabsf(G1) + fabsf(A2));
  const float fe = f0 + G1 + 0.5f * A2;
  const bool vertex_in = G1 < 0.f && G1 + A2 > 0.f;
  return f0 <= margin || fe <= margin || (vertex_in && 2.f * A2 * (f0 - margin) <= G1 * G1);
}

// Support test of PX pixels of one row (columns fl_x + k s, k = 0 .. PX-1, row fl_y,
// relative to the tile origin; s a power of two).  Returns the hit mask; q', r (and y) per
// pixel.  With r = y2 |y2| the single test q' <= r holds exactly when y2 > 0 and
// kp q <= y2^2 (q' = kp q >= 0; y = 0 cannot occur), and r = y2^2 on every hit.
template <int PX>
__device__ __forceinline__ uint32_t eval_pixels(const float4 &A, const float4 &B, float fl_x, float fl_y,
                                                float s, float q[PX], float r[PX], float y0s[PX], float y1s[PX],
                                                float y2s[PX]) {
  const float dy = A.y + fl_y;
  const float dx = A.x + fl_x;
  float y0 = fmaf(A.z, dx, A.w * dy);
  float y1 = fmaf(B.x, dx, B.y * dy);
  float y2 = fmaf(B.z, dx, fmaf(B.w, dy, 1.f));
  const float st0 = s * A.z, st1 = s * B.x, st2 = s * B.z;
  uint32_t hit = 0;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    if (k) { y0 += st0; y1 += st1; y2 += st2; }
    q[k] = fmaf(y0, y0, y1 * y1);
    r[k] = y2 * fabsf(y2);
    y0s[k] = y0; y1s[k] = y1; y2s[k] = y2;
    if (q[k] <= r[k]) hit |= 1u << k;
  }
  return hit;
}

// Rendered opacity before the clamp (fragment formula + Eq. rend_opacity), from the staged
// C and a hit's q' and r.  D_ray (DIV = 0): D log2(e) / 2 = c2h q / (q + r) = c2h q' /
// (q' + kp r).  D_gs (DIV = 1, records with h = 0 so that r = 1): D log2(e) / 2 = c2h q =
// (c2h / kp) q', with c2h / kp staged in C.y.
template <int DIV>
__device__ __forceinline__ float pixel_opacity(const float4 &C, float q, float r) {
  if (DIV == 1) return ex2_approx(fmaf(-C.y, q, C.z));
  const float t = __fdividef(q, fmaf(C.x, r, q));
  return ex2_approx(fmaf(-C.y, t, C.z));
}

}  // namespace raygs
