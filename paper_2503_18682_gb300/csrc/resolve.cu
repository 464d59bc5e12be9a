// Box-filter resolve of a supersampled render: every output pixel is the mean of the
// factor x factor block of pixels rendered for it at factor-times the resolution (the
// cameras' sizes, focal lengths and principal points scaled by factor, so that the block's
// rays are the pixel's sub-pixel rays).  Colour and transmittance are averaged alike.
#include "raygs_internal.cuh"

namespace raygs {

__global__ void __launch_bounds__(256) resolve_kernel(const float *rgb_hi, const float *T_hi, float *rgb_lo,
                                                      float *T_lo, int w_lo, int h_lo, int factor,
                                                      long long base_hi, long long base_lo) {
  const long long n = (long long)w_lo * h_lo;
  const int w_hi = w_lo * factor;
  const float inv = 1.f / float(factor * factor);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const int y = int(p / w_lo), x = int(p - (long long)y * w_lo);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, t = 0.f;
    for (int j = 0; j < factor; ++j) {
      const long long row = base_hi + (long long)(y * factor + j) * w_hi + (long long)x * factor;
      for (int i = 0; i < factor; ++i) {
        const long long q = row + i;
        c0 += rgb_hi[3 * q];
        c1 += rgb_hi[3 * q + 1];
        c2 += rgb_hi[3 * q + 2];
        if (T_hi) t += T_hi[q];
      }
    }
    const long long o = base_lo + p;
    rgb_lo[3 * o] = c0 * inv;
    rgb_lo[3 * o + 1] = c1 * inv;
    rgb_lo[3 * o + 2] = c2 * inv;
    if (T_lo && T_hi) T_lo[o] = t * inv;
  }
}

cudaError_t launch_resolve(const float *rgb_hi, const float *T_hi, float *rgb_lo, float *T_lo, int w_lo, int h_lo,
                           int factor, long long base_hi, long long base_lo, cudaStream_t st) {
  const long long n = (long long)w_lo * h_lo;
  if (n == 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  resolve_kernel<<<unsigned(blocks < 65535 ? blocks : 65535), 256, 0, st>>>(rgb_hi, T_hi, rgb_lo, T_lo, w_lo, h_lo,
                                                                           factor, base_hi, base_lo);
  return cudaGetLastError();
}

}  // namespace raygs
