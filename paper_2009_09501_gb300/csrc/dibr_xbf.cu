// dibr_xbf.cu -- cross-bilateral smoothing of the luminance depth map (Sec. 3 "Filtered
// Depth Map", Sec. 4 "GPU Cross Bilateral Filtering").
//
// Guide = the RGB image.  For pixel p the window is the square |dx|,|dy| <= r clipped to
// the image; sample q has weight exp(-(dx^2+dy^2)/(2 s_s^2) - |RGB(p)-RGB(q)|^2/(2 s_r^2))
// and D(p) = round-half-up(sum w Y(q) / sum w).  FP32 with expf; the sums are taken
// relative to Y(p) (sum w (Y(q) - Y(p))), which is the same quotient and keeps the
// rounding error of the accumulation small next to the final half-integer decision.
//
// One CTA computes a 32 x 8 tile; the tile plus an r-pixel apron of colours and
// luminances is staged in shared memory once, then every thread runs its (2r+1)^2 taps.
#include "dibr_internal.h"

namespace dibr {
namespace {

constexpr int kTX = 32, kTY = 8, kMaxR = 8;
constexpr int kAX = kTX + 2 * kMaxR, kAY = kTY + 2 * kMaxR;

__device__ __forceinline__ uint32_t luma8x(uint32_t r, uint32_t g, uint32_t b) {
  return (299u * r + 587u * g + 114u * b + 500u) / 1000u;
}

__global__ void __launch_bounds__(kTX *kTY) xbf_kernel(const uint8_t *__restrict__ rgb, int64_t pitch,
                                                       int W, int H, int R, float as, float ar,
                                                       uint8_t *__restrict__ D, int64_t dpitch) {
  __shared__ uint32_t col[kAY][kAX];  // 0x00BBGGRR, bit 31 set outside the image
  __shared__ float lum[kAY][kAX];
  const int bx = blockIdx.x * kTX, by = blockIdx.y * kTY;
  const int ax = kTX + 2 * R, ay = kTY + 2 * R;
  for (int i = threadIdx.x; i < ax * ay; i += blockDim.x) {
    const int ty = i / ax, tx = i - ty * ax;
    const int gx = bx - R + tx, gy = by - R + ty;
    uint32_t c = 0x80000000u;
    float l = 0.f;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const uint8_t *p = rgb + static_cast<int64_t>(gy) * pitch + 3 * static_cast<int64_t>(gx);
      const uint32_t r = p[0], g = p[1], b = p[2];
      c = r | (g << 8) | (b << 16);
      l = static_cast<float>(luma8x(r, g, b));
    }
    col[ty][tx] = c;
    lum[ty][tx] = l;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int x = bx + tx, y = by + ty;
  if (x >= W || y >= H) return;
  const uint32_t cp = col[ty + R][tx + R];
  const float yp = lum[ty + R][tx + R];
  const int pr = cp & 255, pg = (cp >> 8) & 255, pb = (cp >> 16) & 255;
  float num = 0.f, den = 0.f;
  for (int dy = -R; dy <= R; ++dy) {
    for (int dx = -R; dx <= R; ++dx) {
      const uint32_t cq = col[ty + R + dy][tx + R + dx];
      if (cq & 0x80000000u) continue;
      const int er = pr - static_cast<int>(cq & 255), eg = pg - static_cast<int>((cq >> 8) & 255),
                eb = pb - static_cast<int>((cq >> 16) & 255);
      const float d2 = static_cast<float>(er * er + eg * eg + eb * eb);
      const float s2 = static_cast<float>(dx * dx + dy * dy);
      const float w = expf(-fmaf(s2, as, d2 * ar));
      num = fmaf(w, lum[ty + R + dy][tx + R + dx] - yp, num);
      den += w;
    }
  }
  const float q = floorf(num / den + 0.5f);
  const int v = static_cast<int>(yp) + static_cast<int>(q);
  D[static_cast<int64_t>(y) * dpitch + x] = static_cast<uint8_t>(min(max(v, 0), 255));
}

}  // namespace

cudaError_t launch_xbf(const uint8_t *rgb, int64_t pitch, int W, int H, int radius, float sigma_s,
                       float sigma_r, uint8_t *D, int64_t dpitch, cudaStream_t st) {
  if (radius < 1 || radius > kMaxR) return cudaErrorInvalidValue;
  const double as = 1.0 / (2.0 * static_cast<double>(sigma_s) * sigma_s);
  const double ar = 1.0 / (2.0 * static_cast<double>(sigma_r) * sigma_r);
  dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY);
  xbf_kernel<<<grid, kTX * kTY, 0, st>>>(rgb, pitch, W, H, radius, static_cast<float>(as),
                                         static_cast<float>(ar), D, dpitch);
  return cudaGetLastError();
}

}  // namespace dibr
