// dibr_xbf.cu -- cross-bilateral smoothing of the luminance depth map (Sec. 3 "Filtered
// Depth Map", Sec. 4 "GPU Cross Bilateral Filtering").
//
// Guide = the RGB image.  For pixel p the window is the square |dx|,|dy| <= r clipped to
// the image; sample q has weight exp(-(dx^2+dy^2)/(2 s_s^2) - |RGB(p)-RGB(q)|^2/(2 s_r^2))
// and D(p) = round-half-up(sum w Y(q) / sum w).  FP32; the sums are taken relative to
// Y(p) (sum w (Y(q) - Y(p))), which is the same quotient and keeps the rounding error of
// the accumulation small next to the final half-integer decision.
//
// One CTA computes a 32 x 16 tile (two vertically adjacent pixels per thread); the tile plus
// an r-pixel apron is staged in shared memory once, one 8-byte cell per pixel: the colour (RGB in the low three bytes) and the
// luminance (as a float).  Per tap: one shared load, the squared colour distance exactly
// in two integer instructions (per-byte absolute differences, then a byte dot product of
// that word with itself), one FMA for the exponent (the spatial part is a per-tap
// constant: the radius is a template parameter, so the taps unroll), one exp2 on the
// special-function unit (the constants are pre-scaled by log2 e), and two accumulations.
// The distance's integer-to-float conversion shares the special-function unit's rate: the
// kernel is bound by instruction issue, not by that unit, and the conversion takes one issue
// slot where an exact mantissa trick (OR into 2^23, subtract 2^23) takes two.
#include "dibr_internal.h"
#include "dibr_ptx.cuh"

namespace dibr {
namespace {

constexpr int kTX = 32, kTY = 8;  // threads per CTA: kTX x kTY; tiles of kTX x kPY kTY pixels; radius 1..8
constexpr int kPY = 4;             // pixels per thread, vertically adjacent

__device__ __forceinline__ uint32_t luma8x(uint32_t r, uint32_t g, uint32_t b) {
  return (299u * r + 587u * g + 114u * b + 500u) / 1000u;
}

// 2^x on the special-function unit (results below 2^-126 flush to zero).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One tap: q's colour cq and luminance yq against the centre's colour cp and luminance yp;
// es = -(dx^2+dy^2) as log2(e).
__device__ __forceinline__ void xbf_tap(uint32_t cp, uint32_t cq, float yq, float es, float nar, float yp, float &num,
                                        float &den) {
  const uint32_t v = __vabsdiffu4(cp, cq);
  const uint32_t d2 = __dp4a(v, v, 0u);  // |RGB(p) - RGB(q)|^2, exact, < 2^18
  const float fd2 = __uint2float_rn(d2);  // exact (d2 < 2^24)
  const float w = ex2(fmaf(fd2, nar, es));
  num = fmaf(w, yq - yp, num);
  den += w;
}

// The depth of one pixel from the staged tile, window clipped to the image (cell (cy, cx) of
// the tile holds the pixel itself).
template <int R>
__device__ __forceinline__ float xbf_clipped(const uint2 (*px)[kTX + 2 * R], int cy, int cx, int x, int y, int W, int H,
                                             float nas, float nar, float &yp_out) {
  const uint2 pc = px[cy][cx];
  const float yp = __uint_as_float(pc.y);
  float num = 0.f, den = 0.f;
  const int x0 = max(-R, -x), x1 = min(R, W - 1 - x), y0 = max(-R, -y), y1 = min(R, H - 1 - y);
  for (int dy = y0; dy <= y1; ++dy)
    for (int dx = x0; dx <= x1; ++dx) {
      const uint2 q = px[cy + dy][cx + dx];
      xbf_tap(pc.x, q.x, __uint_as_float(q.y), static_cast<float>(dx * dx + dy * dy) * nas, nar, yp, num, den);
    }
  yp_out = yp;
  return num / den;
}

__device__ __forceinline__ void xbf_store(uint8_t *D, int64_t dpitch, int x, int y, float yp, float rel) {
  const float q = floorf(rel + 0.5f);
  const int v = static_cast<int>(yp) + static_cast<int>(q);
  D[static_cast<int64_t>(y) * dpitch + x] = static_cast<uint8_t>(min(max(v, 0), 255));
}

// One CTA: a 32 x (8 kPY) tile, each thread kPY vertically adjacent pixels (x, y0 + i),
// whose windows share rows: a cell of the 2R + kPY rows they span is loaded once for all of
// the pixels whose window holds it.
template <int R>
__global__ void __launch_bounds__(kTX *kTY) xbf_kernel(const uint8_t *__restrict__ rgb, int64_t pitch, int W, int H,
                                                       float as, float ar, uint8_t *__restrict__ D, int64_t dpitch,
                                                       int after) {
  constexpr int kRows = kPY * kTY;  // tile rows
  __shared__ uint2 px[kRows + 2 * R][kTX + 2 * R];  // colour 0x00BBGGRR, luminance as float bits
  const int bx = blockIdx.x * kTX, by = blockIdx.y * kRows;
  constexpr int ax = kTX + 2 * R, ay = kRows + 2 * R;
  for (int i = threadIdx.x; i < ax * ay; i += blockDim.x) {
    const int ty = i / ax, tx = i - ty * ax;
    const int gx = bx - R + tx, gy = by - R + ty;
    uint32_t c = 0u;  // outside the image: never read (the window is clipped)
    uint32_t l = 0u;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const uint8_t *p = rgb + static_cast<int64_t>(gy) * pitch + 3 * static_cast<int64_t>(gx);
      const uint32_t r = p[0], g = p[1], b = p[2];
      c = r | (g << 8) | (b << 16);
      l = luma8x(r, g, b);
    }
    px[ty][tx] = make_uint2(c, __float_as_uint(static_cast<float>(l)));
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = kPY * (threadIdx.x / kTX);
  const int x = bx + tx, y = by + ty;
  if (x >= W || y >= H) {
    if (after) griddep_wait();
    return;
  }
  // exponents in base 2: w = 2^(-(s2 * as + d2 * ar) * log2 e)
  constexpr float kLog2e = 1.4426950408889634f;
  const float nas = -as * kLog2e, nar = -ar * kLog2e;
  if (x >= R && x + R < W && y >= R && y + kPY - 1 + R < H) {
    uint32_t cp[kPY];
    float yp[kPY], num[kPY], den[kPY];
#pragma unroll
    for (int i = 0; i < kPY; ++i) {
      const uint2 pc = px[ty + i + R][tx + R];
      cp[i] = pc.x;
      yp[i] = __uint_as_float(pc.y);
      num[i] = den[i] = 0.f;
    }
#pragma unroll
    for (int dy = -R; dy <= R + kPY - 1; ++dy)
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        const uint2 q = px[ty + R + dy][tx + R + dx];
#pragma unroll
        for (int i = 0; i < kPY; ++i)
          if (dy - i >= -R && dy - i <= R)  // row dy of pixel i's window (compile time)
            xbf_tap(cp[i], q.x, __uint_as_float(q.y), static_cast<float>(dx * dx + (dy - i) * (dy - i)) * nas, nar,
                    yp[i], num[i], den[i]);
      }
#pragma unroll
    for (int i = 0; i < kPY; ++i) xbf_store(D, dpitch, x, y + i, yp[i], num[i] / den[i]);
  } else {  // a window clipped to the image
    for (int i = 0; i < kPY && y + i < H; ++i) {
      float yp;
      const float r = xbf_clipped<R>(px, ty + i + R, tx + R, x, y + i, W, H, nas, nar, yp);
      xbf_store(D, dpitch, x, y + i, yp, r);
    }
  }
  // launched to run beside the previous launch on the stream (whose buffers the host found
  // disjoint from this one's): complete only after it, so that the stream order holds
  if (after) griddep_wait();
}

template <int R>
cudaError_t launch_r(const uint8_t *rgb, int64_t pitch, int W, int H, float as, float ar, uint8_t *D, int64_t dpitch,
                     cudaStream_t st, bool after) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((W + kTX - 1) / kTX, (H + kPY * kTY - 1) / (kPY * kTY));
  cfg.blockDim = dim3(kTX * kTY);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = after ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, xbf_kernel<R>, rgb, pitch, W, H, as, ar, D, dpitch, after ? 1 : 0);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_xbf(const uint8_t *rgb, int64_t pitch, int W, int H, int radius, float sigma_s,
                       float sigma_r, uint8_t *D, int64_t dpitch, cudaStream_t st, bool after) {
  const float as = static_cast<float>(1.0 / (2.0 * static_cast<double>(sigma_s) * sigma_s));
  const float ar = static_cast<float>(1.0 / (2.0 * static_cast<double>(sigma_r) * sigma_r));
  switch (radius) {
    case 1: return launch_r<1>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 2: return launch_r<2>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 3: return launch_r<3>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 4: return launch_r<4>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 5: return launch_r<5>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 6: return launch_r<6>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 7: return launch_r<7>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    case 8: return launch_r<8>(rgb, pitch, W, H, as, ar, D, dpitch, st, after);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dibr
