// dibr_internal.h -- declarations shared by the CUDA kernels and the C-ABI host code of
// libdibr.  Not part of the public interface (that is include/dibr.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dibr {

constexpr int kChunk = 16;          // pixels owned by one consumer thread per pass
constexpr int kMaxRing = 8;         // TMA row-ring slots at most
constexpr int kYRing = 6;           // luminance rows kept for the 5-row binomial
constexpr int kBoxBytes = 256;      // TMA box width (bytes) for one input row segment
constexpr int kMaxConsumers = 512;  // consumer threads per CTA at most
constexpr int kMaxWidth = 7680;   // 8K UHD: the widest row whose z-buffers and ring fit on chip

// How the depth of a row is obtained inside the band kernel.
enum DepthSource : int {
  DS_BINOM5 = 0,  // luminance + 5x5 binomial, computed on chip (rows +-2 of context)
  DS_LUMA = 1,    // luminance only
  DS_GLOBAL = 2   // read from a depth map in device memory (cross-bilateral pre-pass)
};

// Bits of the device status word.
enum : int { ST_TIMEOUT_FULL = 1, ST_TIMEOUT_EMPTY = 2, ST_BAD_ARGS = 4, ST_TIMEOUT_DRAIN = 8 };

// Output slots, in the order of dibr_outputs.
enum { O_ANA = 0, O_LEFT = 1, O_RIGHT = 2, O_HSBS = 3, O_DEPTH = 4, O_COUNT = 5 };

// Per-image arguments of the band kernel.  The tensor map comes first for its 64-byte
// alignment; the kernel receives the whole record as a __grid_constant__ parameter.
struct BandArgs {
  CUtensorMap tmap;  // input as a 2-D uint8 tensor {3W, H}, row stride = pitch
  const uint8_t *depth_in;
  uint8_t *out[O_COUNT];
  int64_t out_pitch, depth_pitch, depth_in_pitch;
  int32_t W, H;
  int32_t nbox;      // TMA boxes per row
  int32_t srow;      // bytes per ring slot
  int32_t nb;        // ring slots
  int32_t ystride;   // bytes per luminance row (16-byte pads on both sides)
  int32_t nch;       // 16-pixel chunks per row
  int32_t nc;        // consumer threads (multiple of 32); block = nc + 32
  int32_t grid;      // CTAs; CTA b owns rows [b*H/grid, (b+1)*H/grid)
  uint32_t outputs;  // DIBR_OUT_* bits
  int32_t warp_mode; // DIBR_WARP_*
  int32_t depth_src; // DepthSource
  int *status;
  unsigned long long timeout_ns;
  int32_t lut_h[256];  // low 16 bits: hL[d], high 16 bits: hR[d] (signed)
  int32_t lut_n[256];  // 510 * s_L(d): Fig. 3 shift numerator for the literal gather
};

// Shared-memory layout of the band kernel (bytes from the dynamic smem base).
struct BandSmem {
  int bar, flags, lut, ring, yring, drow, zb, total;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

__host__ __device__ inline BandSmem band_smem_layout(int nb, int srow, int ystride, int nch,
                                                    int depth_src) {
  BandSmem s;
  s.bar = 0;                       // full[kMaxRing], empty[kMaxRing] mbarriers
  s.flags = 16 * kMaxRing;         // abort flag
  s.lut = s.flags + 128;           // lut_h[256]
  s.ring = round_up(s.lut + 1024, 256);
  s.yring = s.ring + nb * srow;
  int ybytes = depth_src == DS_BINOM5 ? kYRing * ystride : 0;
  s.drow = round_up(s.yring + ybytes, 16);
  // z-buffers of the forward warp; the literal gather keeps lut_n[256] here instead
  s.zb = round_up(s.drow + nch * kChunk, 16);
  s.total = s.zb + (2 * nch * kChunk * 4 > 1024 ? 2 * nch * kChunk * 4 : 1024);
  return s;
}

// Host launchers (dibr_band.cu, dibr_xbf.cu).
cudaError_t launch_band(const BandArgs &a, int smem_bytes, cudaStream_t st);
cudaError_t launch_xbf(const uint8_t *rgb, int64_t pitch, int W, int H, int radius,
                       float sigma_s, float sigma_r, uint8_t *D, int64_t dpitch,
                       cudaStream_t st);

}  // namespace dibr
