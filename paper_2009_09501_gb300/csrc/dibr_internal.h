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
constexpr int kBoxBytes = 256;      // 2-D TMA box width (bytes) for rows with 3*W not a multiple of 16
constexpr int kMaxConsumers = 512;  // threads per CTA at most (8K rows use 480)
constexpr int kMaxWidth = 7680;   // 8K UHD: the widest row whose z-buffers and ring fit on chip

// How the depth of a row is obtained inside the band kernel.
enum DepthSource : int {
  DS_BINOM5 = 0,  // luminance + 5x5 binomial, computed on chip (rows +-2 of context)
  DS_LUMA = 1,    // luminance only
  DS_GLOBAL = 2   // read from a depth map in device memory (cross-bilateral pre-pass)
};

// How input rows reach shared memory.
enum LoadMode : int {
  LM_AUTO = 0,
  LM_BULK = 1,   // one contiguous bulk copy (cp.async.bulk) per row
  LM_T3 = 2,     // 3-D tensor {inner, 3W/inner, H}, boxes {inner, step, 1} (cp.async.bulk.tensor)
  LM_T2 = 3      // 2-D tensor {3W, H}, boxes {256, 1}: any width
};

// Bits of the device status word.
enum : int { ST_TIMEOUT_FULL = 1, ST_TIMEOUT_EMPTY = 2, ST_BAD_ARGS = 4, ST_TIMEOUT_DRAIN = 8 };

// Output slots, in the order of dibr_outputs.
enum { O_ANA = 0, O_LEFT = 1, O_RIGHT = 2, O_HSBS = 3, O_DEPTH = 4, O_COUNT = 5 };

// Per-image arguments of the band kernel.  The tensor map comes first for its 64-byte
// alignment; the kernel receives the whole record as a __grid_constant__ parameter.
struct BandArgs {
  // input rows: a 3-D uint8 tensor {16, 3W/16, H} (strides 16, pitch) loaded in boxes of
  // {16, box_step, 1} when 3W is a multiple of 16, else a 2-D tensor {3W, H} loaded in
  // boxes of {256, 1}
  CUtensorMap tmap;
  const uint8_t *in;  // input base (bulk mode)
  int64_t in_pitch;
  const uint8_t *depth_in;
  uint8_t *out[O_COUNT];
  int64_t out_pitch, depth_pitch, depth_in_pitch;
  int32_t W, H;
  int32_t nbox;      // TMA boxes per row
  int32_t box_bytes; // bytes per box
  int32_t box_step;  // box-to-box step of the tensor coordinate that walks along the row
  int32_t tinner;    // LM_T3: bytes of a box's inner rows
  int32_t load_mode; // LM_BULK, LM_T3 or LM_T2
  int32_t row_bytes; // bytes of one input row (3W)
  int32_t l2_prefetch; // prefetch the CTA's later rows into L2 at launch
  int32_t srow;      // bytes per ring slot
  int32_t nb;        // ring slots
  int32_t nch;       // 16-pixel chunks per row
  int32_t nc;        // threads per CTA, one 16-pixel chunk each (multiple of 32)
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
  int bar, flags, lut, ring, drow, zb, total;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

__host__ __device__ inline BandSmem band_smem_layout(int nb, int srow, int nch, int depth_src) {
  (void)depth_src;
  BandSmem s;
  s.bar = 0;                       // full[kMaxRing] mbarriers
  s.flags = 8 * kMaxRing;          // batched launches: the current work unit
  s.lut = s.flags + 64;            // int4 lut[256]: {-hL[d], -hR[d], (255 - d) << 24, 0}
  s.ring = round_up(s.lut + 4096, 128);
  // depth of the current row, one byte per column (read back by the scatter)
  s.drow = round_up(s.ring + nb * srow, 16);
  // z-buffers of the forward warp, double buffered across rows: [2][L, R][nch * 16]
  // (the literal gather keeps lut_n[256] here instead)
  s.zb = round_up(s.drow + nch * kChunk, 16);
  const int zbytes = 4 * nch * kChunk * 4;
  s.total = s.zb + (zbytes > 1024 ? zbytes : 1024);
  return s;
}

// One image of a batched launch, in device memory.
struct alignas(16) ImageDesc {
  const uint8_t *in;
  int64_t in_pitch;
  const uint8_t *depth_in;
  int64_t depth_in_pitch;
  uint8_t *out[O_COUNT];
  int64_t out_pitch, depth_pitch;
  int32_t W, H, nch, row_bytes;
  uint32_t outputs;
  int32_t warp_mode, depth_src, pad;
  int32_t lut_h[256];
  int32_t lut_n[256];
};

static_assert(sizeof(ImageDesc) % 16 == 0, "descriptors are read as an array");

// Arguments of the batched kernel: descriptors, work units {image, first row, end row,
// 0} in the order they are handed out, and the counter the CTAs take units from.
struct BatchArgs {
  const ImageDesc *descs;
  const int4 *units;
  int32_t n_units;
  int *counter;
  int *status;
  unsigned long long timeout_ns;
  int32_t nb, srow, nch_max, nc;
};

// Host launchers (dibr_band.cu, dibr_xbf.cu).
cudaError_t launch_band(const BandArgs &a, int smem_bytes, int ctas_per_sm, cudaStream_t st);
cudaError_t launch_batch(const BatchArgs &b, int grid, int smem_bytes, cudaStream_t st);
int band_max_threads(int ctas_per_sm);
cudaError_t launch_xbf(const uint8_t *rgb, int64_t pitch, int W, int H, int radius,
                       float sigma_s, float sigma_r, uint8_t *D, int64_t dpitch,
                       cudaStream_t st);

}  // namespace dibr
