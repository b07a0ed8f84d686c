// dibr_internal.h -- declarations shared by the CUDA kernels and the C-ABI host code of
// libdibr.  Not part of the public interface (that is include/dibr.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dibr.h"

namespace dibr {

constexpr int kChunk = 16;          // pixels owned by one consumer thread per pass
constexpr int kMaxRing = 8;         // TMA row-ring slots at most
constexpr int kFramesInFlight = 7;  // consecutive independent frames side by side (automatic)
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

// Output slots, in the order of dibr_outputs; depth and holes are one-byte maps (row
// pitch depth_pitch), the others RGB (row pitch pitch).
enum { O_ANA = 0, O_LEFT = 1, O_RIGHT = 2, O_HSBS = 3, O_DEPTH = 4, O_HOLES = 5, O_COUNT = 6 };
constexpr uint32_t kOutBits[O_COUNT] = {DIBR_OUT_ANAGLYPH, DIBR_OUT_LEFT, DIBR_OUT_RIGHT,
                                        DIBR_OUT_HSBS,     DIBR_OUT_DEPTH, DIBR_OUT_HOLES};
constexpr uint32_t kAllOutputs =
    DIBR_OUT_ANAGLYPH | DIBR_OUT_LEFT | DIBR_OUT_RIGHT | DIBR_OUT_HSBS | DIBR_OUT_DEPTH | DIBR_OUT_HOLES;
__host__ __device__ constexpr bool is_map_output(int i) { return i == O_DEPTH || i == O_HOLES; }
inline uint8_t *&out_slot(dibr_outputs &o, int i) {
  uint8_t **s[O_COUNT] = {&o.anaglyph, &o.left, &o.right, &o.hsbs, &o.depth, &o.holes};
  return *s[i];
}
inline uint8_t *out_slot(const dibr_outputs &o, int i) {
  uint8_t *const s[O_COUNT] = {o.anaglyph, o.left, o.right, o.hsbs, o.depth, o.holes};
  return s[i];
}

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
  int32_t zguard;    // guard targets on each side of a z-buffer row (>= the largest shift)
  int32_t grid;      // CTAs; CTA b owns rows row0 + [b*n/grid, (b+1)*n/grid), n = row1 - row0
  int32_t row0, row1;  // the rows this launch computes (all of them: 0, H)
  int32_t overlap;   // 1: independent of the previous launch on the stream (start at once;
                     // wait for it only before exiting); 0: wait for it before any global access
  uint32_t outputs;  // DIBR_OUT_* bits
  int32_t warp_mode; // DIBR_WARP_*
  int32_t depth_src; // DepthSource
  int32_t fast_store;  // every RGB output base and the output pitch are 16-byte aligned
  int *status;
  unsigned long long timeout_ns;
  int32_t lut_h[256];  // low 16 bits: hL[d], high 16 bits: hR[d] (signed)
  int32_t lut_n[256];  // 510 * s_L(d): Fig. 3 shift numerator for the literal gather
};

// Shared-memory layout of the band kernel (bytes from the dynamic smem base).
//   bar   ring-slot mbarriers full[kMaxRing]
//   flags +0: the batch's current work unit; +8, +16: the per-row mbarriers (every warp
//         has scattered the row / has published its summary and cleared its targets)
//   lut   uint2 per value of 255 - depth: byte offsets of the left / right target
//   wsum  per row parity, view and warp: {has a filled target, first, last filled entry}
//   ring  input rows;  drow  255 - depth of the current row, one byte per column
//   zb    z-buffers, [parity][view] rows of zlen targets separated by zguard guard targets
//         (targets a shift moves outside the row land in a guard and are never read);
//         the literal gather keeps int32 lut_n[256] here instead
struct BandSmem {
  int bar, flags, lut, wsum, ring, drow, zb, zstride, total;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

__host__ __device__ inline BandSmem band_smem_layout(int nb, int srow, int nch, int nwarps, int zguard) {
  BandSmem s;
  s.bar = 0;
  s.flags = 8 * kMaxRing;
  s.lut = s.flags + 64;
  s.wsum = s.lut + 2048;
  s.ring = round_up(s.wsum + 2 * 2 * nwarps * 16, 128);
  s.drow = round_up(s.ring + nb * srow, 16);
  s.zb = round_up(s.drow + nch * kChunk, 16);
  const int zlen = nch * kChunk;  // a multiple of 16 targets: rows stay 16-byte aligned
  s.zstride = zlen + zguard;      // words from one row's target 0 to the next row's
  const int zbytes = 4 * (4 * zlen + 5 * zguard);
  s.total = s.zb + (zbytes > 1024 ? zbytes : 1024);
  return s;
}

// Guard targets on each side of a z-buffer row for the shift tables lut_h (low / high 16
// bits: hL, hR): the largest |h|, rounded up to whole 16-byte groups.
inline int zguard_of(const int32_t *lut_h) {
  int g = 0;
  for (int d = 0; d < 256; ++d) {
    const int hl = static_cast<int16_t>(lut_h[d] & 0xFFFF), hr = lut_h[d] >> 16;
    g = g > (hl < 0 ? -hl : hl) ? g : (hl < 0 ? -hl : hl);
    g = g > (hr < 0 ? -hr : hr) ? g : (hr < 0 ? -hr : hr);
  }
  return round_up(g + 1, 4);
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

// Arguments of one batched launch: descriptors, work units {image, first row, end row,
// 0} in the order they are handed out, and the counter the CTAs take units from.
struct BatchArgs {
  const ImageDesc *descs;
  const int4 *units;
  int32_t n_units;
  int *counter;
  int *status;
  unsigned long long timeout_ns;
  int32_t nb, srow, nch_max, nc, zguard;
  uint32_t outs;  // kSetStereo / kSetAnaglyph: every image is of that kind (fixed_set); 0: any
};

// Output sets with kernel instances of their own (outputs fixed at compile time): binomial
// depth, forward warp, and every requested RGB output and the output pitch 16-byte aligned.
constexpr uint32_t kSetStereo = DIBR_OUT_ANAGLYPH | DIBR_OUT_LEFT | DIBR_OUT_RIGHT;
constexpr uint32_t kSetAnaglyph = DIBR_OUT_ANAGLYPH;

// The fixed set an image belongs to (kSetStereo, kSetAnaglyph), else 0.
inline uint32_t fixed_set(uint32_t outputs, int depth_src, int warp_mode, const uint8_t *const *out, int64_t pitch) {
  if (depth_src != DS_BINOM5 || warp_mode != DIBR_WARP_FORWARD) return 0u;
  if (outputs != kSetStereo && outputs != kSetAnaglyph) return 0u;
  const uintptr_t bits = reinterpret_cast<uintptr_t>(out[O_ANA]) | reinterpret_cast<uintptr_t>(out[O_LEFT]) |
                         reinterpret_cast<uintptr_t>(out[O_RIGHT]) | static_cast<uintptr_t>(pitch);
  return (bits & 15u) == 0 ? outputs : 0u;
}

// ---- planning a batch (host; no allocation, so the no-allocation entry point shares it)
//
// A block of the band kernel is as wide as its widest row needs (one thread per 16
// columns, whole warps).  A batch mixing 720p and 8K frames in one launch would run every
// 720p row on an 8K-wide block, most of it idle, at the 8K block's one CTA per SM.  So the
// images are grouped by block width and each group gets a launch of its own plan; the
// launches follow one another on the stream, widest first, each allowed to start while
// the previous one finishes its last units (programmatic dependent launch).
constexpr int kMaxClasses = 16;  // distinct block widths: 32 .. 480 threads in steps of 32

struct BatchClass {
  int nc;          // threads per block
  int nch_max;     // 16-column chunks of the widest row in the group
  int srow;        // bytes per ring slot
  int nb, per;     // ring slots; CTAs per SM
  int smem;        // dynamic shared memory per block
  int rows;        // rows per work unit
  int unit_begin, n_units;
};

struct BatchLimits {
  int max_smem, smem_per_sm;  // device limits
  int ring_slots, ctas_per_sm;  // tuning caps (0: none)
  int zguard;                   // z-buffer guard of every image of the batch (the largest)
};

inline int chunks_of(int width) { return (width + kChunk - 1) / kChunk; }
inline int block_of(int width) { return round_up(chunks_of(width), 32); }

// Ring depth and CTAs per SM of one group (nc, nch_max and srow set): the deepest ring at
// the most CTAs per SM within the limits.  Returns false if no plan fits.
inline bool plan_class(BatchClass &k, const BatchLimits &lim) {
  const int max_nb = lim.ring_slots > 0 ? (lim.ring_slots < 4 ? 4 : lim.ring_slots < kMaxRing ? lim.ring_slots : kMaxRing)
                                        : kMaxRing;
  const int by_regs = 65536 / (k.nc * 128), by_threads = 2048 / k.nc;
  const int max_per = by_regs < by_threads ? by_regs : by_threads;
  k.per = 0;
  for (int nb = 4; nb <= max_nb; ++nb) {
    const int tot = band_smem_layout(nb, k.srow, k.nch_max, k.nc / 32, lim.zguard).total;
    if (tot > lim.max_smem) continue;
    int per = lim.smem_per_sm / (tot + 1024);
    if (per > max_per) per = max_per;
    if (lim.ctas_per_sm > 0 && per > lim.ctas_per_sm) per = lim.ctas_per_sm;
    if (per >= 1 && per >= k.per) {  // the deepest ring at the best CTAs per SM
      k.per = per;
      k.nb = nb;
    }
  }
  if (k.per < 1) return false;
  k.smem = band_smem_layout(k.nb, k.srow, k.nch_max, k.nc / 32, lim.zguard).total;
  return true;
}

// Groups the n images by block width (widest first), plans each group's ring and CTAs per
// SM, and sets class_of[i].  Returns the number of groups, or -1 if some group fits no plan.
inline int plan_batch_classes(int n, const int *width, const int *row_bytes, const BatchLimits &lim,
                              int *class_of, BatchClass *cls) {
  int nclass = 0;
  for (int i = 0; i < n; ++i) {
    const int nc = block_of(width[i]);
    int c = 0;
    while (c < nclass && cls[c].nc > nc) ++c;
    if (c == nclass || cls[c].nc != nc) {
      if (nclass == kMaxClasses) return -1;
      for (int k = nclass; k > c; --k) cls[k] = cls[k - 1];
      cls[c] = BatchClass{nc, 1, 128, 4, 0, 0, 0, 0, 0};
      ++nclass;
    }
  }
  for (int i = 0; i < n; ++i) {
    int c = 0;
    while (cls[c].nc != block_of(width[i])) ++c;
    class_of[i] = c;
    const int nch = chunks_of(width[i]);
    const int need = row_bytes[i] > 48 * nch ? row_bytes[i] : 48 * nch;
    if (nch > cls[c].nch_max) cls[c].nch_max = nch;
    if (round_up(need, 128) > cls[c].srow) cls[c].srow = round_up(need, 128);
  }
  for (int c = 0; c < nclass; ++c)
    if (!plan_class(cls[c], lim)) return -1;
  return nclass;
}

// Rows per work unit of each group: a group whose rows fill the SM slots (sms x CTAs per
// SM) at most kUnitRows deep gets one unit per slot -- e.g. one 4K frame: 2160 rows over 304
// slots, 8 rows each -- so that every slot has work; a larger group gets kUnitRows-row units,
// enough of them for the slots to stay balanced.  A fixed size (rows > 0) overrides.  Each
// unit recomputes the two rows of context above it, so units are not made smaller than
// needed.
constexpr int kUnitRows = 32;
inline void plan_unit_rows(int n, const int *height, const int *class_of, int nclass, int sms, int rows,
                           BatchClass *cls) {
  for (int c = 0; c < nclass; ++c) {
    if (rows > 0) {
      cls[c].rows = rows;
      continue;
    }
    int64_t total = 0;
    for (int i = 0; i < n; ++i)
      if (class_of[i] == c) total += height[i];
    const int64_t slots = static_cast<int64_t>(sms) * (cls[c].per > 0 ? cls[c].per : 1);
    cls[c].rows = total <= slots * kUnitRows ? static_cast<int>((total + slots - 1) / slots) : kUnitRows;
    if (cls[c].rows < 1) cls[c].rows = 1;
  }
}

// order[0..n) = image indices, largest area first (stable insertion sort, no allocation)
inline void order_by_area(int n, const int *width, const int *height, int *order) {
  for (int i = 0; i < n; ++i) {
    const int64_t a = static_cast<int64_t>(width[i]) * height[i];
    int k = i;
    while (k > 0 && static_cast<int64_t>(width[order[k - 1]]) * height[order[k - 1]] < a) {
      order[k] = order[k - 1];
      --k;
    }
    order[k] = i;
  }
}

// Arguments of the 2-D block inpainting (dibr_inpaint.cu): both views are repaired in
// place; anaglyph and HSBS (either may be null) are rewritten where a view changed.
struct InpaintArgs {
  uint8_t *view[2];       // left, right: row-filled views, W x H x 3, row pitch `pitch`
  int64_t pitch;
  const uint8_t *holes;   // bit 0: hole of the left view, bit 1: of the right view
  int64_t holes_pitch;
  uint8_t *ana, *hsbs;    // row pitch out_pitch
  int64_t out_pitch;
  int32_t W, H, block, nbx, nblocks, sms;
  int32_t *order;         // device scratch of 2 nblocks + 3 ints: the work items (2 block +
                          // view) in processing order, the two fill counters of that order and
                          // the next item to take (zeroed before the launch)
};

// Host launchers (dibr_band.cu, dibr_xbf.cu, dibr_inpaint.cu).
cudaError_t launch_band(const BandArgs &a, int smem_bytes, int ctas_per_sm, cudaStream_t st);
// chained: may start while the previous launch on the stream finishes (the previous
// launch is a batch launch of the same call).
cudaError_t launch_batch(const BatchArgs &b, int grid, int smem_bytes, bool chained, cudaStream_t st);
cudaError_t launch_inpaint(const InpaintArgs &a, cudaStream_t st);
// after: may start beside the previous launch on the stream (its buffers are disjoint from
// this launch's), completing only after it.
cudaError_t launch_xbf(const uint8_t *rgb, int64_t pitch, int W, int H, int radius,
                       float sigma_s, float sigma_r, uint8_t *D, int64_t dpitch,
                       cudaStream_t st, bool after = false);

}  // namespace dibr
