// dibr_band.cu -- the fused per-frame DIBR kernel for sm_103a.
//
// One CTA owns a contiguous range of rows of one image and streams them through shared
// memory.  Per row it runs every stage of the pipeline of Sec. 3 / Sec. 4 of the paper:
//   depth (luminance) -> depth smoothing -> depth-to-shift table (Fig. 3) -> forward warp
//   of the left and right views with occlusion -> row-local hole fill (inpainting) ->
//   stereo formatting (anaglyph, L/R pair, half side-by-side, depth).
// Nothing but the input and the requested outputs touches HBM: luminance, depth, the
// z-buffers and the shift tables live in registers and shared memory.
//
// Thread c owns the 16 columns 16c .. 16c+15 of every row.  Input rows stream into a
// ring of shared-memory slots (one bulk copy per row, cp.async.bulk, or tensor boxes,
// cp.async.bulk.tensor), each slot's completion tracked by an mbarrier; the middle warp
// refills a slot once every warp has scattered the row it held.
//
// Per consumer thread and row y:
//   A  luminance of row y+2 for its 16 columns plus 2 on each side, fed into a cascade
//      of four [1 1] row sums held in registers, which yields the vertical binomial of
//      row y; the horizontal binomial gives D(y) for the 16 columns, stored as 255 - D.
//   B  the warp scatters its 512 sources (lane-interleaved) into the left and right
//      z-buffers with a shared-memory atomic minimum of ((255 - D) << 24 | RGB).  The
//      z-buffer rows carry guard targets on both sides, as wide as the largest shift,
//      so a source whose target falls outside the row lands in a guard: no bounds test.
//   C  reads its 16 targets' entries, fills holes (register sweeps; the entries carried
//      across chunks come from the neighbouring lanes by shuffle, across warps from a
//      per-warp summary in shared memory), formats and stores the outputs, and clears
//      its warp's targets for the row two rows later.
// Rows interleave as A(y+1), B(y+1), C(y).  There is no CTA-wide barrier per row: C of a
// row waits on an mbarrier every warp arrives on after B of that row (a row earlier), B of
// a row waits on one every warp arrives on once it has published its summary of the row
// two rows before and cleared its targets there (the same z-buffer), and a warp that needs
// an entry from outside its own targets waits on that second one for its own row.  The
// barriers come in pairs used by alternate rows.  Every wait is bounded (%globaltimer); a
// wait that gives up sets a bit of the status word and the CTA unwinds after letting its
// own copies land.
//
// Instances: the requested outputs are read from the arguments, or fixed at compile time for
// the two sets the workloads use (left + right + anaglyph, anaglyph alone; binomial depth,
// forward warp, 16-byte aligned rows), which drops the output branches and the state they
// keep live.  The fixed-set instances in bands of kTmemMinRows rows or more keep the vertical
// cascade's 32 words per thread in tensor memory between one row's A and the next, so that B
// and C have those registers.
#include <atomic>

#include "dibr.h"
#include "dibr_internal.h"
#include "dibr_ptx.cuh"

namespace dibr {
namespace {

constexpr uint32_t kAll = 0xFFFFFFFFu;
constexpr int kTmemMinRows = 8;  // rows per CTA from which the fixed-set instances use tensor memory

// The wait for a CTA's own copies in flight before it exits after a failed wait: always the
// full 2 s, whatever limit the other waits have, so that no copy lands in shared memory
// the CTA has given up.
constexpr unsigned long long kDrainLimitNs = 2000000000ull;

// z-buffer entry: ((255 - depth) << 24) | RGB of the source, reduced with an atomic
// minimum into a buffer initialised to kEmpty.  The smallest entry has the largest depth
// (nearest source).  Two sources with equal depth have equal shifts and so never meet on
// one target, so the colour bits never decide a collision; the winner's colour is read
// straight from its entry.  kEmpty cannot be a real entry: it would need depth 0 for a
// white pixel, and every depth rule gives a white pixel a depth of at least 1 (binomial:
// its own weight 36/256; luminance: 255; cross-bilateral: its own weight 1 among at most
// 289).
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t bsel(const uint32_t *w, int j) {
  return (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
}

// BT.601 luminance in exact thousandths, rounded half up (the depth-map reading):
// (299 R + 587 G + 114 B + 500) / 1000, the division as a multiply-high by
// ceil(2^32 / 1000), exact for numerators below 6.1e6.
__device__ __forceinline__ uint32_t luma8(uint32_t r, uint32_t g, uint32_t b) {
  return __umulhi(299u * r + 587u * g + 114u * b + 500u, 4294968u);
}

// The same luminance of a pixel word holding R, G, B, G in bytes 0..3: two byte dot
// products, 255 R + 510 G + 114 B and 44 R + 77 G (299 = 255 + 44, 587 = 2 * 255 + 77).
__device__ __forceinline__ uint32_t luma_rgbg(uint32_t w) {
  const uint32_t n = __dp4a(w, 0xFF72FFFFu, 500u);
  return __umulhi(__dp4a(w, 0x00004D2Cu, n), 4294968u);
}

// Pixel word (R, G, B, G) of the colour at byte offset r (0..3) of the byte pair lo, hi.
template <int R>
__device__ __forceinline__ uint32_t rgbg_at(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, R | ((R + 1) << 4) | ((R + 2) << 8) | ((R + 1) << 12));
}

// Luminance of columns x0-2 .. x0+17 (clamped to [0, W-1]) of one input row held in
// shared memory, as 10 words of two 16-bit lanes: yp[2q] = columns (4q, 4q+2) and
// yp[2q+1] = (4q+1, 4q+3) of the window, the layout the vertical cascade works on.
__device__ __forceinline__ void luma20(const uint8_t *row, int x0, int W, uint32_t (&yp)[10]) {
  // bytes 3*x0-8 .. 3*x0+55 (8-byte and 16-byte aligned loads); column j of the window at
  // byte 2+3j.  At the row's ends the loads reach past it into neighbouring shared memory
  // (another ring slot, the summaries before the ring, the depth row after it); those
  // columns are replaced below by the row's first or last column.
  uint32_t b[17];
  const uint2 l = *reinterpret_cast<const uint2 *>(row + 3 * x0 - 8);
  const uint4 m0 = *reinterpret_cast<const uint4 *>(row + 3 * x0);
  const uint4 m1 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 16);
  const uint4 m2 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 32);
  const uint2 r = *reinterpret_cast<const uint2 *>(row + 3 * x0 + 48);
  b[0] = l.x; b[1] = l.y;
  b[2] = m0.x; b[3] = m0.y; b[4] = m0.z; b[5] = m0.w;
  b[6] = m1.x; b[7] = m1.y; b[8] = m1.z; b[9] = m1.w;
  b[10] = m2.x; b[11] = m2.y; b[12] = m2.z; b[13] = m2.w;
  b[14] = r.x; b[15] = r.y; b[16] = r.y;
  uint32_t y[20];
#pragma unroll
  for (int j = 0; j < 20; ++j) {
    const int o = 2 + 3 * j, q = o >> 2;
    uint32_t w;
    switch (o & 3) {
      case 0: w = rgbg_at<0>(b[q], b[q + 1]); break;
      case 1: w = rgbg_at<1>(b[q], b[q + 1]); break;
      case 2: w = rgbg_at<2>(b[q], b[q + 1]); break;
      default: w = rgbg_at<3>(b[q], b[q + 1]); break;
    }
    y[j] = luma_rgbg(w);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    yp[2 * q] = __byte_perm(y[4 * q], y[4 * q + 2], 0x5410);
    yp[2 * q + 1] = __byte_perm(y[4 * q + 1], y[4 * q + 3], 0x5410);
  }
  // clamp to the row: the columns before 0 and after W-1 take column 0 and column W-1
  // (window column j sits in word 2 * (j / 4) + j % 2, high lane when j / 2 is odd)
  if (__any_sync(0xFFFFFFFFu, x0 == 0 || x0 + 18 > W)) {
    if (x0 == 0) {  // window columns 0 and 1 (low lanes of words 0 and 1) <- window column 2
      const uint32_t yf = yp[0] >> 16;
      yp[0] = (yp[0] & 0xFFFF0000u) | yf;
      yp[1] = (yp[1] & 0xFFFF0000u) | yf;
    }
    if (x0 + 16 == W) {  // window columns 18 and 19 (high lanes of words 8, 9) <- column 17
      const uint32_t yl = yp[9] << 16;
      yp[8] = (yp[8] & 0xFFFFu) | yl;
      yp[9] = (yp[9] & 0xFFFFu) | yl;
    } else if (x0 + 18 > W) {
      const uint8_t *pl = row + 3 * (W - 1);
      const uint32_t ylast = luma8(pl[0], pl[1], pl[2]);
#pragma unroll
      for (int j = 3; j < 20; ++j) {
        const int w = 2 * (j >> 2) + (j & 1), sh = 16 * ((j >> 1) & 1);
        if (x0 - 2 + j > W - 1) yp[w] = (yp[w] & ~(0xFFFFu << sh)) | (ylast << sh);
      }
    }
  }
}

// Luminance of the 16 columns x0 .. x0+15 of a row in shared memory, packed 4 per word
// (columns past the row's end take whatever their bytes give: they are never used).
__device__ __forceinline__ uint4 luma16(const uint8_t *row, int x0) {
  const uint4 m0 = *reinterpret_cast<const uint4 *>(row + 3 * x0);
  const uint4 m1 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 16);
  const uint4 m2 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 32);
  const uint32_t b[13] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y, m2.z, m2.w, m2.w};
  uint32_t y[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int o = 3 * j, q = o >> 2;
    uint32_t w;
    switch (o & 3) {
      case 0: w = rgbg_at<0>(b[q], b[q + 1]); break;
      case 1: w = rgbg_at<1>(b[q], b[q + 1]); break;
      case 2: w = rgbg_at<2>(b[q], b[q + 1]); break;
      default: w = rgbg_at<3>(b[q], b[q + 1]); break;
    }
    y[j] = luma_rgbg(w);
  }
  uint32_t d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    d[k] = __byte_perm(__byte_perm(y[4 * k], y[4 * k + 1], 0x0040), __byte_perm(y[4 * k + 2], y[4 * k + 3], 0x0040),
                       0x5410);
  return make_uint4(d[0], d[1], d[2], d[3]);
}

// Horizontal binomial [1 4 6 4 1] of one row's luminance, before rounding: from the 10
// pair words of the window x0-2 .. x0+17 (luma20's layout) to the 16 own columns as 8 pair
// words, h[2k] = columns (4k, 4k+2), h[2k+1] = (4k+1, 4k+3).  Sums stay below 16 * 255.
__device__ __forceinline__ void binom_h(const uint32_t (&Y)[10], uint32_t (&h)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t E0 = Y[2 * k], O0 = Y[2 * k + 1], E1 = Y[2 * k + 2], O1 = Y[2 * k + 3];
    const uint32_t se = __byte_perm(E0, E1, 0x5432);  // window columns (4k+2, 4k+4)
    const uint32_t so = __byte_perm(O0, O1, 0x5432);  // (4k+3, 4k+5)
    h[2 * k] = E0 + E1 + 4u * (O0 + so) + 6u * se;      // own columns 4k, 4k+2
    h[2 * k + 1] = O0 + O1 + 4u * (se + E1) + 6u * so;  // own columns 4k+1, 4k+3
  }
}

// Vertical binomial [1 4 6 4 1] of the row sums as four cascaded [1 1] sums over the
// stream of rows, on the 8 pair words of binom_h.  After row n is fed, p0 = h(n),
// p1 = h(n-1) + h(n), p2 and p3 the next sums; feeding row n+1 returns
// sum_i C(4,i) h(n-3+i), the full 5x5 sum centred on row n-1 (at most 256 * 255, so the
// lanes never carry into each other).  The state is updated in place: the new p3 is the
// sum minus the old p3, each lower level the level above minus its old value.
struct VCascade {
  uint32_t p0[8], p1[8], p2[8], p3[8];

  // the state as 32 words (kept in tensor memory between rows by the fixed-set instances)
  __device__ __forceinline__ void get(uint32_t (&t)[32]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      t[i] = p0[i];
      t[8 + i] = p1[i];
      t[16 + i] = p2[i];
      t[24 + i] = p3[i];
    }
  }
  __device__ __forceinline__ void set(const uint32_t (&t)[32]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      p0[i] = t[i];
      p1[i] = t[8 + i];
      p2[i] = t[16 + i];
      p3[i] = t[24 + i];
    }
  }

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 8; ++i) p0[i] = p1[i] = p2[i] = p3[i] = 0u;
  }
  __device__ __forceinline__ void feed(const uint32_t (&h)[8], uint32_t (&V)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t v = p3[i] + p2[i] + p1[i] + p0[i] + h[i];
      p3[i] = v - p3[i];
      p2[i] = p3[i] - p2[i];
      p1[i] = p2[i] - p1[i];
      p0[i] = p1[i] - p0[i];
      V[i] = v;
    }
  }
  // feeds the newest row again (the image's last row repeated below the image)
  __device__ __forceinline__ void feed_repeat(uint32_t (&V)[8]) {
    uint32_t h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = p0[i];
    feed(h, V);
  }
};

// The depth of the 16 own columns from the 5x5 sums: D = (sum + 128) >> 8, packed 4 per
// word.  Both lanes of a sum word stay below 65536 after the rounding offset, so byte 1 of
// each lane is its rounded result.
__device__ __forceinline__ uint4 round_depth(const uint32_t (&V)[8]) {
  uint32_t d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = __byte_perm(V[2 * k] + 0x00800080u, V[2 * k + 1] + 0x00800080u, 0x7351);
  return make_uint4(d[0], d[1], d[2], d[3]);
}

// Packed RGB (3 bytes) of column x of a row in global memory (byte loads: nothing past the
// pixel is read).
__device__ __forceinline__ uint32_t rgb_at_global(const uint8_t *row, int x) {
  const uint8_t *p = row + 3 * static_cast<int64_t>(x);
  return static_cast<uint32_t>(p[0]) | (static_cast<uint32_t>(p[1]) << 8) | (static_cast<uint32_t>(p[2]) << 16);
}

// Sixteen 3-byte colours (low bytes of c[i]) packed into 12 words.
__device__ __forceinline__ void pack16(const uint32_t (&c)[16], uint32_t (&w)[12]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[3 * k] = __byte_perm(c[4 * k], c[4 * k + 1], 0x4210);
    w[3 * k + 1] = __byte_perm(c[4 * k + 1], c[4 * k + 2], 0x5421);
    w[3 * k + 2] = __byte_perm(c[4 * k + 2], c[4 * k + 3], 0x6542);
  }
}

// Rounded-up per-byte mean of two packed colours: (a + b + 1) >> 1 in every byte.
__device__ __forceinline__ uint32_t avg_up(uint32_t a, uint32_t b) {
  return (a | b) - (((a ^ b) >> 1) & 0x7F7F7F7Fu);
}

template <int N>
__device__ __forceinline__ void store_bytes(uint8_t *p, const uint32_t (&w)[N], int nbytes) {
#pragma unroll
  for (int b = 0; b < 4 * N; ++b)
    if (b < nbytes) p[b] = static_cast<uint8_t>(bsel(w, b));
}

// 16 packed colours (48 bytes) at p: three 16-byte stores when the chunk is whole and
// the row 16-byte aligned (`fast`), else byte stores of the npx pixels.
__device__ __forceinline__ void store48(uint8_t *p, const uint32_t (&w)[12], int npx, bool fast) {
  if (fast) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    q[0] = make_uint4(w[0], w[1], w[2], w[3]);
    q[1] = make_uint4(w[4], w[5], w[6], w[7]);
    q[2] = make_uint4(w[8], w[9], w[10], w[11]);
  } else {
    store_bytes(p, w, 3 * npx);
  }
}

__device__ __forceinline__ void store24(uint8_t *p, const uint32_t (&w)[6], int npx) {
  if (npx == 8 && (reinterpret_cast<uintptr_t>(p) & 7u) == 0) {
    uint2 *q = reinterpret_cast<uint2 *>(p);
    q[0] = make_uint2(w[0], w[1]);
    q[1] = make_uint2(w[2], w[3]);
    q[2] = make_uint2(w[4], w[5]);
  } else {
    store_bytes(p, w, 3 * npx);
  }
}

__device__ __forceinline__ void store16(uint8_t *p, uint4 v, int npx) {
  if (npx == 16 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
    *reinterpret_cast<uint4 *>(p) = v;
  } else {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    store_bytes(p, w, npx);
  }
}

// Bit j of m set for every entry of k that is not kEmpty: a compare and a predicated OR
// per entry.
__device__ __forceinline__ uint32_t filled_mask(const uint32_t (&k)[16]) {
  uint32_t m = 0u;
#pragma unroll
  for (int j = 0; j < 16; ++j)
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, -1;\n\t@p or.b32 %0, %0, %2;\n\t}" : "+r"(m) : "r"(k[j]), "r"(1u << j));
  return m;
}

// Left to right over the 16 entries of both views (two independent chains): an empty
// entry takes the last filled entry before it (c0, c1: the entries carried in).  Columns
// past the row's end come last, so whatever they hold changes no column of the row.
__device__ __forceinline__ void carry_right2(uint32_t (&k0)[16], uint32_t (&k1)[16], uint32_t c0, uint32_t c1) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, -1;\n\tselp.b32 %1, %0, %1, p;\n\tmov.b32 %0, %1;\n\t}"
        : "+r"(k0[j]), "+r"(c0));
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, -1;\n\tselp.b32 %1, %0, %1, p;\n\tmov.b32 %0, %1;\n\t}"
        : "+r"(k1[j]), "+r"(c1));
  }
}

// Right to left over both views: c carries the last entry whose bit of m is set (the
// filled targets of the row; c0, c1: the entries carried in), and an entry whose bit is
// clear takes c where c is strictly farther (c > (k | 0xFFFFFF)).
__device__ __forceinline__ void carry_left_farther2(uint32_t (&k0)[16], uint32_t (&k1)[16], uint32_t m0, uint32_t m1,
                                                    uint32_t c0, uint32_t c1) {
#pragma unroll
  for (int j = 15; j >= 0; --j) {
    asm("{\n\t.reg .pred p, q;\n\t.reg .b32 t;\n\tand.b32 t, %2, %3;\n\tsetp.ne.u32 p, t, 0;\n\t"
        "selp.b32 %1, %0, %1, p;\n\tor.b32 t, %0, 0xFFFFFF;\n\tsetp.gt.u32 q, %1, t;\n\t"
        "selp.b32 %0, %1, %0, q;\n\t}"
        : "+r"(k0[j]), "+r"(c0) : "r"(m0), "r"(1u << j));
    asm("{\n\t.reg .pred p, q;\n\t.reg .b32 t;\n\tand.b32 t, %2, %3;\n\tsetp.ne.u32 p, t, 0;\n\t"
        "selp.b32 %1, %0, %1, p;\n\tor.b32 t, %0, 0xFFFFFF;\n\tsetp.gt.u32 q, %1, t;\n\t"
        "selp.b32 %0, %1, %0, q;\n\t}"
        : "+r"(k1[j]), "+r"(c1) : "r"(m1), "r"(1u << j));
  }
}

// A red.shared.min at a + OFF when pred holds (no branch).
template <int OFF>
__device__ __forceinline__ void reds_min_at_if(uint32_t a, uint32_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %2, 0;\n\t"
      "@p red.shared.min.u32 [%0+%3], %1;\n\t}" ::"r"(a),
      "r"(v), "r"(static_cast<uint32_t>(pred)), "n"(OFF)
      : "memory");
}

// Four consecutive 32-column steps G*4 .. G*4+3 of a lane's sources in the forward warp:
// 255 - depth from the depth row (ds), colour words from the input row (cws, the colour
// at bit offset sh), the two target offsets from the table (ls), atomics into the left
// (bl) and right (br) z-buffers at the sources' own columns plus the offsets.  All
// shared loads come before the atomics.
template <int G>
__device__ __forceinline__ void scatter4(uint32_t ds, uint32_t cws, uint32_t sh, uint32_t ls, uint32_t bl,
                                         uint32_t br) {
  uint32_t fv[4], cw[8];
  lds_u8_step32x4(ds + 128 * G, fv);
  lds_u32_pair_step96x4(cws + 384 * G, cw);
  uint2 lt[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) lt[j] = lds_u32x2(ls + 8u * fv[j]);
  uint32_t e[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) e[j] = __byte_perm(__funnelshift_r(cw[2 * j], cw[2 * j + 1], sh), fv[j], 0x4210);
  reds_min_at<128 * (4 * G + 0)>(bl + lt[0].x, e[0]);
  reds_min_at<128 * (4 * G + 0)>(br + lt[0].y, e[0]);
  reds_min_at<128 * (4 * G + 1)>(bl + lt[1].x, e[1]);
  reds_min_at<128 * (4 * G + 1)>(br + lt[1].y, e[1]);
  reds_min_at<128 * (4 * G + 2)>(bl + lt[2].x, e[2]);
  reds_min_at<128 * (4 * G + 2)>(br + lt[2].y, e[2]);
  reds_min_at<128 * (4 * G + 3)>(bl + lt[3].x, e[3]);
  reds_min_at<128 * (4 * G + 3)>(br + lt[3].y, e[3]);
}

// One image's arguments as the band routine sees them (built from the kernel
// parameters for a single image, from a descriptor in device memory for a batch).
struct Job {
  const uint8_t *in;
  int64_t in_pitch;
  const CUtensorMap *tmap;  // tensor-box load modes only
  const uint8_t *depth_in;
  int64_t depth_in_pitch;
  uint8_t *out[O_COUNT];
  int64_t out_pitch, depth_pitch;
  int W, H, nch, row_bytes, load_mode, nbox, box_bytes, box_step;
  uint32_t outputs;
  int l2_prefetch, fast_store;
};

// Shared-memory regions of one CTA.
struct Shm {
  uint64_t *full;   // ring-slot mbarriers
  uint64_t *bdone;  // [2] every warp has scattered the row (B)
  uint64_t *sdone;  // [2] every warp has published its summary and cleared its targets (C)
  uint2 *lut;       // per 255 - depth: byte offsets of the left / right targets
  int32_t *lut_n;   // Fig. 3 gather: 510 * s_L(d) (in the z-buffer region)
  uint8_t *wsum;    // [parity][view][warp] uint4 {has, first entry, last entry, 0}
  uint8_t *ring, *drow;
  uint32_t zb;      // shared address of the z-buffer region
  int nb, srow, zlen, zstride, zguard;
};

__device__ __forceinline__ Shm carve(uint8_t *smem, int nb, int srow, int nch, int nwarps, int zguard) {
  const BandSmem L = band_smem_layout(nb, srow, nch, nwarps, zguard);
  Shm m;
  m.full = reinterpret_cast<uint64_t *>(smem + L.bar);
  m.bdone = reinterpret_cast<uint64_t *>(smem + L.flags + 8);
  m.sdone = reinterpret_cast<uint64_t *>(smem + L.flags + 24);
  m.lut = reinterpret_cast<uint2 *>(smem + L.lut);
  m.wsum = smem + L.wsum;
  m.ring = smem + L.ring;
  m.drow = smem + L.drow;
  m.zb = smem_addr(smem + L.zb);
  m.lut_n = reinterpret_cast<int32_t *>(smem + L.zb);
  m.nb = nb;
  m.srow = srow;
  m.zlen = nch * kChunk;
  m.zstride = L.zstride;
  m.zguard = zguard;
  return m;
}

// Shift tables into shared memory (all threads; a barrier must follow).  lut[255 - d] =
// {4 * (-hL[d]), 4 * (-hR[d])}: a source at column x with depth d lands on target x - h.
template <bool FWD>
__device__ __forceinline__ void fill_luts(const Shm &m, const int32_t *lut_h, const int32_t *lut_n) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    if (FWD) {
      const int32_t h = lut_h[255 - i];
      const int nl = -static_cast<int16_t>(h & 0xFFFF), nr = -(h >> 16);  // |h| <= 512
      m.lut[i] = make_uint2(static_cast<uint32_t>(4 * nl), static_cast<uint32_t>(4 * nr));
    } else {
      m.lut_n[i] = lut_n[i];
    }
  }
}

// Every thread's wait on an mbarrier phase, the outcome agreed within the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, unsigned long long timeout_ns) {
  if (__all_sync(kAll, mbar_attempt(bar, parity, timeout_ns))) return true;
  const unsigned long long t0 = __shfl_sync(kAll, global_ns(), 0);
  while (true) {
    if (__all_sync(kAll, mbar_attempt(bar, parity, timeout_ns))) return true;
    if (__shfl_sync(kAll, global_ns(), 0) - t0 > timeout_ns) return false;
  }
}

// Rows [ys, ye) of one image, every stage of the pipeline (see the file comment).  All
// threads of the CTA call it together.  kbase counts the ring loads this CTA issued
// before (the slot and mbarrier phase of a load follow from it), nrows the rows the CTA
// processed before (each per-row mbarrier completes one phase per row); both are advanced
// here.  Returns false when a bounded wait gave up (the status word is set and the copies
// in flight have landed).
// OUTS: the requested outputs when fixed at compile time (the stereo set, every output row
// 16-byte aligned: whole chunks stored as 16-byte words), 0 when read from the arguments.
//
// TM: the vertical cascade's 32 words wait in tensor memory (at tmem, this thread's lane)
// between one row's A and the next, so that B and C have those registers.
template <int DS, bool FWD, uint32_t OUTS = 0, bool TM = false>
__device__ __forceinline__ bool run_band(const Job &a, const Shm &m, int ys, int ye, uint32_t &kbase,
                                         uint32_t &nrows, int *status,
                                         unsigned long long timeout_ns, uint32_t tmem = 0u) {
  constexpr bool binom = DS == DS_BINOM5;
  const int tid = threadIdx.x, nc = blockDim.x, W = a.W, H = a.H, nb = m.nb;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nc >> 5;
  const int halo = binom ? 2 : 0;
  const int la = max(ys - halo, 0), lb = min(ye + halo, H);
  const int nload = lb - la;
  const uint32_t k0 = kbase;
  // g / nb as umulhi(g, ceil(2^32 / nb)): exact while g * (nb - 1) < 2^32, far beyond the
  // loads one CTA makes in a launch
  const uint32_t ring_rcp = 0xFFFFFFFFu / static_cast<uint32_t>(nb) + 1u;
  auto ring_div = [&](uint32_t g) { return __umulhi(g, ring_rcp); };

  // Row k = r - la of the band is the (k0 + k)-th load of this CTA: slot (k0+k) % nb.
  // The middle warp issues the loads of rows [issued, upto) (the warps at the row's ends
  // have the most fill work); every earlier occupant of those slots has been released by
  // all warps (every warp has scattered it: the bdone mbarrier, or a CTA barrier).
  int issued = 0;
  const int lw = 32 * (nwarps >> 1);  // first thread of the loading warp
  const bool loader = __shfl_sync(kAll, (tid >> 5) == (nwarps >> 1), 0);
  auto issue_loads = [&](int upto) {
    upto = min(upto, nload);
    if (tid == lw && issued == 0 && a.load_mode != LM_BULK) prefetch_tensormap(a.tmap);
    for (int k = issued; k < upto; ++k) {
      const uint32_t g = k0 + k;
      const int s = static_cast<int>(g - ring_div(g) * nb);
      uint8_t *dst = m.ring + s * m.srow;
      if (a.load_mode == LM_BULK) {
        if (tid == lw) {
          mbar_arrive_expect_tx(&m.full[s], static_cast<uint32_t>(a.row_bytes));
          bulk_load(dst, a.in + static_cast<int64_t>(la + k) * a.in_pitch, static_cast<uint32_t>(a.row_bytes),
                    &m.full[s]);
        }
      } else {
        if (tid == lw) mbar_arrive_expect_tx(&m.full[s], static_cast<uint32_t>(a.nbox * a.box_bytes));
        __syncwarp();
        for (int i = tid - lw; i < a.nbox; i += 32) {
          if (a.load_mode == LM_T3)
            tma_load_3d(dst + i * a.box_bytes, a.tmap, 0, i * a.box_step, la + k, &m.full[s]);
          else
            tma_load_2d(dst + i * a.box_bytes, a.tmap, i * a.box_step, la + k, &m.full[s]);
        }
      }
    }
    if (upto > issued) issued = upto;
  };
  if (loader) {
    issue_loads(nb);
    // optionally, the band's later rows go to L2 now
    if (a.l2_prefetch) {
      if (a.load_mode == LM_BULK) {
        for (int k = nb + lane; k < nload; k += 32)
          bulk_prefetch_l2(a.in + static_cast<int64_t>(la + k) * a.in_pitch, static_cast<uint32_t>(a.row_bytes));
      } else {
        for (int j = lane; j < (nload - nb) * a.nbox; j += 32) {
          const int k = nb + j / a.nbox, i = j % a.nbox;
          if (a.load_mode == LM_T3) tma_prefetch_3d(a.tmap, 0, i * a.box_step, la + k);
          else tma_prefetch_2d(a.tmap, i * a.box_step, la + k);
        }
      }
    }
  }

  const int x0 = tid * kChunk;
  const int npx = max(0, min(kChunk, W - x0));
  const bool active = npx > 0;
  const bool own_chunk = tid < a.nch;            // the thread's chunk exists (active or not)
  // the warp's 32 chunks are all whole (every warp of a row but possibly the last):
  // warp-uniform fast paths for its depth row, clears and stores
  const bool wfull = __all_sync(kAll, npx == kChunk);
  const bool fast_store = OUTS ? true : a.fast_store != 0;
  const bool wfast = wfull && fast_store;
  const int x0c = min(x0, (a.nch - 1) * kChunk);  // clamped: loads stay inside the buffers
  const int warp_lo = (tid & ~31) * kChunk;
  const int warp_hi = min(W, warp_lo + 32 * kChunk);
  bool timed_out = false;
  auto slot = [&](int r) {
    const uint32_t g = k0 + (r - la);
    return m.ring + (g - ring_div(g) * nb) * m.srow;
  };
  auto wait_row = [&](int r) {
    const uint32_t g = k0 + (r - la), q = ring_div(g);
    if (!warp_wait(&m.full[g - q * nb], q & 1, timeout_ns)) timed_out = true;
  };
  // shared address of target 0 of the z-buffer row of parity p, view v
  auto zrow = [&](int p, int v) { return m.zb + 4u * static_cast<uint32_t>(m.zguard + (2 * p + v) * m.zstride); };

  const uint32_t outs = OUTS ? OUTS : a.outputs;
  const bool want_depth = (outs & DIBR_OUT_DEPTH) != 0;
  const bool want_holes = (outs & DIBR_OUT_HOLES) != 0;
  const bool want_ana = (outs & DIBR_OUT_ANAGLYPH) != 0;
  const bool want_l = (outs & DIBR_OUT_LEFT) != 0;
  const bool want_r = (outs & DIBR_OUT_RIGHT) != 0;
  const bool want_hsbs = (outs & DIBR_OUT_HSBS) != 0;

  // every z-buffer target empty (later rows: C clears its targets once it has read them)
  if (FWD) {
    const uint4 e = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
    for (int i = tid; 4 * i < m.zlen; i += nc) {  // groups of 4 targets
#pragma unroll
      for (int r = 0; r < 4; ++r) sts_u32x4(zrow(r >> 1, r & 1) + 16u * i, e);
    }
  }
  VCascade vc;
  vc.clear();
  if (binom) {
    // rows clamp(ys-2) .. clamp(ys+1) into the cascade, each as soon as it has landed
#pragma unroll 1
    for (int i = -2; i <= 1; ++i) {
      const int r = min(max(ys + i, 0), H - 1);
      if (r >= la && r < lb && (i == -2 || r != min(max(ys + i - 1, 0), H - 1))) wait_row(r);
      uint32_t yq[10], hq[8], V[8];
      luma20(slot(r), x0c, W, yq);
      binom_h(yq, hq);
      vc.feed(hq, V);
    }
    if (TM) {
      uint32_t t[32];
      vc.get(t);
      tmem_store32(tmem, t);
    }
  }
  // the cleared z-buffers (and, with the binomial, the rows above the band) are done with
  bool aborted = consumer_sync_or(timed_out, nc);
  if (!aborted && loader) issue_loads((ys - la) + nb);

  const uint32_t ltm = lanemask_lt(), gtm = lanemask_gt();

  // The per-row mbarriers come in pairs: the CTA's r-th row (r = nrows + y - ys) uses
  // barrier r & 1 of a pair, phase r >> 1, so that phases of rows two apart never meet.
  auto rix = [&](int y) { return nrows + static_cast<uint32_t>(y - ys); };
  auto bbar = [&](int y) { return m.bdone + (rix(y) & 1u); };
  auto sbar = [&](int y) { return m.sdone + (rix(y) & 1u); };
  auto par = [&](int y) { return (rix(y) >> 1) & 1u; };
  auto arrive_b = [&](int y) { mbar_arrive(bbar(y)); };

  // ---- A: the depth of row y (registers, 4 per word), 255 - depth into the depth row
  auto phase_a = [&](int y) -> uint4 {
    uint4 d;
    if (binom) {
      const int r2 = y + 2;
      uint32_t t[32];
      if (TM) tmem_load32(tmem, t);  // the cascade back (waited for just before it is fed)
      if (r2 < lb) wait_row(r2);
      uint32_t V[8];
      if (r2 < H) {
        uint32_t yq[10], hq[8];
        luma20(slot(r2), x0c, W, yq);
        binom_h(yq, hq);
        if (TM) {
          tmem_load_wait32(t);
          vc.set(t);
        }
        vc.feed(hq, V);
      } else {
        if (TM) {
          tmem_load_wait32(t);
          vc.set(t);
        }
        vc.feed_repeat(V);  // rows below the image repeat row H-1
      }
      if (TM) {
        vc.get(t);
        tmem_store32(tmem, t);
      }
      d = round_depth(V);
    } else if (DS == DS_LUMA) {
      wait_row(y);
      d = luma16(slot(y), x0c);
    } else {
      wait_row(y);  // B reads the row's colours
      d = make_uint4(0u, 0u, 0u, 0u);
      if (active) {
        const uint8_t *dp = a.depth_in + static_cast<int64_t>(y) * a.depth_in_pitch + x0;
        if (npx == kChunk && (reinterpret_cast<uintptr_t>(dp) & 15u) == 0) {
          d = *reinterpret_cast<const uint4 *>(dp);
        } else {
          uint32_t w[4] = {0u, 0u, 0u, 0u};
          for (int i = 0; i < npx; ++i) w[i >> 2] |= static_cast<uint32_t>(dp[i]) << (8 * (i & 3));
          d = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    if (want_depth && active) store16(a.out[O_DEPTH] + static_cast<int64_t>(y) * a.depth_pitch + x0, d, npx);
    if (FWD && (wfull || own_chunk)) *reinterpret_cast<uint4 *>(m.drow + x0) = make_uint4(~d.x, ~d.y, ~d.z, ~d.w);
    return d;
  };

  // ---- B: the forward warp of row y: the warp's 512 sources, consecutive lanes on
  // consecutive columns, so that the atomics of one instruction land on distinct banks
  // (shifts vary slowly); all shared loads of four steps are issued before their atomics
  auto phase_b = [&](int y) {
    if (!FWD) return;
    // every warp has cleared its targets of row y - 2, the previous user of this z-buffer
    // (the band's first two rows use the buffers cleared before the band)
    if (y >= ys + 2 && !warp_wait(m.sdone + (rix(y - 2) & 1u), par(y - 2), timeout_ns)) timed_out = true;
    const int xb = warp_lo + lane;
    const uint32_t ob = 3u * static_cast<uint32_t>(xb);
    const uint32_t cws = smem_addr(slot(y)) + (ob & ~3u);  // the lane's colours: +96 bytes per step
    const uint32_t sh = (ob & 3u) * 8u;
    const uint32_t ds = smem_addr(m.drow) + static_cast<uint32_t>(xb);
    const uint32_t ls = smem_addr(m.lut);
    const int p = y & 1;
    const uint32_t bl = zrow(p, 0) + 4u * static_cast<uint32_t>(xb);
    const uint32_t br = zrow(p, 1) + 4u * static_cast<uint32_t>(xb);
    if (warp_hi - warp_lo == 32 * kChunk) {
      scatter4<0>(ds, cws, sh, ls, bl, br);
      scatter4<1>(ds, cws, sh, ls, bl, br);
      scatter4<2>(ds, cws, sh, ls, bl, br);
      scatter4<3>(ds, cws, sh, ls, bl, br);
    } else {
      // the row's last, partial warp: columns from warp_hi on do not exist (their loads
      // read column warp_hi - 1, so that they stay in the row; their atomics are skipped)
      const uint32_t rs = smem_addr(slot(y)), dr = smem_addr(m.drow);
      const int ng = (warp_hi - warp_lo + 127) >> 7;  // groups of 4 x 32 columns holding some
#pragma unroll 1
      for (int g = 0; g < ng; ++g) {
        uint32_t fv[4], cw[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t xc = static_cast<uint32_t>(min(xb + 32 * (4 * g + j), warp_hi - 1));
          const uint32_t ca = rs + ((3u * xc) & ~3u);
          fv[j] = lds_u8(dr + xc);
          cw[2 * j] = lds_u32(ca);
          cw[2 * j + 1] = lds_u32(ca + 4);
        }
        uint2 lt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) lt[j] = lds_u32x2(ls + 8u * fv[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = xb + 32 * (4 * g + j) < warp_hi;
          const uint32_t e = __byte_perm(__funnelshift_r(cw[2 * j], cw[2 * j + 1], sh), fv[j], 0x4210);
          const uint32_t off = 512u * static_cast<uint32_t>(g) + 128u * j;
          reds_min_at_if<0>(bl + off + lt[j].x, e, in);
          reds_min_at_if<0>(br + off + lt[j].y, e, in);
        }
      }
    }
  };

  // ---- C: row y's targets: winners, hole fill, formatting, stores
  auto wsum_at = [&](int p, int v, int w) { return smem_addr(m.wsum) + 16u * static_cast<uint32_t>((p * 2 + v) * nwarps + w); };

  // this lane's clears: 16 bytes at warp_lo + 4 * lane + 128 q targets, q = 0..3
  const uint32_t clr_off = 4u * static_cast<uint32_t>(warp_lo + 4 * lane);
  auto phase_c = [&](int y, uint4 d) {
    // every warp has scattered row y: its targets are final and its ring slot is free
    if (!warp_wait(bbar(y), par(y), timeout_ns)) timed_out = true;
    if (loader) issue_loads((y - la) + 1 + nb);
    const uint8_t *grow = a.in + static_cast<int64_t>(y) * a.in_pitch;
    const int p = y & 1;
    // Formatting and stores of one view's 16 targets: the view itself, its half of the
    // side-by-side frame and, after the right view, the anaglyph (red from the left view,
    // green and blue from the right: in the packed words, the bytes at offsets 0 mod 3).
    const int64_t ro = static_cast<int64_t>(y) * a.out_pitch;
    const bool fast = wfast || (fast_store && npx == kChunk);
    uint32_t wl[12];
    auto emit_view = [&](int v, const uint32_t (&kv)[16]) {
      if (!wfull && !active) return;
      uint32_t w[12];
      pack16(kv, w);
      if (v == 0) {
        if (want_l) store48(a.out[O_LEFT] + ro + 3 * x0, w, npx, fast);
#pragma unroll
        for (int i = 0; i < 12; ++i) wl[i] = w[i];
      } else {
        if (want_r) store48(a.out[O_RIGHT] + ro + 3 * x0, w, npx, fast);
        if (want_ana) {
          uint32_t wa[12];
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            const uint32_t M = i % 3 == 0 ? 0xFF0000FFu : i % 3 == 1 ? 0x00FF0000u : 0x0000FF00u;
            wa[i] = (wl[i] & M) | (w[i] & ~M);
          }
          store48(a.out[O_ANA] + ro + 3 * x0, wa, npx, fast);
        }
      }
      if (want_hsbs) {
        uint32_t c8[8], h6[6];
#pragma unroll
        for (int j = 0; j < 8; ++j) c8[j] = avg_up(kv[2 * j], kv[2 * j + 1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          h6[3 * q] = __byte_perm(c8[4 * q], c8[4 * q + 1], 0x4210);
          h6[3 * q + 1] = __byte_perm(c8[4 * q + 1], c8[4 * q + 2], 0x5421);
          h6[3 * q + 2] = __byte_perm(c8[4 * q + 2], c8[4 * q + 3], 0x6542);
        }
        // W is even, so chunks hold whole pairs; the left view fills the left half
        store24(a.out[O_HSBS] + ro + 3 * ((v == 0 ? 0 : W / 2) + x0 / 2), h6, npx / 2);
      }
    };
    uint32_t k[2][16];
    uint32_t hole[2] = {0u, 0u};
    if (FWD) {
      const uint32_t rowmask = npx >= kChunk ? 0xFFFFu : ((1u << npx) - 1u);
      uint32_t mm[2], fe[2], cl[2], cr[2], lanes[2];

#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const uint32_t za = zrow(p, v) + 4u * static_cast<uint32_t>(x0c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 u = lds_u32x4(za + 16u * q);
          k[v][4 * q] = u.x; k[v][4 * q + 1] = u.y; k[v][4 * q + 2] = u.z; k[v][4 * q + 3] = u.w;
        }
        const uint32_t mk = filled_mask(k[v]) & rowmask;
        // the chunk's first and last filled entries, for the neighbouring lanes
        const int fj = __ffs(mk) - 1, lj = 31 - __clz(mk);
        fe[v] = lds_u32(za + 4u * static_cast<uint32_t>(fj & 15));
        const uint32_t le = lds_u32(za + 4u * static_cast<uint32_t>(lj & 15));
        const uint32_t ln = __ballot_sync(kAll, mk != 0u);
        const uint32_t lower = ln & ltm, upper = ln & gtm;
        cl[v] = __shfl_sync(kAll, le, (31 - __clz(lower)) & 31);
        cr[v] = __shfl_sync(kAll, fe[v], (__ffs(upper) - 1) & 31);
        const uint32_t wf = __shfl_sync(kAll, fe[v], (__ffs(ln) - 1) & 31);
        const uint32_t wl = __shfl_sync(kAll, le, (31 - __clz(ln)) & 31);
        sts_u32x4(wsum_at(p, v, warp), make_uint4(ln != 0u ? 1u : 0u, wf, wl, 0u));  // (same value, every lane)
        mm[v] = mk;
        lanes[v] = ln;
      }
      // this warp's targets are read: clear them for row y + 2 (consecutive lanes on
      // consecutive 16-byte words: no bank conflicts), then tell the other warps that its
      // summary is published and its targets are clear
      __syncwarp();
      const uint4 e4 = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
      const uint32_t c0 = zrow(p, 0) + clr_off, c1 = zrow(p, 1) + clr_off;
      if (wfull) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sts_u32x4(c0 + 512u * q, e4);
          sts_u32x4(c1 + 512u * q, e4);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (warp_lo + 4 * (32 * q + lane) < m.zlen) {
            sts_u32x4(c0 + 512u * q, e4);
            sts_u32x4(c1 + 512u * q, e4);
          }
      }
      mbar_arrive(sbar(y));
      // entries from outside the warp, for lanes whose leading (trailing) holes have no
      // filled target below (above) them in the warp: the nearest warp's last (first)
      // filled entry, from the summaries -- only where a warp below (above) exists: the
      // holes at the row's ends need nothing from the other warps
      bool need = false;
      const bool below_exists = warp_lo > 0, above_exists = warp_hi < W;
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const uint32_t lower = lanes[v] & ltm, upper = lanes[v] & gtm;
        need |= active && ((below_exists && lower == 0u && !(mm[v] & 1u)) ||
                           (above_exists && upper == 0u && !((mm[v] >> ((npx - 1) & 15)) & 1u)));
      }
      uint32_t wle[2] = {0u, 0u}, wre[2] = {0u, 0u};
      bool wlh[2] = {false, false}, wrh[2] = {false, false};
      if (__any_sync(kAll, need)) {
        if (!warp_wait(sbar(y), par(y), timeout_ns)) timed_out = true;
        // lane w reads warp w's summary; the nearest warp below / above with a filled target
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const uint4 sm = lds_u32x4(wsum_at(p, v, lane < nwarps ? lane : 0));
          const uint32_t has = __ballot_sync(kAll, lane < nwarps && sm.x != 0u);
          const uint32_t below = has & ((1u << warp) - 1u), above = has & ~((2u << warp) - 1u);
          const uint32_t el = __shfl_sync(kAll, sm.z, (31 - __clz(below)) & 31);
          const uint32_t er = __shfl_sync(kAll, sm.y, (__ffs(above) - 1) & 31);
          wlh[v] = below != 0u;
          wrh[v] = above != 0u;
          wle[v] = below ? el : 0u;
          wre[v] = above ? er : 0u;
        }
      }
      // Hole fill: a hole shows the winner of the nearest filled target on its farther
      // side -- of the nearest filled targets to its left and right, the one whose winner
      // has the smaller depth (the left one on a tie, the only one at a row edge); the
      // input pixel when the row has no filled target.  Two register sweeps: left to right
      // carrying the last filled entry into the holes, then right to left carrying the
      // last filled entry and keeping it where it is strictly farther (entries are
      // (255 - depth) << 24 | colour, so "c strictly farther than k" is the unsigned
      // compare c > (k | 0xFFFFFF)).  A missing right entry carries in as 0, which is never
      // strictly farther; holes with no filled target on their left (the row's start)
      // carry in the first filled entry on their right from the start.  Both views'
      // sweeps run interleaved.
      uint32_t lin[2], rin[2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const uint32_t lower = lanes[v] & ltm, upper = lanes[v] & gtm, mk = mm[v];
        rin[v] = upper ? cr[v] : wre[v];
        lin[v] = lower ? cl[v] : (wlh[v] ? wle[v] : (mk ? fe[v] : rin[v]));
        hole[v] = ~mk & rowmask;
      }
      carry_right2(k[0], k[1], lin[0], lin[1]);
      carry_left_farther2(k[0], k[1], mm[0], mm[1], rin[0], rin[1]);
      // a view of a row without any filled target shows the input row (warp-uniform)
      const bool none0 = lanes[0] == 0u && !wlh[0] && !wrh[0], none1 = lanes[1] == 0u && !wlh[1] && !wrh[1];
      if (none0 || none1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t c = active ? rgb_at_global(grow, min(x0 + j, W - 1)) : 0u;
          if (none0) k[0][j] = c;
          if (none1) k[1][j] = c;
        }
      }
      emit_view(0, k[0]);
      emit_view(1, k[1]);
    } else {
      // Fig. 3 literally: sample trunc(x + s(d)); out of range -> own column
      mbar_arrive(sbar(y));
      const uint32_t dw[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int i = 0; i < kChunk; ++i) {
        const int x = min(x0 + i, W - 1);
        const int n = m.lut_n[bsel(dw, i)];
        int sl = (510 * x + n) / 510, sr = (510 * x - n) / 510;
        if (static_cast<unsigned>(sl) >= static_cast<unsigned>(W)) sl = x;
        if (static_cast<unsigned>(sr) >= static_cast<unsigned>(W)) sr = x;
        k[0][i] = active ? rgb_at_global(grow, sl) : 0u;
        k[1][i] = active ? rgb_at_global(grow, sr) : 0u;
      }
      emit_view(0, k[0]);
      emit_view(1, k[1]);
    }
    if (active && want_holes) {
      // one byte per target: bit 0 a hole of the left view, bit 1 of the right view
      auto spread4 = [](uint32_t x) { return ((x & 0xFu) * 0x00204081u) & 0x01010101u; };
      uint4 hv;
      hv.x = spread4(hole[0]) | (spread4(hole[1]) << 1);
      hv.y = spread4(hole[0] >> 4) | (spread4(hole[1] >> 4) << 1);
      hv.z = spread4(hole[0] >> 8) | (spread4(hole[1] >> 8) << 1);
      hv.w = spread4(hole[0] >> 12) | (spread4(hole[1] >> 12) << 1);
      store16(a.out[O_HOLES] + static_cast<int64_t>(y) * a.depth_pitch + x0, hv, npx);
    }
  };

  uint4 dcur = make_uint4(0u, 0u, 0u, 0u);
  if (!aborted) {
    dcur = phase_a(ys);
    phase_b(ys);
    arrive_b(ys);
  }
  for (int y = ys; y < ye && !aborted && !timed_out; ++y) {
    // the loader refills the slot of row y as soon as every warp has scattered it
    if (loader && __any_sync(kAll, mbar_test(bbar(y), par(y)))) issue_loads((y - la) + 1 + nb);
    const bool more = y + 1 < ye;
    uint4 dnext = make_uint4(0u, 0u, 0u, 0u);
    if (more) {
      dnext = phase_a(y + 1);
      phase_b(y + 1);
      arrive_b(y + 1);
    }
    phase_c(y, dcur);
    dcur = dnext;
  }

  // every thread agrees whether the band completed
  aborted = consumer_sync_or(aborted || timed_out, nc);
  if (aborted) {
    if (tid == lw) {
      atomicOr(status, ST_TIMEOUT_FULL);
      // let every copy this CTA issued land before its shared memory goes away
      for (int k = max(0, issued - nb); k < issued; ++k) {
        const uint32_t g = k0 + k;
        if (!mbar_wait_bounded(&m.full[g % nb], (g / nb) & 1, kDrainLimitNs)) atomicOr(status, ST_TIMEOUT_DRAIN);
      }
    }
    return false;
  }
  kbase = k0 + static_cast<uint32_t>(nload);
  nrows += static_cast<uint32_t>(ye - ys);
  return true;
}

__device__ __forceinline__ void init_barriers(const Shm &m, int nb) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < nb; ++i) mbar_init(&m.full[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(m.bdone + i, blockDim.x);
      mbar_init(m.sdone + i, blockDim.x);
    }
    fence_mbar_init();
  }
}

// ---------------------------------------------------------------------------------
// One image: CTA b owns the rows row0 + [b*n/grid, (b+1)*n/grid), n = row1 - row0.
// TM (fixed-set instances with the binomial depth, bands of kTmemMinRows rows or more): the
// cascade waits in tensor memory between rows.
template <int DS, bool FWD, uint32_t OUTS, bool TM>
__global__ void __launch_bounds__(kMaxConsumers, 1) band_kernel(const __grid_constant__ BandArgs a) {
  static_assert(!TM || (OUTS != 0 && DS == DS_BINOM5), "tensor memory only in the fixed-set binomial instances");
  // The next launch on the stream may start its set-up while this one runs (programmatic
  // dependent launch); it waits below for this one to complete before any global access.
  griddep_launch_dependents();
  extern __shared__ __align__(128) uint8_t smem[];
  const Shm m = carve(smem, a.nb, a.srow, a.nch, blockDim.x >> 5, a.zguard);
  fill_luts<FWD>(m, a.lut_h, a.lut_n);
  init_barriers(m, a.nb);
  __syncthreads();
  // the work before this launch on the stream (whose results may be this launch's inputs,
  // or whose inputs this launch's outputs may overwrite) has completed -- unless the host
  // knows this launch touches none of that launch's buffers; then the wait moves to the
  // end, so that this launch still completes after the previous one
  if (!a.overlap) griddep_wait();
  const int nr = a.row1 - a.row0;
  const int ys = a.row0 + static_cast<int>(static_cast<int64_t>(blockIdx.x) * nr / a.grid);
  const int ye = a.row0 + static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * nr / a.grid);
  if (ys < ye) {
    Job j;
    j.in = a.in;
    j.in_pitch = a.in_pitch;
    j.tmap = &a.tmap;
    j.depth_in = a.depth_in;
    j.depth_in_pitch = a.depth_in_pitch;
#pragma unroll
    for (int i = 0; i < O_COUNT; ++i) j.out[i] = a.out[i];
    j.out_pitch = a.out_pitch;
    j.depth_pitch = a.depth_pitch;
    j.W = a.W; j.H = a.H; j.nch = a.nch; j.row_bytes = a.row_bytes; j.load_mode = a.load_mode;
    j.nbox = a.nbox; j.box_bytes = a.box_bytes; j.box_step = a.box_step;
    j.outputs = a.outputs; j.l2_prefetch = a.l2_prefetch; j.fast_store = a.fast_store;
    uint32_t kbase = 0, nrows = 0;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // 32 columns per group of four warps (a warp reaches only its quarter of the lanes),
    // rounded up to a power of two: at most 128 of the SM's 512 columns per CTA, and
    // 512 / 128 = 4 CTAs of 16 warps would not fit an SM's 2048 threads anyway
    const uint32_t ncols = nwarps <= 4 ? 32u : nwarps <= 8 ? 64u : 128u;
    uint32_t tbase = 0u;
    if (TM) {
      const uint32_t slot_addr = smem_addr(smem + band_smem_layout(a.nb, a.srow, a.nch, nwarps, a.zguard).flags + 48);
      if (warp == 0) tmem_alloc(slot_addr, ncols);
      tmem_fence_before_sync();
      __syncthreads();
      tmem_fence_after_sync();
      tbase = lds_u32(slot_addr);
    }
    const uint32_t tmem = tbase + ((32u * (warp & 3)) << 16) + 32u * (warp >> 2);
    run_band<DS, FWD, OUTS, TM>(j, m, ys, ye, kbase, nrows, a.status, a.timeout_ns, tmem);
    if (TM) {  // every thread's stores have completed (each store waits for itself)
      tmem_fence_before_sync();
      __syncthreads();
      tmem_fence_after_sync();
      if (warp == 0) tmem_dealloc(tbase, ncols);
    }
  }
  if (a.overlap) griddep_wait();
}

// ---------------------------------------------------------------------------------
// A batch of images in one persistent launch: CTAs pull work units (an image and a
// range of its rows) from a device counter until none is left.
// OUTS: every image of the launch has this fixed output set (binomial depth, forward warp,
// aligned rows); 0: each image's own choices.
template <uint32_t OUTS>
__global__ void __launch_bounds__(kMaxConsumers, 1) batch_kernel(BatchArgs b) {
  // The next launch of the batch (another group of images, independent of this one) may be
  // placed as soon as every CTA of this one runs: its CTAs take the SM slots this launch
  // frees while its last units finish, instead of waiting for the last of them.
  griddep_launch_dependents();
  extern __shared__ __align__(128) uint8_t smem[];
  const int nwarps = blockDim.x >> 5;
  // the barriers and the unit word sit at the same place in every image's layout
  const Shm m0 = carve(smem, b.nb, b.srow, b.nch_max, nwarps, b.zguard);
  const int flags = band_smem_layout(b.nb, b.srow, b.nch_max, nwarps, b.zguard).flags;
  int *unit_s = reinterpret_cast<int *>(smem + flags);
  init_barriers(m0, b.nb);
  // a fixed-set batch keeps each unit's binomial cascade in tensor memory between rows
  // (allocated once per CTA, as in the band kernel)
  constexpr bool TM = OUTS != 0;
  const int warp = threadIdx.x >> 5;
  const uint32_t ncols = nwarps <= 4 ? 32u : nwarps <= 8 ? 64u : 128u;
  const uint32_t tslot = smem_addr(smem + flags + 48);
  uint32_t tbase = 0u;
  if (TM) {
    if (warp == 0) tmem_alloc(tslot, ncols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    tbase = lds_u32(tslot);
  }
  const uint32_t tmem = tbase + ((32u * (warp & 3)) << 16) + 32u * (warp >> 2);
  uint32_t kbase = 0, nrows = 0;
  while (true) {
    __syncthreads();  // the previous unit is done with the ring, tables and unit_s
    if (threadIdx.x == 0) *unit_s = atomicAdd(b.counter, 1);
    __syncthreads();
    const int u = *unit_s;
    if (u >= b.n_units) break;
    const int4 un = b.units[u];  // {image, first row, end row}
    const ImageDesc &dsc = b.descs[un.x];
    // this image's layout (its z-buffer rows as wide as its own row, so that its targets
    // past the row's end are the ones its C clears)
    const Shm m = carve(smem, b.nb, b.srow, dsc.nch, nwarps, b.zguard);
    Job j;
    j.in = dsc.in;
    j.in_pitch = dsc.in_pitch;
    j.tmap = nullptr;
    j.depth_in = dsc.depth_in;
    j.depth_in_pitch = dsc.depth_in_pitch;
#pragma unroll
    for (int i = 0; i < O_COUNT; ++i) j.out[i] = dsc.out[i];
    j.out_pitch = dsc.out_pitch;
    j.depth_pitch = dsc.depth_pitch;
    j.W = dsc.W; j.H = dsc.H; j.nch = dsc.nch; j.row_bytes = dsc.row_bytes; j.load_mode = LM_BULK;
    j.nbox = 1; j.box_bytes = dsc.row_bytes; j.box_step = 0;
    j.outputs = dsc.outputs; j.l2_prefetch = 0;
    j.fast_store = ((reinterpret_cast<uintptr_t>(dsc.out[O_ANA]) | reinterpret_cast<uintptr_t>(dsc.out[O_LEFT]) |
                     reinterpret_cast<uintptr_t>(dsc.out[O_RIGHT]) | static_cast<uintptr_t>(dsc.out_pitch)) & 15u) == 0;
    const bool fwd = OUTS ? true : dsc.warp_mode == DIBR_WARP_FORWARD;
    if (fwd) fill_luts<true>(m, dsc.lut_h, dsc.lut_n);
    else fill_luts<false>(m, dsc.lut_h, dsc.lut_n);
    __syncthreads();
    bool ok;
    if (OUTS) ok = run_band<DS_BINOM5, true, OUTS, TM>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns, tmem);
    else switch (dsc.depth_src * 2 + (fwd ? 0 : 1)) {
      case DS_BINOM5 * 2: ok = run_band<DS_BINOM5, true>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
      case DS_BINOM5 * 2 + 1: ok = run_band<DS_BINOM5, false>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
      case DS_LUMA * 2: ok = run_band<DS_LUMA, true>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
      case DS_LUMA * 2 + 1: ok = run_band<DS_LUMA, false>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
      case DS_GLOBAL * 2: ok = run_band<DS_GLOBAL, true>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
      default: ok = run_band<DS_GLOBAL, false>(j, m, un.y, un.z, kbase, nrows, b.status, b.timeout_ns); break;
    }
    if (!ok) break;
  }
  if (TM) {  // every thread's stores have completed (each store waits for itself)
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, ncols);
  }
  // A chained launch's CTAs wait for the previous launch to complete before they exit, so
  // that the work after the batch in stream order still follows all of it.
  griddep_wait();
}

// The dynamic shared-memory limit of a kernel is raised once per device (the attribute
// is per function and device); bit d of `done` records device d.
template <typename K>
cudaError_t allow_smem(K kernel, std::atomic<uint64_t> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <int DS, bool FWD, uint32_t OUTS = 0, bool TM = false>
cudaError_t launch_band_t(const BandArgs &a, int smem_bytes, cudaStream_t st) {
  static std::atomic<uint64_t> done{0};
  cudaError_t e = allow_smem(band_kernel<DS, FWD, OUTS, TM>, done);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.grid);
  cfg.blockDim = dim3(a.nc);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, band_kernel<DS, FWD, OUTS, TM>, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_band(const BandArgs &a, int smem_bytes, int ctas_per_sm, cudaStream_t st) {
  (void)ctas_per_sm;
  const bool fwd = a.warp_mode == DIBR_WARP_FORWARD;
  // the stereo set (left, right, anaglyph) and the anaglyph alone, with 16-byte aligned
  // rows: instances of their own
  if (a.depth_src == DS_BINOM5 && fwd && a.fast_store) {
    // bands of a few rows do not repay a CTA's tensor-memory allocation
    const bool tm = a.row1 - a.row0 >= kTmemMinRows * a.grid;
    if (a.outputs == kSetStereo)
      return tm ? launch_band_t<DS_BINOM5, true, kSetStereo, true>(a, smem_bytes, st)
                : launch_band_t<DS_BINOM5, true, kSetStereo, false>(a, smem_bytes, st);
    if (a.outputs == kSetAnaglyph)
      return tm ? launch_band_t<DS_BINOM5, true, kSetAnaglyph, true>(a, smem_bytes, st)
                : launch_band_t<DS_BINOM5, true, kSetAnaglyph, false>(a, smem_bytes, st);
  }
  switch (a.depth_src) {
    case DS_BINOM5: return fwd ? launch_band_t<DS_BINOM5, true>(a, smem_bytes, st) : launch_band_t<DS_BINOM5, false>(a, smem_bytes, st);
    case DS_LUMA: return fwd ? launch_band_t<DS_LUMA, true>(a, smem_bytes, st) : launch_band_t<DS_LUMA, false>(a, smem_bytes, st);
    default: return fwd ? launch_band_t<DS_GLOBAL, true>(a, smem_bytes, st) : launch_band_t<DS_GLOBAL, false>(a, smem_bytes, st);
  }
}

template <uint32_t OUTS>
static cudaError_t launch_batch_t(const BatchArgs &b, int grid, int smem_bytes, bool chained, cudaStream_t st) {
  static std::atomic<uint64_t> done{0};
  cudaError_t e = allow_smem(batch_kernel<OUTS>, done);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(b.nc);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, batch_kernel<OUTS>, b);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &b, int grid, int smem_bytes, bool chained, cudaStream_t st) {
  if (b.outs == kSetStereo) return launch_batch_t<kSetStereo>(b, grid, smem_bytes, chained, st);
  if (b.outs == kSetAnaglyph) return launch_batch_t<kSetAnaglyph>(b, grid, smem_bytes, chained, st);
  return launch_batch_t<0>(b, grid, smem_bytes, chained, st);
}

}  // namespace dibr
