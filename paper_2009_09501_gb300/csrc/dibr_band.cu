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
// refills a slot right after the row barrier that proves every thread is done with it.
// Every wait is bounded (%globaltimer); a wait that gives up sets a bit of the status word
// and the CTA unwinds after letting its own copies land.
//
// Per consumer thread and row y:
//   A  luminance of row y+2 for its 16 columns plus 2 on each side, fed into a cascade
//      of four [1 1] row sums held in registers, which yields the vertical binomial of
//      row y; the horizontal binomial gives D(y) for the 16 columns; clears its 16
//      targets of this row's z-buffers (double buffered across rows).
//   B  the warp scatters its 512 sources (lane-interleaved) into the left and right
//      z-buffers with atomicMin on a ((255 - depth) << 24 | RGB) entry; needs A of the
//      row done by every warp.
//   C  reads its 16 targets' entries, fills holes (warp scans for the nearest filled
//      target on each side), formats and stores the outputs; needs B of the row done by
//      every warp.
// Rows interleave as A(y+1), C(y), B(y+1): a split barrier (an mbarrier every warp arrives
// on after A and waits on before B) and a full barrier per row.
#include "dibr.h"
#include "dibr_internal.h"
#include "dibr_ptx.cuh"

namespace dibr {
namespace {

constexpr int kNoTarget = 0x7FFFFFFF;

__device__ __forceinline__ uint32_t bsel(const uint32_t *w, int j) {
  return (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
}

// BT.601 luminance in exact thousandths, rounded half up (the depth-map reading):
// (299 R + 587 G + 114 B + 500) / 1000, the division as a multiply-high by
// ceil(2^32 / 1000), exact for numerators below 6.1e6.
__device__ __forceinline__ uint32_t luma8(uint32_t r, uint32_t g, uint32_t b) {
  return __umulhi(299u * r + 587u * g + 114u * b + 500u, 4294968u);
}

// The same luminance of the pixel held in bytes 0..2 (S = 0) or 1..3 (S = 8) of w, as
// three byte dot products: 299 = 255 + 44, 587 = 255 + 255 + 77, 114.
template <int S>
__device__ __forceinline__ uint32_t luma_dp(uint32_t w) {
  uint32_t n = __dp4a(w, 0x0072FFFFu << S, 500u);
  n = __dp4a(w, 0x0000FF2Cu << S, n);
  n = __dp4a(w, 0x00004D00u << S, n);
  return __umulhi(n, 4294968u);
}

// Luminance of one packed pixel word (R, G, B in the low three bytes).
__device__ __forceinline__ uint32_t luma_px(uint32_t c) { return luma_dp<0>(c); }

// Luminance of columns x0-2 .. x0+17 (clamped to [0, W-1]) of one input row held in
// shared memory, as 10 words of two 16-bit lanes: yp[2q] = columns (4q, 4q+2) and
// yp[2q+1] = (4q+1, 4q+3) of the window, the layout the vertical cascade works on.
__device__ __forceinline__ void luma20(const uint8_t *row, int x0, int W, uint32_t (&yp)[10]) {
  // bytes 3*x0-8 .. 3*x0+55 (8-byte and 16-byte aligned loads); column j of the window at
  // byte 2+3j.  At the row's ends the loads reach past it into neighbouring shared memory
  // (the ring's other slots, the table before it, the depth row after it); those columns
  // are replaced below by the row's first or last column.
  uint32_t y[20];
  uint32_t b[16];
  const uint2 l = *reinterpret_cast<const uint2 *>(row + 3 * x0 - 8);
  const uint4 m0 = *reinterpret_cast<const uint4 *>(row + 3 * x0);
  const uint4 m1 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 16);
  const uint4 m2 = *reinterpret_cast<const uint4 *>(row + 3 * x0 + 32);
  const uint2 r = *reinterpret_cast<const uint2 *>(row + 3 * x0 + 48);
  b[0] = l.x; b[1] = l.y;
  b[2] = m0.x; b[3] = m0.y; b[4] = m0.z; b[5] = m0.w;
  b[6] = m1.x; b[7] = m1.y; b[8] = m1.z; b[9] = m1.w;
  b[10] = m2.x; b[11] = m2.y; b[12] = m2.z; b[13] = m2.w;
  b[14] = r.x; b[15] = r.y;
#pragma unroll
  for (int j = 0; j < 20; ++j) {
    const int o = 2 + 3 * j, q = o >> 2;
    if ((o & 3) == 0) y[j] = luma_dp<0>(b[q]);
    else if ((o & 3) == 1) y[j] = luma_dp<8>(b[q]);
    else y[j] = luma_dp<0>(__funnelshift_r(b[q], b[q + 1], 8 * (o & 3)));
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    yp[2 * q] = y[4 * q] | (y[4 * q + 2] << 16);
    yp[2 * q + 1] = y[4 * q + 1] | (y[4 * q + 3] << 16);
  }
  // clamp to the row: the columns before 0 and after W-1 take column 0 and column W-1
  // (window column j sits in word 2 * (j / 4) + j % 2, high lane when j / 2 is odd)
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

// Vertical binomial [1 4 6 4 1] as four cascaded [1 1] sums over the stream of
// luminance rows.  The 20 columns are held as 10 words of two 16-bit lanes: lo[q] =
// columns (4q, 4q+2), hi[q] = (4q+1, 4q+3) of the window x0-2 .. x0+17.  After a row n
// is fed, p0 = Y(n), p1 = Y(n-1)+Y(n), p2 and p3 the next sums; feeding row n+1 returns
// sum_i C(4,i) Y(n-3+i), the vertical binomial centred on row n-1.  All sums stay below
// 16 * 255, so the lanes never carry into each other.
struct VCascade {
  uint32_t p0[10], p1[10], p2[10], p3[10];

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 10; ++i) p0[i] = p1[i] = p2[i] = p3[i] = 0u;
  }
  // feeds one row (16-bit lane pairs); V receives the vertical sums (valid from the
  // fifth row on)
  __device__ __forceinline__ void feed(const uint32_t (&y)[10], uint32_t (&V)[10]) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const uint32_t a1 = p0[i] + y[i];
      const uint32_t a2 = p1[i] + a1;
      const uint32_t a3 = p2[i] + a2;
      V[i] = p3[i] + a3;
      p0[i] = y[i];
      p1[i] = a1;
      p2[i] = a2;
      p3[i] = a3;
    }
  }
  // feeds the newest row again (the image's last row repeated below the image)
  __device__ __forceinline__ void feed_repeat(uint32_t (&V)[10]) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const uint32_t a1 = p0[i] + p0[i];
      const uint32_t a2 = p1[i] + a1;
      const uint32_t a3 = p2[i] + a2;
      V[i] = p3[i] + a3;
      p1[i] = a1;
      p2[i] = a2;
      p3[i] = a3;
    }
  }
};

// Horizontal binomial of the vertical sums and rounding: D = (sum + 128) >> 8 for the 16
// own columns (window columns 2..17), packed 4 per word.
__device__ __forceinline__ uint4 binom_h(const uint32_t (&V)[10]) {
  uint32_t d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t E0 = V[2 * k], O0 = V[2 * k + 1], E1 = V[2 * k + 2], O1 = V[2 * k + 3];
    const uint32_t se = __byte_perm(E0, E1, 0x5432);  // (V[4k+2], V[4k+4])
    const uint32_t so = __byte_perm(O0, O1, 0x5432);  // (V[4k+3], V[4k+5])
    const uint32_t pe = E0 + E1 + 4u * (O0 + so) + 6u * se;  // columns 4k, 4k+2
    const uint32_t po = O0 + O1 + 4u * (se + E1) + 6u * so;  // columns 4k+1, 4k+3
    const uint32_t de = ((pe + 0x00800080u) >> 8) & 0x00FF00FFu;
    const uint32_t dd = ((po + 0x00800080u) >> 8) & 0x00FF00FFu;
    d[k] = de | (dd << 8);
  }
  return make_uint4(d[0], d[1], d[2], d[3]);
}

// Target offsets of a source from its packed table entry: -hL (low half) and -hR (high
// half), both sign-extended.
__device__ __forceinline__ int shift_l(uint32_t w) { return static_cast<int>(w << 16) >> 16; }
__device__ __forceinline__ int shift_r(uint32_t w) { return static_cast<int>(w) >> 16; }

// z-buffer entry: ((255 - depth) << 24) | RGB of the source, reduced with atomicMin
// into a buffer initialised to kEmpty.  The smallest entry has the largest depth
// (nearest source).  Two sources with equal depth have equal shifts and so never meet
// on one target, so the colour bits never decide a collision; the winner's colour is
// read straight from its entry.  kEmpty cannot be a real entry: it would need depth 0
// for a white pixel, and every depth rule gives a white pixel a depth of at least 1
// (binomial: its own weight 36/256; luminance: 255; cross-bilateral: its own weight 1
// among at most 289).
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// Packed RGB (3 bytes) of column x of a row in global memory (byte loads: nothing past the
// pixel is read).
__device__ __forceinline__ uint32_t rgb_at_global(const uint8_t *row, int x) {
  const uint8_t *p = row + 3 * static_cast<int64_t>(x);
  return static_cast<uint32_t>(p[0]) | (static_cast<uint32_t>(p[1]) << 8) | (static_cast<uint32_t>(p[2]) << 16);
}

// Packed RGB (3 bytes) of column x of a row held in shared memory.
__device__ __forceinline__ uint32_t rgb_at(const uint8_t *row, int x) {
  const uint32_t off = 3u * static_cast<uint32_t>(x);
  const uint32_t *wp = reinterpret_cast<const uint32_t *>(row + (off & ~3u));
  return __funnelshift_r(wp[0], wp[1], (off & 3u) * 8u) & 0xFFFFFFu;
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

// Nearest filled target at or below t (or -1) / at or above t (or kNoTarget), searched
// by the whole warp 32 targets at a time (all lanes call it together): the path for
// holes whose neighbours lie outside the warp's own targets.
__device__ __noinline__ int warp_walk_left(const uint32_t *zb, int t, int lane) {
  for (int base = t; base >= 0; base -= 32) {
    const int i = base - lane;
    const uint32_t b = __ballot_sync(0xffffffffu, i >= 0 && zb[i] != kEmpty);
    if (b) return base - (__ffs(b) - 1);
  }
  return -1;
}

__device__ __noinline__ int warp_walk_right(const uint32_t *zb, int t, int W, int lane) {
  for (int base = t; base < W; base += 32) {
    const int i = base + lane;
    const uint32_t b = __ballot_sync(0xffffffffu, i < W && zb[i] != kEmpty);
    if (b) return base + (__ffs(b) - 1);
  }
  return kNoTarget;
}

// Entries shown by the 16 targets of this thread in one view: the z-buffer winner, or
// for a hole the winner of the nearest filled target on its farther side -- of the
// nearest filled targets to its left and right, the one whose winner has the smaller
// depth (the left one on a tie, the only one at a row edge); the input pixel at the hole
// when the row has no filled target.
//
// Two register sweeps: left to right carrying the last filled key into the holes, then
// right to left carrying the last filled key and keeping it where it is strictly
// farther.  Entries are (255 - depth) << 24 | colour, so "c strictly farther than k" is
// the unsigned compare c > (k | 0xFFFFFF).  The keys carried into the chunk come from
// the nearest lane on each side with a filled target (ballot + shuffle) or, past the
// warp's 512 targets, from a warp-wide search of the z-buffer.  A missing right key
// carries in as 0, which is never strictly farther; holes with no left key (row starts)
// are set afterwards on a path of their own.
// Returns the thread's hole bits (bit j: no source reached target x0 + j).
__device__ __forceinline__ uint32_t resolve_view(const uint32_t *zb, const uint8_t *grow, int x0, int npx, int W,
                                                 int lane, int warp_lo, int warp_hi, uint32_t (&k)[16]) {
  const uint32_t zs = smem_addr(zb);
  if (npx > 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 u = lds_u32x4(zs + 4u * (x0 + 4 * q));
      k[4 * q] = u.x; k[4 * q + 1] = u.y; k[4 * q + 2] = u.z; k[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) k[i] = 0u;
  }
  const uint32_t rowmask = npx >= 16 ? 0xFFFFu : ((1u << max(npx, 0)) - 1u);
  uint32_t m = 0u;
#pragma unroll
  for (int i = 0; i < 16; ++i)
    if (k[i] != kEmpty) m |= 1u << i;
  m &= rowmask;
  const uint32_t holes = ~m & rowmask;
  if (!__any_sync(0xffffffffu, holes != 0u)) return holes;

  const int first = m ? x0 + __ffs(m) - 1 : kNoTarget;  // this chunk's first / last filled target
  const int last = m ? x0 + 31 - __clz(m) : -1;
  // holes before the chunk's first filled target need the key carried in from the left,
  // holes after its last one the key carried in from the right
  const uint32_t before = m ? holes & ((1u << (first - x0)) - 1u) : holes;
  const uint32_t after = m ? holes & ~((2u << (last - x0)) - 1u) : holes;
  const uint32_t lanes = __ballot_sync(0xffffffffu, m != 0u);
  const uint32_t lower = lanes & ((1u << lane) - 1u);
  const uint32_t upper = lanes & ~((2u << lane) - 1u);
  int nl = __shfl_sync(0xffffffffu, last, lower ? 31 - __clz(lower) : lane);
  int nr = __shfl_sync(0xffffffffu, first, upper ? __ffs(upper) - 1 : lane);
  if (!lower) nl = -1;
  if (!upper) nr = kNoTarget;
  if (__any_sync(0xffffffffu, before && !lower)) {
    const int w = warp_lo > 0 ? warp_walk_left(zb, warp_lo - 1, lane) : -1;
    if (!lower) nl = w;
  }
  if (__any_sync(0xffffffffu, after && !upper)) {
    const int w = warp_hi < W ? warp_walk_right(zb, warp_hi, W, lane) : kNoTarget;
    if (!upper) nr = w;
  }
  // left to right: every hole takes the last filled key (entries past the row's end take
  // whatever they take: they are never stored and this sweep carries nothing leftwards)
  uint32_t c = nl >= 0 ? lds_u32(zs + 4u * nl) : kEmpty;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (k[j] != kEmpty) c = k[j];
    k[j] = c;
  }
  // right to left: a hole keeps the right key where it is strictly farther
  c = nr < W ? lds_u32(zs + 4u * nr) : 0u;
#pragma unroll
  for (int j = 15; j >= 0; --j) {
    if ((m >> j) & 1u) c = k[j];
    else if (c > (k[j] | 0xFFFFFFu)) k[j] = c;
  }
  // holes before the first filled target of the row: the right key, or the input pixel
  // when the row has no filled target at all
  const bool row_start = nl < 0 && before != 0u;
  if (__any_sync(0xffffffffu, row_start) && row_start) {
    const int r = m ? first : nr;
    if (r < W) {
      const uint32_t cr = lds_u32(zs + 4u * r);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if ((before >> j) & 1u) k[j] = cr;
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)  // (no bit is set past the row's end)
        if ((before >> j) & 1u) k[j] = rgb_at_global(grow, x0 + j);
    }
  }
  return holes;
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

__device__ __forceinline__ void store48(uint8_t *p, const uint32_t (&w)[12], int npx) {
  if (npx == 16 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
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
  int warp_mode, depth_src, l2_prefetch;
};

// Shared-memory regions of one CTA (laid out for the widest image of the launch).
struct Shm {
  uint64_t *full;  // ring-slot mbarriers
  uint64_t *adone; // every warp has stored the next row's depths and cleared its z-buffers
  uint32_t *lut;   // per depth: -hL in the low 16 bits, -hR in the high 16 bits (two's complement)
  int32_t *lut_n;  // Fig. 3 gather: 510 * s_L(d) (in the z-buffer region)
  uint8_t *ring, *drow;
  uint32_t *zb0;   // [2 rows][L, R][zlen]
  int nb, srow, zlen;
};

__device__ __forceinline__ Shm carve(uint8_t *smem, int nb, int srow, int nch_max, int depth_src) {
  const BandSmem L = band_smem_layout(nb, srow, nch_max, depth_src);
  Shm m;
  m.full = reinterpret_cast<uint64_t *>(smem + L.bar);
  m.adone = reinterpret_cast<uint64_t *>(smem + L.flags + 8);
  m.lut = reinterpret_cast<uint32_t *>(smem + L.lut);
  m.ring = smem + L.ring;
  m.drow = smem + L.drow;
  m.zb0 = reinterpret_cast<uint32_t *>(smem + L.zb);
  m.lut_n = reinterpret_cast<int32_t *>(smem + L.zb);
  m.nb = nb;
  m.srow = srow;
  m.zlen = nch_max * kChunk;
  return m;
}

// Shift tables into shared memory (all threads; a barrier must follow).
__device__ __forceinline__ void fill_luts(const Shm &m, const int32_t *lut_h, const int32_t *lut_n, bool forward) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const int32_t h = lut_h[i];
    const int nl = -static_cast<int16_t>(h & 0xFFFF), nr = -(h >> 16);  // |h| <= 512
    m.lut[i] = (static_cast<uint32_t>(nr) << 16) | (static_cast<uint32_t>(nl) & 0xFFFFu);
    if (!forward) m.lut_n[i] = lut_n[i];
  }
}

// Rows [ys, ye) of one image, every stage of the pipeline (see the file comment).  All
// threads of the CTA call it together.  kbase counts the ring loads this CTA issued
// before (the slot and mbarrier phase of a load follow from it); it is advanced by the
// loads issued here.  Returns false when a bounded wait gave up (the status word is
// set and the copies in flight have been waited for).
__device__ __forceinline__ bool run_band(const Job &a, const Shm &m, int ys, int ye, uint32_t &kbase,
                                         uint32_t &abase, int *status, unsigned long long timeout_ns) {
  const int tid = threadIdx.x, nc = blockDim.x, W = a.W, H = a.H, nb = m.nb;
  const bool binom = a.depth_src == DS_BINOM5;
  const bool forward = a.warp_mode == DIBR_WARP_FORWARD;
  const int halo = binom ? 2 : 0;
  const int la = max(ys - halo, 0), lb = min(ye + halo, H);
  const int nload = lb - la;
  const int zimg = a.nch * kChunk;  // this image's targets, rounded up to whole chunks
  const uint32_t k0 = kbase;
  // g / nb as umulhi(g, ceil(2^32 / nb)): exact while g * (nb - 1) < 2^32, far beyond the
  // loads one CTA makes in a launch
  const uint32_t ring_rcp = 0xFFFFFFFFu / static_cast<uint32_t>(nb) + 1u;
  auto ring_div = [&](uint32_t g) { return __umulhi(g, ring_rcp); };

  // Row k = r - la of the band is the (k0 + k)-th load of this CTA: slot (k0+k) % nb.
  // The middle warp issues the loads of rows [issued, upto) (the warps at the row's ends
  // have the most fill work); the caller guarantees every earlier occupant of those slots
  // has been released by all threads (a barrier separates the last use from the call).
  int issued = 0;
  const int lw = 32 * ((nc >> 5) >> 1);  // first thread of the loading warp
  auto issue_loads = [&](int upto) {
    upto = min(upto, nload);
    if (tid - lw >= 0 && tid - lw < 32) {
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
    }
    issued = max(issued, upto);
  };
  issue_loads(nb);
  // optionally, the band's later rows go to L2 now
  if (a.l2_prefetch && tid - lw >= 0 && tid - lw < 32) {
    if (a.load_mode == LM_BULK) {
      for (int k = nb + tid - lw; k < nload; k += 32)
        bulk_prefetch_l2(a.in + static_cast<int64_t>(la + k) * a.in_pitch, static_cast<uint32_t>(a.row_bytes));
    } else {
      for (int j = tid - lw; j < (nload - nb) * a.nbox; j += 32) {
        const int k = nb + j / a.nbox, i = j % a.nbox;
        if (a.load_mode == LM_T3) tma_prefetch_3d(a.tmap, 0, i * a.box_step, la + k);
        else tma_prefetch_2d(a.tmap, i * a.box_step, la + k);
      }
    }
  }

  const int lane = tid & 31;
  const int x0 = tid * kChunk;
  const int npx = max(0, min(kChunk, W - x0));
  const bool active = npx > 0;
  const int warp_lo = (tid & ~31) * kChunk;
  const int warp_hi = min(W, warp_lo + 32 * kChunk);
  bool timed_out = false;
  auto slot = [&](int r) {
    const uint32_t g = k0 + (r - la);
    return m.ring + (g - ring_div(g) * nb) * m.srow;
  };
  auto wait_row = [&](int r) {
    const uint32_t g = k0 + (r - la), q = ring_div(g);
    if (!mbar_wait_bounded(&m.full[g - q * nb], q & 1, timeout_ns)) timed_out = true;
  };

  const bool want_depth = (a.outputs & DIBR_OUT_DEPTH) != 0;
  const bool want_holes = (a.outputs & DIBR_OUT_HOLES) != 0;
  const bool want_ana = (a.outputs & DIBR_OUT_ANAGLYPH) != 0;
  const bool want_l = (a.outputs & DIBR_OUT_LEFT) != 0;
  const bool want_r = (a.outputs & DIBR_OUT_RIGHT) != 0;
  const bool want_hsbs = (a.outputs & DIBR_OUT_HSBS) != 0;
  bool aborted = false;

  VCascade vc;
  vc.clear();
  if (binom) {
    // rows clamp(ys-2) .. clamp(ys+1) into the cascade
    const int pend = min(ys + 1, lb - 1);
    for (int r = la; r <= pend; ++r) wait_row(r);
#pragma unroll 1
    for (int i = -2; i <= 1; ++i) {
      const int r = min(max(ys + i, 0), H - 1);
      uint32_t yq[10] = {0u}, V[10];
      if (active) luma20(slot(r), x0, W, yq);
      vc.feed(yq, V);
    }
    if (consumer_sync_or(timed_out, nc)) aborted = true;
    else issue_loads((ys - la) + nb);  // the rows above the band are done with
  }

  // Per row, three phases: A (depth of the row into shared memory, its z-buffers cleared),
  // B (the forward warp: every source's entry reduced into the z-buffers), C (winners, hole
  // fill, formatting, stores).  B of a row needs A of that row done by every warp (a split
  // barrier: each warp arrives after its A and waits before its B), and C of a row needs B
  // of that row done by every warp (a full barrier).  A of the next row comes before C of
  // this one, so a warp that finishes C early scatters the next row while the others still
  // resolve this one.  C reads this row's input from global memory (the rare cases that
  // need it), so its ring slot is refilled as soon as B of the row is done.
  auto phase_a = [&](int y) -> uint4 {
    uint4 d = make_uint4(0u, 0u, 0u, 0u);
    uint32_t *zl = m.zb0 + (y & 1) * 2 * m.zlen;
    uint32_t *zr = zl + m.zlen;
    if (binom) {
      const int r2 = y + 2;
      if (r2 < lb) wait_row(r2);
      uint32_t V[10];
      if (r2 < H) {
        uint32_t yq[10] = {0u};
        if (active) luma20(slot(r2), x0, W, yq);
        vc.feed(yq, V);
      } else {
        vc.feed_repeat(V);  // rows below the image repeat row H-1
      }
      d = binom_h(V);
    } else {
      wait_row(y);
      if (active) {
        if (a.depth_src == DS_LUMA) {
          const uint8_t *row = slot(y);
          uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
          for (int j = 0; j < 16; ++j) w[j >> 2] |= luma_px(rgb_at(row, min(x0 + j, W - 1))) << (8 * (j & 3));
          d = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
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
    }
    if (active && want_depth)
      store16(a.out[O_DEPTH] + static_cast<int64_t>(y) * a.depth_pitch + x0, d, npx);
    if (forward) {
      if (active) *reinterpret_cast<uint4 *>(m.drow + x0) = d;
      // clear this warp's 512 targets of both views, consecutive lanes on consecutive
      // 16-byte words (no bank conflicts)
      const uint4 e = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = warp_lo + 4 * (32 * q + lane);
        if (t < zimg) {
          *reinterpret_cast<uint4 *>(zl + t) = e;
          *reinterpret_cast<uint4 *>(zr + t) = e;
        }
      }
    }
    return d;
  };
  auto phase_b = [&](int y) {
    const uint8_t *rgbrow = slot(y);
    uint32_t *zl = m.zb0 + (y & 1) * 2 * m.zlen;
    uint32_t *zr = zl + m.zlen;
    if (forward) {
      // the warp's 512 sources, consecutive lanes on consecutive columns, so that the
      // atomics of one instruction land on distinct banks (shifts vary slowly)
      const int xb = warp_lo + lane;
      const uint32_t ob = 3u * static_cast<uint32_t>(xb);
      const uint32_t cws = smem_addr(rgbrow) + (ob & ~3u);  // the lane's colours: +96 bytes per step
      const uint32_t sh = (ob & 3u) * 8u;
      const uint32_t ds = smem_addr(m.drow) + static_cast<uint32_t>(xb);
      const uint32_t ls = smem_addr(m.lut);
      const uint32_t zls = smem_addr(zl), zrs = smem_addr(zr);
      const bool full_warp = warp_hi - warp_lo == 32 * kChunk;
      if (full_warp) {
        // four steps at a time: all their shared loads are issued before their atomics
#pragma unroll
        for (int g = 0; g < kChunk / 4; ++g) {
          uint32_t dv[4], cw[8];
          lds_u8_step32x4(ds + 128 * g, dv);
          lds_u32_pair_step96x4(cws + 384 * g, cw);
          uint32_t lh[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) lh[j] = lds_u32(ls + 4u * dv[j]);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int x = xb + 32 * (4 * g + j);
            const uint32_t e = (__funnelshift_r(cw[2 * j], cw[2 * j + 1], sh) & 0xFFFFFFu) | (~dv[j] << 24);
            const int tl = x + shift_l(lh[j]), tr = x + shift_r(lh[j]);
            if (static_cast<unsigned>(tl) < static_cast<unsigned>(W)) reds_min(zls + 4u * tl, e);
            if (static_cast<unsigned>(tr) < static_cast<unsigned>(W)) reds_min(zrs + 4u * tr, e);
          }
        }
      } else {
        // the row's last, partial warp: columns from warp_hi on do not exist (their loads
        // read column warp_hi - 1, so that they stay in the row; their atomics are skipped)
        const uint32_t rs = smem_addr(rgbrow), dr = smem_addr(m.drow);
        const int ng = (warp_hi - warp_lo + 127) >> 7;  // groups of 4 x 32 columns holding some
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
          uint32_t dv[4], cw[8];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t xc = static_cast<uint32_t>(min(xb + 32 * (4 * g + j), warp_hi - 1));
            const uint32_t ca = rs + ((3u * xc) & ~3u);
            dv[j] = lds_u8(dr + xc);
            cw[2 * j] = lds_u32(ca);
            cw[2 * j + 1] = lds_u32(ca + 4);
          }
          uint32_t lh[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) lh[j] = lds_u32(ls + 4u * dv[j]);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int x = xb + 32 * (4 * g + j);
            if (x < warp_hi) {
              const uint32_t e = (__funnelshift_r(cw[2 * j], cw[2 * j + 1], sh) & 0xFFFFFFu) | (~dv[j] << 24);
              const int tl = x + shift_l(lh[j]), tr = x + shift_r(lh[j]);
              if (static_cast<unsigned>(tl) < static_cast<unsigned>(W)) reds_min(zls + 4u * tl, e);
              if (static_cast<unsigned>(tr) < static_cast<unsigned>(W)) reds_min(zrs + 4u * tr, e);
            }
          }
        }
      }
    }
  };
  auto phase_c = [&](int y, uint4 d) {
    uint32_t *zl = m.zb0 + (y & 1) * 2 * m.zlen;
    uint32_t *zr = zl + m.zlen;
    const uint32_t dw[4] = {d.x, d.y, d.z, d.w};
    // this row's input from global memory: its ring slot is refilled while this runs
    const uint8_t *grow = a.in + static_cast<int64_t>(y) * a.in_pitch;
    uint32_t kl[16], kr[16];
    uint32_t hole_l = 0u, hole_r = 0u;
    if (forward) {
      hole_l = resolve_view(zl, grow, x0, npx, W, lane, warp_lo, warp_hi, kl);
      hole_r = resolve_view(zr, grow, x0, npx, W, lane, warp_lo, warp_hi, kr);
    } else {
      // Fig. 3 literally: sample trunc(x + s(d)); out of range -> own column
#pragma unroll
      for (int i = 0; i < kChunk; ++i) {
        const int x = min(x0 + i, W - 1);
        const int n = m.lut_n[bsel(dw, i)];
        int sl = (510 * x + n) / 510, sr = (510 * x - n) / 510;
        if (static_cast<unsigned>(sl) >= static_cast<unsigned>(W)) sl = x;
        if (static_cast<unsigned>(sr) >= static_cast<unsigned>(W)) sr = x;
        kl[i] = active ? rgb_at_global(grow, sl) : 0u;
        kr[i] = active ? rgb_at_global(grow, sr) : 0u;
      }
    }
    if (active && want_holes) {
      // one byte per target: bit 0 a hole of the left view, bit 1 of the right view
      auto spread4 = [](uint32_t x) { return ((x & 0xFu) * 0x00204081u) & 0x01010101u; };
      uint4 hv;
      hv.x = spread4(hole_l) | (spread4(hole_r) << 1);
      hv.y = spread4(hole_l >> 4) | (spread4(hole_r >> 4) << 1);
      hv.z = spread4(hole_l >> 8) | (spread4(hole_r >> 8) << 1);
      hv.w = spread4(hole_l >> 12) | (spread4(hole_r >> 12) << 1);
      store16(a.out[O_HOLES] + static_cast<int64_t>(y) * a.depth_pitch + x0, hv, npx);
    }
    if (active) {
      const int64_t ro = static_cast<int64_t>(y) * a.out_pitch;
      uint32_t w[12];
      if (want_l) {
        pack16(kl, w);
        store48(a.out[O_LEFT] + ro + 3 * x0, w, npx);
      }
      if (want_r) {
        pack16(kr, w);
        store48(a.out[O_RIGHT] + ro + 3 * x0, w, npx);
      }
      if (want_ana) {
        uint32_t c[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = __byte_perm(kl[i], kr[i], 0x3650);  // R from L; G, B from R
        pack16(c, w);
        store48(a.out[O_ANA] + ro + 3 * x0, w, npx);
      }
      if (want_hsbs) {
        uint32_t cl8[8], cr8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          cl8[j] = avg_up(kl[2 * j], kl[2 * j + 1]);
          cr8[j] = avg_up(kr[2 * j], kr[2 * j + 1]);
        }
        uint32_t wl[6], wr[6];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          wl[3 * k] = __byte_perm(cl8[4 * k], cl8[4 * k + 1], 0x4210);
          wl[3 * k + 1] = __byte_perm(cl8[4 * k + 1], cl8[4 * k + 2], 0x5421);
          wl[3 * k + 2] = __byte_perm(cl8[4 * k + 2], cl8[4 * k + 3], 0x6542);
          wr[3 * k] = __byte_perm(cr8[4 * k], cr8[4 * k + 1], 0x4210);
          wr[3 * k + 1] = __byte_perm(cr8[4 * k + 1], cr8[4 * k + 2], 0x5421);
          wr[3 * k + 2] = __byte_perm(cr8[4 * k + 2], cr8[4 * k + 3], 0x6542);
        }
        const int np = npx / 2;  // W is even, so chunks hold whole pairs
        store24(a.out[O_HSBS] + ro + 3 * (x0 / 2), wl, np);
        store24(a.out[O_HSBS] + ro + 3 * (W / 2 + x0 / 2), wr, np);
      }
    }
  };
  // the split barrier: warps arrive after A of a row; it completes once per row
  auto a_arrive = [&]() {
    __syncwarp();
    if (lane == 0) mbar_arrive(m.adone);
  };
  auto a_wait = [&]() {
    if (!mbar_wait_bounded(m.adone, abase & 1u, timeout_ns)) timed_out = true;
    ++abase;
  };

  uint4 dcur = make_uint4(0u, 0u, 0u, 0u);
  if (!aborted && ys < ye) {
    dcur = phase_a(ys);
    if (consumer_sync_or(timed_out, nc)) aborted = true;
    else {
      phase_b(ys);
      if (consumer_sync_or(timed_out, nc)) aborted = true;
    }
  }
  for (int y = ys; y < ye && !aborted; ++y) {
    // every thread is past B of row y: the slots of rows <= y can be refilled
    issue_loads((y - la) + 1 + nb);
    const bool more = y + 1 < ye;
    uint4 dnext = make_uint4(0u, 0u, 0u, 0u);
    if (more) {
      dnext = phase_a(y + 1);
      a_arrive();
    }
    phase_c(y, dcur);
    if (more) {
      a_wait();
      phase_b(y + 1);
    }
    if (consumer_sync_or(timed_out, nc)) {
      aborted = true;
      break;
    }
    dcur = dnext;
  }

  kbase = k0 + issued;
  if (aborted) {
    if (tid == 0) {
      atomicOr(status, ST_TIMEOUT_FULL);
      // let every copy already issued land before the CTA's shared memory goes away
      for (int k = max(0, issued - nb); k < issued; ++k) {
        const uint32_t g = k0 + k;
        if (!mbar_wait_bounded(&m.full[g % nb], (g / nb) & 1, timeout_ns)) atomicOr(status, ST_TIMEOUT_DRAIN);
      }
    }
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------
// One image: CTA b owns the rows [b*H/grid, (b+1)*H/grid).
__global__ void __launch_bounds__(kMaxConsumers, 1) band_kernel(const __grid_constant__ BandArgs a) {
  // The next launch on the stream may start its set-up while this one runs (programmatic
  // dependent launch); it waits below for this one to complete before any global access.
  griddep_launch_dependents();
  extern __shared__ __align__(128) uint8_t smem[];
  const Shm m = carve(smem, a.nb, a.srow, a.nch, a.depth_src);
  fill_luts(m, a.lut_h, a.lut_n, a.warp_mode == DIBR_WARP_FORWARD);
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nb; ++i) mbar_init(&m.full[i], 1);
    mbar_init(m.adone, blockDim.x / 32);
    fence_mbar_init();
  }
  __syncthreads();
  // the work before this launch on the stream (whose results may be this launch's inputs,
  // or whose inputs this launch's outputs may overwrite) has completed -- unless the host
  // knows this launch touches none of that launch's buffers; then the wait moves to the
  // end, so that this launch still completes after the previous one
  if (!a.overlap) griddep_wait();
  const int nr = a.row1 - a.row0;
  const int ys = a.row0 + static_cast<int>(static_cast<int64_t>(blockIdx.x) * nr / a.grid);
  const int ye = a.row0 + static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * nr / a.grid);
  if (ys >= ye) {
    if (a.overlap) griddep_wait();
    return;
  }
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
  j.outputs = a.outputs; j.warp_mode = a.warp_mode; j.depth_src = a.depth_src; j.l2_prefetch = a.l2_prefetch;
  uint32_t kbase = 0, abase = 0;
  run_band(j, m, ys, ye, kbase, abase, a.status, a.timeout_ns);
  if (a.overlap) griddep_wait();
}

// ---------------------------------------------------------------------------------
// A batch of images in one persistent launch: CTAs pull work units (an image and a
// range of its rows) from a device counter until none is left.
__global__ void __launch_bounds__(kMaxConsumers, 1) batch_kernel(BatchArgs b) {
  // The next launch of the batch (another group of images, independent of this one) may be
  // placed as soon as every CTA of this one runs: its CTAs take the SM slots this launch
  // frees while its last units finish, instead of waiting for the last of them.
  griddep_launch_dependents();
  extern __shared__ __align__(128) uint8_t smem[];
  int *unit_s = reinterpret_cast<int *>(smem + band_smem_layout(b.nb, b.srow, b.nch_max, DS_BINOM5).flags);
  const Shm m = carve(smem, b.nb, b.srow, b.nch_max, DS_BINOM5);
  if (threadIdx.x == 0) {
    for (int i = 0; i < b.nb; ++i) mbar_init(&m.full[i], 1);
    mbar_init(m.adone, blockDim.x / 32);
    fence_mbar_init();
  }
  uint32_t kbase = 0, abase = 0;
  while (true) {
    __syncthreads();  // the previous unit is done with the ring, tables and unit_s
    if (threadIdx.x == 0) *unit_s = atomicAdd(b.counter, 1);
    __syncthreads();
    const int u = *unit_s;
    if (u >= b.n_units) break;
    const int4 un = b.units[u];  // {image, first row, end row}
    const ImageDesc &dsc = b.descs[un.x];
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
    j.outputs = dsc.outputs; j.warp_mode = dsc.warp_mode; j.depth_src = dsc.depth_src; j.l2_prefetch = 0;
    fill_luts(m, dsc.lut_h, dsc.lut_n, j.warp_mode == DIBR_WARP_FORWARD);
    __syncthreads();
    if (!run_band(j, m, un.y, un.z, kbase, abase, b.status, b.timeout_ns)) break;
  }
  // A chained launch's CTAs wait for the previous launch to complete before they exit, so
  // that the work after the batch in stream order still follows all of it.
  griddep_wait();
}

template <typename K>
cudaError_t allow_smem(K kernel, bool &done) {
  if (done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace


cudaError_t launch_band(const BandArgs &a, int smem_bytes, int ctas_per_sm, cudaStream_t st) {
  (void)ctas_per_sm;
  static bool done = false;  // per process: the attribute is per function
  cudaError_t e = allow_smem(band_kernel, done);
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
  e = cudaLaunchKernelEx(&cfg, band_kernel, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &b, int grid, int smem_bytes, bool chained, cudaStream_t st) {
  static bool done = false;
  cudaError_t e = allow_smem(batch_kernel, done);
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
  e = cudaLaunchKernelEx(&cfg, batch_kernel, b);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace dibr
