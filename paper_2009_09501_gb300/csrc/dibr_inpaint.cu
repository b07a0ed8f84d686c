// dibr_inpaint.cu -- the iterative 2-D block inpainting of Fig. 3 (left column), run over
// the holes of both reconstructed views after the band kernel (hole fill DIBR_FILL_INPAINT2D).
//
// Per block of B x B pixels and per view, one warp.  The figure's algorithm visits the
// block's damaged pixels block column by block column, in passes that repeat while some
// pixel is repaired, and repairs a pixel once two or more of its 8 neighbours are
// undamaged; a repair is visible at once to the visits after it.  The warp runs that order
// as a wavefront with the passes pipelined: lane x owns block column x, and pass p visits
// row y of it at step 2x + y + 4p.  Every visit sees exactly the state the sequential
// passes would show it, and the visits of one step are never neighbours (see the loop), so
// a block whose repairs creep one column per pass (the undamaged side to the right of a
// wide hole) takes about 2B + B + 4 x passes steps instead of B steps per pass.
//
// The damage flags of a column live in a 64-bit register of its lane (bit j = block row
// j - 1, with the rows above and below the block at bits 0 and B + 1); a lane reads its
// neighbours' columns with shuffles at the step it needs them.  Colours live in shared
// memory with a one-pixel frame around the block.  Pixels outside the block are read as
// the band kernel left them (they are never written by this block, and their damage
// flags come from the holes map, which nothing changes), so blocks are independent.
// Repaired pixels are written back into the view in place; then the anaglyph and HSBS
// outputs are rewritten where a view changed.
#include "dibr_internal.h"

namespace dibr {
namespace {

constexpr int kMaxBlock = 32;
constexpr int kStride = kMaxBlock + 2;  // cells per row of a block's colour frame
// One warp per CTA, one image block per warp; the warp takes the block's two views in turn
// (a finished block frees its slot at once; no warp waits for another)

// floor(v / (2n)) for v < 4096 and n = 2..8 as (v * ceil(65536 / 2n)) >> 16 (exact over that
// range); index n.
__constant__ uint32_t kHalfRecip[9] = {0, 0, 16384, 10923, 8192, 6554, 5462, 4682, 4096};

__device__ __forceinline__ void store_rgb(uint8_t *p, uint32_t c) {
  p[0] = static_cast<uint8_t>(c);
  p[1] = static_cast<uint8_t>(c >> 8);
  p[2] = static_cast<uint8_t>(c >> 16);
}

__global__ void __launch_bounds__(32, 32) inpaint_kernel(const __grid_constant__ InpaintArgs a) {
  __shared__ uint32_t cell[kStride * kStride];
  const int lane = threadIdx.x;
  const int blk = blockIdx.x;
  const int B = a.block, W = a.W, H = a.H;
  int bx0 = 0, by0 = 0, bw = 0, bh = 0;
  if (blk < a.nblocks) {
    // the blocks of the first and last block columns go first: the whole background moves
    // there, so their holes are the widest (up to P/2 columns) and they take longest
    const int nbx = a.nbx, nby = a.nblocks / a.nbx;
    int bx, by;
    if (nbx <= 2) {
      bx = blk % nbx;
      by = blk / nbx;
    } else if (blk < 2 * nby) {
      bx = (blk & 1) ? nbx - 1 : 0;
      by = blk >> 1;
    } else {
      const int i = blk - 2 * nby;
      bx = 1 + i % (nbx - 2);
      by = i / (nbx - 2);
    }
    bx0 = bx * B;
    by0 = by * B;
    bw = min(B, W - bx0);
    bh = min(B, H - by0);
  }
  // ---- the holes of both views inside the block (lane x: column x), every row's load in
  // flight
  uint64_t own_l = 0, own_r = 0;
  {
    // (addresses of lanes and rows outside the block are clamped to the block's corner)
    const uint8_t *hp = a.holes + static_cast<int64_t>(by0) * a.holes_pitch + bx0 + (lane < bw ? lane : 0);
    uint32_t hb[kMaxBlock];
#pragma unroll
    for (int r = 0; r < kMaxBlock; ++r) {
      const bool in = lane < bw && r < bh;
      const uint32_t v8 = hp[static_cast<int64_t>(r < bh ? r : 0) * a.holes_pitch];
      hb[r] = in ? v8 : 0u;
    }
#pragma unroll
    for (int r = 0; r < kMaxBlock; ++r) {
      if (hb[r] & 1u) own_l |= 2ull << r;
      if (hb[r] & 2u) own_r |= 2ull << r;
    }
  }
  uint64_t rep_l = 0, rep_r = 0;  // per view, the repaired frame rows of this lane's column
#pragma unroll 1
  for (int v = 0; v < 2; ++v) {
  uint8_t *view = a.view[v];
  const uint32_t vbit = 1u << v;
  uint64_t own = v ? own_r : own_l;
  if (!__any_sync(0xffffffffu, own != 0)) continue;
  uint64_t own0 = own;
  {
    // ---- colours of the block and its one-pixel frame, damage flags of the frame
    // (pixels outside the image count as damaged); eight rows of loads in flight at a time
    uint64_t col_a = 0, col_b = 0;  // flags of frame columns lane and lane + 32
    for (int i = lane; i < bw + 2; i += 32) {
      const int x = bx0 - 1 + i;
      const bool xin = x >= 0 && x < W;
      uint64_t flags = 0;
      for (int j0 = 0; j0 < bh + 2; j0 += 8) {
        uint32_t hv[8], c0[8], c1[8], c2[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = j0 + t, y = by0 - 1 + j;
          const bool in = xin && j < bh + 2 && y >= 0 && y < H;
          const int64_t yy = in ? y : by0, xx = in ? x : bx0;  // pixels outside: read (bx0, by0), unused
          const uint8_t *px = view + yy * a.pitch + 3 * xx;
          const uint32_t h8 = a.holes[yy * a.holes_pitch + xx];
          hv[t] = in ? h8 : 0xFFu;
          c0[t] = px[0];
          c1[t] = px[1];
          c2[t] = px[2];
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = j0 + t;
          if (j >= bh + 2) break;
          const bool bad = (hv[t] & vbit) != 0;
          cell[j * kStride + i] = bad ? 0u : (c0[t] | (c1[t] << 8) | (c2[t] << 16));
          if (bad) flags |= 1ull << j;
        }
      }
      if (i < 32) col_a = flags;
      else col_b = flags;
    }
    // lane x (< bw) owns frame column x + 1; the frame columns 0 and bw + 1 are the halo
    const uint64_t next_a = __shfl_sync(0xffffffffu, col_a, (lane + 1) & 31);
    const uint64_t first_b = __shfl_sync(0xffffffffu, col_b, 0);
    own = lane < bw ? (lane < 31 ? next_a : first_b) : ~0ull;
    own0 = own;
    const uint64_t halo_l = __shfl_sync(0xffffffffu, col_a, 0);
    const int hr = bw + 1;
    const uint64_t hr_a = __shfl_sync(0xffffffffu, col_a, hr & 31);
    const uint64_t hr_b = __shfl_sync(0xffffffffu, col_b, hr & 31);
    const uint64_t halo_r = hr < 32 ? hr_a : hr_b;
    __syncwarp();

    const uint64_t rows = ((1ull << bh) - 1ull) << 1;  // the block's own rows in a column mask
    uint64_t lm = 0, rm = 0;  // damage flags of the neighbouring columns
    auto refresh = [&]() {
      lm = __shfl_up_sync(0xffffffffu, own, 1);
      rm = __shfl_down_sync(0xffffffffu, own, 1);
      if (lane == 0) lm = halo_l;
      if (lane == bw - 1) rm = halo_r;
    };
    // The visit of damaged block row r of this lane's column: with two or more undamaged
    // neighbours the pixel takes their mean colour and is no longer damaged.
    auto visit = [&](int r) -> bool {
      // frame rows r, r + 1 (the pixel's own), r + 2 of the three columns
      const uint32_t bl = static_cast<uint32_t>(lm >> r) & 7u;
      const uint32_t bo = static_cast<uint32_t>(own >> r) & 5u;
      const uint32_t br = static_cast<uint32_t>(rm >> r) & 7u;
      const int n = 8 - __popc(bl) - __popc(bo) - __popc(br);
      if (n < 2) return false;
      // A damaged cell holds 0 until it is repaired (and then its flag is cleared with the
      // same visit), so the sums over all eight neighbours are the sums over the undamaged
      // ones.  Per channel at most 8 * 255 < 2^11: the red and blue sums fit 16-bit lanes
      // of one word, and the green sum is what the plain word sum has beyond them.
      const uint32_t *c0 = cell + r * kStride + lane;
      const uint32_t c[8] = {c0[0], c0[1], c0[2], c0[kStride], c0[kStride + 2], c0[2 * kStride],
                             c0[2 * kStride + 1], c0[2 * kStride + 2]};
      const uint32_t all = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
      const uint32_t srb = (((c[0] & 0x00FF00FFu) + (c[1] & 0x00FF00FFu)) + ((c[2] & 0x00FF00FFu) + (c[3] & 0x00FF00FFu))) +
                           (((c[4] & 0x00FF00FFu) + (c[5] & 0x00FF00FFu)) + ((c[6] & 0x00FF00FFu) + (c[7] & 0x00FF00FFu)));
      const uint32_t sg = (all - srb) >> 8;
      // per channel floor((2 sum + n) / 2n): the mean rounded half up
      const uint32_t rc = kHalfRecip[n];
      const uint32_t mr = ((2u * (srb & 0xFFFFu) + n) * rc) >> 16, mb = ((2u * (srb >> 16) + n) * rc) >> 16;
      const uint32_t mg = ((2u * sg + n) * rc) >> 16;
      cell[(r + 1) * kStride + lane + 1] = mr | (mg << 8) | (mb << 16);
      own &= ~(1ull << (r + 1));
      return true;
    };
    // ---- the passes, pipelined.  Pass p visits block pixel (x, y) at step 2x + y + 4p.
    // A visit reads only the eight neighbours; in the sequential order those earlier in the
    // list (column x-1, and (x, y-1)) were last visited by the same pass at a smaller step,
    // and those later in it (column x+1, and (x, y+1)) by the previous pass at most 3 steps
    // later in the wavefront than (x, y) itself, i.e. at a step 1 or more below this visit's,
    // and by this pass at a larger step.  So every visit sees exactly the state the
    // sequential passes would show it.  Two visits of one step are never neighbours (same
    // column: rows 4 apart; adjacent columns: rows 2 apart modulo 4), so each step's visits
    // are independent, and lane x makes those of its column: rows y = T - 2x - 4p, p >= 0.
    // A damaged pixel whose neighbourhood has not changed since it last failed the test
    // fails it again, so only "dirty" pixels are visited (never visited yet, or next to a
    // repair since their last visit); when no damaged pixel is dirty nothing can change any
    // more, which is where the figure's loop ends too (a pass that repairs nothing).  Steps
    // at which no lane has a dirty pixel to visit are skipped.
    uint64_t dirty = own & rows;
    refresh();
    const int x2 = 2 * lane;
    // frame rows j (block row j - 1) that lane x has reached by step t: j - 1 <= t - 2x
    auto reached = [&](int t) -> uint64_t {
      const int b = t - x2;
      return b < 0 ? 0ull : b >= 32 ? ~0ull : (4ull << b) - 1ull;
    };
    // the first step at or after t with a visit to make, over the warp (INT_MAX: none)
    auto next_step = [&](int t) -> int {
      const uint64_t dd = lane < bw ? own & dirty & rows : 0ull;
      int n = 0x7FFFFFFF;
      if (dd & reached(t)) n = t;                                 // visited within 4 steps
      else if (dd) n = x2 + __ffsll(static_cast<long long>(dd)) - 2;  // its first visit
      return __reduce_min_sync(0xffffffffu, n);
    };
    for (int t = next_step(0); t != 0x7FFFFFFF; t = next_step(t + 1)) {
      const int b = t - x2;
      // damaged, dirty rows of this lane's column visited at step t: y = b - 4p, p >= 0
      uint64_t cand = lane < bw && b >= 0 ? own & dirty & reached(t) & (0x2222222222222222ull << (b & 3)) : 0ull;
      uint64_t mine = 0;
      while (cand) {
        const int j = __ffsll(static_cast<long long>(cand)) - 1;  // frame row; block row j - 1
        cand &= cand - 1;
        dirty &= ~(1ull << j);
        if (visit(j - 1)) mine |= 1ull << j;
      }
      __syncwarp();
      if (__any_sync(0xffffffffu, mine != 0)) {
        // new neighbour columns; the damaged neighbours of every repair become dirty
        const uint64_t ol = lm, orr = rm;
        refresh();
        const uint64_t gone = (ol & ~lm) | (orr & ~rm) | mine;
        dirty |= (gone | (gone << 1) | (gone >> 1)) & own & rows;
      }
    }
    // ---- repaired pixels back into the view
    const uint64_t rep = lane < bw ? (own0 & ~own & rows) : 0ull;
    uint64_t left = rep;
    while (left) {
      const int j = __ffsll(static_cast<long long>(left)) - 1;  // frame row; block row j - 1
      left &= left - 1;
      store_rgb(view + static_cast<int64_t>(by0 + j - 1) * a.pitch + 3 * static_cast<int64_t>(bx0 + lane),
                cell[j * kStride + lane + 1]);
    }
    if (v) rep_r = rep;
    else rep_l = rep;
  }
  __syncwarp();  // the frame of the next view goes into the same cells
  }
  __syncwarp();  // both views are final in memory for every lane

  // ---- formatted outputs where a view changed
  const uint64_t rl = rep_l, rr = rep_r;
  // rows where x or x + 1 changed, per view
  const uint64_t pair_l = rl | __shfl_down_sync(0xffffffffu, rl, 1);
  const uint64_t pair_r = rr | __shfl_down_sync(0xffffffffu, rr, 1);
  if (lane < bw) {
    const int x = bx0 + lane;
    if (a.ana) {
      uint64_t m = rl | rr;
      while (m) {
        const int j = __ffsll(static_cast<long long>(m)) - 1;
        m &= m - 1;
        const int64_t o = static_cast<int64_t>(by0 + j - 1) * a.pitch + 3 * static_cast<int64_t>(x);
        uint8_t *d = a.ana + static_cast<int64_t>(by0 + j - 1) * a.out_pitch + 3 * static_cast<int64_t>(x);
        d[0] = a.view[0][o];
        d[1] = a.view[1][o + 1];
        d[2] = a.view[1][o + 2];
      }
    }
    for (int v = 0; a.hsbs && (lane & 1) == 0 && v < 2; ++v) {
      // pairs (x, x + 1) of each view; blocks start at even columns and have even widths
      uint64_t m = v ? pair_r : pair_l;
      const uint8_t *src = a.view[v];
      while (m) {
        const int j = __ffsll(static_cast<long long>(m)) - 1;
        m &= m - 1;
        const int y = by0 + j - 1;
        const uint8_t *p = src + static_cast<int64_t>(y) * a.pitch + 3 * static_cast<int64_t>(x);
        uint8_t *d = a.hsbs + static_cast<int64_t>(y) * a.out_pitch + 3 * static_cast<int64_t>((v ? W / 2 : 0) + x / 2);
        for (int c = 0; c < 3; ++c) d[c] = static_cast<uint8_t>((p[c] + p[3 + c] + 1) >> 1);
      }
    }
  }
}

}  // namespace

cudaError_t launch_inpaint(const InpaintArgs &a, cudaStream_t st) {
  if (a.nblocks <= 0) return cudaSuccess;
  inpaint_kernel<<<a.nblocks, 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dibr
