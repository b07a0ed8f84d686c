// dibr_inpaint.cu -- the iterative 2-D block inpainting of Fig. 3 (left column), run over
// the holes of both reconstructed views after the band kernel (hole fill DIBR_FILL_INPAINT2D).
//
// One warp per work item: a B x B block in one view.  The figure's algorithm visits the
// block's damaged pixels block column by block column, in passes that repeat while some
// pixel is repaired, and repairs a pixel once two or more of its 8 neighbours are
// undamaged; a repair is visible at once to the visits after it.  The warp runs that order
// as a wavefront with the passes pipelined: lane x owns block column x, and pass p visits
// row y of it at step 2x + y + 4p.  Every visit sees exactly the state the sequential
// passes would show it, and the visits of one step are never neighbours (see the loop), so
// a block whose repairs creep one column per pass (the undamaged side to the right of a
// wide hole) takes about 2B + B + 4 x passes steps instead of B steps per pass.
//
// The damage flags of a column live in a 32-bit register of its lane (bit y = block row
// y; the rows above and below the block never change and are kept apart); a lane reads its
// neighbours' columns with shuffles after each step.  Colours live in shared memory with a
// one-pixel frame around the block.  Pixels outside the block are read as the band kernel
// left them (undamaged ones are never written; damaged ones are never read), so the items are
// independent.  Repaired pixels are written back into the view in place, with the view's own
// anaglyph bytes and its half of the side-by-side frame.  A rank pass orders the items
// heavily damaged first; a persistent kernel takes them in that order.
#include "dibr_internal.h"
#include "dibr_ptx.cuh"

namespace dibr {
namespace {

constexpr int kMaxBlock = 32;
constexpr int kStride = kMaxBlock + 2;  // cells per row of a block's colour frame

// floor(v / (2n)) for v < 4096 and n = 2..8 as (v * ceil(65536 / 2n)) >> 16 (exact over that
// range); index n.
__constant__ uint32_t kHalfRecip[9] = {0, 0, 16384, 10923, 8192, 6554, 5462, 4682, 4096};

__device__ __forceinline__ void store_rgb(uint8_t *p, uint32_t c) {
  p[0] = static_cast<uint8_t>(c);
  p[1] = static_cast<uint8_t>(c >> 8);
  p[2] = static_cast<uint8_t>(c >> 16);
}

// The order in which the work items (a block in one view) are taken: an item with many
// damaged pixels takes the most steps (one pass per column when its repairs creep across a
// wide hole), so items with at least kHeavyDamage damaged pixels go first and the others after
// them; a heavy item that started late would otherwise finish well after the rest.  One warp
// per block counts the damaged pixels of both views (lane x: block column x) and places the
// two items at the front (heavy) or at the back of the order; an item without damage is not
// placed (nothing in it changes).
constexpr int kHeavyDamage = 256;

__global__ void __launch_bounds__(256) inpaint_rank_kernel(const __grid_constant__ InpaintArgs a) {
  const int lane = threadIdx.x & 31;
  const int blk = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (blk >= a.nblocks) return;
  const int B = a.block, bx0 = (blk % a.nbx) * B, by0 = (blk / a.nbx) * B;
  const int bw = min(B, a.W - bx0), bh = min(B, a.H - by0);
  const bool col = lane < bw;
  const uint8_t *hp = a.holes + static_cast<int64_t>(by0) * a.holes_pitch + bx0 + (col ? lane : 0);
  uint32_t hb[kMaxBlock];
#pragma unroll
  for (int r = 0; r < kMaxBlock; ++r) hb[r] = col && r < bh ? hp[static_cast<int64_t>(r) * a.holes_pitch] : 0u;
  uint32_t nl = 0, nr = 0;
#pragma unroll
  for (int r = 0; r < kMaxBlock; ++r) {
    nl += hb[r] & 1u;
    nr += (hb[r] >> 1) & 1u;
  }
  nl = __reduce_add_sync(0xffffffffu, nl);
  nr = __reduce_add_sync(0xffffffffu, nr);
  const uint32_t n = lane ? nr : nl;
  if (lane < 2 && n > 0) {  // lane v places the work item of view v (2 blk + v), if damaged
    const int items = 2 * a.nblocks;
    int32_t *heads = a.order + items;
    const bool heavy = n >= static_cast<uint32_t>(kHeavyDamage);
    const int pos = heavy ? atomicAdd(&heads[0], 1) : items - 1 - atomicAdd(&heads[1], 1);
    a.order[pos] = 2 * blk + lane;
  }
}

// One work item (a block in one view) by one warp; cell is the warp's colour frame in shared
// memory.  The two views of a block are independent: a view's repairs change only that view
// and its own bytes of the anaglyph (red from the left view, green and blue from the right)
// and its half of the side-by-side frame.
__device__ __forceinline__ void inpaint_block(const InpaintArgs &a, int item, uint32_t *cell) {
  const int blk = item >> 1, v = item & 1;
  const int lane = threadIdx.x;
  const int B = a.block, W = a.W, H = a.H;
  int bx0 = 0, by0 = 0, bw = 0, bh = 0;
  {
    const int bx = blk % a.nbx, by = blk / a.nbx;
    bx0 = bx * B;
    by0 = by * B;
    bw = min(B, W - bx0);
    bh = min(B, H - by0);
  }
  // ---- damage flags, both views (bit j = frame row j, block row j - 1; pixels outside the
  // image count as damaged): of this lane's own column (lane x < bw: image column bx0 + x)
  // over the frame rows 0 .. bh + 1, and of the halo columns bx0 - 1 and bx0 + bw, whose
  // frame row j is read by lane j (rows 32 and 33 by lanes 0 and 1) and gathered by ballot.
  // Every load in flight at once.
  const int x = bx0 + lane;
  const bool col = lane < bw;
  uint64_t fl0 = 0, fl1 = 0;
  {
    uint32_t hb[kMaxBlock + 2];
#pragma unroll
    for (int j = 0; j < kMaxBlock + 2; ++j) {
      const int y = by0 - 1 + j;
      const bool frame = col && j < bh + 2, in = frame && y >= 0 && y < H;
      const uint32_t h8 = a.holes[static_cast<int64_t>(in ? y : by0) * a.holes_pitch + (col ? x : bx0)];
      hb[j] = in ? h8 : frame ? 3u : 0u;
    }
#pragma unroll
    for (int j = 0; j < kMaxBlock + 2; ++j) {
      if (hb[j] & 1u) fl0 |= 1ull << j;
      if (hb[j] & 2u) fl1 |= 1ull << j;
    }
  }
  // halo pixels of this lane: frame rows hj[k], left (column bx0 - 1) and right (bx0 + bw)
  const int hj[2] = {lane, 32 + lane};
  uint32_t hl8[2], hr8[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = hj[k], y = by0 - 1 + j;
    const bool frame = j < bh + 2, rin = frame && y >= 0 && y < H;
    const bool lin = rin && bx0 > 0, rinr = rin && bx0 + bw < W;
    const int64_t yy = rin ? y : by0;
    const uint32_t l8 = a.holes[yy * a.holes_pitch + (lin ? bx0 - 1 : bx0)];
    const uint32_t r8 = a.holes[yy * a.holes_pitch + (rinr ? bx0 + bw : bx0)];
    hl8[k] = lin ? l8 : frame ? 3u : 0u;
    hr8[k] = rinr ? r8 : frame ? 3u : 0u;
  }
  const uint32_t rows = bh >= 32 ? 0xFFFFFFFFu : (1u << bh) - 1u;  // the block's rows (bit y = row y)
  // a column's damage in the frame rows (bit 0: the row above the block, bit 1: the row below)
  auto frame_bits = [&](uint64_t f) -> uint32_t {
    return static_cast<uint32_t>(f & 1ull) | (static_cast<uint32_t>((f >> (bh + 1)) & 1ull) << 1);
  };
  // ... and as a mask of frame rows, to be OR-ed with a column's block rows shifted up by one
  auto frame_mask = [&](uint32_t fb) -> uint64_t {
    return static_cast<uint64_t>(fb & 1u) | (static_cast<uint64_t>(fb >> 1) << (bh + 1));
  };
  do {
  uint8_t *view = a.view[v];
  const uint64_t fl = col ? (v ? fl1 : fl0) : ~0ull;  // frame rows
  // damaged block rows of this lane's column (bit y = block row y); every row beyond a
  // real column counts as damaged
  uint32_t own = col ? static_cast<uint32_t>(fl >> 1) & rows : 0xFFFFFFFFu;
  if (!__any_sync(0xffffffffu, col && own != 0u)) continue;
  const uint32_t own0 = own;
  const uint64_t halo_l = __ballot_sync(0xffffffffu, (hl8[0] >> v) & 1u) |
                          (static_cast<uint64_t>(__ballot_sync(0xffffffffu, (hl8[1] >> v) & 1u) & 3u) << 32);
  const uint64_t halo_r = __ballot_sync(0xffffffffu, (hr8[0] >> v) & 1u) |
                          (static_cast<uint64_t>(__ballot_sync(0xffffffffu, (hr8[1] >> v) & 1u) & 3u) << 32);
  {
    // ---- colours of the frame into the cells: undamaged pixels their colour, damaged ones
    // 0; kBatch rows of loads in flight at a time
    constexpr int kBatch = 10;
    for (int j0 = 0; j0 < bh + 2; j0 += kBatch) {
      uint32_t c0[kBatch], c1[kBatch], c2[kBatch];
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        const int j = j0 + t;
        const bool need = col && j < bh + 2 && !((fl >> j) & 1ull);
        c0[t] = c1[t] = c2[t] = 0u;
        if (need) {
          const uint8_t *px = view + static_cast<int64_t>(by0 - 1 + j) * a.pitch + 3 * static_cast<int64_t>(x);
          c0[t] = px[0];
          c1[t] = px[1];
          c2[t] = px[2];
        }
      }
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        const int j = j0 + t;
        if (col && j < bh + 2) cell[j * kStride + lane + 1] = c0[t] | (c1[t] << 8) | (c2[t] << 16);
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int j = hj[k];
      if (j < bh + 2) {
        const int64_t ro = static_cast<int64_t>(by0 - 1 + j) * a.pitch;
        uint32_t cl = 0u, cr = 0u;
        if (!((halo_l >> j) & 1ull)) {
          const uint8_t *px = view + ro + 3 * static_cast<int64_t>(bx0 - 1);
          cl = px[0] | (px[1] << 8) | (px[2] << 16);
        }
        if (!((halo_r >> j) & 1ull)) {
          const uint8_t *px = view + ro + 3 * static_cast<int64_t>(bx0 + bw);
          cr = px[0] | (px[1] << 8) | (px[2] << 16);
        }
        cell[j * kStride] = cl;
        cell[j * kStride + bw + 1] = cr;
      }
    }
    __syncwarp();

    // the neighbouring columns' damage (block rows, from their lanes or the halo) and the
    // frame rows of all three columns (constant)
    const uint32_t fo = col ? frame_bits(fl) : 3u;
    uint32_t fl_l = __shfl_up_sync(0xffffffffu, fo, 1), fl_r = __shfl_down_sync(0xffffffffu, fo, 1);
    if (lane == 0) fl_l = frame_bits(halo_l);
    if (lane == bw - 1) fl_r = frame_bits(halo_r);
    const uint64_t F_l = frame_mask(fl_l), F_o = frame_mask(fo), F_r = frame_mask(fl_r);
    const uint32_t hl = static_cast<uint32_t>(halo_l >> 1) & rows, hr = static_cast<uint32_t>(halo_r >> 1) & rows;
    uint32_t lm = 0, rm = 0;
    auto refresh = [&]() {
      lm = __shfl_up_sync(0xffffffffu, own, 1);
      rm = __shfl_down_sync(0xffffffffu, own, 1);
      if (lane == 0) lm = hl;
      if (lane == bw - 1) rm = hr;
    };
    // The visit of damaged block row r of this lane's column: with two or more undamaged
    // neighbours the pixel takes their mean colour and is no longer damaged.
    auto visit = [&](int r) -> bool {
      // rows r - 1, r (the pixel's own), r + 1 of the three columns (row -1 and row bh are
      // the frame rows: bit k of a column mask shifted up by one is frame row k)
      const uint32_t bl = static_cast<uint32_t>(((static_cast<uint64_t>(lm) << 1) | F_l) >> r) & 7u;
      const uint32_t bo = static_cast<uint32_t>(((static_cast<uint64_t>(own) << 1) | F_o) >> r) & 5u;
      const uint32_t br = static_cast<uint32_t>(((static_cast<uint64_t>(rm) << 1) | F_r) >> r) & 7u;
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
      own &= ~(1u << r);
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
    // dirty damaged rows of this lane's column (always a subset of own; none past a real
    // column)
    const uint32_t live = col ? rows : 0u;  // the rows that can be dirty in this lane
    uint32_t dirty = own & live;
    refresh();
    const int x2 = 2 * lane;
    // block rows of this lane's column visited at step t: y = t - 2x - 4p, p >= 0, y >= 0
    auto window = [&](int t) -> uint32_t {
      const int b = t - x2;
      return b < 0 ? 0u : (0x11111111u << (b & 3)) & (b >= 31 ? 0xFFFFFFFFu : (2u << b) - 1u);
    };
    // the first step at or after t with a visit to make, over the warp (INT_MAX: none): t
    // when the lane has a dirty row it has reached (visited within 4 steps), else the first
    // visit of its lowest dirty row, 2x + y; both are max(t, 2x + lowest dirty row)
    auto next_step = [&](int t) -> int {
      const int n = dirty ? max(t, x2 + __ffs(dirty) - 1) : 0x7FFFFFFF;
      return __reduce_min_sync(0xffffffffu, n);
    };
    int t = next_step(0);
    uint32_t win = window(t);
    while (t != 0x7FFFFFFF) {
      uint32_t cand = dirty & win;
      // a step with visits goes on to the next step; after a step without any, the warp
      // jumps to the first step with a visit to make (or ends)
      if (__any_sync(0xffffffffu, cand != 0u)) {
        uint32_t mine = 0;
        while (cand) {
          const int y = __ffs(cand) - 1;
          cand &= cand - 1;
          dirty &= ~(1u << y);
          if (visit(y)) mine |= 1u << y;
        }
        __syncwarp();
        // new neighbour columns; the damaged neighbours of every repair become dirty
        const uint32_t ol = lm, orr = rm;
        refresh();
        const uint32_t gone = (ol & ~lm) | (orr & ~rm) | mine;
        dirty |= (gone | (gone << 1) | (gone >> 1)) & own & live;
        ++t;
        // the window of step t + 1: one row further, and row 0 when t + 1 - 2x is 0 mod 4
        win = (win << 1) | (((t - x2) & static_cast<int>(0x80000003u)) == 0 ? 1u : 0u);
      } else {
        t = next_step(t + 1);
        win = window(t);
      }
    }
    // ---- repaired pixels back into the view, and the formatted outputs where it changed:
    // the anaglyph takes red from the left view and green, blue from the right one; a
    // half side-by-side pixel is the rounded-up mean of the pair (x, x + 1) of its view
    // (blocks start at even columns and have even widths), from the cells, or from the view
    // for a pixel left damaged (it keeps the colour of the row fill)
    const uint32_t rep = col ? (own0 & ~own & rows) : 0u;
    const uint32_t pair = rep | __shfl_down_sync(0xffffffffu, rep, 1);
    const uint32_t own_n = __shfl_down_sync(0xffffffffu, own, 1);
    uint32_t left = rep;
    while (left) {
      const int y = __ffs(left) - 1;  // block row; frame row y + 1
      left &= left - 1;
      const int64_t iy = by0 + y;
      const uint32_t c = cell[(y + 1) * kStride + lane + 1];
      store_rgb(view + iy * a.pitch + 3 * static_cast<int64_t>(x), c);
      if (a.ana) {
        uint8_t *d = a.ana + iy * a.out_pitch + 3 * static_cast<int64_t>(x);
        if (v == 0) {
          d[0] = static_cast<uint8_t>(c);
        } else {
          d[1] = static_cast<uint8_t>(c >> 8);
          d[2] = static_cast<uint8_t>(c >> 16);
        }
      }
    }
    if (a.hsbs && col && (lane & 1) == 0) {
      uint32_t m = pair;
      while (m) {
        const int y = __ffs(m) - 1;
        m &= m - 1;
        const int64_t iy = by0 + y;
        const uint8_t *p = view + iy * a.pitch + 3 * static_cast<int64_t>(x);
        const uint32_t ca = ((own >> y) & 1u) ? (p[0] | (p[1] << 8) | (p[2] << 16)) : cell[(y + 1) * kStride + lane + 1];
        const uint32_t cb = ((own_n >> y) & 1u) ? (p[3] | (p[4] << 8) | (p[5] << 16)) : cell[(y + 1) * kStride + lane + 2];
        const uint32_t mean = (ca | cb) - (((ca ^ cb) >> 1) & 0x7F7F7F7Fu);  // per byte (a + b + 1) >> 1
        store_rgb(a.hsbs + iy * a.out_pitch + 3 * static_cast<int64_t>((v ? W / 2 : 0) + x / 2), mean);
      }
    }
  }
  } while (false);
}

// Persistent: one warp per CTA and as many CTAs as fit the GPU at once; each takes the next
// work item of the order (heaviest first) until none is left.
__global__ void __launch_bounds__(32, 32) inpaint_kernel(const __grid_constant__ InpaintArgs a) {
  // The next band launch on the stream may start as soon as every CTA of this one runs: its
  // CTAs take the SM slots that this launch's finished warps leave while its longest items
  // finish (it waits for this launch before any global access unless the host knows their
  // buffers are disjoint).
  griddep_launch_dependents();
  __shared__ uint32_t cell[kStride * kStride];
  // the order holds nh heavy items at its front and nl others at its back
  const int items = 2 * a.nblocks, nh = a.order[items], nl = a.order[items + 1];
  int *next = a.order + items + 2;
  while (true) {
    int i = 0;
    if (threadIdx.x == 0) i = atomicAdd(next, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= nh + nl) break;
    inpaint_block(a, a.order[i < nh ? i : items - nl + (i - nh)], cell);
    __syncwarp();  // the cells are reused by the next item
  }
}

}  // namespace

cudaError_t launch_inpaint(const InpaintArgs &a, cudaStream_t st) {
  if (a.nblocks <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.order + 2 * a.nblocks, 0, 3 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  inpaint_rank_kernel<<<(a.nblocks + 7) / 8, 256, 0, st>>>(a);
  inpaint_kernel<<<std::min(2 * a.nblocks, 32 * a.sms), 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dibr
