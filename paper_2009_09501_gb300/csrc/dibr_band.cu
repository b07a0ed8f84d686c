// dibr_band.cu -- the fused per-frame DIBR kernel for sm_103a.
//
// One CTA owns a contiguous range of rows of one image and streams them through shared
// memory.  Per row it runs every stage of the pipeline of Sec. 3 / Sec. 4 of the paper:
//   depth (luminance) -> depth smoothing -> depth-to-shift table (Fig. 3) -> forward warp
//   of the left and right views with occlusion -> row-local hole fill (inpainting) ->
//   stereo formatting (anaglyph, L/R pair, half side-by-side, depth).
// Nothing but the input and the requested outputs touches HBM: luminance, depth, the
// z-buffers and the shift tables live in shared memory and registers.
//
// Warp roles: warps 0..nc/32-1 are consumers (each thread owns 16-pixel chunks of a
// row); the last warp is the producer, which streams input rows into a ring of
// shared-memory slots with 2-D TMA tensor loads (cp.async.bulk.tensor), completion
// tracked by mbarriers.  Every wait is bounded (%globaltimer); a wait that gives up sets
// a bit of the status word and the CTA unwinds.
#include "dibr.h"
#include "dibr_internal.h"
#include "dibr_ptx.cuh"

namespace dibr {
namespace {

__device__ __forceinline__ uint32_t bsel(const uint32_t *w, int j) {
  return (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
}

__device__ __forceinline__ void lds48(const uint8_t *s, uint32_t (&w)[12]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(s);
  const uint4 a = p[0], b = p[1], c = p[2];
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
  w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
}

// BT.601 luminance in exact thousandths, rounded half up (the depth-map reading).
__device__ __forceinline__ uint32_t luma8(uint32_t r, uint32_t g, uint32_t b) {
  return (299u * r + 587u * g + 114u * b + 500u) / 1000u;
}

__device__ __forceinline__ uint4 luma_chunk(const uint32_t (&w)[12]) {
  uint32_t y[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 16; ++i)
    y[i >> 2] |= luma8(bsel(w, 3 * i), bsel(w, 3 * i + 1), bsel(w, 3 * i + 2)) << (8 * (i & 3));
  return make_uint4(y[0], y[1], y[2], y[3]);
}

// 5x5 binomial smoothing of the luminance for the 16 pixels of one chunk:
// D = (sum_ij b_i b_j Y[clamp(y+i)][clamp(x+j)] + 128) >> 8, b = (1 4 6 4 1).
__device__ __forceinline__ uint4 binom5_chunk(const uint8_t *yring, int ystride, int y, int H,
                                              int W, int x0) {
  const uint8_t *rows[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int r = min(max(y + i - 2, 0), H - 1);
    rows[i] = yring + (r % kYRing) * ystride;
  }
  const uint32_t kb[5] = {1u, 4u, 6u, 4u, 1u};
  uint32_t V[20];
#pragma unroll
  for (int j = 0; j < 20; ++j) V[j] = 0u;
  if (x0 >= 4 && x0 + 18 <= W) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint8_t *p = rows[i] + x0;
      const uint32_t l = *reinterpret_cast<const uint32_t *>(p - 4);
      const uint4 m = *reinterpret_cast<const uint4 *>(p);
      const uint32_t r = *reinterpret_cast<const uint32_t *>(p + 16);
      const uint32_t w[6] = {l, m.x, m.y, m.z, m.w, r};
#pragma unroll
      for (int j = 0; j < 20; ++j) V[j] += kb[i] * bsel(w, j + 2);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 20; ++j) {
      const int xc = min(max(x0 - 2 + j, 0), W - 1);
#pragma unroll
      for (int i = 0; i < 5; ++i) V[j] += kb[i] * rows[i][xc];
    }
  }
  uint32_t d[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t s = V[i] + 4u * V[i + 1] + 6u * V[i + 2] + 4u * V[i + 3] + V[i + 4];
    d[i >> 2] |= ((s + 128u) >> 8) << (8 * (i & 3));
  }
  return make_uint4(d[0], d[1], d[2], d[3]);
}

// z-buffer key: (depth + 1) in the high half (0 = empty target), source column in the
// low half, reversed in the left view so that atomicMax prefers the smaller column.
__device__ __forceinline__ int key_src(uint32_t k, bool left) {
  const uint32_t lo = k & 0xFFFFu;
  return left ? static_cast<int>(0xFFFFu - lo) : static_cast<int>(lo);
}

// Row-local hole fill: nearest filled target on each side; the one with the smaller
// depth (background) wins, the left one on a tie; a single side wins alone; with none,
// the target keeps its own input column.
__device__ __noinline__ int fill_src(const uint32_t *zb, int t, int W, bool left) {
  int l = t - 1;
  while (l >= 0 && zb[l] == 0u) --l;
  int r = t + 1;
  while (r < W && zb[r] == 0u) ++r;
  const uint32_t kl = l >= 0 ? zb[l] : 0u, kr = r < W ? zb[r] : 0u;
  uint32_t k;
  if (kl && kr) k = (kl >> 16) <= (kr >> 16) ? kl : kr;
  else if (kl) k = kl;
  else if (kr) k = kr;
  else return t;
  return key_src(k, left);
}

// Packed RGB (3 bytes) of column x of a row held in shared memory.
__device__ __forceinline__ uint32_t rgb_at(const uint8_t *row, int x) {
  const uint32_t off = 3u * static_cast<uint32_t>(x);
  const uint32_t *wp = reinterpret_cast<const uint32_t *>(row + (off & ~3u));
  return __funnelshift_r(wp[0], wp[1], (off & 3u) * 8u) & 0xFFFFFFu;
}

// Places the 3 bytes of c at pixel i of a packed RGB word array.
template <int N>
__device__ __forceinline__ void put3(uint32_t (&w)[N], int i, uint32_t c) {
  const int o = 3 * i, j = o >> 2, s = (o & 3) * 8;
  w[j] |= c << s;
  if (s > 8) w[j + 1] |= c >> (32 - s);
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

__global__ void __launch_bounds__(kMaxConsumers + 32, 1)
    band_kernel(const __grid_constant__ BandArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const BandSmem L = band_smem_layout(a.nb, a.srow, a.ystride, a.nch, a.depth_src);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bar);
  uint64_t *empty = full + kMaxRing;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.flags);
  int32_t *lut_h = reinterpret_cast<int32_t *>(smem + L.lut);
  int32_t *lut_n = reinterpret_cast<int32_t *>(smem + L.zb);  // gather mode only
  uint8_t *ring = smem + L.ring;
  uint8_t *yring = smem + L.yring;
  uint8_t *drow = smem + L.drow;
  uint32_t *zbL = reinterpret_cast<uint32_t *>(smem + L.zb);
  uint32_t *zbR = zbL + a.nch * kChunk;

  const int tid = threadIdx.x, nc = a.nc, W = a.W, H = a.H, nb = a.nb;
  const int ys = static_cast<int>(static_cast<int64_t>(blockIdx.x) * H / a.grid);
  const int ye = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * H / a.grid);
  const bool binom = a.depth_src == DS_BINOM5;
  const int halo = binom ? 2 : 0;
  const int la = max(ys - halo, 0), lb = min(ye + halo, H);

  const bool forward = a.warp_mode == DIBR_WARP_FORWARD;
  for (int i = tid; i < 256; i += blockDim.x) {
    lut_h[i] = a.lut_h[i];
    if (!forward) lut_n[i] = a.lut_n[i];
  }
  if (tid == 0) {
    for (int i = 0; i < nb; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (ys >= ye) return;

  // ------------------------------------------------------------------ producer warp
  if (tid >= nc) {
    const int lane = tid - nc;
    if (lane == 0) prefetch_tensormap(&a.tmap);
    int issued = 0;
    bool ok = true;
    for (int k = 0; k < lb - la; ++k) {
      const int s = k % nb;
      if (k >= nb) {
        int got = 1;
        if (lane == 0) {
          const unsigned long long t0 = global_ns();
          while (!mbar_try_wait(&empty[s], ((k / nb) - 1) & 1)) {
            if (*abort_flag || global_ns() - t0 > a.timeout_ns) {
              got = 0;
              break;
            }
          }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
      }
      if (lane == 0) mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>(a.nbox * kBoxBytes));
      __syncwarp();
      uint8_t *dst = ring + s * a.srow;
      for (int i = lane; i < a.nbox; i += 32)
        tma_load_2d(dst + i * kBoxBytes, &a.tmap, i * kBoxBytes, la + k, &full[s]);
      issued = k + 1;
    }
    if (!ok && lane == 0) {
      if (!*abort_flag) atomicOr(a.status, ST_TIMEOUT_EMPTY);
      // let every copy already issued land before the CTA's shared memory goes away
      for (int k = max(0, issued - nb); k < issued; ++k)
        if (!mbar_wait_bounded(&full[k % nb], (k / nb) & 1, a.timeout_ns))
          atomicOr(a.status, ST_TIMEOUT_DRAIN);
    }
    return;
  }

  // ---------------------------------------------------------------------- consumers
  bool timed_out = false;
  auto slot = [&](int r) { return ring + ((r - la) % nb) * a.srow; };
  auto wait_row = [&](int r) {
    const int k = r - la;
    if (!mbar_wait_bounded(&full[k % nb], (k / nb) & 1, a.timeout_ns)) timed_out = true;
  };
  auto release_row = [&](int r) {
    if (tid == 0) mbar_arrive(&empty[(r - la) % nb]);
  };
  auto luma_row = [&](int r) {
    const uint8_t *src = slot(r);
    uint8_t *yd = yring + (r % kYRing) * a.ystride;
    for (int c = tid; c < a.nch; c += nc) {
      uint32_t w[12];
      lds48(src + 48 * c, w);
      *reinterpret_cast<uint4 *>(yd + 16 * c) = luma_chunk(w);
    }
  };

  const bool want_depth = (a.outputs & DIBR_OUT_DEPTH) != 0;
  const bool want_ana = (a.outputs & DIBR_OUT_ANAGLYPH) != 0;
  const bool want_l = (a.outputs & DIBR_OUT_LEFT) != 0;
  const bool want_r = (a.outputs & DIBR_OUT_RIGHT) != 0;
  const bool want_hsbs = (a.outputs & DIBR_OUT_HSBS) != 0;
  bool aborted = false;

  if (binom) {
    // luminance of the rows above the band and of the first rows of the band
    const int pend = min(ys + 2, lb - 1);
    for (int r = la; r <= pend; ++r) {
      wait_row(r);
      luma_row(r);
    }
    if (consumer_sync_or(timed_out, nc)) aborted = true;
    else
      for (int r = la; r <= pend; ++r)
        if (r < ys || r >= ye) release_row(r);
  }

  for (int y = ys; y < ye && !aborted; ++y) {
    // ---- phase A: depth of row y (and luminance of row y+3), clear the z-buffers
    if (binom) {
      const int r3 = y + 3;
      if (r3 < lb) {
        wait_row(r3);
        luma_row(r3);
      }
    } else {
      wait_row(y);
    }
    for (int c = tid; c < a.nch; c += nc) {
      const int x0 = c * kChunk;
      uint4 d;
      if (binom) {
        d = binom5_chunk(yring, a.ystride, y, H, W, x0);
      } else if (a.depth_src == DS_LUMA) {
        uint32_t w[12];
        lds48(slot(y) + 48 * c, w);
        d = luma_chunk(w);
      } else {
        const uint8_t *dp = a.depth_in + static_cast<int64_t>(y) * a.depth_in_pitch + x0;
        const int npx = min(kChunk, W - x0);
        if (npx == kChunk && (reinterpret_cast<uintptr_t>(dp) & 15u) == 0) {
          d = *reinterpret_cast<const uint4 *>(dp);
        } else {
          uint32_t w[4] = {0u, 0u, 0u, 0u};
          for (int i = 0; i < npx; ++i) w[i >> 2] |= static_cast<uint32_t>(dp[i]) << (8 * (i & 3));
          d = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      *reinterpret_cast<uint4 *>(drow + x0) = d;
      if (want_depth)
        store16(a.out[O_DEPTH] + static_cast<int64_t>(y) * a.depth_pitch + x0, d,
                min(kChunk, W - x0));
      if (forward) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        uint4 *zl = reinterpret_cast<uint4 *>(zbL + x0);
        uint4 *zr = reinterpret_cast<uint4 *>(zbR + x0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          zl[q] = z;
          zr[q] = z;
        }
      }
    }
    if (consumer_sync_or(timed_out, nc)) {
      aborted = true;
      break;
    }

    // ---- phase B: forward warp, occlusion by atomicMax on (depth, column) keys
    if (forward) {
      for (int c = tid; c < a.nch; c += nc) {
        const int x0 = c * kChunk;
        const uint4 dq = *reinterpret_cast<const uint4 *>(drow + x0);
        const uint32_t dw[4] = {dq.x, dq.y, dq.z, dq.w};
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
          const int x = x0 + i;
          if (x < W) {
            const uint32_t d = bsel(dw, i);
            const int32_t lh = lut_h[d];
            const int hl = static_cast<int16_t>(lh & 0xFFFF), hr = lh >> 16;
            const int tl = x - hl, tr = x - hr;
            if (static_cast<unsigned>(tl) < static_cast<unsigned>(W))
              atomicMax(&zbL[tl], ((d + 1u) << 16) | (0xFFFFu - static_cast<uint32_t>(x)));
            if (static_cast<unsigned>(tr) < static_cast<unsigned>(W))
              atomicMax(&zbR[tr], ((d + 1u) << 16) | static_cast<uint32_t>(x));
          }
        }
      }
    }
    consumer_sync(nc);

    // ---- phase C: resolve winners, fill holes, compose and store the outputs
    const uint8_t *rgbrow = slot(y);
    for (int c = tid; c < a.nch; c += nc) {
      const int x0 = c * kChunk;
      const int npx = min(kChunk, W - x0);
      uint32_t cl[16], cr[16];
      if (forward) {
        const uint4 *zl = reinterpret_cast<const uint4 *>(zbL + x0);
        const uint4 *zr = reinterpret_cast<const uint4 *>(zbR + x0);
        uint32_t kL[16], kR[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 u = zl[q], v = zr[q];
          kL[4 * q] = u.x; kL[4 * q + 1] = u.y; kL[4 * q + 2] = u.z; kL[4 * q + 3] = u.w;
          kR[4 * q] = v.x; kR[4 * q + 1] = v.y; kR[4 * q + 2] = v.z; kR[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
          if (i < npx) {
            const int sl = kL[i] ? key_src(kL[i], true) : fill_src(zbL, x0 + i, W, true);
            const int sr = kR[i] ? key_src(kR[i], false) : fill_src(zbR, x0 + i, W, false);
            cl[i] = rgb_at(rgbrow, sl);
            cr[i] = rgb_at(rgbrow, sr);
          } else {
            cl[i] = 0u;
            cr[i] = 0u;
          }
        }
      } else {
        // Fig. 3 literally: sample trunc(x + s(d)); out of range -> own column
        const uint4 dq = *reinterpret_cast<const uint4 *>(drow + x0);
        const uint32_t dw[4] = {dq.x, dq.y, dq.z, dq.w};
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
          if (i < npx) {
            const int x = x0 + i;
            const int n = lut_n[bsel(dw, i)];
            int sl = (510 * x + n) / 510, sr = (510 * x - n) / 510;
            if (static_cast<unsigned>(sl) >= static_cast<unsigned>(W)) sl = x;
            if (static_cast<unsigned>(sr) >= static_cast<unsigned>(W)) sr = x;
            cl[i] = rgb_at(rgbrow, sl);
            cr[i] = rgb_at(rgbrow, sr);
          } else {
            cl[i] = 0u;
            cr[i] = 0u;
          }
        }
      }
      const int64_t ro = static_cast<int64_t>(y) * a.out_pitch;
      if (want_l) {
        uint32_t w[12] = {0u};
#pragma unroll
        for (int i = 0; i < 16; ++i) put3(w, i, cl[i]);
        store48(a.out[O_LEFT] + ro + 3 * x0, w, npx);
      }
      if (want_r) {
        uint32_t w[12] = {0u};
#pragma unroll
        for (int i = 0; i < 16; ++i) put3(w, i, cr[i]);
        store48(a.out[O_RIGHT] + ro + 3 * x0, w, npx);
      }
      if (want_ana) {
        uint32_t w[12] = {0u};
#pragma unroll
        for (int i = 0; i < 16; ++i) put3(w, i, (cl[i] & 0x0000FFu) | (cr[i] & 0xFFFF00u));
        store48(a.out[O_ANA] + ro + 3 * x0, w, npx);
      }
      if (want_hsbs) {
        uint32_t wl[6] = {0u}, wr[6] = {0u};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          put3(wl, j, avg_up(cl[2 * j], cl[2 * j + 1]) & 0xFFFFFFu);
          put3(wr, j, avg_up(cr[2 * j], cr[2 * j + 1]) & 0xFFFFFFu);
        }
        const int np = npx / 2;  // W is even, so chunks hold whole pairs
        store24(a.out[O_HSBS] + ro + 3 * (x0 / 2), wl, np);
        store24(a.out[O_HSBS] + ro + 3 * (W / 2 + x0 / 2), wr, np);
      }
    }
    consumer_sync(nc);
    release_row(y);
    if (binom && y + 3 < lb && y + 3 >= ye) release_row(y + 3);
  }

  if (aborted && tid == 0) {
    *abort_flag = 1;
    atomicOr(a.status, ST_TIMEOUT_FULL);
  }
}

}  // namespace

cudaError_t launch_band(const BandArgs &a, int smem_bytes, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  band_kernel<<<a.grid, a.nc + 32, smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dibr
