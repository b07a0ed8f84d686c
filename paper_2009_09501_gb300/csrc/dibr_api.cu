// dibr_api.cu -- the C-ABI of libdibr (declared in include/dibr.h): contexts, argument
// checks, the depth-to-shift tables of Fig. 3, TMA descriptors, staging of host
// buffers, and the launches of the fused kernels.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dibr.h"
#include "dibr_context.h"
#include "dibr_internal.h"

using namespace dibr;

// ------------------------------------------------------------------------ helpers
void dibr_ctx::set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::lock_guard<std::mutex> g(err_mu);
  last_error = buf;
}

dibr_status dibr_ctx::cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return DIBR_E_CUDA;
}

void *dibr_ctx::dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (alloc_hook) return alloc_hook(bytes, alloc_user);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dibr_ctx::dev_free(void *p) {
  if (!p) return;
  if (free_hook) free_hook(p, alloc_user);
  else cudaFreeAsync(p, stream);
}

dibr_status dibr_ctx::ensure(DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes && b.ptr) return DIBR_OK;
  prev_band = false;  // the stream-ordered free and allocation below are work on the stream
  if (b.ptr) {
    cudaStreamSynchronize(stream);
    dev_free(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  b.ptr = static_cast<uint8_t *>(dev_alloc(bytes));
  if (!b.ptr) {
    set_error("device allocation of %zu bytes failed", bytes);
    return DIBR_E_NOMEM;
  }
  b.bytes = bytes;
  return DIBR_OK;
}

// ------------------------------------------------------------- parameter checking
static bool valid_enum(int v, int lo, int hi) { return v >= lo && v <= hi; }

static dibr_status check_params(const dibr_params *p, const dibr_image *img, std::string *why) {
  if (!p) { *why = "params is NULL"; return DIBR_E_INVALID; }
  if (!valid_enum(p->depth_rule, 0, 2)) { *why = "unknown depth_rule"; return DIBR_E_INVALID; }
  if (!valid_enum(p->disparity_rule, 0, 1)) { *why = "unknown disparity_rule"; return DIBR_E_INVALID; }
  if (!valid_enum(p->warp_mode, 0, 1)) { *why = "unknown warp_mode"; return DIBR_E_INVALID; }
  if (p->warp_mode == DIBR_WARP_GATHER_FIG3 && p->disparity_rule != DIBR_DISP_PAPER) {
    *why = "the Fig. 3 gather mode is defined for the paper's disparity rule only";
    return DIBR_E_INVALID;
  }
  if (p->max_parallax_px < 0 || p->max_parallax_px > 1024) { *why = "max_parallax_px outside 0..1024"; return DIBR_E_INVALID; }
  if (p->threshold < 0 || p->threshold > 255) { *why = "threshold outside 0..255"; return DIBR_E_INVALID; }
  if (p->depth_rule == DIBR_DEPTH_LUMA_XBF) {
    if (!(p->xbf_sigma_s > 0.f) || !(p->xbf_sigma_r > 0.f) || p->xbf_radius < 1 || p->xbf_radius > 8) {
      *why = "cross-bilateral parameters out of range (sigmas > 0, radius 1..8)";
      return DIBR_E_INVALID;
    }
  }
  if (p->outputs == 0 || (p->outputs & ~kAllOutputs)) { *why = "outputs must be a non-empty set of DIBR_OUT_* bits"; return DIBR_E_INVALID; }
  if (!valid_enum(p->hole_fill, 0, 1)) { *why = "unknown hole_fill"; return DIBR_E_INVALID; }
  if (p->hole_fill == DIBR_FILL_INPAINT2D) {
    if (p->inpaint_block < 1 || p->inpaint_block > 32) { *why = "inpaint_block outside 1..32"; return DIBR_E_INVALID; }
    if ((p->outputs & DIBR_OUT_HSBS) && (p->inpaint_block & 1)) {
      *why = "the 2-D fill with HSBS needs an even inpaint_block";
      return DIBR_E_INVALID;
    }
  }
  if (img) {
    if (img->width < 1 || img->height < 1 || img->width > kMaxWidth || img->height > 65535) {
      *why = "image size outside 1..7680 x 1..65535";
      return DIBR_E_INVALID;
    }
    if (!img->rgb) { *why = "image pointer is NULL"; return DIBR_E_INVALID; }
    if (img->pitch < 3 * static_cast<int64_t>(img->width)) { *why = "pitch < 3*width"; return DIBR_E_INVALID; }
    if ((p->outputs & DIBR_OUT_HSBS) && (img->width & 1)) { *why = "HSBS needs an even width"; return DIBR_E_INVALID; }
  }
  return DIBR_OK;
}

static dibr_status check_outputs(const dibr_params *p, const dibr_image *img, const dibr_outputs *o,
                                 std::string *why) {
  if (!o) { *why = "outputs is NULL"; return DIBR_E_INVALID; }
  bool rgb_out = false, map_out = false;
  for (int i = 0; i < O_COUNT; ++i) {
    if (!(p->outputs & kOutBits[i])) continue;
    if (!out_slot(*o, i)) { *why = "a requested output pointer is NULL"; return DIBR_E_INVALID; }
    (is_map_output(i) ? map_out : rgb_out) = true;
  }
  if (rgb_out && o->pitch < 3 * static_cast<int64_t>(img->width)) { *why = "output pitch < 3*width"; return DIBR_E_INVALID; }
  if (map_out && o->depth_pitch < img->width) { *why = "depth_pitch < width"; return DIBR_E_INVALID; }
  return DIBR_OK;
}

// ----------------------------------------------------- depth -> shift tables (Fig. 3)
static int64_t floor_div510(int64_t a) {  // floor(a / 510)
  int64_t q = a / 510;
  if (a % 510 != 0 && a < 0) --q;
  return q;
}

// Fig. 3: s_L(d) = -(P/2) d/255 (d > T) or (P/2)(1 - d/255); numerator over 510.
static int64_t shift_num510(int d, int P, int T) {
  return d > T ? -static_cast<int64_t>(P) * d : static_cast<int64_t>(P) * (255 - d);
}

static void build_tables(const dibr_params *p, int16_t *hL, int16_t *hR, int32_t *num) {
  for (int d = 0; d < 256; ++d) {
    if (p->disparity_rule == DIBR_DISP_PAPER) {
      const int64_t n = shift_num510(d, p->max_parallax_px, p->threshold);
      hL[d] = static_cast<int16_t>(floor_div510(n));
      hR[d] = static_cast<int16_t>(floor_div510(-n));
      if (num) num[d] = static_cast<int32_t>(n);
    } else {
      const int64_t m = static_cast<int64_t>(p->max_parallax_px) * d / 510;
      hL[d] = static_cast<int16_t>(-m);
      hR[d] = static_cast<int16_t>(m);
      if (num) num[d] = static_cast<int32_t>(-510 * m);
    }
  }
}

namespace dibr {
// Argument checks of one image (params, input, outputs), for the batch entry points.
dibr_status check_image_args(const dibr_params *p, const dibr_image *img, const dibr_outputs *o, std::string *why) {
  dibr_status s = check_params(p, img, why);
  if (s == DIBR_OK) s = check_outputs(p, img, o, why);
  return s;
}

// The kernels' packed tables: lut_h[d] = (hR << 16) | (hL & 0xFFFF); lut_n[d] = 510 * s_L(d).
void shift_tables(const dibr_params *p, int32_t *lut_h, int32_t *lut_n) {
  int16_t hL[256], hR[256];
  build_tables(p, hL, hR, lut_n);
  for (int d = 0; d < 256; ++d)
    lut_h[d] = static_cast<int32_t>((static_cast<uint32_t>(static_cast<uint16_t>(hR[d])) << 16) |
                                    static_cast<uint16_t>(hL[d]));
}
}  // namespace dibr

// ---------------------------------------------------------------- launch planning
static PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

int dibr_ctx::band_tables(const dibr_params *p) {
  const int32_t key[3] = {p->disparity_rule, p->max_parallax_px, p->threshold};
  if (key[0] != args_tables_key[0] || key[1] != args_tables_key[1] || key[2] != args_tables_key[2]) {
    shift_tables(p, args.lut_h, args.lut_n);
    args_zguard = zguard_of(args.lut_h);
    for (int i = 0; i < 3; ++i) args_tables_key[i] = key[i];
  }
  return args_zguard;
}

dibr_status dibr_ctx::plan_band(int W, int H, int depth_src, const uint8_t *in, int64_t pitch, int zguard,
                               BandArgs &a, int &smem, int &per_sm) {
  a.W = W;
  a.H = H;
  a.nch = (W + kChunk - 1) / kChunk;
  a.nc = round_up(a.nch, 32);  // one 16-pixel chunk per consumer thread
  a.zguard = zguard;
  // how rows reach shared memory: the tuned mode when the image allows it, else the
  // automatic choice (one bulk copy per row when rows are whole 16-byte units)
  const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15u) == 0 && (pitch & 15) == 0;
  int mode = tuning.load_mode;
  const int row = 3 * W;
  auto fits = [&](int m) {
    if (m == 1) return aligned && row % 16 == 0;
    if (m == 2) return aligned && row % 16 == 0;
    if (m == 3) return aligned && row % 128 == 0;
    if (m == 4) return aligned && row % 256 == 0;
    return m == 5;
  };
  if (mode == 0) mode = fits(1) ? 1 : 5;
  if (!fits(mode)) mode = 5;
  a.row_bytes = row;
  a.in = in;
  a.in_pitch = pitch;
  if (mode == 1) {
    a.load_mode = LM_BULK;
    a.nbox = 1;
    a.box_bytes = row;
    a.box_step = 0;
  } else if (mode <= 4) {
    const int inner = mode == 2 ? 16 : mode == 3 ? 128 : 256;
    const int n = row / inner;
    a.load_mode = LM_T3;
    a.tinner = inner;
    a.nbox = (n + 255) / 256;
    a.box_step = round_up((n + a.nbox - 1) / a.nbox, inner >= 128 ? 1 : 128 / inner);  // 128-byte aligned boxes
    a.box_bytes = inner * a.box_step;
  } else {
    a.load_mode = LM_T2;
    a.nbox = (row + kBoxBytes - 1) / kBoxBytes;
    a.box_step = kBoxBytes;
    a.box_bytes = kBoxBytes;
  }
  a.l2_prefetch = tuning.l2_prefetch == 1 ? 1 : 0;
  a.srow = round_up(std::max(a.nbox * a.box_bytes, 48 * a.nch), 128);
  a.depth_src = depth_src;
  const int min_nb = depth_src == DS_BINOM5 ? 4 : 2;
  const int max_nb = tuning.ring_slots > 0 ? std::max(min_nb, std::min(kMaxRing, tuning.ring_slots)) : kMaxRing;
  // at most 128 registers per thread (the kernel's launch bound) and 2048 threads per SM
  const int max_per = std::max(1, std::min(65536 / (a.nc * 128), 2048 / a.nc));
  auto per_for = [&](int nb) {
    const int tot = band_smem_layout(nb, a.srow, a.nch, a.nc / 32, zguard).total;
    if (tot > max_smem) return 0;
    int per = std::min(max_per, smem_per_sm / (tot + 1024));
    if (tuning.ctas_per_sm > 0) per = std::min(per, tuning.ctas_per_sm);
    return per;
  };
  int best = 0;
  for (int nb = min_nb; nb <= max_nb; ++nb) best = std::max(best, per_for(nb));
  if (best < 1) {
    set_error("width %d needs more shared memory than the device offers", W);
    return DIBR_E_INVALID;
  }
  int nb = min_nb;
  for (int k = min_nb; k <= max_nb; ++k)
    if (per_for(k) == best) nb = k;
  a.nb = nb;
  smem = band_smem_layout(nb, a.srow, a.nch, a.nc / 32, zguard).total;
  per_sm = best;
  a.grid = std::max(1, std::min(H, num_sms * per_sm));
  a.row0 = 0;
  a.row1 = H;
  a.overlap = 0;
  a.status = status_dev;
  a.timeout_ns = timeout_ns;
  return DIBR_OK;
}

dibr_status dibr_ctx::encode_input(BandArgs &a, const uint8_t *dev_rgb, int64_t pitch) {
  auto enc = get_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return DIBR_E_CUDA;
  }
  if (a.load_mode == LM_BULK) return DIBR_OK;  // no tensor map needed
  CUresult r;
  if (a.load_mode == LM_T3) {
    const cuuint64_t inner = static_cast<cuuint64_t>(a.tinner);
    cuuint64_t dims[3] = {inner, static_cast<cuuint64_t>(3) * a.W / inner, static_cast<cuuint64_t>(a.H)};
    cuuint64_t strides[2] = {inner, static_cast<cuuint64_t>(pitch)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(inner), static_cast<cuuint32_t>(a.box_step), 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(dev_rgb), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(3) * a.W, static_cast<cuuint64_t>(a.H)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kBoxBytes), 1u};
    cuuint32_t estr[2] = {1u, 1u};
    r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(dev_rgb), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return DIBR_E_CUDA;
  }
  return DIBR_OK;
}

// Every requested RGB output and the output pitch are 16-byte aligned: whole 16-column
// chunks are stored as three 16-byte words.
static int aligned_rgb_outputs(const BandArgs &a) {
  uintptr_t bits = static_cast<uintptr_t>(a.out_pitch);
  for (int i = 0; i < O_COUNT; ++i)
    if (!is_map_output(i) && (a.outputs & kOutBits[i])) bits |= reinterpret_cast<uintptr_t>(a.out[i]);
  return (bits & 15u) == 0 ? 1 : 0;
}

static bool tma_ok(const uint8_t *p, int64_t pitch) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (pitch & 15) == 0;
}

// Enqueues the whole pipeline for one image whose input and outputs are in device memory.
dibr_status dibr_ctx::enqueue_device(const dibr_image *img, const dibr_params *p, const dibr_outputs *o) {
  const int W = img->width, H = img->height;
  const uint8_t *in = img->rgb;
  int64_t pitch = img->pitch;
  // this launch may overlap the previous one (see below) only if that was the last work
  // on a stream the context owns
  const bool may_overlap = owns_stream && prev_band;
  prev_band = false;
  auto span = [](const uint8_t *ptr, int64_t row_pitch, int rows, int64_t row_bytes) {
    Span sp;
    sp.lo = reinterpret_cast<uintptr_t>(ptr);
    sp.hi = sp.lo + static_cast<uintptr_t>(row_pitch) * (rows - 1) + static_cast<uintptr_t>(row_bytes);
    return sp;
  };
  auto meets = [](const Span &x, const Span &y) { return x.lo < y.hi && y.lo < x.hi; };
  bool scratch = false;  // context buffers written before the band kernel
  bool realigned = false;
  if (!tma_ok(in, pitch)) {
    scratch = true;
    realigned = true;
    // TMA needs a 16-byte aligned base and pitch: repack into an aligned device buffer
    const int64_t ap = round_up(3 * W, 16);
    dibr_status s = ensure(realign, static_cast<size_t>(ap) * H);
    if (s != DIBR_OK) return s;
    cudaError_t e = cudaMemcpy2DAsync(realign.ptr, ap, in, pitch, 3 * static_cast<size_t>(W), H,
                                      cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "repacking the input");
    in = realign.ptr;
    pitch = ap;
  }
  int depth_src = p->depth_rule == DIBR_DEPTH_LUMA_BINOM5 ? DS_BINOM5
                  : p->depth_rule == DIBR_DEPTH_LUMA     ? DS_LUMA
                                                         : DS_GLOBAL;
  BandArgs &a = args;
  int smem = 0, per_sm = 1;
  const int zguard = band_tables(p);
  dibr_status s = plan_band(W, H, depth_src, in, pitch, zguard, a, smem, per_sm);
  if (s != DIBR_OK) return s;
  if ((s = encode_input(a, in, pitch)) != DIBR_OK) return s;
  Span cur_depth;  // the cross-bilateral depth this frame's band launch reads
  if (depth_src == DS_GLOBAL) {
    scratch = true;  // the band launch waits for the cross-bilateral one
    // two halves used by alternate frames, so that this frame's cross-bilateral launch may
    // start beside the previous frame's band launch: it reads this frame's input and writes
    // a half that launch does not read, when neither meets that launch's outputs
    const int64_t dp = round_up(W, 16);
    const size_t half = static_cast<size_t>(dp) * H;
    if ((s = ensure(xbf_depth, 2 * half)) != DIBR_OK) return s;
    uint8_t *dd = xbf_depth.ptr + xbf_half * half;
    xbf_half ^= 1;
    cur_depth = span(dd, dp, H, W);
    const Span xin = span(in, pitch, H, 3 * static_cast<int64_t>(W));
    bool after = may_overlap && !realigned && !meets(cur_depth, prev_in) && !meets(cur_depth, prev_depth);
    for (int i = 0; i < O_COUNT; ++i)
      if (prev_out[i].hi && (meets(xin, prev_out[i]) || meets(cur_depth, prev_out[i]))) after = false;
    cudaError_t e = launch_xbf(in, pitch, W, H, p->xbf_radius, p->xbf_sigma_s, p->xbf_sigma_r, dd, dp, stream,
                               after);
    if (e != cudaSuccess) return cuda_fail(e, "cross-bilateral launch");
    ++launches;
    a.depth_in = dd;
    a.depth_in_pitch = dp;
  } else {
    a.depth_in = nullptr;
    a.depth_in_pitch = 0;
  }
  for (int i = 0; i < O_COUNT; ++i) a.out[i] = out_slot(*o, i);
  a.out_pitch = o->pitch;
  a.depth_pitch = o->depth_pitch;
  a.outputs = p->outputs;
  a.warp_mode = p->warp_mode;
  // The 2-D fill inpaints both views in place after the band kernel, so that kernel also
  // writes both views and the holes map: into the caller's buffers when requested, else
  // into context scratch with the same row pitches (two halves used by alternate frames,
  // so that a frame's band launch may overlap the previous frame's inpainting).
  const bool inpaint = p->hole_fill == DIBR_FILL_INPAINT2D && p->warp_mode == DIBR_WARP_FORWARD;
  if (inpaint) {
    const uint32_t rgb = DIBR_OUT_ANAGLYPH | DIBR_OUT_LEFT | DIBR_OUT_RIGHT | DIBR_OUT_HSBS;
    const uint32_t maps = DIBR_OUT_DEPTH | DIBR_OUT_HOLES;
    const int64_t vp = (p->outputs & rgb) ? o->pitch : round_up(3 * W, 16);
    const int64_t hp = (p->outputs & maps) ? o->depth_pitch : round_up(W, 16);
    size_t need = 0;
    if (!(p->outputs & DIBR_OUT_LEFT)) need += static_cast<size_t>(vp) * H;
    if (!(p->outputs & DIBR_OUT_RIGHT)) need += static_cast<size_t>(vp) * H;
    if (!(p->outputs & DIBR_OUT_HOLES)) need += static_cast<size_t>(hp) * H;
    if (need && (s = ensure(inpaint_scratch, 2 * need)) != DIBR_OK) return s;
    size_t off = inpaint_half * need;
    inpaint_half ^= 1;
    auto take = [&](int slot, uint32_t bit, int64_t rows_pitch) {
      if (p->outputs & bit) return;
      a.out[slot] = inpaint_scratch.ptr + off;
      off += static_cast<size_t>(rows_pitch) * H;
    };
    take(O_LEFT, DIBR_OUT_LEFT, vp);
    take(O_RIGHT, DIBR_OUT_RIGHT, vp);
    take(O_HOLES, DIBR_OUT_HOLES, hp);
    a.out_pitch = vp;
    a.depth_pitch = hp;
    a.outputs |= DIBR_OUT_LEFT | DIBR_OUT_RIGHT | DIBR_OUT_HOLES;
  }
  a.fast_store = aligned_rgb_outputs(a);
  // Overlap with the previous band launch on the stream when neither reads or writes what
  // the other writes: this launch then starts in the SMs the previous one leaves and only
  // its exit waits for it.
  Span cur_in = span(in, pitch, H, 3 * static_cast<int64_t>(W)), cur_out[O_COUNT];
  for (int i = 0; i < O_COUNT; ++i)
    cur_out[i] = (a.outputs & kOutBits[i]) && a.out[i]
                     ? span(a.out[i], is_map_output(i) ? a.depth_pitch : a.out_pitch, H,
                            is_map_output(i) ? static_cast<int64_t>(W) : 3 * static_cast<int64_t>(W))
                     : Span{};
  bool disjoint = may_overlap && !scratch;
  for (int i = 0; i < O_COUNT; ++i) {
    if (prev_out[i].hi && meets(cur_in, prev_out[i])) disjoint = false;  // reads what it wrote
    if (!cur_out[i].hi) continue;
    if (meets(cur_out[i], prev_in) || meets(cur_out[i], prev_depth)) disjoint = false;  // writes what it read
    for (int j = 0; j < O_COUNT; ++j)
      if (prev_out[j].hi && meets(cur_out[i], prev_out[j])) disjoint = false;  // writes what it wrote
  }
  a.overlap = disjoint ? 1 : 0;
  // A frame enqueued behind queued work: consecutive independent frames run side by side
  // in a share of the SM slots each, in taller row bands (fewer band start-ups, whose
  // first input rows arrive while another frame's CTA on the SM computes), instead of
  // one after the other across every SM.  Both CTAs of an SM must fit at once.
  const int fif = tuning.frames_in_flight > 0 ? tuning.frames_in_flight : kFramesInFlight;
  const int full_grid = a.grid;
  if (disjoint && fif > 1 && per_sm >= 2 && cudaStreamQuery(stream) == cudaErrorNotReady) {
    if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();  // (not an error)
    a.grid = std::max(1, std::min(a.grid, (num_sms * per_sm + fif - 1) / fif));
  }
  cudaError_t e = launch_band(a, smem, per_sm, stream);
  a.overlap = 0;
  a.grid = full_grid;
  if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
  ++launches;
  if (!inpaint) {
    prev_band = true;
    prev_in = cur_in;
    prev_depth = cur_depth;
    for (int i = 0; i < O_COUNT; ++i) prev_out[i] = cur_out[i];
  }
  if (inpaint) {
    InpaintArgs ia;
    ia.view[0] = a.out[O_LEFT];
    ia.view[1] = a.out[O_RIGHT];
    ia.pitch = a.out_pitch;
    ia.holes = a.out[O_HOLES];
    ia.holes_pitch = a.depth_pitch;
    ia.ana = (p->outputs & DIBR_OUT_ANAGLYPH) ? a.out[O_ANA] : nullptr;
    ia.hsbs = (p->outputs & DIBR_OUT_HSBS) ? a.out[O_HSBS] : nullptr;
    ia.out_pitch = a.out_pitch;
    ia.W = W;
    ia.H = H;
    ia.block = p->inpaint_block;
    ia.nbx = (W + ia.block - 1) / ia.block;
    ia.nblocks = ia.nbx * ((H + ia.block - 1) / ia.block);
    if ((s = ensure(inpaint_order, sizeof(int32_t) * (2 * static_cast<size_t>(ia.nblocks) + 3))) != DIBR_OK) return s;
    ia.sms = num_sms;
    ia.order = reinterpret_cast<int32_t *>(inpaint_order.ptr);
    e = launch_inpaint(ia, stream);
    if (e != cudaSuccess) return cuda_fail(e, "inpainting launch");
    ++launches;
    // the inpainting reads and writes the band launch's outputs (views, holes map,
    // anaglyph, side-by-side) and nothing else the next frame's band launch could touch
    prev_band = true;
    prev_in = Span{};
    prev_depth = Span{};
    for (int i = 0; i < O_COUNT; ++i) prev_out[i] = cur_out[i];
  }
  return DIBR_OK;
}

dibr_status dibr_ctx::read_status() {
  prev_band = false;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, status_dev, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronising the context stream");
  if (st) {
    cudaMemsetAsync(status_dev, 0, sizeof(int), stream);
    cudaStreamSynchronize(stream);
    set_error("a bounded device-side wait gave up (status 0x%x)", st);
    return DIBR_E_TIMEOUT;
  }
  return DIBR_OK;
}

// ------------------------------------------------------------------- the C-ABI
extern "C" {

dibr_status dibr_params_default(dibr_params *p) {
  if (!p) return DIBR_E_INVALID;
  p->depth_rule = DIBR_DEPTH_LUMA_BINOM5;
  p->disparity_rule = DIBR_DISP_PAPER;
  p->warp_mode = DIBR_WARP_FORWARD;
  p->max_parallax_px = 16;
  p->threshold = 150;
  p->xbf_sigma_s = 1.5f;
  p->xbf_sigma_r = 16.0f;
  p->xbf_radius = 2;
  p->outputs = DIBR_OUT_ANAGLYPH;
  p->hole_fill = DIBR_FILL_ROW;
  p->inpaint_block = 32;
  return DIBR_OK;
}

dibr_status dibr_set_wait_limit(dibr_ctx *c, uint64_t limit_ns) {
  if (!c) return DIBR_E_INVALID;
  c->timeout_ns = limit_ns ? static_cast<unsigned long long>(limit_ns) : 2000000000ull;
  return DIBR_OK;
}

dibr_status dibr_validate(const dibr_params *p, const dibr_image *img) {
  std::string why;
  return check_params(p, img, &why);
}

dibr_status dibr_shift_tables(const dibr_params *p, int16_t hL[256], int16_t hR[256]) {
  std::string why;
  dibr_status s = check_params(p, nullptr, &why);
  if (s != DIBR_OK) return s;
  if (!hL || !hR) return DIBR_E_INVALID;
  build_tables(p, hL, hR, nullptr);
  return DIBR_OK;
}

dibr_status dibr_create(const dibr_config *cfg_in, dibr_ctx **out) {
  if (!out) return DIBR_E_INVALID;
  *out = nullptr;
  dibr_config cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  if (cfg_in) cfg = *cfg_in;
  if ((cfg.alloc == nullptr) != (cfg.free == nullptr)) return DIBR_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return DIBR_E_CUDA;
  }
  if (cfg.device < 0 || cfg.device >= ndev) return DIBR_E_INVALID;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) return DIBR_E_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return DIBR_E_CUDA;  // built for sm_103a only
  if (cudaSetDevice(cfg.device) != cudaSuccess) return DIBR_E_CUDA;
  dibr_ctx *c = new dibr_ctx();
  c->device = cfg.device;
  c->num_sms = prop.multiProcessorCount;
  c->max_smem = static_cast<int>(prop.sharedMemPerBlockOptin);
  c->smem_per_sm = static_cast<int>(prop.sharedMemPerMultiprocessor);
  c->alloc_hook = cfg.alloc;
  c->free_hook = cfg.free;
  c->alloc_user = cfg.user;
  c->mem_budget = cfg.mem_budget_bytes;
  c->max_streams = cfg.max_streams > 0 ? cfg.max_streams : 64;
  c->max_batch = cfg.max_batch > 0 ? cfg.max_batch : 256;
  if (cfg.cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cfg.cuda_stream);
    c->owns_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return DIBR_E_CUDA;
    }
    c->owns_stream = true;
  }
  c->status_dev = static_cast<int *>(c->dev_alloc(64));
  if (!c->status_dev) {
    if (c->owns_stream) cudaStreamDestroy(c->stream);
    delete c;
    return DIBR_E_NOMEM;
  }
  cudaMemsetAsync(c->status_dev, 0, 64, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    c->dev_free(c->status_dev);
    if (c->owns_stream) cudaStreamDestroy(c->stream);
    delete c;
    return DIBR_E_CUDA;
  }
  *out = c;
  return DIBR_OK;
}

void dibr_destroy(dibr_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  c->shutdown_serving();
  cudaStreamSynchronize(c->stream);
  c->release_buffers();
  c->dev_free(c->status_dev);
  cudaStreamSynchronize(c->stream);
  if (c->owns_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char *dibr_last_error(dibr_ctx *c) {
  if (!c) return "null context";
  std::lock_guard<std::mutex> g(c->err_mu);
  c->last_error_copy = c->last_error;
  return c->last_error_copy.c_str();
}

void *dibr_stream(dibr_ctx *c) { return c ? static_cast<void *>(c->stream) : nullptr; }

dibr_status dibr_set_tuning(dibr_ctx *c, const dibr_tuning *t) {
  if (!c || !t) return DIBR_E_INVALID;
  if (t->ring_slots < 0 || t->ring_slots > kMaxRing || (t->ring_slots > 0 && t->ring_slots < 2) ||
      t->ctas_per_sm < 0 || t->ctas_per_sm > 32 || t->load_mode < 0 || t->load_mode > 5 ||
      t->l2_prefetch < 0 || t->l2_prefetch > 2 || t->rows_per_unit < 0 || t->rows_per_unit > 4096 ||
      t->host_bands < 0 || t->host_bands > dibr_ctx::kMaxBands || t->frames_in_flight < 0 ||
      t->frames_in_flight > 16) {
    c->set_error("tuning value out of range");
    return DIBR_E_INVALID;
  }
  c->tuning = *t;
  return DIBR_OK;
}

dibr_status dibr_get_tuning(dibr_ctx *c, dibr_tuning *t) {
  if (!c || !t) return DIBR_E_INVALID;
  *t = c->tuning;
  return DIBR_OK;
}

dibr_status dibr_enqueue_image(dibr_ctx *c, const dibr_image *img, const dibr_params *p,
                               const dibr_outputs *o) {
  if (!c || !img) return DIBR_E_INVALID;
  std::string why;
  dibr_status s = check_params(p, img, &why);
  if (s == DIBR_OK) s = check_outputs(p, img, o, &why);
  if (s != DIBR_OK) {
    c->set_error("%s", why.c_str());
    return s;
  }
  if (!img->on_device || !o->on_device) {
    c->set_error("dibr_enqueue_image needs device buffers");
    return DIBR_E_INVALID;
  }
  cudaSetDevice(c->device);
  return c->enqueue_device(img, p, o);
}

dibr_status dibr_synchronize(dibr_ctx *c) {
  if (!c) return DIBR_E_INVALID;
  cudaSetDevice(c->device);
  return c->read_status();
}

dibr_status dibr_synthesize_image(dibr_ctx *c, const dibr_image *img, const dibr_params *p,
                                  const dibr_outputs *o) {
  if (!c || !img) return DIBR_E_INVALID;
  std::string why;
  dibr_status s = check_params(p, img, &why);
  if (s == DIBR_OK) s = check_outputs(p, img, o, &why);
  if (s != DIBR_OK) {
    c->set_error("%s", why.c_str());
    return s;
  }
  cudaSetDevice(c->device);
  return c->synthesize_staged(img, p, o);
}

}  // extern "C"

// Blocking single-frame path with the input and every output in host memory: the frame is
// cut into row bands; band k's input copy (copy_in stream), its kernel (the context's
// stream, once the copies of bands k and k+1 -- two rows of depth context -- have landed)
// and its output copies (copy_out stream) overlap with the other bands'.  The host link,
// not the GPU, bounds such a call (about 100 MB cross it per 4K stereo frame), and this
// keeps both directions of the link busy together.
dibr_status dibr_ctx::synthesize_banded(const dibr_image *img, const dibr_params *p, const dibr_outputs *o,
                                        int bands) {
  const int W = img->width, H = img->height;
  prev_band = false;
  cudaError_t e;
  dibr_status s;
  if (!copy_in) {
    if (cudaStreamCreateWithFlags(&copy_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&copy_out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "creating the copy streams");
    for (int k = 0; k < kMaxBands; ++k)
      if (cudaEventCreateWithFlags(&ev_in[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_comp[k], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "creating the band events");
  }
  const int64_t ap = round_up(3 * W, 16), op = round_up(3 * W, 16), dp = round_up(W, 16);
  if ((s = ensure(stage_in, static_cast<size_t>(ap) * H)) != DIBR_OK) return s;
  size_t total = 0, offs[O_COUNT];
  for (int i = 0; i < O_COUNT; ++i) {
    offs[i] = total;
    if (p->outputs & kOutBits[i]) total += static_cast<size_t>(is_map_output(i) ? dp : op) * H;
  }
  if ((s = ensure(stage_out, total)) != DIBR_OK) return s;
  BandArgs &a = args;
  int smem = 0, per_sm = 1;
  const int depth_src = p->depth_rule == DIBR_DEPTH_LUMA_BINOM5 ? DS_BINOM5 : DS_LUMA;
  const int zguard = band_tables(p);
  if ((s = plan_band(W, H, depth_src, stage_in.ptr, ap, zguard, a, smem, per_sm)) != DIBR_OK) return s;
  if ((s = encode_input(a, stage_in.ptr, ap)) != DIBR_OK) return s;
  a.depth_in = nullptr;
  a.depth_in_pitch = 0;
  for (int i = 0; i < O_COUNT; ++i) a.out[i] = (p->outputs & kOutBits[i]) ? stage_out.ptr + offs[i] : nullptr;
  a.out_pitch = op;
  a.depth_pitch = dp;
  a.outputs = p->outputs;
  a.warp_mode = p->warp_mode;
  a.fast_store = aligned_rgb_outputs(a);
  const int slots = a.grid;  // CTAs of a whole-frame launch
  auto band_row = [&](int k) { return static_cast<int>(static_cast<int64_t>(k) * H / bands); };
  // the copy streams start after the work already queued on the context's stream
  if ((e = cudaEventRecord(ev_out, stream)) != cudaSuccess) return cuda_fail(e, "ordering the copies");
  cudaStreamWaitEvent(copy_in, ev_out, 0);
  cudaStreamWaitEvent(copy_out, ev_out, 0);
  for (int k = 0; k < bands; ++k) {
    const int y0 = band_row(k), y1 = band_row(k + 1);
    e = cudaMemcpy2DAsync(stage_in.ptr + static_cast<int64_t>(y0) * ap, ap, img->rgb + static_cast<int64_t>(y0) * img->pitch,
                          img->pitch, 3 * static_cast<size_t>(W), y1 - y0, cudaMemcpyHostToDevice, copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], copy_in);
    if (e != cudaSuccess) return cuda_fail(e, "input upload");
  }
  for (int k = 0; k < bands; ++k) {
    const int y0 = band_row(k), y1 = band_row(k + 1);
    // rows y0 - 2 .. y1 + 1 of the input: the uploads up to the band holding row y1 + 1
    // (they complete in order on one stream)
    int kl = k;
    while (kl + 1 < bands && band_row(kl + 1) <= std::min(y1 + 1, H - 1)) ++kl;
    cudaStreamWaitEvent(stream, ev_in[kl], 0);
    a.row0 = y0;
    a.row1 = y1;
    a.grid = std::max(1, std::min(y1 - y0, slots));
    e = launch_band(a, smem, per_sm, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp[k], stream);
    if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
    ++launches;
    cudaStreamWaitEvent(copy_out, ev_comp[k], 0);
    for (int i = 0; i < O_COUNT; ++i) {
      if (!(p->outputs & kOutBits[i])) continue;
      const bool map = is_map_output(i);
      const int64_t hp = map ? o->depth_pitch : o->pitch, sp = map ? dp : op;
      e = cudaMemcpy2DAsync(out_slot(*o, i) + static_cast<int64_t>(y0) * hp, hp, a.out[i] + static_cast<int64_t>(y0) * sp,
                            sp, map ? static_cast<size_t>(W) : 3 * static_cast<size_t>(W), y1 - y0,
                            cudaMemcpyDeviceToHost, copy_out);
      if (e != cudaSuccess) return cuda_fail(e, "output download");
    }
  }
  a.row0 = 0;
  a.row1 = H;
  a.grid = slots;
  // the call's end: everything on the context's stream after the last download
  if ((e = cudaEventRecord(ev_out, copy_out)) != cudaSuccess) return cuda_fail(e, "ordering the copies");
  cudaStreamWaitEvent(stream, ev_out, 0);
  return read_status();
}

void dibr_ctx::release_band_pipeline() {
  if (!copy_in) return;
  cudaStreamSynchronize(copy_in);
  cudaStreamSynchronize(copy_out);
  for (int k = 0; k < kMaxBands; ++k) {
    if (ev_in[k]) cudaEventDestroy(ev_in[k]);
    if (ev_comp[k]) cudaEventDestroy(ev_comp[k]);
    ev_in[k] = ev_comp[k] = nullptr;
  }
  if (ev_out) cudaEventDestroy(ev_out);
  ev_out = nullptr;
  cudaStreamDestroy(copy_in);
  cudaStreamDestroy(copy_out);
  copy_in = copy_out = nullptr;
}

// Blocking single-frame path: host buffers are staged through context-owned device
// memory (input H2D, outputs D2H) on the context's stream.
dibr_status dibr_ctx::synthesize_staged(const dibr_image *img, const dibr_params *p, const dibr_outputs *o) {
  const int W = img->width, H = img->height;
  prev_band = false;  // copies precede the launch
  // row bands when both sides of the call are in host memory and every row band is
  // independent of the others' results (not with the 2-D fill or the cross-bilateral depth,
  // which need the whole frame first)
  const int bands = tuning.host_bands > 0 ? std::min(tuning.host_bands, H) : H >= 2048 ? 4 : H >= 512 ? 2 : 1;
  if (bands > 1 && !img->on_device && !o->on_device && p->hole_fill == DIBR_FILL_ROW &&
      p->depth_rule != DIBR_DEPTH_LUMA_XBF)
    return synthesize_banded(img, p, o, bands);
  dibr_image din = *img;
  dibr_outputs dout = *o;
  cudaError_t e;
  dibr_status s;
  if (!img->on_device) {
    const int64_t ap = round_up(3 * W, 16);
    if ((s = ensure(stage_in, static_cast<size_t>(ap) * H)) != DIBR_OK) return s;
    e = cudaMemcpy2DAsync(stage_in.ptr, ap, img->rgb, img->pitch, 3 * static_cast<size_t>(W), H,
                          cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "input upload");
    din.rgb = stage_in.ptr;
    din.pitch = ap;
    din.on_device = 1;
  }
  const int64_t op = round_up(3 * W, 16), dp = round_up(W, 16);
  if (!o->on_device) {
    size_t total = 0;
    size_t offs[O_COUNT];
    for (int i = 0; i < O_COUNT; ++i) {
      offs[i] = total;
      if (p->outputs & kOutBits[i]) total += static_cast<size_t>(is_map_output(i) ? dp : op) * H;
    }
    if ((s = ensure(stage_out, total)) != DIBR_OK) return s;
    for (int i = 0; i < O_COUNT; ++i) out_slot(dout, i) = (p->outputs & kOutBits[i]) ? stage_out.ptr + offs[i] : nullptr;
    dout.pitch = op;
    dout.depth_pitch = dp;
    dout.on_device = 1;
  }
  if ((s = enqueue_device(&din, p, &dout)) != DIBR_OK) return s;
  if (!o->on_device) {
    for (int i = 0; i < O_COUNT; ++i) {
      if (!(p->outputs & kOutBits[i])) continue;
      const bool map = is_map_output(i);
      e = cudaMemcpy2DAsync(out_slot(*o, i), map ? o->depth_pitch : o->pitch, out_slot(dout, i), map ? dp : op,
                            map ? static_cast<size_t>(W) : 3 * static_cast<size_t>(W), H,
                            cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) return cuda_fail(e, "output download");
    }
  }
  return read_status();
}

void dibr_ctx::release_buffers() {
  release_band_pipeline();
  for (DevBuf *b : {&stage_in, &stage_out, &realign, &xbf_depth, &inpaint_scratch, &inpaint_order}) {
    dev_free(b->ptr);
    b->ptr = nullptr;
    b->bytes = 0;
  }
  release_batch_buffers();
}
