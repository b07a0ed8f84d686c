// dibr_batch.cu -- images of uneven sizes in one call (dibr_synthesize_batch,
// dibr_enqueue_batch; also the serving loop's batches).
//
// Images that fill the GPU on their own get a band launch each, back to back.  The others
// are cut into work units of a few rows (plan_unit_rows); the host writes one descriptor
// per image (pointers, sizes, shift tables) and the unit list, largest images first, into
// device memory with a single copy; the persistent CTAs of the batch kernel (one chained
// launch per block-width group) take units from a device counter until none is left, so
// the launches balance themselves over images of any mix of sizes.
#include <algorithm>
#include <cstdio>
#include <map>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dibr.h"
#include "dibr_context.h"
#include "dibr_internal.h"

using namespace dibr;

namespace dibr {
dibr_status check_image_args(const dibr_params *p, const dibr_image *img, const dibr_outputs *o,
                             std::string *why);
void shift_tables(const dibr_params *p, int32_t *lut_h, int32_t *lut_n);
}  // namespace dibr

// The z-buffer guard every image of a batch fits in: the largest shift of their tables.
static int batch_zguard(const dibr_params *p, int n_params) {
  int g = 4;
  for (int i = 0; i < n_params; ++i) {
    int32_t lh[256], ln[256];
    shift_tables(&p[i], lh, ln);
    g = std::max(g, zguard_of(lh));
  }
  return g;
}

void dibr_ctx::release_batch_buffers() {
  for (DevBuf *b : {&batch_desc, &batch_img, &batch_depth}) {
    dev_free(b->ptr);
    b->ptr = nullptr;
    b->bytes = 0;
  }
  if (batch_pinned) {
    if (batch_copy_done) cudaEventSynchronize(batch_copy_done);
    cudaFreeHost(batch_pinned);
    batch_pinned = nullptr;
    batch_pinned_bytes = 0;
  }
  if (batch_copy_done) {
    cudaEventDestroy(batch_copy_done);
    batch_copy_done = nullptr;
  }
}

// All buffers in device memory.  Images large enough to fill the GPU on their own (at
// least kOwnLaunchRows rows per CTA slot of their launch plan; e.g. 4K and 8K frames) get a
// band launch each, back to back, overlapping one another when their buffers are disjoint;
// measured, that beats the persistent launch for them.  The others (e.g. 1080p, 720p) share
// the grouped persistent launches, which beat per-image launches for them.
constexpr int kOwnLaunchRows = 4;

dibr_status dibr_ctx::enqueue_batch_device(int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                                           const dibr_outputs *outs) {
  if (n == 0) return DIBR_OK;
  std::vector<int> own, shared;
  const BatchLimits lim{max_smem, smem_per_sm, tuning.ring_slots, tuning.ctas_per_sm, batch_zguard(p, n_params)};
  for (int i = 0; i < n; ++i) {
    const int w = imgs[i].width, rb = round_up(3 * w, 16);
    int cl = 0;
    BatchClass c[1];
    const bool fits = plan_batch_classes(1, &w, &rb, lim, &cl, c) == 1;
    const int64_t slots = static_cast<int64_t>(num_sms) * (fits ? c[0].per : 1);
    bool big = fits && tuning.rows_per_unit == 0 && imgs[i].height >= kOwnLaunchRows * slots;
    const auto t = class_tune.find(block_of(w));
    if (fits && tuning.rows_per_unit == 0 && t != class_tune.end() && t->second.own >= 0) big = t->second.own == 1;
    (big ? own : shared).push_back(i);
  }
  dibr_status s = DIBR_OK;
  if (!shared.empty()) {
    if (own.empty()) {
      s = enqueue_grouped(n, imgs, p, n_params, outs);
    } else {
      std::vector<dibr_image> si;
      std::vector<dibr_params> sp;
      std::vector<dibr_outputs> so;
      for (int i : shared) {
        si.push_back(imgs[i]);
        so.push_back(outs[i]);
        if (n_params != 1) sp.push_back(p[i]);
      }
      s = enqueue_grouped(static_cast<int>(si.size()), si.data(), n_params == 1 ? p : sp.data(),
                          n_params == 1 ? 1 : static_cast<int>(sp.size()), so.data());
    }
    if (s != DIBR_OK) return s;
  }
  std::stable_sort(own.begin(), own.end(), [&](int a, int b) {
    return static_cast<int64_t>(imgs[a].width) * imgs[a].height > static_cast<int64_t>(imgs[b].width) * imgs[b].height;
  });
  for (int i : own)
    if ((s = enqueue_device(&imgs[i], &p[n_params == 1 ? 0 : i], &outs[i])) != DIBR_OK) return s;
  return DIBR_OK;
}

// The grouped persistent launches (all buffers in device memory).
dibr_status dibr_ctx::enqueue_grouped(int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                                      const dibr_outputs *outs) {
  prev_band = false;
  if (n == 0) return DIBR_OK;
  // --- inputs that a bulk row copy cannot read directly are repacked (16-byte rows)
  std::vector<const uint8_t *> in(n);
  std::vector<int64_t> in_pitch(n);
  std::vector<int> row_bytes(n);
  size_t realign_bytes = 0, depth_bytes = 0;
  for (int i = 0; i < n; ++i) {
    const dibr_image &im = imgs[i];
    const bool ok = (reinterpret_cast<uintptr_t>(im.rgb) & 15u) == 0 && (im.pitch & 15) == 0 && (3 * im.width) % 16 == 0;
    if (!ok) realign_bytes += static_cast<size_t>(round_up(3 * im.width, 16)) * im.height;
    if (p[n_params == 1 ? 0 : i].depth_rule == DIBR_DEPTH_LUMA_XBF)
      depth_bytes += static_cast<size_t>(round_up(im.width, 16)) * im.height;
  }
  dibr_status s;
  if (realign_bytes && (s = ensure(batch_img, realign_bytes)) != DIBR_OK) return s;
  if (depth_bytes && (s = ensure(batch_depth, depth_bytes)) != DIBR_OK) return s;
  size_t ro = 0, dof = 0;
  std::vector<const uint8_t *> depth_in(n, nullptr);
  std::vector<int64_t> depth_pitch_in(n, 0);
  for (int i = 0; i < n; ++i) {
    const dibr_image &im = imgs[i];
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    const bool ok = (reinterpret_cast<uintptr_t>(im.rgb) & 15u) == 0 && (im.pitch & 15) == 0 && (3 * im.width) % 16 == 0;
    if (ok) {
      in[i] = im.rgb;
      in_pitch[i] = im.pitch;
      row_bytes[i] = 3 * im.width;
    } else {
      const int64_t ap = round_up(3 * im.width, 16);
      uint8_t *dst = batch_img.ptr + ro;
      cudaError_t e = cudaMemcpy2DAsync(dst, ap, im.rgb, im.pitch, 3 * static_cast<size_t>(im.width), im.height,
                                        cudaMemcpyDeviceToDevice, stream);
      if (e != cudaSuccess) return cuda_fail(e, "repacking a batch input");
      in[i] = dst;
      in_pitch[i] = ap;
      row_bytes[i] = static_cast<int>(ap);  // whole 16-byte units; the padding is never used
      ro += static_cast<size_t>(ap) * im.height;
    }
    if (pp.depth_rule == DIBR_DEPTH_LUMA_XBF) {
      const int64_t dp = round_up(im.width, 16);
      uint8_t *dd = batch_depth.ptr + dof;
      cudaError_t e = launch_xbf(in[i], in_pitch[i], im.width, im.height, pp.xbf_radius, pp.xbf_sigma_s,
                                 pp.xbf_sigma_r, dd, dp, stream);
      if (e != cudaSuccess) return cuda_fail(e, "cross-bilateral launch");
      ++launches;
      depth_in[i] = dd;
      depth_pitch_in[i] = dp;
      dof += static_cast<size_t>(dp) * im.height;
    }
  }
  // --- one launch per group of images of equal block width, widest first
  std::vector<int> widths(n), heights(n), class_of(n), order(n);
  for (int i = 0; i < n; ++i) {
    widths[i] = imgs[i].width;
    heights[i] = imgs[i].height;
  }
  BatchClass cls[kMaxClasses];
  const BatchLimits lim{max_smem, smem_per_sm, tuning.ring_slots, tuning.ctas_per_sm, batch_zguard(p, n_params)};
  const int nclass = plan_batch_classes(n, widths.data(), row_bytes.data(), lim, class_of.data(), cls);
  if (nclass < 1) {
    set_error("batch images too wide for shared memory");
    return DIBR_E_INVALID;
  }
  // the autotuner's choices for tuned classes (where the context's knobs are automatic)
  for (int c = 0; c < nclass; ++c) {
    const auto t = class_tune.find(cls[c].nc);
    if (t == class_tune.end()) continue;
    BatchLimits l2 = lim;
    if (lim.ring_slots == 0 && t->second.nb > 0) l2.ring_slots = t->second.nb;
    if (lim.ctas_per_sm == 0 && t->second.per > 0) l2.ctas_per_sm = t->second.per;
    if (!plan_class(cls[c], l2)) plan_class(cls[c], lim);
  }
  order_by_area(n, widths.data(), heights.data(), order.data());
  plan_unit_rows(n, heights.data(), class_of.data(), nclass, num_sms, tuning.rows_per_unit, cls);
  if (tuning.rows_per_unit == 0)
    for (int c = 0; c < nclass; ++c) {
      const auto t = class_tune.find(cls[c].nc);
      if (t != class_tune.end() && t->second.rows > 0) cls[c].rows = t->second.rows;
    }

  // --- descriptors and units, staged in pinned memory; each group's units are
  // contiguous, largest images first
  int n_units = 0;
  for (int i = 0; i < n; ++i) n_units += (imgs[i].height + cls[class_of[i]].rows - 1) / cls[class_of[i]].rows;
  // [counters][pad] [descs] [units]: every part 256-byte aligned (the kernel reads the
  // units as int4 and the descriptors' 64-bit fields)
  const size_t off_desc = 256;
  const size_t off_units = (off_desc + sizeof(ImageDesc) * n + 255) / 256 * 256;
  const size_t total = off_units + sizeof(int4) * static_cast<size_t>(n_units);
  if (batch_copy_done) cudaEventSynchronize(batch_copy_done);  // the previous copy has read the staging
  if (batch_pinned_bytes < total) {
    if (batch_pinned) cudaFreeHost(batch_pinned);
    batch_pinned = nullptr;
    batch_pinned_bytes = 0;
    if (cudaHostAlloc(reinterpret_cast<void **>(&batch_pinned), total, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      set_error("pinned allocation of %zu bytes failed", total);
      return DIBR_E_NOMEM;
    }
    batch_pinned_bytes = total;
  }
  if (!batch_copy_done && cudaEventCreateWithFlags(&batch_copy_done, cudaEventDisableTiming) != cudaSuccess)
    return DIBR_E_CUDA;
  if ((s = ensure(batch_desc, total)) != DIBR_OK) return s;
  std::memset(batch_pinned, 0, off_desc);  // the groups' unit counters start at zero
  ImageDesc *descs = reinterpret_cast<ImageDesc *>(batch_pinned + off_desc);
  int4 *units = reinterpret_cast<int4 *>(batch_pinned + off_units);
  for (int i = 0; i < n; ++i) {
    const dibr_image &im = imgs[i];
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    const dibr_outputs &o = outs[i];
    ImageDesc &d = descs[i];
    std::memset(&d, 0, sizeof(d));
    d.in = in[i];
    d.in_pitch = in_pitch[i];
    d.depth_in = depth_in[i];
    d.depth_in_pitch = depth_pitch_in[i];
    for (int k = 0; k < O_COUNT; ++k) d.out[k] = out_slot(o, k);
    d.out_pitch = o.pitch;
    d.depth_pitch = o.depth_pitch;
    d.W = im.width;
    d.H = im.height;
    d.nch = chunks_of(im.width);
    d.row_bytes = row_bytes[i];
    d.outputs = pp.outputs;
    d.warp_mode = pp.warp_mode;
    d.depth_src = pp.depth_rule == DIBR_DEPTH_LUMA_BINOM5 ? DS_BINOM5 : pp.depth_rule == DIBR_DEPTH_LUMA ? DS_LUMA : DS_GLOBAL;
    shift_tables(&pp, d.lut_h, d.lut_n);
  }
  // every image of one fixed output set: the launches use that set's kernel instance
  uint32_t fixed = 0;
  for (int i = 0; i < n; ++i) {
    const ImageDesc &d = descs[i];
    const uint32_t f = fixed_set(d.outputs, d.depth_src, d.warp_mode, d.out, d.out_pitch);
    fixed = i == 0 ? f : (f == fixed ? fixed : 0u);
  }
  int u = 0;
  for (int c = 0; c < nclass; ++c) {
    cls[c].unit_begin = u;
    for (int oi = 0; oi < n; ++oi) {
      const int i = order[oi];
      if (class_of[i] != c) continue;
      const int rpu = cls[c].rows;
      for (int y0 = 0; y0 < imgs[i].height; y0 += rpu)
        units[u++] = make_int4(i, y0, std::min(imgs[i].height, y0 + rpu), 0);
    }
    cls[c].n_units = u - cls[c].unit_begin;
  }
  cudaError_t e = cudaMemcpyAsync(batch_desc.ptr, batch_pinned, total, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaEventRecord(batch_copy_done, stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
  for (int c = 0; c < nclass; ++c) {
    BatchArgs b;
    b.descs = reinterpret_cast<const ImageDesc *>(batch_desc.ptr + off_desc);
    b.units = reinterpret_cast<const int4 *>(batch_desc.ptr + off_units) + cls[c].unit_begin;
    b.n_units = cls[c].n_units;
    b.counter = reinterpret_cast<int *>(batch_desc.ptr) + c;
    b.status = status_dev;
    b.timeout_ns = timeout_ns;
    b.nb = cls[c].nb;
    b.srow = cls[c].srow;
    b.nch_max = cls[c].nch_max;
    b.nc = cls[c].nc;
    b.zguard = lim.zguard;
    b.outs = fixed;
    const int grid = std::max(1, std::min(cls[c].n_units, num_sms * cls[c].per));
    e = launch_batch(b, grid, cls[c].smem, c > 0, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    ++launches;
  }
  return DIBR_OK;
}

static dibr_status check_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                               const dibr_outputs *outs) {
  if (!c || n < 0 || (n > 0 && (!imgs || !p || !outs))) return DIBR_E_INVALID;
  if (n > 0 && n_params != 1 && n_params != n) {
    c->set_error("n_params must be 1 or n");
    return DIBR_E_INVALID;
  }
  if (n > c->max_batch) {
    c->set_error("batch of %d images exceeds max_batch %d", n, c->max_batch);
    return DIBR_E_INVALID;
  }
  for (int i = 0; i < n; ++i) {
    std::string why;
    const dibr_status s = check_image_args(&p[n_params == 1 ? 0 : i], &imgs[i], &outs[i], &why);
    if (s != DIBR_OK) {
      c->set_error("image %d: %s", i, why.c_str());
      return s;
    }
    if (p[n_params == 1 ? 0 : i].hole_fill != DIBR_FILL_ROW) {
      c->set_error("image %d: the 2-D fill runs on single-image calls only", i);
      return DIBR_E_INVALID;
    }
  }
  return DIBR_OK;
}

extern "C" {

dibr_status dibr_enqueue_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                               const dibr_outputs *outs) {
  dibr_status s = check_batch(c, n, imgs, p, n_params, outs);
  if (s != DIBR_OK) return s;
  for (int i = 0; i < n; ++i)
    if (!imgs[i].on_device || !outs[i].on_device) {
      c->set_error("dibr_enqueue_batch needs device buffers");
      return DIBR_E_INVALID;
    }
  cudaSetDevice(c->device);
  return c->enqueue_batch_device(n, imgs, p, n_params, outs);
}

dibr_status dibr_autotune_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                                const dibr_outputs *outs, int reps) {
  dibr_status s = check_batch(c, n, imgs, p, n_params, outs);
  if (s != DIBR_OK) return s;
  for (int i = 0; i < n; ++i)
    if (!imgs[i].on_device || !outs[i].on_device) {
      c->set_error("dibr_autotune_batch needs device buffers");
      return DIBR_E_INVALID;
    }
  if (reps < 1) reps = 1;
  cudaSetDevice(c->device);
  // the images of each size class (block width), timed alone under every candidate plan
  std::map<int, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) groups[block_of(imgs[i].width)].push_back(i);
  std::vector<ClassTune> cands;
  cands.push_back(ClassTune{0, 0, 0, 1});  // a band launch per image
  for (int rows : {0, 2, 4, 8, 16, 32, 64})
    for (int per : {0, 1})
      for (int nb : {0, 4}) cands.push_back(ClassTune{rows, per, nb, 0});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return c->cuda_fail(cudaGetLastError(), "creating the autotuner's events");
  }
  for (auto &g : groups) {
    std::vector<dibr_image> gi;
    std::vector<dibr_params> gp;
    std::vector<dibr_outputs> go;
    for (int i : g.second) {
      gi.push_back(imgs[i]);
      gp.push_back(p[n_params == 1 ? 0 : i]);
      go.push_back(outs[i]);
    }
    const int m = static_cast<int>(gi.size());
    float best = -1.f;
    ClassTune pick;
    for (const ClassTune &cand : cands) {
      c->class_tune[g.first] = cand;
      if ((s = c->enqueue_batch_device(m, gi.data(), gp.data(), m, go.data())) != DIBR_OK) break;  // warm-up
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && s == DIBR_OK; ++r) s = c->enqueue_batch_device(m, gi.data(), gp.data(), m, go.data());
      cudaEventRecord(e1, c->stream);
      if (s != DIBR_OK) break;
      if ((s = c->read_status()) != DIBR_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0.f || ms < best) {
        best = ms;
        pick = cand;
      }
    }
    if (s != DIBR_OK) {
      c->class_tune.erase(g.first);
      break;
    }
    c->class_tune[g.first] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

dibr_status dibr_tuning_save(dibr_ctx *c, const char *path) {
  if (!c || !path) return DIBR_E_INVALID;
  FILE *f = std::fopen(path, "w");
  if (!f) {
    c->set_error("cannot write %s", path);
    return DIBR_E_INVALID;
  }
  std::fprintf(f, "{\"batch_classes\": [");
  bool first = true;
  for (const auto &kv : c->class_tune) {
    std::fprintf(f, "%s\n  {\"block_threads\": %d, \"rows_per_unit\": %d, \"ctas_per_sm\": %d, \"ring_slots\": %d, "
                 "\"own_launch\": %d}",
                 first ? "" : ",", kv.first, kv.second.rows, kv.second.per, kv.second.nb, kv.second.own);
    first = false;
  }
  std::fprintf(f, "\n]}\n");
  const bool ok = std::fclose(f) == 0;
  return ok ? DIBR_OK : DIBR_E_INVALID;
}

dibr_status dibr_tuning_load(dibr_ctx *c, const char *path) {
  if (!c || !path) return DIBR_E_INVALID;
  FILE *f = std::fopen(path, "r");
  if (!f) {
    c->set_error("cannot read %s", path);
    return DIBR_E_INVALID;
  }
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
  std::fclose(f);
  // entries as dibr_tuning_save writes them; anything else is rejected
  std::map<int, ClassTune> table;
  size_t pos = 0;
  while ((pos = text.find("{\"block_threads\":", pos)) != std::string::npos) {
    int nc, rows, per, nb, own;
    if (std::sscanf(text.c_str() + pos,
                    "{\"block_threads\": %d, \"rows_per_unit\": %d, \"ctas_per_sm\": %d, \"ring_slots\": %d, "
                    "\"own_launch\": %d}",
                    &nc, &rows, &per, &nb, &own) != 5 ||
        nc < 32 || nc > kMaxConsumers || nc % 32 || rows < 0 || per < 0 || nb < 0 || nb > kMaxRing || own < -1 || own > 1) {
      c->set_error("%s: malformed tuning entry", path);
      return DIBR_E_INVALID;
    }
    table[nc] = ClassTune{rows, per, nb, own};
    ++pos;
  }
  c->class_tune = table;
  return DIBR_OK;
}

dibr_status dibr_synthesize_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                                  const dibr_outputs *outs) {
  dibr_status s = check_batch(c, n, imgs, p, n_params, outs);
  if (s != DIBR_OK) return s;
  cudaSetDevice(c->device);
  // host buffers are staged through one device area: inputs, then outputs
  std::vector<dibr_image> di(imgs, imgs + n);
  std::vector<dibr_outputs> dout(outs, outs + n);
  size_t need = 0;
  const uint32_t *bits = kOutBits;
  for (int i = 0; i < n; ++i) {
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    if (!imgs[i].on_device) need += static_cast<size_t>(round_up(3 * imgs[i].width, 16)) * imgs[i].height;
    if (!outs[i].on_device)
      for (int k = 0; k < O_COUNT; ++k)
        if (pp.outputs & bits[k])
          need += static_cast<size_t>(round_up(is_map_output(k) ? imgs[i].width : 3 * imgs[i].width, 16)) * imgs[i].height;
  }
  if (need && (s = c->ensure(c->stage_in, need)) != DIBR_OK) return s;
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    const int W = imgs[i].width, H = imgs[i].height;
    if (!imgs[i].on_device) {
      const int64_t ap = round_up(3 * W, 16);
      e = cudaMemcpy2DAsync(c->stage_in.ptr + off, ap, imgs[i].rgb, imgs[i].pitch, 3 * static_cast<size_t>(W), H,
                            cudaMemcpyHostToDevice, c->stream);
      di[i].rgb = c->stage_in.ptr + off;
      di[i].pitch = ap;
      di[i].on_device = 1;
      off += static_cast<size_t>(ap) * H;
    }
    if (!outs[i].on_device) {
      const int64_t op = round_up(3 * W, 16), dpp = round_up(W, 16);
      for (int k = 0; k < O_COUNT; ++k) {
        if (!(pp.outputs & bits[k])) continue;
        out_slot(dout[i], k) = c->stage_in.ptr + off;
        off += static_cast<size_t>(is_map_output(k) ? dpp : op) * H;
      }
      dout[i].pitch = op;
      dout[i].depth_pitch = dpp;
      dout[i].on_device = 1;
    }
  }
  if (e != cudaSuccess) return c->cuda_fail(e, "batch input upload");
  if ((s = c->enqueue_batch_device(n, di.data(), p, n_params, dout.data())) != DIBR_OK) return s;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (outs[i].on_device) continue;
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    const int W = imgs[i].width, H = imgs[i].height;
    for (int k = 0; k < O_COUNT && e == cudaSuccess; ++k) {
      if (!(pp.outputs & bits[k])) continue;
      const bool dep = is_map_output(k);
      e = cudaMemcpy2DAsync(out_slot(outs[i], k), dep ? outs[i].depth_pitch : outs[i].pitch, out_slot(dout[i], k),
                            dep ? dout[i].depth_pitch : dout[i].pitch, dep ? W : 3 * static_cast<size_t>(W), H,
                            cudaMemcpyDeviceToHost, c->stream);
    }
  }
  if (e != cudaSuccess) return c->cuda_fail(e, "batch output download");
  return c->read_status();
}

}  // extern "C"
