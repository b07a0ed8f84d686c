// dibr_context.h -- the library context behind the opaque dibr_ctx handle.
#pragma once

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dibr.h"
#include "dibr_internal.h"

namespace dibr {

struct DevBuf {
  uint8_t *ptr = nullptr;
  size_t bytes = 0;
};

struct ServeState;  // dibr_serve.cu

// A batched launch plan chosen by the autotuner for one size class (the block width, in
// threads, of the images' rows); a zero field (own: -1) keeps the automatic choice.
struct ClassTune {
  int rows = 0;  // rows per work unit
  int per = 0;   // CTAs per SM at most
  int nb = 0;    // ring slots at most
  int own = -1;  // 1: every image of the class in a band launch of its own; 0: shared launches
};

}  // namespace dibr

struct dibr_ctx {
  int device = 0;
  int num_sms = 1;
  int max_smem = 0;
  int smem_per_sm = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  void *(*alloc_hook)(size_t, void *) = nullptr;
  void (*free_hook)(void *, void *) = nullptr;
  void *alloc_user = nullptr;
  uint64_t mem_budget = 0;
  int max_streams = 64;
  int max_batch = 256;
  int *status_dev = nullptr;
  unsigned long long timeout_ns = 2000000000ull;  // 2 s per bounded device-side wait
  dibr_tuning tuning{};      // zero fields: automatic
  std::map<int, dibr::ClassTune> class_tune;  // per block width: the autotuner's choices
  uint64_t launches = 0;     // kernels launched by this context

  std::mutex err_mu;
  std::string last_error, last_error_copy;

  dibr::DevBuf stage_in, stage_out, realign, xbf_depth, inpaint_scratch, inpaint_order;
  dibr::BandArgs args;  // scratch for one launch (large: keeps it off the stack)
  // the shift tables in args (and their guard width) were built for these disparity
  // parameters {rule, P, T}; rebuilt only when a call brings others
  int32_t args_tables_key[3] = {-1, -1, -1};
  int args_zguard = 0;
  int band_tables(const dibr_params *p);  // fills args.lut_h / lut_n, returns the guard width

  // batched launches (dibr_batch.cu)
  dibr::DevBuf batch_desc, batch_img, batch_depth;
  uint8_t *batch_pinned = nullptr;         // descriptor staging (pinned host memory)
  size_t batch_pinned_bytes = 0;
  cudaEvent_t batch_copy_done = nullptr;   // the last descriptor upload has read the staging

  // the buffers of the last single-frame launch (a band launch, or the inpainting launch
  // after one), when it is the last work on a stream the context owns: the next band launch
  // may overlap it if their buffers are disjoint
  struct Span {
    uintptr_t lo = 0, hi = 0;
  };
  bool prev_band = false;
  Span prev_in, prev_depth, prev_out[dibr::O_COUNT];  // read: input, cross-bilateral depth
  int inpaint_half = 0;  // the half of inpaint_scratch the next 2-D fill frame uses
  int xbf_half = 0;      // the half of xbf_depth the next cross-bilateral frame uses

  // blocking calls with host buffers: copies and kernels of row bands overlap
  static constexpr int kMaxBands = 8;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_in[kMaxBands] = {}, ev_comp[kMaxBands] = {}, ev_out = nullptr;

  // serving loop (dibr_serve.cu)
  dibr::ServeState *serve = nullptr;

  void set_error(const char *fmt, ...);
  dibr_status cuda_fail(cudaError_t e, const char *what);
  void *dev_alloc(size_t bytes);
  void dev_free(void *p);
  dibr_status ensure(dibr::DevBuf &b, size_t bytes);
  dibr_status plan_band(int W, int H, int depth_src, const uint8_t *in, int64_t pitch, int zguard,
                        dibr::BandArgs &a, int &smem, int &per_sm);
  dibr_status encode_input(dibr::BandArgs &a, const uint8_t *dev_rgb, int64_t pitch);
  dibr_status enqueue_device(const dibr_image *img, const dibr_params *p, const dibr_outputs *o);
  dibr_status synthesize_staged(const dibr_image *img, const dibr_params *p, const dibr_outputs *o);
  dibr_status synthesize_banded(const dibr_image *img, const dibr_params *p, const dibr_outputs *o, int bands);
  void release_band_pipeline();
  dibr_status enqueue_batch_device(int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                                   const dibr_outputs *outs);
  dibr_status enqueue_grouped(int n, const dibr_image *imgs, const dibr_params *p, int n_params,
                              const dibr_outputs *outs);
  dibr_status read_status();
  void release_buffers();
  void release_batch_buffers();
  void shutdown_serving();
};
