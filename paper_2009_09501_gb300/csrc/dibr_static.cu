// dibr_static.cu -- dibr_synthesize_batch_static: the batched synthesis for callers that
// must not allocate memory.
//
// The batch kernel needs a little device memory beside the caller's images: a work
// counter, one descriptor per image and the list of work units.  dibr_synthesize_batch
// takes it from a context, which allocates.  This entry point instead uses one array in
// the library's own device data (file-scope, fixed size), so it needs no context and
// calls no allocation routine: no cudaMalloc, no cudaFree, no pinned or pageable host
// allocation.  The descriptors are written into a fixed host array and copied to the
// device array before the launch.
#include <cstring>
#include <mutex>

#include "dibr.h"
#include "dibr_internal.h"

namespace dibr {
void shift_tables(const dibr_params *p, int32_t *lut_h, int32_t *lut_n);
}

using namespace dibr;

namespace {

constexpr int kStaticMaxImages = 64;
constexpr int kStaticMaxUnits = 8192;
constexpr int kStaticMaxDevices = 64;
constexpr size_t kDescOff = 256;  // [group counters][status] ... [descriptors] [units]
constexpr int kStatusWord = kMaxClasses;  // int index of the status word in the header
constexpr size_t kUnitsOff = (kDescOff + sizeof(ImageDesc) * kStaticMaxImages + 255) / 256 * 256;
constexpr size_t kStaticBytes = kUnitsOff + sizeof(int4) * kStaticMaxUnits;  // 267,008 bytes

// Device scratch shared by every call on a device (each GPU that loads the library holds
// it until the process exits).  Host code must not use its name as an address: the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_scratch[kStaticBytes];

// Host staging of the descriptors, guarded by g_mu.
static uint8_t g_staging[kStaticBytes];
static std::mutex g_mu;

struct DeviceSetup {
  bool done = false;
  uint8_t *scratch = nullptr;  // device address of g_scratch on this device
  int sms = 0, smem_per_sm = 0, max_smem = 0;
};
static DeviceSetup g_dev[kStaticMaxDevices];

// Once per device, with that device current: the scratch array's device address and the
// device limits the launch plan needs.
dibr_status setup_device(int dev) {
  DeviceSetup &d = g_dev[dev];
  if (d.done) return DIBR_OK;
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return DIBR_E_CUDA;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return DIBR_E_CUDA;
  }
  if (!(major == 10 && minor == 3)) return DIBR_E_CUDA;  // built for sm_103a only
  d.scratch = static_cast<uint8_t *>(ptr);
  d.done = true;
  return DIBR_OK;
}

// Argument checks without any allocation (status codes only).
bool valid_image(const dibr_params *p, const dibr_image *im, const dibr_outputs *o) {
  if (!p || !im || !o) return false;
  if (p->depth_rule != DIBR_DEPTH_LUMA && p->depth_rule != DIBR_DEPTH_LUMA_BINOM5) return false;
  if (p->disparity_rule < 0 || p->disparity_rule > 1 || p->warp_mode < 0 || p->warp_mode > 1) return false;
  if (p->warp_mode == DIBR_WARP_GATHER_FIG3 && p->disparity_rule != DIBR_DISP_PAPER) return false;
  if (p->max_parallax_px < 0 || p->max_parallax_px > 1024 || p->threshold < 0 || p->threshold > 255) return false;
  if (p->outputs == 0 || (p->outputs & ~kAllOutputs)) return false;
  if (p->hole_fill != DIBR_FILL_ROW) return false;  // the 2-D fill needs scratch views
  if (!im->rgb || !im->on_device || !o->on_device) return false;
  if (im->width < 1 || im->height < 1 || im->width > kMaxWidth || im->height > 65535) return false;
  if (im->pitch < 3 * static_cast<int64_t>(im->width)) return false;
  // rows are read with one bulk copy each: 16-byte aligned rows of whole 16-byte units
  if ((reinterpret_cast<uintptr_t>(im->rgb) & 15u) || (im->pitch & 15) || (3 * im->width) % 16) return false;
  if ((p->outputs & DIBR_OUT_HSBS) && (im->width & 1)) return false;
  for (int k = 0; k < O_COUNT; ++k)
    if ((p->outputs & kOutBits[k]) && !out_slot(*o, k)) return false;
  const uint32_t maps = DIBR_OUT_DEPTH | DIBR_OUT_HOLES;
  if ((p->outputs & ~maps) && o->pitch < 3 * static_cast<int64_t>(im->width)) return false;
  if ((p->outputs & maps) && o->depth_pitch < im->width) return false;
  return true;
}

}  // namespace

extern "C" dibr_status dibr_synthesize_batch_static(int n, const dibr_image *imgs, const dibr_params *p,
                                                    int n_params, const dibr_outputs *outs, void *cuda_stream) {
  if (n < 1 || n > kStaticMaxImages || !imgs || !p || !outs || (n_params != 1 && n_params != n))
    return DIBR_E_INVALID;
  int widths[kStaticMaxImages], heights[kStaticMaxImages], row_bytes[kStaticMaxImages];
  for (int i = 0; i < n; ++i) {
    if (!valid_image(&p[n_params == 1 ? 0 : i], &imgs[i], &outs[i])) return DIBR_E_INVALID;
    widths[i] = imgs[i].width;
    heights[i] = imgs[i].height;
    row_bytes[i] = 3 * imgs[i].width;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
    cudaGetLastError();
    return DIBR_E_CUDA;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  std::lock_guard<std::mutex> lk(g_mu);
  dibr_status s = setup_device(dev);
  if (s != DIBR_OK) return s;
  const DeviceSetup &d = g_dev[dev];

  // one launch per group of equal block width (the context's batched launch plan)
  BatchClass cls[kMaxClasses];
  int class_of[kStaticMaxImages], order[kStaticMaxImages];
  // the z-buffer guard every image fits in: the largest shift of their tables
  int zguard = 4;
  for (int i = 0; i < n_params; ++i) {
    int32_t lh[256], ln[256];
    shift_tables(&p[i], lh, ln);
    const int g = zguard_of(lh);
    if (g > zguard) zguard = g;
  }
  const BatchLimits lim{d.max_smem, d.smem_per_sm, 0, 0, zguard};
  const int nclass = plan_batch_classes(n, widths, row_bytes, lim, class_of, cls);
  if (nclass < 1) return DIBR_E_INVALID;
  order_by_area(n, widths, heights, order);
  // rows per unit as for the context's batches, larger while the unit list would not fit
  plan_unit_rows(n, heights, class_of, nclass, d.sms, 0, cls);
  auto count_units = [&]() {
    int64_t u = 0;
    for (int i = 0; i < n; ++i) u += (heights[i] + cls[class_of[i]].rows - 1) / cls[class_of[i]].rows;
    return u;
  };
  while (count_units() > kStaticMaxUnits)
    for (int c = 0; c < nclass; ++c) cls[c].rows *= 2;

  // descriptors and units into the host staging; the header zeroes the groups' unit
  // counters and the status word, which every call needs to start at zero
  std::memset(g_staging, 0, kDescOff);
  ImageDesc *descs = reinterpret_cast<ImageDesc *>(g_staging + kDescOff);
  int4 *units = reinterpret_cast<int4 *>(g_staging + kUnitsOff);
  for (int i = 0; i < n; ++i) {
    const dibr_image &im = imgs[i];
    const dibr_params &pp = p[n_params == 1 ? 0 : i];
    const dibr_outputs &o = outs[i];
    ImageDesc &dd = descs[i];
    std::memset(&dd, 0, sizeof(dd));
    dd.in = im.rgb;
    dd.in_pitch = im.pitch;
    for (int k = 0; k < O_COUNT; ++k) dd.out[k] = out_slot(o, k);
    dd.out_pitch = o.pitch;
    dd.depth_pitch = o.depth_pitch;
    dd.W = im.width;
    dd.H = im.height;
    dd.nch = chunks_of(im.width);
    dd.row_bytes = 3 * im.width;
    dd.outputs = pp.outputs;
    dd.warp_mode = pp.warp_mode;
    dd.depth_src = pp.depth_rule == DIBR_DEPTH_LUMA_BINOM5 ? DS_BINOM5 : DS_LUMA;
    shift_tables(&pp, dd.lut_h, dd.lut_n);
  }
  // every image of one fixed output set: the launches use that set's kernel instance
  uint32_t fixed = 0;
  for (int i = 0; i < n; ++i) {
    const uint32_t f = fixed_set(descs[i].outputs, descs[i].depth_src, descs[i].warp_mode, descs[i].out,
                                 descs[i].out_pitch);
    fixed = i == 0 ? f : (f == fixed ? fixed : 0u);
  }
  int n_units = 0;
  for (int c = 0; c < nclass; ++c) {
    cls[c].unit_begin = n_units;
    for (int oi = 0; oi < n; ++oi) {
      const int i = order[oi];
      if (class_of[i] != c) continue;
      const int rpu = cls[c].rows;
      for (int y0 = 0; y0 < imgs[i].height; y0 += rpu)
        units[n_units++] = make_int4(i, y0, y0 + rpu < imgs[i].height ? y0 + rpu : imgs[i].height, 0);
    }
    cls[c].n_units = n_units - cls[c].unit_begin;
  }
  // From pageable memory the copy has left g_staging when the call returns.
  const size_t bytes = kUnitsOff + sizeof(int4) * static_cast<size_t>(n_units);
  cudaError_t e = cudaMemcpyAsync(d.scratch, g_staging, bytes, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return DIBR_E_CUDA;
  int *status_dev = reinterpret_cast<int *>(d.scratch) + kStatusWord;
  for (int c = 0; c < nclass; ++c) {
    BatchArgs b;
    b.descs = reinterpret_cast<const ImageDesc *>(d.scratch + kDescOff);
    b.units = reinterpret_cast<const int4 *>(d.scratch + kUnitsOff) + cls[c].unit_begin;
    b.n_units = cls[c].n_units;
    b.counter = reinterpret_cast<int *>(d.scratch) + c;
    b.status = status_dev;
    b.timeout_ns = 2000000000ull;
    b.nb = cls[c].nb;
    b.srow = cls[c].srow;
    b.nch_max = cls[c].nch_max;
    b.nc = cls[c].nc;
    b.zguard = zguard;
    b.outs = fixed;
    const int grid = cls[c].n_units < d.sms * cls[c].per ? cls[c].n_units : d.sms * cls[c].per;
    e = launch_batch(b, grid > 0 ? grid : 1, cls[c].smem, c > 0, stream);
    if (e != cudaSuccess) return DIBR_E_CUDA;
  }
  // blocking: wait for the batch, then read the device status word
  int status = 0;
  e = cudaMemcpyAsync(&status, status_dev, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return DIBR_E_CUDA;
  return status ? DIBR_E_TIMEOUT : DIBR_OK;
}
