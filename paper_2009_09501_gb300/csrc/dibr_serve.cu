// dibr_serve.cu -- serving loop: concurrent video streams with continuous batching.
//
// Each open stream owns kSlots frame slots of resident device memory (input + requested
// outputs).  dibr_submit_frame() queues a host frame.  A scheduler thread repeatedly
// takes every queued frame that has a free slot (across all streams, up to max_batch),
// uploads them on an H2D copy stream, runs them as one batched launch on the compute
// stream once the uploads are done, and downloads the outputs on a D2H copy stream.  It
// does not wait for a batch to finish before forming the next one, so frames that arrive
// while others are on the GPU join the next launch as soon as their stream has a free
// slot.  A completion thread waits for each batch's download, stamps the completion
// time and hands the completions to dibr_poll().
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dibr.h"
#include "dibr_context.h"
#include "dibr_internal.h"

namespace dibr {

dibr_status check_image_args(const dibr_params *p, const dibr_image *img, const dibr_outputs *o,
                             std::string *why);

constexpr int kSlots = 3;       // frames in flight per stream: upload, compute, download
constexpr int kMaxQueued = 16;  // frames queued per stream beyond the slots

static uint64_t now_ns() {
  timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return static_cast<uint64_t>(t.tv_sec) * 1000000000ull + static_cast<uint64_t>(t.tv_nsec);
}

struct Frame {
  uint64_t seq, t_submit;
  dibr_image in;
  dibr_outputs out;
};

struct Slot {
  uint8_t *in = nullptr, *out[O_COUNT] = {};
  bool busy = false;
};

struct Stream {
  int id, W, H;
  dibr_params p;
  int64_t in_pitch, out_pitch, depth_pitch;
  size_t bytes = 0;
  Slot slots[kSlots];
  std::deque<Frame> queue;
  int in_flight = 0;
  bool closed = false;
};

constexpr int kStatusRing = 1024;  // > streams x slots: one entry per batch in flight

struct InFlight {  // one batched launch
  cudaEvent_t done;
  int status_slot;  // this batch's status word on the device and its pinned copy
  std::vector<std::pair<int, int>> frames;  // (stream id, slot)
  std::vector<Frame> meta;
  dibr_status status;
};

struct ServeState {
  dibr_ctx *owner = nullptr;
  dibr_ctx *gpu = nullptr;  // private context: compute stream, batch buffers, status word
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_poll;
  std::map<int, std::unique_ptr<Stream>> streams;
  std::deque<InFlight> inflight;
  std::deque<dibr_completion> done;
  int next_id = 1;
  uint64_t resident = 0;
  int *status_host = nullptr;  // pinned [kStatusRing]
  int *status_ring = nullptr;  // device [kStatusRing]: one status word per batch, zeroed before it
  int *gpu_status = nullptr;   // the private context's own status word (restored at shutdown)
  cudaEvent_t ev_up = nullptr, ev_comp = nullptr;  // re-recorded by every batch
  std::vector<cudaEvent_t> ev_free;                 // batch completion events for reuse (under mu)
  uint64_t batches = 0;
  bool stop = false;
  std::thread sched, compl_thread;
};

static size_t stream_bytes(const Stream &s) {
  size_t b = static_cast<size_t>(s.in_pitch) * s.H;
  for (int k = 0; k < O_COUNT; ++k)
    if (s.p.outputs & kOutBits[k]) b += static_cast<size_t>(is_map_output(k) ? s.depth_pitch : s.out_pitch) * s.H;
  return b * kSlots;
}

static void free_stream(ServeState *st, Stream &s) {
  for (Slot &sl : s.slots) {
    st->gpu->dev_free(sl.in);
    for (uint8_t *&o : sl.out) {
      st->gpu->dev_free(o);
      o = nullptr;
    }
    sl.in = nullptr;
  }
  st->resident -= s.bytes;
}

// Scheduler: forms and enqueues batches.
static void scheduler_loop(ServeState *st) {
  cudaSetDevice(st->gpu->device);
  const uint32_t *bits = kOutBits;
  std::vector<dibr_image> imgs;
  std::vector<dibr_params> prms;
  std::vector<dibr_outputs> outs;
  while (true) {
    InFlight b;
    {
      std::unique_lock<std::mutex> lk(st->mu);
      auto ready = [&] {
        if (st->stop) return true;
        for (auto &kv : st->streams) {
          Stream &s = *kv.second;
          if (s.queue.empty()) continue;
          for (const Slot &sl : s.slots)
            if (!sl.busy) return true;
        }
        return false;
      };
      st->cv_sched.wait(lk, ready);
      if (st->stop) return;
      // gather: round-robin over streams, one frame per free slot, up to max_batch
      const int cap = st->owner->max_batch;
      bool more = true;
      while (more && static_cast<int>(b.frames.size()) < cap) {
        more = false;
        for (auto &kv : st->streams) {
          Stream &s = *kv.second;
          if (s.queue.empty() || static_cast<int>(b.frames.size()) >= cap) continue;
          int free_slot = -1;
          for (int i = 0; i < kSlots; ++i)
            if (!s.slots[i].busy) {
              free_slot = i;
              break;
            }
          if (free_slot < 0) continue;
          s.slots[free_slot].busy = true;
          ++s.in_flight;
          b.frames.emplace_back(s.id, free_slot);
          b.meta.push_back(s.queue.front());
          s.queue.pop_front();
          more = true;
        }
      }
      // descriptors of the batch (stream objects stay alive while they have frames in flight)
      imgs.clear();
      prms.clear();
      outs.clear();
      for (size_t f = 0; f < b.frames.size(); ++f) {
        Stream &s = *st->streams[b.frames[f].first];
        Slot &sl = s.slots[b.frames[f].second];
        imgs.push_back(dibr_image{sl.in, s.W, s.H, s.in_pitch, 1});
        prms.push_back(s.p);
        dibr_outputs o;
        std::memset(&o, 0, sizeof(o));
        for (int k = 0; k < O_COUNT; ++k) out_slot(o, k) = sl.out[k];
        o.pitch = s.out_pitch;
        o.depth_pitch = s.depth_pitch;
        o.on_device = 1;
        outs.push_back(o);
      }
    }
    // uploads (copy stream) -> batched launch (compute stream) -> downloads (copy stream)
    dibr_status status = DIBR_OK;
    cudaEvent_t up = st->ev_up, comp = st->ev_comp;
    b.done = nullptr;
    {
      std::lock_guard<std::mutex> lk(st->mu);
      if (!st->ev_free.empty()) {
        b.done = st->ev_free.back();
        st->ev_free.pop_back();
      }
    }
    if (!b.done) cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    // the batch reports bounded-wait failures in a status word of its own, zeroed before its
    // launch on the compute stream, so that one batch's failure never shows on later ones
    b.status_slot = static_cast<int>(st->batches++ % kStatusRing);
    int *status_word = st->status_ring + b.status_slot;
    cudaMemsetAsync(status_word, 0, sizeof(int), st->gpu->stream);
    st->gpu->status_dev = status_word;
    st->gpu->timeout_ns = st->owner->timeout_ns;
    st->gpu->prev_band = false;  // (the memset is other work on the stream)
    for (size_t f = 0; f < b.frames.size(); ++f) {
      const Frame &fr = b.meta[f];
      if (cudaMemcpy2DAsync(const_cast<uint8_t *>(imgs[f].rgb), imgs[f].pitch, fr.in.rgb, fr.in.pitch,
                            3 * static_cast<size_t>(imgs[f].width), imgs[f].height, cudaMemcpyHostToDevice,
                            st->h2d) != cudaSuccess)
        status = DIBR_E_CUDA;
    }
    cudaEventRecord(up, st->h2d);
    cudaStreamWaitEvent(st->gpu->stream, up, 0);
    if (status == DIBR_OK)
      status = st->gpu->enqueue_batch_device(static_cast<int>(imgs.size()), imgs.data(), prms.data(),
                                             static_cast<int>(prms.size()), outs.data());
    cudaEventRecord(comp, st->gpu->stream);
    cudaStreamWaitEvent(st->d2h, comp, 0);
    for (size_t f = 0; f < b.frames.size() && status == DIBR_OK; ++f) {
      const Frame &fr = b.meta[f];
      for (int k = 0; k < O_COUNT; ++k) {
        if (!(prms[f].outputs & bits[k])) continue;
        const bool dep = is_map_output(k);
        if (cudaMemcpy2DAsync(out_slot(fr.out, k), dep ? fr.out.depth_pitch : fr.out.pitch, out_slot(outs[f], k),
                              dep ? outs[f].depth_pitch : outs[f].pitch,
                              dep ? imgs[f].width : 3 * static_cast<size_t>(imgs[f].width), imgs[f].height,
                              cudaMemcpyDeviceToHost, st->d2h) != cudaSuccess)
          status = DIBR_E_CUDA;
      }
    }
    cudaMemcpyAsync(&st->status_host[b.status_slot], status_word, sizeof(int), cudaMemcpyDeviceToHost, st->d2h);
    cudaEventRecord(b.done, st->d2h);
    b.status = status;
    {
      std::lock_guard<std::mutex> lk(st->mu);
      st->inflight.push_back(std::move(b));
    }
    st->cv_done.notify_one();
  }
}

// Completion thread: finishes batches in launch order.
static void completion_loop(ServeState *st) {
  cudaSetDevice(st->gpu->device);
  while (true) {
    InFlight b;
    {
      std::unique_lock<std::mutex> lk(st->mu);
      st->cv_done.wait(lk, [&] { return st->stop || !st->inflight.empty(); });
      if (st->inflight.empty()) return;  // stop requested and nothing left
      b = std::move(st->inflight.front());
      st->inflight.pop_front();
    }
    cudaError_t e = cudaEventSynchronize(b.done);
    dibr_status status = b.status;
    if (e != cudaSuccess && status == DIBR_OK) status = DIBR_E_CUDA;
    // device-side bounded waits report through the batch's own status word, copied behind
    // the batch's downloads
    if (status == DIBR_OK && st->status_host[b.status_slot] != 0) status = DIBR_E_TIMEOUT;
    const uint64_t t = now_ns();
    {
      std::lock_guard<std::mutex> lk(st->mu);
      st->ev_free.push_back(b.done);
      for (size_t f = 0; f < b.frames.size(); ++f) {
        auto it = st->streams.find(b.frames[f].first);
        if (it != st->streams.end()) {
          Stream &s = *it->second;
          s.slots[b.frames[f].second].busy = false;
          --s.in_flight;
          if (s.closed && s.in_flight == 0 && s.queue.empty()) {
            free_stream(st, s);
            st->streams.erase(it);
          }
        }
        dibr_completion c;
        c.stream_id = b.frames[f].first;
        c.status = status;
        c.seq = b.meta[f].seq;
        c.t_submit_ns = b.meta[f].t_submit;
        c.t_done_ns = t;
        st->done.push_back(c);
      }
    }
    st->cv_poll.notify_all();
    st->cv_sched.notify_one();
  }
}

static dibr_status ensure_serving(dibr_ctx *c) {
  if (c->serve) return DIBR_OK;
  auto *st = new ServeState();
  st->owner = c;
  dibr_config cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.device = c->device;
  cfg.alloc = c->alloc_hook;
  cfg.free = c->free_hook;
  cfg.user = c->alloc_user;
  cfg.max_batch = c->max_batch;
  dibr_status s = dibr_create(&cfg, &st->gpu);
  if (s != DIBR_OK) {
    delete st;
    return s;
  }
  st->gpu->tuning = c->tuning;
  st->gpu_status = st->gpu->status_dev;
  st->status_ring = static_cast<int *>(st->gpu->dev_alloc(sizeof(int) * kStatusRing));
  if (!st->status_ring) {
    dibr_destroy(st->gpu);
    delete st;
    c->set_error("device allocation of the serving status words failed");
    return DIBR_E_NOMEM;
  }
  if (cudaStreamCreateWithFlags(&st->h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st->d2h, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&st->ev_up, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&st->ev_comp, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&st->status_host), sizeof(int) * kStatusRing, cudaHostAllocDefault) !=
          cudaSuccess) {
    if (st->h2d) cudaStreamDestroy(st->h2d);
    if (st->d2h) cudaStreamDestroy(st->d2h);
    if (st->ev_up) cudaEventDestroy(st->ev_up);
    if (st->ev_comp) cudaEventDestroy(st->ev_comp);
    cudaStreamSynchronize(st->gpu->stream);
    st->gpu->dev_free(st->status_ring);
    dibr_destroy(st->gpu);
    delete st;
    return DIBR_E_CUDA;
  }
  c->serve = st;
  st->sched = std::thread(scheduler_loop, st);
  st->compl_thread = std::thread(completion_loop, st);
  return DIBR_OK;
}

}  // namespace dibr

using namespace dibr;

void dibr_ctx::shutdown_serving() {
  ServeState *st = serve;
  if (!st) return;
  {
    // let queued frames finish: wait until nothing is queued or in flight
    std::unique_lock<std::mutex> lk(st->mu);
    st->cv_poll.wait_for(lk, std::chrono::seconds(30), [&] {
      for (auto &kv : st->streams)
        if (!kv.second->queue.empty() || kv.second->in_flight) return false;
      return st->inflight.empty();
    });
    st->stop = true;
  }
  st->cv_sched.notify_all();
  st->cv_done.notify_all();
  st->sched.join();
  st->compl_thread.join();
  cudaStreamSynchronize(st->h2d);
  cudaStreamSynchronize(st->d2h);
  for (auto &kv : st->streams) free_stream(st, *kv.second);
  st->streams.clear();
  cudaStreamDestroy(st->h2d);
  cudaStreamDestroy(st->d2h);
  cudaFreeHost(st->status_host);
  for (cudaEvent_t e : st->ev_free) cudaEventDestroy(e);
  cudaEventDestroy(st->ev_up);
  cudaEventDestroy(st->ev_comp);
  cudaStreamSynchronize(st->gpu->stream);
  st->gpu->dev_free(st->status_ring);
  st->gpu->status_dev = st->gpu_status;
  dibr_destroy(st->gpu);
  delete st;
  serve = nullptr;
}

extern "C" {

dibr_status dibr_open_stream(dibr_ctx *c, int width, int height, const dibr_params *p, int *stream_id) {
  if (!c || !p || !stream_id) return DIBR_E_INVALID;
  *stream_id = -1;
  dibr_image probe{reinterpret_cast<const uint8_t *>(16), width, height, 3 * static_cast<int64_t>(width), 0};
  std::string why;
  dibr_outputs po;
  std::memset(&po, 0, sizeof(po));
  uint8_t *nonnull = reinterpret_cast<uint8_t *>(16);
  for (int k = 0; k < O_COUNT; ++k) out_slot(po, k) = nonnull;
  po.pitch = 3 * static_cast<int64_t>(width);
  po.depth_pitch = width;
  dibr_status s = check_image_args(p, &probe, &po, &why);
  if (s != DIBR_OK) {
    c->set_error("%s", why.c_str());
    return s;
  }
  if (p->hole_fill != DIBR_FILL_ROW) {
    c->set_error("the 2-D fill runs on single-image calls only");
    return DIBR_E_INVALID;
  }
  cudaSetDevice(c->device);
  if ((s = ensure_serving(c)) != DIBR_OK) return s;
  ServeState *st = c->serve;
  auto strm = std::make_unique<Stream>();
  strm->W = width;
  strm->H = height;
  strm->p = *p;
  strm->in_pitch = round_up(3 * width, 16);
  strm->out_pitch = round_up(3 * width, 16);
  strm->depth_pitch = round_up(width, 16);
  strm->bytes = stream_bytes(*strm);
  std::lock_guard<std::mutex> lk(st->mu);
  int open = 0;
  for (auto &kv : st->streams)
    if (!kv.second->closed) ++open;
  if (open >= c->max_streams) {
    c->set_error("stream limit %d reached", c->max_streams);
    return DIBR_E_BUSY;
  }
  if (c->mem_budget && st->resident + strm->bytes > c->mem_budget) {
    c->set_error("stream needs %zu bytes; %llu of the %llu-byte budget in use", strm->bytes,
                 static_cast<unsigned long long>(st->resident), static_cast<unsigned long long>(c->mem_budget));
    return DIBR_E_BUSY;
  }
  const uint32_t *bits = kOutBits;
  bool ok = true;
  for (Slot &sl : strm->slots) {
    sl.in = static_cast<uint8_t *>(st->gpu->dev_alloc(static_cast<size_t>(strm->in_pitch) * height));
    ok = ok && sl.in;
    for (int k = 0; k < O_COUNT; ++k)
      if (p->outputs & bits[k]) {
        sl.out[k] = static_cast<uint8_t *>(
            st->gpu->dev_alloc(static_cast<size_t>(is_map_output(k) ? strm->depth_pitch : strm->out_pitch) * height));
        ok = ok && sl.out[k];
      }
  }
  st->resident += strm->bytes;
  if (!ok) {
    free_stream(st, *strm);
    c->set_error("device allocation for the stream's buffers failed");
    return DIBR_E_NOMEM;
  }
  cudaStreamSynchronize(st->gpu->stream);  // allocations ordered before first use
  strm->id = st->next_id++;
  *stream_id = strm->id;
  st->streams[strm->id] = std::move(strm);
  return DIBR_OK;
}

dibr_status dibr_submit_frame(dibr_ctx *c, int stream_id, uint64_t seq, const dibr_image *host_in,
                              const dibr_outputs *host_out) {
  if (!c || !host_in || !host_out) return DIBR_E_INVALID;
  ServeState *st = c->serve;
  if (!st) return DIBR_E_CLOSED;
  {
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->streams.find(stream_id);
    if (it == st->streams.end() || it->second->closed) return DIBR_E_CLOSED;
    Stream &s = *it->second;
    std::string why;
    dibr_status v = check_image_args(&s.p, host_in, host_out, &why);
    if (v == DIBR_OK && (host_in->width != s.W || host_in->height != s.H)) v = DIBR_E_INVALID;
    if (v == DIBR_OK && (host_in->on_device || host_out->on_device)) v = DIBR_E_INVALID;
    if (v != DIBR_OK) return v;
    if (static_cast<int>(s.queue.size()) >= kMaxQueued) return DIBR_E_BUSY;
    s.queue.push_back(Frame{seq, now_ns(), *host_in, *host_out});
  }
  st->cv_sched.notify_one();
  return DIBR_OK;
}

dibr_status dibr_poll(dibr_ctx *c, dibr_completion *out, int max, int *n_out, int timeout_us) {
  if (!c || !n_out || max < 0 || (max > 0 && !out)) return DIBR_E_INVALID;
  *n_out = 0;
  ServeState *st = c->serve;
  if (!st) return DIBR_NOT_READY;
  std::unique_lock<std::mutex> lk(st->mu);
  if (st->done.empty() && timeout_us > 0)
    st->cv_poll.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !st->done.empty(); });
  int n = 0;
  while (n < max && !st->done.empty()) {
    out[n++] = st->done.front();
    st->done.pop_front();
  }
  *n_out = n;
  return n ? DIBR_OK : DIBR_NOT_READY;
}

dibr_status dibr_close_stream(dibr_ctx *c, int stream_id) {
  if (!c) return DIBR_E_INVALID;
  ServeState *st = c->serve;
  if (!st) return DIBR_E_CLOSED;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->streams.find(stream_id);
  if (it == st->streams.end() || it->second->closed) return DIBR_E_CLOSED;
  Stream &s = *it->second;
  s.closed = true;
  if (s.in_flight == 0 && s.queue.empty()) {
    free_stream(st, s);
    st->streams.erase(it);
  }
  return DIBR_OK;
}

}  // extern "C"
