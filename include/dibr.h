/*
 * dibr.h -- C-ABI of libdibr, GB300 (sm_103a) depth-image-based rendering for 2D-to-3D
 * pseudo-stereo synthesis.
 *
 * The pipeline is the one of "3D Pseudo Stereo Visualization with GPGPU Support"
 * (Al-Oraiqat, Zori; arXiv 2009.09501):
 *   Sec. 3 / Fig. 1  depth map -> filtered depth map -> left frame / right frame ->
 *                    post-processed (inpainted) left / right frame;
 *   Sec. 4           the GPU stages: cross-bilateral filtering, left/right frame
 *                    reconstruction, left/right inpainting, stereo-pair formatting;
 *   Fig. 3           the shift rule (threshold on the filtered depth, Base/2 scaling,
 *                    out-of-range fallback) and the red-cyan channel map.
 * The parameters follow the paper's statement of the problem: the input frame, the
 * depth-map rule, the maximum parallax (Fig. 3's "Base") and the output format
 * (anaglyph, anamorphic half side-by-side pair; Figs. 4-5).
 *
 * Conventions shared by every entry point
 *  - Images are interleaved 8-bit RGB, row-major; a row holds 3*width bytes and rows are
 *    `pitch` bytes apart (pitch >= 3*width).  Depth maps are 8-bit, one byte per pixel.
 *  - Buffers belong to the caller.  The library never frees or retains a caller pointer
 *    beyond the call, except frames submitted to a stream, which must stay valid until
 *    dibr_poll() has returned their completion.
 *  - Every function returns a dibr_status; no exception or abort crosses the ABI.  The
 *    text of the last error of a context is available from dibr_last_error().
 *  - There is no CPU fallback: every pixel is computed by the library's CUDA kernels.
 *    A context cannot be created without a usable sm_103a device.
 *  - Thread safety: dibr_submit_frame() and dibr_poll() may be called from any thread;
 *    every other call on one context must come from one thread at a time.
 */
#ifndef DIBR_H
#define DIBR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIBR_ABI_VERSION 1

typedef enum {
    DIBR_OK = 0,
    DIBR_NOT_READY = 1,     /* dibr_poll: nothing completed within the timeout */
    DIBR_E_INVALID = -1,    /* an argument is out of range or inconsistent */
    DIBR_E_NOMEM = -2,      /* a device or pinned host allocation failed */
    DIBR_E_CUDA = -3,       /* a CUDA runtime/driver call failed */
    DIBR_E_BUSY = -4,       /* admission refused: memory budget or slot limit reached */
    DIBR_E_TIMEOUT = -5,    /* a bounded device-side wait gave up (status word set) */
    DIBR_E_CLOSED = -6      /* the stream is closed or unknown */
} dibr_status;

/* Depth map and its smoothing (Sec. 3 "Depth Map", "Filtered Depth Map").  The paper's
 * depth generator (an edge-based method of its earlier work) is not given; the depth
 * used here is the BT.601 luminance Y = (299 R + 587 G + 114 B + 500) / 1000 (integer
 * division).  Smoothing: none; a 5x5 binomial [1 4 6 4 1]^2/256 with clamp-to-edge,
 * rounded half up (default); or the cross-bilateral filter the paper names (RGB guide,
 * square window of half width xbf_radius clipped to the image, Gaussian spatial weight
 * sigma xbf_sigma_s, Gaussian range weight sigma xbf_sigma_r on the RGB distance,
 * evaluated in FP32, rounded half up). */
enum { DIBR_DEPTH_LUMA = 0, DIBR_DEPTH_LUMA_BINOM5 = 1, DIBR_DEPTH_LUMA_XBF = 2 };

/* Depth -> shift (Fig. 3).  With P = max_parallax_px and T = threshold,
 *   s_L(d) = -(P/2) d/255 if d > T, else (P/2)(1 - d/255);   s_R(d) = -s_L(d).
 * DIBR_DISP_PAPER uses this rule; DIBR_DISP_LINEAR uses s_L(d) = -floor(P d/510), which
 * gives zero shift at zero depth. */
enum { DIBR_DISP_PAPER = 0, DIBR_DISP_LINEAR = 1 };

/* Left/right frame reconstruction (Sec. 3, Sec. 4).
 * DIBR_WARP_FORWARD: source column x moves to target column x - floor(s(d)); per target
 *   the largest depth wins (nearer), ties go to the smaller source column in the left
 *   view and the larger one in the right view; holes take the colour of the nearest
 *   filled target on the background (smaller depth) side of the same row, the left one
 *   on a tie, the only one at a border, the input pixel if the row has none (the
 *   row-local "simplified" inpainting Sec. 4 refers to).
 * DIBR_WARP_GATHER_FIG3: Fig. 3 literally: target x samples column trunc(x + s(d)) of
 *   the input, d being the target's own filtered depth; out-of-range samples copy the
 *   input pixel at x.  Only with DIBR_DISP_PAPER. */
enum { DIBR_WARP_FORWARD = 0, DIBR_WARP_GATHER_FIG3 = 1 };

/* Output formats (Sec. 4 "GPU-Stereo 3D Pair formatting"; Fig. 3 channel map; Figs. 4-5).
 * ANAGLYPH: red-cyan, R from the left view, G and B from the right view.
 * LEFT/RIGHT: the two full-resolution views.
 * HSBS: anamorphic half side-by-side; each view squeezed 2:1 by pairwise channel means
 *   rounded half up, left view in the left half (requires an even width).
 * DEPTH: the filtered depth map (one byte per pixel).
 * HOLES: the holes of the forward warp, one byte per pixel: bit 0 set where no source
 *   reached the target in the left view, bit 1 the same for the right view (zero
 *   everywhere with DIBR_WARP_GATHER_FIG3). */
enum { DIBR_OUT_ANAGLYPH = 1, DIBR_OUT_LEFT = 2, DIBR_OUT_RIGHT = 4, DIBR_OUT_HSBS = 8,
       DIBR_OUT_DEPTH = 16, DIBR_OUT_HOLES = 32 };

/* Hole fill (Sec. 3: post-processed left / right frames; Fig. 3, left column: the
 * iterative inpainting algorithm).
 * DIBR_FILL_ROW: the row-local copy described under DIBR_WARP_FORWARD.
 * DIBR_FILL_INPAINT2D: the row-local copy, then Fig. 3's iterative block inpainting over
 *   the holes of each view: the frame is cut into inpaint_block x inpaint_block blocks;
 *   in each block the holes are visited block column by block column, and a hole with at
 *   least two non-hole 8-neighbours takes the mean of their colours (per channel, rounded
 *   half up) and stops being a hole at once for the holes after it; the visits repeat
 *   while one of them repairs something.  A block sees pixels outside it as the row-local
 *   copy left them.  Holes never repaired keep the row-local colour.  Anaglyph and HSBS
 *   are formatted from the inpainted views.  Single-image calls only
 *   (dibr_synthesize_image / dibr_enqueue_image); with DIBR_OUT_HSBS the block side must
 *   be even. */
enum { DIBR_FILL_ROW = 0, DIBR_FILL_INPAINT2D = 1 };

typedef struct {
    int32_t depth_rule;       /* DIBR_DEPTH_* */
    int32_t disparity_rule;   /* DIBR_DISP_* */
    int32_t warp_mode;        /* DIBR_WARP_* */
    int32_t max_parallax_px;  /* P, 0..1024 (Fig. 3's Base) */
    int32_t threshold;        /* T, 0..255 (150 in Fig. 3) */
    float   xbf_sigma_s;      /* > 0, pixels (default 1.5) */
    float   xbf_sigma_r;      /* > 0, RGB units (default 16) */
    int32_t xbf_radius;       /* 1..8 (default 2) */
    uint32_t outputs;         /* OR of DIBR_OUT_*; at least one */
    int32_t hole_fill;        /* DIBR_FILL_* (default DIBR_FILL_ROW) */
    int32_t inpaint_block;    /* DIBR_FILL_INPAINT2D block side, 1..32 (default 32) */
} dibr_params;

/* One input frame.  on_device != 0: rgb is a device pointer of the context's device;
 * otherwise host memory (pinned or pageable). */
typedef struct {
    const uint8_t *rgb;
    int32_t width, height;    /* >= 1; width <= 7680 (8K UHD), height <= 65535 */
    int64_t pitch;            /* bytes between rows, >= 3*width */
    int32_t on_device;
} dibr_image;

/* Where the outputs go.  Pointers for outputs not requested in dibr_params.outputs are
 * ignored and may be NULL; requested ones must be non-NULL.  RGB outputs are width x
 * height x 3 with row pitch `pitch` (>= 3*width); the depth and holes outputs are width x
 * height with row pitch `depth_pitch` (>= width).  on_device as in dibr_image. */
typedef struct {
    uint8_t *anaglyph, *left, *right, *hsbs, *depth, *holes;
    int64_t pitch;
    int64_t depth_pitch;
    int32_t on_device;
} dibr_outputs;

/* Context creation.  alloc/free, when both set, supply all device memory the library
 * uses (e.g. from a framework's caching allocator); a NULL return from alloc is reported
 * as DIBR_E_NOMEM.  When unset, cudaMallocAsync/cudaFreeAsync are used.  cuda_stream,
 * when set, is the cudaStream_t the context's work is ordered on; otherwise the context
 * creates its own non-blocking stream.  mem_budget_bytes bounds the device memory the
 * serving loop may hold for open streams (0: no bound). */
typedef struct {
    int32_t device;
    uint64_t mem_budget_bytes;
    int32_t max_streams;      /* serving: open streams at most (0: 64) */
    int32_t max_batch;        /* batch/serving: images per launch at most (0: 256) */
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
    void *cuda_stream;
} dibr_config;

typedef struct dibr_ctx dibr_ctx;

/* Fills *p with the defaults: BINOM5 smoothing, the Fig. 3 rule with T = 150, forward
 * warp, P = 16, sigma_s 1.5, sigma_r 16, radius 2, outputs = ANAGLYPH. */
dibr_status dibr_params_default(dibr_params *p);

/* Checks *p (and, when img is not NULL, that it is consistent with img). */
dibr_status dibr_validate(const dibr_params *p, const dibr_image *img);

/* The per-depth shift tables the kernels use (Fig. 3, floor reading): target column
 * t = x - hL[d] in the left view, x - hR[d] in the right view.  Host-only, no device. */
dibr_status dibr_shift_tables(const dibr_params *p, int16_t hL[256], int16_t hR[256]);

/* Creates a context on cfg->device (cfg may be NULL for all defaults).  Fails with
 * DIBR_E_CUDA when no sm_103a device is usable. */
dibr_status dibr_create(const dibr_config *cfg, dibr_ctx **out);

/* Waits for the context's work, closes its streams and frees everything it owns. */
void dibr_destroy(dibr_ctx *ctx);

/* Text of the last error recorded on ctx ("" if none).  Valid until the next call. */
const char *dibr_last_error(dibr_ctx *ctx);

/* The context's CUDA stream (a cudaStream_t).  When the context created it
 * (dibr_config.cuda_stream NULL), the caller may record events on it and wait for it but
 * enqueues no work of its own there; consecutive dibr_enqueue_image calls whose buffers
 * are disjoint then overlap: the next frame starts in the SMs the previous one has left
 * (a frame still completes only after the one before it). */
void *dibr_stream(dibr_ctx *ctx);

/* One frame, blocking: returns when the outputs are written (host or device).  Host
 * buffers are staged through device memory the context owns.  Device-side failures
 * (a bounded wait that gave up) are reported as DIBR_E_TIMEOUT. */
dibr_status dibr_synthesize_image(dibr_ctx *ctx, const dibr_image *img, const dibr_params *p,
                                  const dibr_outputs *out);

/* One frame, asynchronous: input and outputs must be device memory; the work is
 * enqueued on the context's stream and the call returns.  Use dibr_synchronize(). */
dibr_status dibr_enqueue_image(dibr_ctx *ctx, const dibr_image *img, const dibr_params *p,
                               const dibr_outputs *out);

/* Waits for all work enqueued on the context's stream and reports device-side failures
 * recorded since the previous call. */
dibr_status dibr_synchronize(dibr_ctx *ctx);

/* n frames of any sizes in one persistent launch (per-image row-band descriptors pulled
 * from a device work counter), blocking.  p points to n parameter records (one per
 * image) or to one record used for all when n_params == 1. */
dibr_status dibr_synthesize_batch(dibr_ctx *ctx, int n, const dibr_image *imgs,
                                  const dibr_params *p, int n_params, const dibr_outputs *outs);

/* As dibr_synthesize_batch, asynchronous; all buffers must be device memory. */
dibr_status dibr_enqueue_batch(dibr_ctx *ctx, int n, const dibr_image *imgs,
                               const dibr_params *p, int n_params, const dibr_outputs *outs);

/* Autotuner of the batched launches (the paper has no counterpart; it changes speed,
 * never results).  The images are grouped by size class -- the block width of their rows,
 * one thread per 16 columns rounded up to whole warps -- and each class is run alone
 * (reps timed repetitions after one warm-up, CUDA events on the context's stream) under
 * every candidate plan: a band launch of its own per image, or the shared persistent
 * launch with rows per work unit in {automatic, 2, 4, 8, 16, 32, 64}, CTAs per SM
 * {automatic, 1} and ring slots {automatic, 4}.  The fastest plan of each class is kept in
 * the context and used by every later dibr_synthesize_batch / dibr_enqueue_batch (and
 * serving batch) whose images fall in that class, where the matching dibr_set_tuning
 * knob is automatic.  All buffers must be device memory; the outputs are written (with
 * the final results) by the timed runs.  Blocking. */
dibr_status dibr_autotune_batch(dibr_ctx *ctx, int n, const dibr_image *imgs, const dibr_params *p,
                                int n_params, const dibr_outputs *outs, int reps);

/* The autotuner's per-class choices as a JSON file ({"batch_classes": [{"block_threads",
 * "rows_per_unit", "ctas_per_sm", "ring_slots", "own_launch"}, ...]}), written by
 * dibr_tuning_save and read back (replacing the context's choices) by dibr_tuning_load.
 * DIBR_E_INVALID if the file cannot be written / read or an entry is malformed. */
dibr_status dibr_tuning_save(dibr_ctx *ctx, const char *path);
dibr_status dibr_tuning_load(dibr_ctx *ctx, const char *path);

/* Batched synthesis that allocates nothing.  The paper has no counterpart: this serves
 * callers that may not allocate memory at the time they call, for example an application
 * that reserves its whole device-memory budget at start-up and forbids allocation later,
 * or code that runs under another framework's memory manager and must not allocate behind
 * its back.  dibr_synthesize_batch needs a context, and creating one allocates; this entry
 * point needs none.  It calls no cudaMalloc, cudaFree or other allocating routine: the
 * small device scratch of the batched launch (a work counter, one descriptor per image, the
 * list of work units) lives in one fixed array of 267,008 bytes in the library's device
 * data, which every GPU that loads the library holds until the process exits.
 *   - Inputs and outputs: device memory of the current device, as for dibr_enqueue_batch.
 *     Input rows must be whole 16-byte units: 16-byte aligned base and pitch, 3*width a
 *     multiple of 16 (other images would need a repacking buffer).
 *   - Limits: 1..64 images; depth rules DIBR_DEPTH_LUMA and DIBR_DEPTH_LUMA_BINOM5 only
 *     (the cross-bilateral rule needs a depth buffer); at most 8192 work units (rows per
 *     unit grow to fit).  Anything beyond returns DIBR_E_INVALID, with no error text.
 *   - cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).  The call
 *     is blocking: it copies the descriptors to the device, launches, waits for the batch
 *     on cuda_stream and reads the status word before it returns; DIBR_E_TIMEOUT reports a
 *     bounded device-side wait that gave up.
 *   - The first call on a device does a one-time set-up on that device (it looks up the
 *     device address of the scratch array); make that first call before any stream
 *     capture.
 *   - Every call shares the scratch array and rewrites it, so calls whose GPU work
 *     overlapped would race.  Within one process that cannot happen: a mutex serialises
 *     the calls and is held until each call's batch has completed. */
dibr_status dibr_synthesize_batch_static(int n, const dibr_image *imgs, const dibr_params *p,
                                         int n_params, const dibr_outputs *outs, void *cuda_stream);

/* Launch tuning: the knobs an autotuner sweeps (the paper has no counterpart; these
 * change speed, never results).  A zero field means "automatic".
 *   ring_slots     input rows staged in shared memory per CTA, 4..8;
 *   ctas_per_sm    CTAs resident per SM at most;
 *   load_mode      1: one bulk copy per input row; 2/3/4: 3-D tensor boxes whose inner
 *                  rows are 16 / 128 / 256 bytes; 5: 2-D tensor boxes of 256 bytes.
 *                  A mode that does not fit an image's width or alignment falls back to
 *                  mode 5, which fits every image;
 *   l2_prefetch    1: each CTA prefetches its later input rows into L2 at launch;
 *                  2: it does not;
 *   rows_per_unit  rows per work unit of a batched launch (dibr_synthesize_batch and
 *                  the serving loop); automatic: one unit per SM slot when an image group
 *                  is small (one 4K frame: 8 rows), 32 rows otherwise;
 *   host_bands     row bands of dibr_synthesize_image with host input and outputs (the
 *                  bands' uploads, kernels and downloads overlap), 1..8; automatic: 4 from
 *                  2048 rows, 2 from 512, else 1;
 *   frames_in_flight  1..16: when a frame is enqueued on the context's own stream while
 *                  earlier work is still queued there, and it shares no buffer with the
 *                  frame before it, its launch takes 1/n of the SM slots (in taller row
 *                  bands), so that n consecutive frames run side by side; 1: every launch
 *                  spreads over all SMs.  A launch on an idle stream always does.
 *                  Automatic: 7.
 * dibr_set_tuning() rejects out-of-range values with DIBR_E_INVALID. */
typedef struct {
    int32_t ring_slots, ctas_per_sm, load_mode, l2_prefetch, rows_per_unit, host_bands;
    int32_t frames_in_flight;
} dibr_tuning;

dibr_status dibr_set_tuning(dibr_ctx *ctx, const dibr_tuning *t);
dibr_status dibr_get_tuning(dibr_ctx *ctx, dibr_tuning *t);

/* The limit of every bounded device-side wait of this context's launches and of its
 * serving loop's batches, in nanoseconds (0: the default, 2 s).  The paper has no
 * counterpart.  The kernels wait on data and on one another only with such a limit; a wait
 * that gives up sets the context's status word, the launch unwinds after letting its own
 * copies in flight land (that wait always uses the full 2 s), and the call -- or every
 * frame of the served batch -- returns DIBR_E_TIMEOUT.  The context stays usable: the
 * status word is cleared once reported.  A very small limit makes waits that would have
 * succeeded give up, which is how the tests exercise this path without any fault.
 * DIBR_E_INVALID if ctx is NULL. */
dibr_status dibr_set_wait_limit(dibr_ctx *ctx, uint64_t limit_ns);

/* ------------------------------------------------------------------ serving loop ---
 * Concurrent video streams with continuous batching: frames submitted on any open
 * stream are gathered by a scheduler thread, copied to per-stream device buffers on a
 * copy stream, synthesized together in one batched launch, and copied back on a second
 * copy stream; completions are returned by dibr_poll(). */
typedef struct {
    int32_t stream_id;
    int32_t status;           /* dibr_status of this frame */
    uint64_t seq;             /* as given to dibr_submit_frame */
    uint64_t t_submit_ns;     /* CLOCK_MONOTONIC at submission */
    uint64_t t_done_ns;       /* CLOCK_MONOTONIC when the outputs were in host memory */
} dibr_completion;

/* Opens a stream of width x height frames.  Admission: DIBR_E_BUSY when the stream
 * limit is reached or the stream's resident device buffers would exceed the budget. */
dibr_status dibr_open_stream(dibr_ctx *ctx, int width, int height, const dibr_params *p,
                             int *stream_id);

/* Queues one host frame; host_in/host_out must stay valid until its completion is
 * polled.  DIBR_E_BUSY when the stream already has its maximum of frames in flight. */
dibr_status dibr_submit_frame(dibr_ctx *ctx, int stream_id, uint64_t seq,
                              const dibr_image *host_in, const dibr_outputs *host_out);

/* Returns up to max completions (any stream); waits up to timeout_us microseconds for
 * the first one (0: do not wait).  DIBR_NOT_READY when none arrived in time. */
dibr_status dibr_poll(dibr_ctx *ctx, dibr_completion *out, int max, int *n_out, int timeout_us);

/* Closes a stream: frames already submitted complete normally (their completions are
 * still delivered); later submissions return DIBR_E_CLOSED.  Its device buffers are
 * released once its last frame has completed. */
dibr_status dibr_close_stream(dibr_ctx *ctx, int stream_id);

#ifdef __cplusplus
}
#endif

#endif /* DIBR_H */
