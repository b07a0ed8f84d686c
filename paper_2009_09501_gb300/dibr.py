"""ctypes binding of libdibr (the C-ABI declared in ``include/dibr.h``).

Argument marshalling only: every pixel is computed by the library's CUDA kernels.  The
functions below carry the C names (``dibr_create``, ``dibr_synthesize_image``, ...); the
``Context`` class wraps them for numpy arrays (host buffers) and torch CUDA tensors
(device buffers).  If the native library is missing or cannot be loaded, every entry
point raises -- there is no fallback.
"""
import ctypes as C
import os

from . import build as _build

# ----------------------------------------------------------------------- constants
DIBR_OK, DIBR_NOT_READY = 0, 1
DIBR_E_INVALID, DIBR_E_NOMEM, DIBR_E_CUDA, DIBR_E_BUSY, DIBR_E_TIMEOUT, DIBR_E_CLOSED = -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "DIBR_OK", 1: "DIBR_NOT_READY", -1: "DIBR_E_INVALID", -2: "DIBR_E_NOMEM",
                -3: "DIBR_E_CUDA", -4: "DIBR_E_BUSY", -5: "DIBR_E_TIMEOUT", -6: "DIBR_E_CLOSED"}
DIBR_DEPTH_LUMA, DIBR_DEPTH_LUMA_BINOM5, DIBR_DEPTH_LUMA_XBF = 0, 1, 2
DIBR_DISP_PAPER, DIBR_DISP_LINEAR = 0, 1
DIBR_WARP_FORWARD, DIBR_WARP_GATHER_FIG3 = 0, 1
DIBR_OUT_ANAGLYPH, DIBR_OUT_LEFT, DIBR_OUT_RIGHT, DIBR_OUT_HSBS, DIBR_OUT_DEPTH, DIBR_OUT_HOLES = 1, 2, 4, 8, 16, 32
OUTPUT_BITS = {"anaglyph": 1, "left": 2, "right": 4, "hsbs": 8, "depth": 16, "holes": 32}
MAP_OUTPUTS = ("depth", "holes")  # one byte per pixel, row pitch depth_pitch
DIBR_FILL_ROW, DIBR_FILL_INPAINT2D = 0, 1

# exported symbols, as declared in include/dibr.h
SYMBOLS = ("dibr_params_default", "dibr_validate", "dibr_shift_tables", "dibr_create",
           "dibr_destroy", "dibr_last_error", "dibr_stream", "dibr_synthesize_image",
           "dibr_enqueue_image", "dibr_synchronize", "dibr_synthesize_batch", "dibr_enqueue_batch",
           "dibr_open_stream", "dibr_submit_frame", "dibr_poll", "dibr_close_stream",
           "dibr_set_tuning", "dibr_get_tuning", "dibr_synthesize_batch_static", "dibr_set_wait_limit",
           "dibr_autotune_batch", "dibr_tuning_save", "dibr_tuning_load")


class dibr_params(C.Structure):
    _fields_ = [("depth_rule", C.c_int32), ("disparity_rule", C.c_int32), ("warp_mode", C.c_int32),
                ("max_parallax_px", C.c_int32), ("threshold", C.c_int32),
                ("xbf_sigma_s", C.c_float), ("xbf_sigma_r", C.c_float), ("xbf_radius", C.c_int32),
                ("outputs", C.c_uint32), ("hole_fill", C.c_int32), ("inpaint_block", C.c_int32)]


class dibr_image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("pitch", C.c_int64), ("on_device", C.c_int32)]


class dibr_outputs(C.Structure):
    _fields_ = [("anaglyph", C.c_void_p), ("left", C.c_void_p), ("right", C.c_void_p),
                ("hsbs", C.c_void_p), ("depth", C.c_void_p), ("holes", C.c_void_p),
                ("pitch", C.c_int64), ("depth_pitch", C.c_int64), ("on_device", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class dibr_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("mem_budget_bytes", C.c_uint64), ("max_streams", C.c_int32),
                ("max_batch", C.c_int32), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("user", C.c_void_p), ("cuda_stream", C.c_void_p)]


class dibr_tuning(C.Structure):
    _fields_ = [("ring_slots", C.c_int32), ("ctas_per_sm", C.c_int32), ("load_mode", C.c_int32),
                ("l2_prefetch", C.c_int32), ("rows_per_unit", C.c_int32), ("host_bands", C.c_int32),
                ("frames_in_flight", C.c_int32)]


class dibr_completion(C.Structure):
    _fields_ = [("stream_id", C.c_int32), ("status", C.c_int32), ("seq", C.c_uint64),
                ("t_submit_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class DibrError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS_NAMES.get(status, str(status)), (": " + msg) if msg else ""))


_lib = None


def library_path():
    return _build.LIB_PATH


def load(build_if_missing=True):
    """Loads libdibr.so (building it first if it is missing and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError("libdibr.so is not built (%s)" % path)
        _build.build()
    L = C.CDLL(path)
    P = C.POINTER
    ctx = C.c_void_p
    sig = {
        "dibr_params_default": (C.c_int, [P(dibr_params)]),
        "dibr_validate": (C.c_int, [P(dibr_params), P(dibr_image)]),
        "dibr_shift_tables": (C.c_int, [P(dibr_params), P(C.c_int16), P(C.c_int16)]),
        "dibr_create": (C.c_int, [P(dibr_config), P(ctx)]),
        "dibr_destroy": (None, [ctx]),
        "dibr_last_error": (C.c_char_p, [ctx]),
        "dibr_stream": (C.c_void_p, [ctx]),
        "dibr_synthesize_image": (C.c_int, [ctx, P(dibr_image), P(dibr_params), P(dibr_outputs)]),
        "dibr_enqueue_image": (C.c_int, [ctx, P(dibr_image), P(dibr_params), P(dibr_outputs)]),
        "dibr_synchronize": (C.c_int, [ctx]),
        "dibr_synthesize_batch": (C.c_int, [ctx, C.c_int, P(dibr_image), P(dibr_params), C.c_int, P(dibr_outputs)]),
        "dibr_enqueue_batch": (C.c_int, [ctx, C.c_int, P(dibr_image), P(dibr_params), C.c_int, P(dibr_outputs)]),
        "dibr_open_stream": (C.c_int, [ctx, C.c_int, C.c_int, P(dibr_params), P(C.c_int)]),
        "dibr_submit_frame": (C.c_int, [ctx, C.c_int, C.c_uint64, P(dibr_image), P(dibr_outputs)]),
        "dibr_poll": (C.c_int, [ctx, P(dibr_completion), C.c_int, P(C.c_int), C.c_int]),
        "dibr_close_stream": (C.c_int, [ctx, C.c_int]),
        "dibr_set_tuning": (C.c_int, [ctx, P(dibr_tuning)]),
        "dibr_get_tuning": (C.c_int, [ctx, P(dibr_tuning)]),
        "dibr_synthesize_batch_static": (C.c_int, [C.c_int, P(dibr_image), P(dibr_params), C.c_int,
                                                   P(dibr_outputs), C.c_void_p]),
        "dibr_set_wait_limit": (C.c_int, [ctx, C.c_uint64]),
        "dibr_autotune_batch": (C.c_int, [ctx, C.c_int, P(dibr_image), P(dibr_params), C.c_int, P(dibr_outputs),
                                          C.c_int]),
        "dibr_tuning_save": (C.c_int, [ctx, C.c_char_p]),
        "dibr_tuning_load": (C.c_int, [ctx, C.c_char_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _fn(name):
    return getattr(load(), name)


# thin wrappers with the C names ----------------------------------------------------
def dibr_params_default(p):
    return _fn("dibr_params_default")(C.byref(p))


def dibr_validate(p, img=None):
    return _fn("dibr_validate")(C.byref(p), C.byref(img) if img is not None else None)


def dibr_shift_tables(p, hL, hR):
    return _fn("dibr_shift_tables")(C.byref(p), hL, hR)


def dibr_create(cfg, out_ctx):
    return _fn("dibr_create")(C.byref(cfg) if cfg is not None else None, C.byref(out_ctx))


def dibr_destroy(ctx):
    return _fn("dibr_destroy")(ctx)


def dibr_last_error(ctx):
    r = _fn("dibr_last_error")(ctx)
    return r.decode() if r else ""


def dibr_stream(ctx):
    return _fn("dibr_stream")(ctx)


def dibr_synthesize_image(ctx, img, p, out):
    return _fn("dibr_synthesize_image")(ctx, C.byref(img), C.byref(p), C.byref(out))


def dibr_enqueue_image(ctx, img, p, out):
    return _fn("dibr_enqueue_image")(ctx, C.byref(img), C.byref(p), C.byref(out))


def dibr_synchronize(ctx):
    return _fn("dibr_synchronize")(ctx)


def dibr_synthesize_batch(ctx, n, imgs, p, n_params, outs):
    return _fn("dibr_synthesize_batch")(ctx, n, imgs, p, n_params, outs)


def dibr_enqueue_batch(ctx, n, imgs, p, n_params, outs):
    return _fn("dibr_enqueue_batch")(ctx, n, imgs, p, n_params, outs)


def dibr_open_stream(ctx, w, h, p, sid):
    return _fn("dibr_open_stream")(ctx, w, h, C.byref(p), C.byref(sid))


def dibr_submit_frame(ctx, sid, seq, img, out):
    return _fn("dibr_submit_frame")(ctx, sid, seq, C.byref(img), C.byref(out))


def dibr_poll(ctx, comps, max_n, n_out, timeout_us):
    return _fn("dibr_poll")(ctx, comps, max_n, C.byref(n_out), timeout_us)


def dibr_close_stream(ctx, sid):
    return _fn("dibr_close_stream")(ctx, sid)


def dibr_set_tuning(ctx, t):
    return _fn("dibr_set_tuning")(ctx, C.byref(t))


def dibr_get_tuning(ctx, t):
    return _fn("dibr_get_tuning")(ctx, C.byref(t))


def dibr_set_wait_limit(ctx, limit_ns):
    return _fn("dibr_set_wait_limit")(ctx, limit_ns)


def dibr_autotune_batch(ctx, n, imgs, p, n_params, outs, reps):
    return _fn("dibr_autotune_batch")(ctx, n, imgs, p, n_params, outs, reps)


def dibr_tuning_save(ctx, path):
    return _fn("dibr_tuning_save")(ctx, path.encode())


def dibr_tuning_load(ctx, path):
    return _fn("dibr_tuning_load")(ctx, path.encode())


def dibr_synthesize_batch_static(n, imgs, p, n_params, outs, stream):
    return _fn("dibr_synthesize_batch_static")(n, imgs, p, n_params, outs, stream)


# ------------------------------------------------------------------ convenience layer
def make_params(depth_rule=DIBR_DEPTH_LUMA_BINOM5, disparity_rule=DIBR_DISP_PAPER,
                warp_mode=DIBR_WARP_FORWARD, max_parallax=16, threshold=150, xbf_sigma_s=1.5,
                xbf_sigma_r=16.0, xbf_radius=2, outputs=("anaglyph",), hole_fill=DIBR_FILL_ROW,
                inpaint_block=32):
    p = dibr_params()
    dibr_params_default(p)
    p.depth_rule, p.disparity_rule, p.warp_mode = depth_rule, disparity_rule, warp_mode
    p.hole_fill, p.inpaint_block = hole_fill, inpaint_block
    p.max_parallax_px, p.threshold = max_parallax, threshold
    p.xbf_sigma_s, p.xbf_sigma_r, p.xbf_radius = xbf_sigma_s, xbf_sigma_r, xbf_radius
    bits = 0
    for o in outputs:
        bits |= OUTPUT_BITS[o]
    p.outputs = bits
    return p


def output_names(p):
    return [n for n, b in OUTPUT_BITS.items() if p.outputs & b]


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def image_struct(img, pitch=None):
    """dibr_image for a (H, W, 3) uint8 numpy array (host) or torch CUDA tensor (device).
    A row pitch other than 3*W may be given for a strided 2-D view of a larger buffer."""
    if _is_torch(img):
        H, W = int(img.shape[0]), int(img.shape[1])
        ptr, dev = img.data_ptr(), 1
        if pitch is None:
            pitch = int(img.stride(0))
    else:
        H, W = img.shape[0], img.shape[1]
        ptr, dev = img.ctypes.data, 0
        if pitch is None:
            pitch = img.strides[0]
    return dibr_image(ptr, W, H, pitch, dev)


def outputs_struct(outs, pitch=None, depth_pitch=None):
    """dibr_outputs for a dict name -> array/tensor (all host or all device)."""
    o = dibr_outputs()
    dev = None
    for name, arr in outs.items():
        if _is_torch(arr):
            setattr(o, name, arr.data_ptr())
            d = 1
            st = int(arr.stride(0))
        else:
            setattr(o, name, arr.ctypes.data)
            d = 0
            st = arr.strides[0]
        if dev is not None and d != dev:
            raise ValueError("outputs must be all host or all device buffers")
        dev = d
        if name in MAP_OUTPUTS:
            if o.depth_pitch and o.depth_pitch != (depth_pitch if depth_pitch is not None else st):
                raise ValueError("depth and holes maps must share one row pitch")
            o.depth_pitch = depth_pitch if depth_pitch is not None else st
        else:
            o.pitch = pitch if pitch is not None else st
    o.on_device = dev or 0
    return o


def block_threads(width):
    """The size class of an image in batched launches: threads per block for its rows (one
    per 16 columns, rounded up to whole warps)."""
    return ((width + 15) // 16 + 31) // 32 * 32


class Context:
    """Owns one dibr_ctx.  Raises DibrError on any non-OK status."""

    def __init__(self, device=0, stream=None, mem_budget_bytes=0, max_streams=0, max_batch=0,
                 alloc=None, free=None):
        """alloc(nbytes) -> device address (0: failure) and free(address): the context's
        device allocations go through them (both or neither)."""
        cfg = dibr_config()
        cfg.device = device
        cfg.mem_budget_bytes = mem_budget_bytes
        cfg.max_streams, cfg.max_batch = max_streams, max_batch
        cfg.cuda_stream = stream
        if alloc is not None or free is not None:
            # the callbacks must outlive the context
            self._hooks = (ALLOC_FN(lambda n, user: alloc(n) or None), FREE_FN(lambda ptr, user: free(ptr)))
            cfg.alloc, cfg.free = self._hooks
        self._ctx = C.c_void_p()
        st = dibr_create(cfg, self._ctx)
        if st != DIBR_OK:
            raise DibrError(st, "dibr_create failed (needs an sm_103a GPU)")

    @property
    def handle(self):
        return self._ctx

    def check(self, st):
        if st not in (DIBR_OK, DIBR_NOT_READY):
            raise DibrError(st, dibr_last_error(self._ctx))
        return st

    def stream(self):
        return dibr_stream(self._ctx)

    @staticmethod
    def _after_torch(*objs):
        # torch's work on CUDA tensors (made or written on torch's stream) completes before
        # the context's own stream touches them
        for o in objs:
            for t in (o.values() if isinstance(o, dict) else o if isinstance(o, (list, tuple)) else (o,)):
                if isinstance(t, dict):
                    Context._after_torch(t)
                elif _is_torch(t) and t.is_cuda:
                    import torch
                    torch.cuda.current_stream(t.device).synchronize()
                    return

    def synthesize_image(self, img, p, outs, in_pitch=None):
        self._after_torch(img, outs)
        return self.check(dibr_synthesize_image(self._ctx, image_struct(img, in_pitch), p, outputs_struct(outs)))

    def enqueue_image(self, img, p, outs, in_pitch=None):
        self._after_torch(img, outs)
        return self.check(dibr_enqueue_image(self._ctx, image_struct(img, in_pitch), p, outputs_struct(outs)))

    def synchronize(self):
        return self.check(dibr_synchronize(self._ctx))

    def _batch_args(self, imgs, params, outs):
        n = len(imgs)
        I = (dibr_image * max(n, 1))(*[image_struct(x) for x in imgs])
        if isinstance(params, dibr_params):
            params = [params]
        Pa = (dibr_params * len(params))(*params)
        O = (dibr_outputs * max(n, 1))(*[outputs_struct(o) for o in outs])
        return n, I, Pa, len(params), O

    def autotune_batch(self, imgs, params, outs, reps=3):
        """Times candidate launch plans per size class on this batch (device buffers) and
        keeps the fastest in the context; returns the chosen plans."""
        self._after_torch(imgs, outs)
        self.check(dibr_autotune_batch(self._ctx, *self._batch_args(imgs, params, outs), reps))
        import json
        import os
        import tempfile
        fd, path = tempfile.mkstemp(suffix=".json")
        os.close(fd)
        try:
            self.check(dibr_tuning_save(self._ctx, path))
            with open(path) as f:
                return json.load(f)["batch_classes"]
        finally:
            os.unlink(path)

    def save_tuning(self, path):
        return self.check(dibr_tuning_save(self._ctx, path))

    def load_tuning(self, path):
        return self.check(dibr_tuning_load(self._ctx, path))

    def synthesize_batch(self, imgs, params, outs):
        self._after_torch(imgs, outs)
        n, I, Pa, npar, O = self._batch_args(imgs, params, outs)
        return self.check(dibr_synthesize_batch(self._ctx, n, I, Pa, npar, O))

    def enqueue_batch(self, imgs, params, outs):
        self._after_torch(imgs, outs)
        n, I, Pa, npar, O = self._batch_args(imgs, params, outs)
        return self.check(dibr_enqueue_batch(self._ctx, n, I, Pa, npar, O))

    def open_stream(self, width, height, p):
        sid = C.c_int(-1)
        self.check(dibr_open_stream(self._ctx, width, height, p, sid))
        return sid.value

    def submit_frame(self, sid, seq, img, outs):
        return dibr_submit_frame(self._ctx, sid, seq, image_struct(img), outputs_struct(outs))

    def poll(self, max_n=64, timeout_us=0):
        comps = (dibr_completion * max_n)()
        n = C.c_int(0)
        st = self.check(dibr_poll(self._ctx, comps, max_n, n, timeout_us))
        return [comps[i] for i in range(n.value)] if st == DIBR_OK else []

    def set_tuning(self, **kw):
        t = dibr_tuning()
        dibr_get_tuning(self._ctx, t)
        for k, v in kw.items():
            setattr(t, k, v)
        return self.check(dibr_set_tuning(self._ctx, t))

    def get_tuning(self):
        t = dibr_tuning()
        self.check(dibr_get_tuning(self._ctx, t))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def set_wait_limit(self, limit_ns):
        """Limit of the device-side bounded waits in ns (0: the default 2 s)."""
        return self.check(dibr_set_wait_limit(self._ctx, limit_ns))

    def close_stream(self, sid):
        return self.check(dibr_close_stream(self._ctx, sid))

    def close(self):
        if self._ctx:
            dibr_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
