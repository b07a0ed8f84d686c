"""ctypes wrapper over the compiled C oracle -- TEST INFRASTRUCTURE ONLY.

Every function takes and returns numpy arrays.  Images are ``(H, W, 3) uint8`` RGB,
depth maps ``(H, W) uint8``.  The pipeline definitions live in ``dibr_oracle.c`` (and
``inpaint2d_oracle.c``), each citing the section of the paper it follows.
"""
import ctypes as C

import numpy as np

from . import build as _build

DEPTH_LUMA, DEPTH_BINOM5, DEPTH_XBF = 0, 1, 2
DISP_PAPER, DISP_LINEAR = 0, 1
WARP_FORWARD, WARP_GATHER_FIG3 = 0, 1
FILL_ROW, FILL_INPAINT2D = 0, 1

OUTPUT_NAMES = ("anaglyph", "left", "right", "hsbs", "depth", "holes")


class _Params(C.Structure):
    _fields_ = [("depth_rule", C.c_int32), ("disparity_rule", C.c_int32),
                ("warp_mode", C.c_int32), ("max_parallax", C.c_int32),
                ("threshold", C.c_int32), ("xbf_sigma_s", C.c_double),
                ("xbf_sigma_r", C.c_double), ("xbf_radius", C.c_int32),
                ("fill_mode", C.c_int32), ("inpaint_block", C.c_int32)]


class _Outputs(C.Structure):
    _fields_ = [("anaglyph", C.c_void_p), ("left", C.c_void_p), ("right", C.c_void_p),
                ("hsbs", C.c_void_p), ("depth", C.c_void_p), ("holes", C.c_void_p),
                ("pitch", C.c_int64),
                ("depth_pitch", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u8p = C.c_void_p
        L.or_luma.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, u8p]
        L.or_smooth_binom5.argtypes = [u8p, C.c_int, C.c_int, u8p]
        L.or_smooth_xbf.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, u8p, C.c_int,
                                    C.c_double, C.c_double, u8p]
        L.or_disparity_lut.argtypes = [C.c_int, C.c_int, C.c_int, u8p, u8p]
        L.or_from_depth.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, u8p,
                                    C.POINTER(_Params), C.POINTER(_Outputs)]
        L.or_from_depth.restype = C.c_int
        L.or_depth.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, C.POINTER(_Params), u8p]
        L.or_depth.restype = C.c_int
        L.or_dibr.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, C.POINTER(_Params),
                              C.POINTER(_Outputs)]
        L.or_dibr.restype = C.c_int
        L.or_dibr_rows.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, C.POINTER(_Params),
                                   C.POINTER(_Outputs), C.c_int, C.c_int]
        L.or_dibr_rows.restype = C.c_int
        L.or_inpaint2d.argtypes = [u8p, C.c_int, C.c_int, C.c_int64, u8p, C.c_int64,
                                   C.c_int, C.c_int, u8p, C.c_int64]
        L.or_inpaint2d.restype = C.c_int64
        _lib = L
    return _lib


def params(depth_rule=DEPTH_BINOM5, disparity_rule=DISP_PAPER, warp_mode=WARP_FORWARD,
           max_parallax=16, threshold=150, xbf_sigma_s=1.5, xbf_sigma_r=16.0, xbf_radius=2,
           fill_mode=FILL_ROW, inpaint_block=32):
    """Oracle parameter record; defaults follow Fig. 3 (T = 150) and the default smoothing."""
    return dict(depth_rule=depth_rule, disparity_rule=disparity_rule, warp_mode=warp_mode,
                max_parallax=max_parallax, threshold=threshold, xbf_sigma_s=xbf_sigma_s,
                xbf_sigma_r=xbf_sigma_r, xbf_radius=xbf_radius, fill_mode=fill_mode,
                inpaint_block=inpaint_block)


def _cparams(p):
    return _Params(p["depth_rule"], p["disparity_rule"], p["warp_mode"], p["max_parallax"],
                   p["threshold"], p["xbf_sigma_s"], p["xbf_sigma_r"], p["xbf_radius"],
                   p.get("fill_mode", FILL_ROW), p.get("inpaint_block", 32))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check_img(img):
    img = np.ascontiguousarray(img)
    assert img.dtype == np.uint8 and img.ndim == 3 and img.shape[2] == 3
    return img


def luma(img):
    img = _check_img(img)
    H, W, _ = img.shape
    Y = np.empty((H, W), np.uint8)
    lib().or_luma(_ptr(img), W, H, 3 * W, _ptr(Y))
    return Y


def smooth_binom5(Y):
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W = Y.shape
    D = np.empty_like(Y)
    lib().or_smooth_binom5(_ptr(Y), W, H, _ptr(D))
    return D


def smooth_xbf(img, Y, radius=2, sigma_s=1.5, sigma_r=16.0):
    img = _check_img(img)
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W = Y.shape
    D = np.empty_like(Y)
    lib().or_smooth_xbf(_ptr(img), W, H, 3 * W, _ptr(Y), radius, sigma_s, sigma_r, _ptr(D))
    return D


def disparity_lut(rule, P, T=150):
    hL = np.empty(256, np.int16)
    hR = np.empty(256, np.int16)
    lib().or_disparity_lut(rule, P, T, _ptr(hL), _ptr(hR))
    return hL, hR


def _alloc_outputs(H, W, want):
    outs = {}
    for name in want:
        if name in ("depth", "holes"):
            outs[name] = np.zeros((H, W), np.uint8)
        else:
            outs[name] = np.zeros((H, W, 3), np.uint8)
    co = _Outputs(*[_ptr(outs.get(n)) for n in OUTPUT_NAMES], 3 * W, W)
    return outs, co


def depth(img, p):
    img = _check_img(img)
    H, W, _ = img.shape
    D = np.empty((H, W), np.uint8)
    cp = _cparams(p)
    rc = lib().or_depth(_ptr(img), W, H, 3 * W, C.byref(cp), _ptr(D))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return D


def from_depth(img, D, p, want=("anaglyph", "left", "right")):
    """Warp, occlusion, fill and formatting for a given depth map (the integer back half)."""
    img = _check_img(img)
    D = np.ascontiguousarray(D, dtype=np.uint8)
    H, W, _ = img.shape
    assert D.shape == (H, W)
    outs, co = _alloc_outputs(H, W, want)
    cp = _cparams(p)
    rc = lib().or_from_depth(_ptr(img), W, H, 3 * W, _ptr(D), C.byref(cp), C.byref(co))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return outs


def dibr(img, p, want=("anaglyph", "left", "right")):
    """The whole pipeline for one image; returns a dict of the requested outputs."""
    img = _check_img(img)
    H, W, _ = img.shape
    outs, co = _alloc_outputs(H, W, want)
    cp = _cparams(p)
    rc = lib().or_dibr(_ptr(img), W, H, 3 * W, C.byref(cp), C.byref(co))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return outs


def dibr_rows(img, p, y0, y1, want=("anaglyph", "left", "right")):
    """Rows [y0, y1) of the whole pipeline (other rows of the outputs stay zero)."""
    img = _check_img(img)
    H, W, _ = img.shape
    outs, co = _alloc_outputs(H, W, want)
    cp = _cparams(p)
    rc = lib().or_dibr_rows(_ptr(img), W, H, 3 * W, C.byref(cp), C.byref(co), y0, y1)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return outs


def alloc_outputs(H, W, want):
    """Zeroed output arrays of the oracle's layout, for dibr_rows_into."""
    return _alloc_outputs(H, W, want)[0]


def dibr_rows_into(img, p, y0, y1, outs):
    """Rows [y0, y1) of the whole pipeline written into the given full-size output arrays
    (from alloc_outputs); disjoint row ranges may be computed by concurrent threads."""
    img = _check_img(img)
    H, W, _ = img.shape
    co = _Outputs(*[_ptr(outs.get(n)) for n in OUTPUT_NAMES], 3 * W, W)
    cp = _cparams(p)
    rc = lib().or_dibr_rows(_ptr(img), W, H, 3 * W, C.byref(cp), C.byref(co), y0, y1)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return outs


def dibr_parallel(img, p, want=("anaglyph", "left", "right"), threads=None, band=64):
    """The whole pipeline for one image computed band by band on several host threads
    (the oracle's row-band entry point; every band is computed exactly as in dibr)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    img = _check_img(img)
    H, W, _ = img.shape
    outs = alloc_outputs(H, W, want)
    n = threads or max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=n) as ex:
        list(ex.map(lambda y: dibr_rows_into(img, p, y, min(H, y + band), outs), range(0, H, band)))
    return outs


def inpaint2d(view, damaged, block=32, block_h=None):
    """The iterative 2-D block inpainting (Fig. 3) of one view; returns (result, pixels
    left damaged)."""
    view = _check_img(view)
    H, W, _ = view.shape
    dmg = np.ascontiguousarray(damaged != 0, dtype=np.uint8)
    assert dmg.shape == (H, W)
    out = np.empty_like(view)
    left = lib().or_inpaint2d(_ptr(view), W, H, 3 * W, _ptr(dmg), W, block,
                              block if block_h is None else block_h, _ptr(out), 3 * W)
    if left < 0:
        raise ValueError("oracle rejected the arguments")
    return out, int(left)
