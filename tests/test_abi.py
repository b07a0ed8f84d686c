"""The C-ABI library without a GPU: it builds, loads, exports every declared entry point,
and its host-side logic (argument checks, Fig. 3 shift tables) is right."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2009_09501_gb300 import dibr as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    """Names of the functions include/dibr.h declares."""
    with open(os.path.join(ROOT, "include", "dibr.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dibr_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = D.load()
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(D.SYMBOLS)


def test_params_default_and_validation():
    p = D.dibr_params()
    assert D.dibr_params_default(p) == D.DIBR_OK
    assert (p.depth_rule, p.disparity_rule, p.warp_mode, p.threshold) == (1, 0, 0, 150)
    assert D.dibr_validate(p) == D.DIBR_OK
    img = D.dibr_image(1, 640, 480, 1920, 1)
    assert D.dibr_validate(p, img) == D.DIBR_OK
    bad = [("depth_rule", 3), ("disparity_rule", 2), ("warp_mode", 2), ("max_parallax_px", -1),
           ("max_parallax_px", 1025), ("threshold", 256), ("outputs", 0), ("outputs", 64),
           ("hole_fill", 2), ("hole_fill", -1)]
    for field, val in bad:
        q = D.dibr_params()
        D.dibr_params_default(q)
        setattr(q, field, val)
        assert D.dibr_validate(q) == D.DIBR_E_INVALID, field
    q = D.make_params(warp_mode=D.DIBR_WARP_GATHER_FIG3, disparity_rule=D.DIBR_DISP_LINEAR)
    assert D.dibr_validate(q) == D.DIBR_E_INVALID
    q = D.make_params(depth_rule=D.DIBR_DEPTH_LUMA_XBF, xbf_radius=9)
    assert D.dibr_validate(q) == D.DIBR_E_INVALID
    q = D.make_params(depth_rule=D.DIBR_DEPTH_LUMA_XBF, xbf_sigma_r=0.0)
    assert D.dibr_validate(q) == D.DIBR_E_INVALID
    for w, h, pitch in [(0, 4, 0), (4, 0, 12), (4, 4, 11), (16385, 1, 50000)]:
        assert D.dibr_validate(p, D.dibr_image(1, w, h, pitch, 1)) == D.DIBR_E_INVALID
    assert D.dibr_validate(p, D.dibr_image(None, 4, 4, 12, 1)) == D.DIBR_E_INVALID
    hs = D.make_params(outputs=("hsbs",))
    assert D.dibr_validate(hs, D.dibr_image(1, 5, 4, 15, 1)) == D.DIBR_E_INVALID
    assert D.dibr_validate(hs, D.dibr_image(1, 6, 4, 18, 1)) == D.DIBR_OK
    # the 2-D fill: block side 1..32, even with HSBS; the holes map is a valid output
    assert (p.hole_fill, p.inpaint_block) == (D.DIBR_FILL_ROW, 32)
    for blk, ok in ((0, False), (1, True), (32, True), (33, False)):
        q = D.make_params(hole_fill=D.DIBR_FILL_INPAINT2D, inpaint_block=blk)
        assert (D.dibr_validate(q) == D.DIBR_OK) == ok, blk
    assert D.dibr_validate(D.make_params(hole_fill=1, inpaint_block=7, outputs=("hsbs",))) == D.DIBR_E_INVALID
    assert D.dibr_validate(D.make_params(hole_fill=1, inpaint_block=8, outputs=("hsbs",))) == D.DIBR_OK
    assert D.dibr_validate(D.make_params(inpaint_block=0, outputs=("holes",))) == D.DIBR_OK  # unused with the row fill


@pytest.mark.parametrize("rule", [0, 1])
def test_shift_tables_match_oracle(oracle, rule):
    for P in [0, 1, 2, 3, 15, 16, 17, 64, 191, 192, 1024]:
        for T in [0, 150, 255]:
            p = D.make_params(disparity_rule=rule, max_parallax=P, threshold=T)
            hL = (C.c_int16 * 256)()
            hR = (C.c_int16 * 256)()
            assert D.dibr_shift_tables(p, hL, hR) == D.DIBR_OK
            oL, oR = oracle.disparity_lut(rule, P, T)
            assert np.array_equal(np.array(hL[:]), oL) and np.array_equal(np.array(hR[:]), oR), (P, T)


def test_create_fails_cleanly_without_sm103():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    st = D.dibr_create(None, ctx)
    assert st in (D.DIBR_E_CUDA, D.DIBR_E_INVALID)
    assert not ctx.value
    with pytest.raises(D.DibrError):
        D.Context()
