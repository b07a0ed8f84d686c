"""dibr_synthesize_batch_static: batched synthesis without any allocation (GPU).

Some callers may not allocate memory when they call into the library -- an application
that reserves all of its device memory at start-up and forbids allocation afterwards, or
code running under another framework's memory manager.  For them the library keeps the
batched launch's small scratch (work counter, per-image descriptors, work units) in a
fixed array of its own device data, and this entry point needs no context at all.

This test calls it through the C-ABI, twice in a row on the same buffers, and checks both
results byte for byte against the context-based dibr_synthesize_batch.  The file is named
to be collected last, so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2009_09501_gb300 import dibr as D
from paper_2009_09501_gb300 import scenes

pytestmark = pytest.mark.gpu

# sizes with 16-byte input rows (3 * width a multiple of 16), as the entry point requires
SPECS = [
    ((640, 480), dict(max_parallax=16), ("anaglyph", "left", "right", "hsbs", "depth")),
    ((1280, 720), dict(max_parallax=32, depth_rule=0), ("anaglyph", "depth")),
    ((96, 64), dict(max_parallax=12, warp_mode=1), ("left", "right")),
    ((1920, 1080), dict(max_parallax=48, disparity_rule=1), ("anaglyph",)),
    ((32, 16), dict(max_parallax=64), ("anaglyph", "left")),
]


def _params(kw, want):
    return D.make_params(depth_rule=kw.get("depth_rule", 1), disparity_rule=kw.get("disparity_rule", 0),
                         warp_mode=kw.get("warp_mode", 0), max_parallax=kw["max_parallax"], outputs=want)


def test_static_batch_matches_context_batch_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    ins, ref_outs, st_outs, prms = [], [], [], []
    for j, ((W, H), kw, want) in enumerate(SPECS):
        img = scenes.Scene(W, H, seed=1200 + j, n_objects=10).frame(0)
        t = torch.from_numpy(img).cuda()
        ins.append(t)
        mk = lambda: {n: torch.zeros((H, W) if n == "depth" else (H, W, 3), dtype=torch.uint8, device="cuda")
                      for n in want}
        ref_outs.append(mk())
        st_outs.append(mk())
        prms.append(_params(kw, want))

    # the existing, context-based batched entry point
    with D.Context(device=0) as ctx:
        ctx.synthesize_batch(ins, prms, ref_outs)

    n = len(SPECS)
    imgs_c = (D.dibr_image * n)(*[D.image_struct(t) for t in ins])
    prms_c = (D.dibr_params * n)(*prms)
    outs_c = (D.dibr_outputs * n)(*[D.outputs_struct(o) for o in st_outs])
    stream = torch.cuda.Stream()
    for call in range(2):
        for o in st_outs:  # the second call must write every output again
            for v in o.values():
                v.fill_(7)
        torch.cuda.synchronize()
        st = D.dibr_synthesize_batch_static(n, imgs_c, prms_c, n, outs_c, C.c_void_p(stream.cuda_stream))
        assert st == D.DIBR_OK, (call, D.STATUS_NAMES.get(st, st))
        for j in range(n):
            for name, v in st_outs[j].items():
                got, ref = v.cpu().numpy(), ref_outs[j][name].cpu().numpy()
                assert np.array_equal(got, ref), (call, j, name, int((got != ref).sum()))


def test_static_batch_equals_oracle(oracle):
    # the same images, checked against the CPU oracle directly
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    imgs, ins, outs, prms = [], [], [], []
    for j, ((W, H), kw, want) in enumerate(SPECS):
        img = scenes.Scene(W, H, seed=1200 + j, n_objects=10).frame(0)
        imgs.append(img)
        ins.append(torch.from_numpy(img).cuda())
        outs.append({n: torch.zeros((H, W) if n == "depth" else (H, W, 3), dtype=torch.uint8, device="cuda")
                     for n in want})
        prms.append(_params(kw, want))
    n = len(SPECS)
    imgs_c = (D.dibr_image * n)(*[D.image_struct(t) for t in ins])
    prms_c = (D.dibr_params * n)(*prms)
    outs_c = (D.dibr_outputs * n)(*[D.outputs_struct(o) for o in outs])
    torch.cuda.synchronize()
    assert D.dibr_synthesize_batch_static(n, imgs_c, prms_c, n, outs_c, None) == D.DIBR_OK
    for j, ((W, H), kw, want) in enumerate(SPECS):
        p = oracle.params(depth_rule=kw.get("depth_rule", 1), disparity_rule=kw.get("disparity_rule", 0),
                          warp_mode=kw.get("warp_mode", 0), max_parallax=kw["max_parallax"])
        ref = oracle.dibr(imgs[j], p, want=want)
        for name in want:
            got = outs[j][name].cpu().numpy()
            assert np.array_equal(got, ref[name]), (j, name, int((got != ref[name]).sum()))


def test_static_batch_unit_limit_and_widest_block(oracle):
    # 60 frames of 7680 x 4320 (the widest block: 480 threads per CTA) and 4 of 1280 x 720:
    # at the automatic rows per unit the list would hold 60 * 135 + 4 * 240 = 9,060 units,
    # more than the 8,192 the scratch array holds, so the rows per unit double until it fits
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    pool = scenes.batch_pool()
    big, small = pool[(7680, 4320)], pool[(1280, 720)]
    tb, ts = torch.from_numpy(big).cuda(), torch.from_numpy(small).cuda()
    ins = [tb] * 60 + [ts] * 4
    prms = [_params(dict(max_parallax=scenes.batch_parallax(t.shape[1])), ("anaglyph",)) for t in ins]
    outs = [{"anaglyph": torch.full_like(t, 3)} for t in ins]
    n = len(ins)
    imgs_c = (D.dibr_image * n)(*[D.image_struct(t) for t in ins])
    prms_c = (D.dibr_params * n)(*prms)
    outs_c = (D.dibr_outputs * n)(*[D.outputs_struct(o) for o in outs])
    torch.cuda.synchronize()
    assert D.dibr_synthesize_batch_static(n, imgs_c, prms_c, n, outs_c, None) == D.DIBR_OK
    # the context-based batch on two of the same entries, byte for byte, and the oracle
    with D.Context(device=0) as ctx:
        ref_outs = [{"anaglyph": torch.zeros_like(ins[j])} for j in (0, 63)]
        ctx.synthesize_batch([ins[0], ins[63]], [prms[0], prms[63]], ref_outs)
    for j, r in zip((0, 63), ref_outs):
        assert torch.equal(outs[j]["anaglyph"], r["anaglyph"]), j
    refs = {w: oracle.dibr_parallel(img, oracle.params(max_parallax=scenes.batch_parallax(w)), want=("anaglyph",))["anaglyph"]
            for w, img in ((7680, big), (1280, small))}
    for j, o in enumerate(outs):
        got = o["anaglyph"].cpu().numpy()
        assert np.array_equal(got, refs[got.shape[1]]), (j, int((got != refs[got.shape[1]]).sum()))


def test_static_batch_rejects_what_it_cannot_do_without_allocating():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    t = torch.zeros((16, 32, 3), dtype=torch.uint8, device="cuda")
    o = {"anaglyph": torch.zeros_like(t)}
    img = D.image_struct(t)
    out = D.outputs_struct(o)
    ok = _params(dict(max_parallax=8), ("anaglyph",))
    xbf = D.make_params(depth_rule=D.DIBR_DEPTH_LUMA_XBF, outputs=("anaglyph",))
    one = lambda i, p: D.dibr_synthesize_batch_static(1, C.byref(i), C.byref(p), 1, C.byref(out), None)
    assert one(img, ok) == D.DIBR_OK
    assert one(img, xbf) == D.DIBR_E_INVALID  # the cross-bilateral depth needs a buffer
    odd = D.dibr_image(t.data_ptr(), 31, 16, 96, 1)  # 3 * 31 bytes: not whole 16-byte rows
    assert one(odd, ok) == D.DIBR_E_INVALID
    many = (D.dibr_image * 65)(*([img] * 65))
    outs = (D.dibr_outputs * 65)(*([out] * 65))
    assert D.dibr_synthesize_batch_static(65, many, C.byref(ok), 1, outs, None) == D.DIBR_E_INVALID
