"""Parity of the holes map and of the 2-D block inpainting fill (Fig. 3, left column) with
the CPU oracle, through the C-ABI, byte for byte."""
import numpy as np
import pytest

from paper_2009_09501_gb300 import dibr as D
from paper_2009_09501_gb300 import scenes

pytestmark = pytest.mark.gpu

RGB = ("anaglyph", "left", "right", "hsbs")


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    return T


@pytest.fixture(scope="module")
def ctx(torch):
    c = D.Context(device=0)
    yield c
    c.close()


def _alloc(torch, H, W, want, device):
    mk = (lambda s: torch.zeros(s, dtype=torch.uint8, device="cuda")) if device else (lambda s: np.zeros(s, np.uint8))
    return {n: mk((H, W) if n in D.MAP_OUTPUTS else (H, W, 3)) for n in want}


def run(ctx, torch, img, want, device=True, **kw):
    H, W, _ = img.shape
    p = D.make_params(max_parallax=kw.get("P", 16), depth_rule=kw.get("depth_rule", 1),
                      disparity_rule=kw.get("rule", 0), warp_mode=kw.get("warp_mode", 0), outputs=want,
                      hole_fill=kw.get("fill", 0), inpaint_block=kw.get("block", 32))
    outs = _alloc(torch, H, W, want, device)
    src = torch.from_numpy(np.ascontiguousarray(img)).cuda() if device else np.ascontiguousarray(img)
    ctx.synthesize_image(src, p, outs)
    return {n: (v.cpu().numpy() if device else v) for n, v in outs.items()}


def ref(oracle, img, want, **kw):
    p = oracle.params(max_parallax=kw.get("P", 16), depth_rule=kw.get("depth_rule", 1),
                      disparity_rule=kw.get("rule", 0), warp_mode=kw.get("warp_mode", 0),
                      fill_mode=kw.get("fill", 0), inpaint_block=kw.get("block", 32))
    return oracle.dibr(img, p, want=want)


def same(got, exp, what):
    for n in exp:
        if not np.array_equal(got[n], exp[n]):
            d = np.argwhere(got[n] != exp[n])
            raise AssertionError("%s %s: %d bytes differ, first at %s" % (what, n, len(d), d[0].tolist()))


def scene(W, H, seed):
    return scenes.Scene(W, H, seed=seed, n_objects=8).frame(0)


@pytest.mark.parametrize("W,H", [(1, 1), (5, 3), (31, 17), (64, 64), (97, 61), (330, 71), (1920, 36)])
@pytest.mark.parametrize("fill", [0, 1])
def test_holes_map(ctx, torch, oracle, W, H, fill):
    img = scene(W, H, W + H)
    want = ("holes", "depth", "anaglyph")
    for P in (0, 16, 90):
        kw = dict(P=P, fill=fill, block=8)
        same(run(ctx, torch, img, want, **kw), ref(oracle, img, want, **kw), "P=%d" % P)


@pytest.mark.parametrize("W,H,block", [(2, 2, 32), (30, 22, 4), (64, 48, 32), (98, 61, 8), (250, 77, 16),
                                       (640, 97, 32), (1282, 33, 2), (512, 40, 30)])
def test_inpaint2d_all_outputs(ctx, torch, oracle, W, H, block):
    img = scene(W, H, 7 * W + H)
    want = RGB + ("holes",)
    for P in (8, 48, 200):
        for rule in (0, 1):
            kw = dict(P=P, rule=rule, fill=1, block=block)
            same(run(ctx, torch, img, want, **kw), ref(oracle, img, want, **kw), "P=%d rule=%d" % (P, rule))


@pytest.mark.parametrize("block", [1, 3, 7, 31])
def test_inpaint2d_odd_blocks_without_hsbs(ctx, torch, oracle, block):
    img = scene(97, 53, block)
    want = ("anaglyph", "left", "right")
    kw = dict(P=40, fill=1, block=block)
    same(run(ctx, torch, img, want, **kw), ref(oracle, img, want, **kw), "block=%d" % block)


def test_inpaint2d_single_output_and_host_buffers(ctx, torch, oracle):
    img = scene(334, 120, 5)
    for want in (("anaglyph",), ("right",), ("hsbs",), ("depth",), ("holes",)):
        kw = dict(P=64, fill=1, block=16)
        exp = ref(oracle, img, want, **kw)
        same(run(ctx, torch, img, want, device=False, **kw), exp, "host %s" % (want,))
        same(run(ctx, torch, img, want, device=True, **kw), exp, "device %s" % (want,))


def test_inpaint2d_gather_mode_has_no_holes(ctx, torch, oracle):
    img = scene(200, 50, 9)
    want = ("anaglyph", "holes")
    kw = dict(P=32, fill=1, warp_mode=1)
    got = run(ctx, torch, img, want, **kw)
    same(got, ref(oracle, img, want, **kw), "gather")
    assert not got["holes"].any()


def test_inpaint2d_4k(ctx, torch, oracle):
    img = scenes.config_scene(2)
    want = ("anaglyph", "left", "right", "holes")
    kw = dict(P=64, fill=1, block=32)
    got = run(ctx, torch, img, want, **kw)
    exp = ref(oracle, img, want, **kw)
    same(got, exp, "4K")
    # the 2-D fill did repair something at this size
    row = ref(oracle, img, ("left",), P=64)
    assert not np.array_equal(row["left"], exp["left"])


def test_inpaint2d_back_to_back_frames(ctx, torch, oracle):
    # asynchronous 2-D fill frames on the context's own stream: a frame whose buffers are
    # disjoint from the previous frame's may start its band kernel while the previous
    # frame's inpainting runs; a frame reading the previous frame's output may not.  The
    # views and the holes map of frames that do not request them go to context scratch.
    H, W, P = 300, 640, 48
    imgs = [scenes.Scene(W, H, seed=700 + k, n_objects=15).frame(0) for k in range(4)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    kinds = [("anaglyph",), ("anaglyph", "left", "right", "holes")]
    outs = [_alloc(torch, H, W, kinds[k % 2], True) for k in range(4)]
    chained = _alloc(torch, H, W, ("anaglyph",), True)
    ps = [D.make_params(max_parallax=P, depth_rule=1, outputs=kinds[k % 2], hole_fill=1, inpaint_block=32)
          for k in range(4)]
    torch.cuda.synchronize()
    lib = D.load()
    for rep in range(3):
        for k in range(4):
            assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k]), ps[k], D.outputs_struct(outs[k])) == 0
        # reads the anaglyph the last frame wrote
        assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(outs[3]["anaglyph"]), ps[0],
                                      D.outputs_struct(chained)) == 0
    ctx.synchronize()
    for k in range(4):
        exp = ref(oracle, imgs[k], kinds[k % 2], P=P, fill=1, block=32)
        same({n: v.cpu().numpy() for n, v in outs[k].items()}, exp, "frame %d" % k)
    exp3 = ref(oracle, imgs[3], ("anaglyph",), P=P, fill=1, block=32)["anaglyph"]
    exp_c = ref(oracle, exp3, ("anaglyph",), P=P, fill=1, block=32)
    same({"anaglyph": chained["anaglyph"].cpu().numpy()}, exp_c, "chained")


def test_inpaint2d_is_refused_where_it_does_not_run(ctx, torch):
    img = torch.zeros((16, 32, 3), dtype=torch.uint8, device="cuda")
    outs = {"anaglyph": torch.zeros_like(img)}
    p = D.make_params(outputs=("anaglyph",), hole_fill=1, inpaint_block=8)
    with pytest.raises(D.DibrError):
        ctx.synthesize_batch([img], [p], [outs])
    with pytest.raises(D.DibrError):
        ctx.open_stream(32, 16, p)
