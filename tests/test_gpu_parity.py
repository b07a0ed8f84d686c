"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, element by element.

Integer pipelines (luminance / binomial smoothing, any shift rule, forward or Fig. 3
gather warp) must be bit-exact.  The cross-bilateral rule is FP32 on the GPU and FP64 in
the oracle: its depth may differ by 1 on at most 0.01 % of pixels, and everything after
the depth is bit-exact when the oracle is fed the GPU's depth.
"""
import numpy as np
import pytest

from paper_2009_09501_gb300 import dibr as D
from paper_2009_09501_gb300 import scenes

pytestmark = pytest.mark.gpu

ALL = ("anaglyph", "left", "right", "hsbs", "depth")


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


def oracle_params(O, **kw):
    m = dict(max_parallax=kw.get("max_parallax", 16), depth_rule=kw.get("depth_rule", 1),
             disparity_rule=kw.get("disparity_rule", 0), warp_mode=kw.get("warp_mode", 0),
             threshold=kw.get("threshold", 150), xbf_radius=kw.get("xbf_radius", 2),
             xbf_sigma_s=kw.get("xbf_sigma_s", 1.5), xbf_sigma_r=kw.get("xbf_sigma_r", 16.0))
    return O.params(**m)


def gpu_params(outputs, **kw):
    return D.make_params(depth_rule=kw.get("depth_rule", 1), disparity_rule=kw.get("disparity_rule", 0),
                         warp_mode=kw.get("warp_mode", 0), max_parallax=kw.get("max_parallax", 16),
                         threshold=kw.get("threshold", 150), xbf_sigma_s=kw.get("xbf_sigma_s", 1.5),
                         xbf_sigma_r=kw.get("xbf_sigma_r", 16.0), xbf_radius=kw.get("xbf_radius", 2),
                         outputs=outputs)


def run_host(ctx, img, outputs, **kw):
    H, W, _ = img.shape
    outs = {n: np.zeros((H, W) if n == "depth" else (H, W, 3), np.uint8) for n in outputs}
    ctx.synthesize_image(np.ascontiguousarray(img), gpu_params(outputs, **kw), outs)
    return outs


def run_device(ctx, torch, img, outputs, **kw):
    H, W, _ = img.shape
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    outs = {n: torch.zeros((H, W) if n == "depth" else (H, W, 3), dtype=torch.uint8, device="cuda")
            for n in outputs}
    ctx.synthesize_image(t, gpu_params(outputs, **kw), outs)
    return {n: v.cpu().numpy() for n, v in outs.items()}


def assert_same(got, ref, what=""):
    for n in ref:
        g, r = got[n], ref[n]
        if not np.array_equal(g, r):
            diff = np.argwhere(g != r)
            raise AssertionError("%s %s: %d differing bytes, first at %s (gpu %s, oracle %s)" % (
                what, n, len(diff), diff[0].tolist(), g[tuple(diff[0])], r[tuple(diff[0])]))


def test_workload1_640x480_anaglyph(ctx, torch, oracle):
    img = scenes.config_scene(1)
    ref = oracle.dibr(img, oracle_params(oracle, max_parallax=16), want=("anaglyph",))
    assert_same(run_host(ctx, img, ("anaglyph",), max_parallax=16), ref, "host")
    assert_same(run_device(ctx, torch, img, ("anaglyph",), max_parallax=16), ref, "device")


def test_workload2_4k_stereo_pair_and_anaglyph(ctx, torch, oracle):
    img = scenes.config_scene(2)
    want = ("anaglyph", "left", "right")
    ref = oracle.dibr(img, oracle_params(oracle, max_parallax=64), want=want)
    assert_same(run_device(ctx, torch, img, want, max_parallax=64), ref, "4K")


def test_workload2_4k_as_the_benchmark_times_it(ctx, torch, oracle):
    # the launch configuration the benchmark times: frames back to back on the context's own
    # stream (consecutive frames overlapping), four rotating input/output sets; every set's
    # final outputs against the oracle
    want = ("anaglyph", "left", "right")
    imgs = [scenes.config_scene(2)] + [scenes.Scene(3840, 2160, seed=900 + k, n_objects=40).frame(0) for k in range(3)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [{n: torch.zeros((2160, 3840, 3), dtype=torch.uint8, device="cuda") for n in want} for _ in imgs]
    p = gpu_params(want, max_parallax=64)
    torch.cuda.synchronize()
    lib = D.load()
    for k in range(12):
        assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k % 4]), p, D.outputs_struct(outs[k % 4])) == 0
    ctx.synchronize()
    for k in range(4):
        ref = oracle.dibr(imgs[k], oracle_params(oracle, max_parallax=64), want=want)
        assert_same({n: v.cpu().numpy() for n, v in outs[k].items()}, ref, "4K set %d" % k)


SIZES = [(1, 1), (2, 1), (1, 5), (7, 3), (16, 16), (17, 9), (33, 20), (48, 7), (100, 37),
         (250, 50), (1000, 13), (3000, 7), (7680, 6)]


@pytest.mark.parametrize("W,H", SIZES)
def test_sizes_all_outputs(ctx, torch, oracle, W, H):
    rng = np.random.default_rng(W * 1000 + H)
    img = scenes.Scene(W, H, seed=W + 7 * H, n_objects=6, texture="uniform32").frame(0)
    img = img ^ rng.integers(0, 2, size=img.shape, dtype=np.uint8)  # break flat areas a little
    want = ALL if W % 2 == 0 else ("anaglyph", "left", "right", "depth")
    for P in (0, 1, 16, 64, 300):
        for rule in (0, 1):
            ref = oracle.dibr(img, oracle_params(oracle, max_parallax=P, disparity_rule=rule), want=want)
            got = run_device(ctx, torch, img, want, max_parallax=P, disparity_rule=rule)
            assert_same(got, ref, "W=%d H=%d P=%d rule=%d" % (W, H, P, rule))


@pytest.mark.parametrize("depth_rule", [0, 1])
def test_depth_rules_and_thresholds(ctx, torch, oracle, depth_rule):
    img = scenes.Scene(333, 41, seed=5, n_objects=10).frame(0)
    for T in (0, 100, 150, 255):
        kw = dict(max_parallax=40, depth_rule=depth_rule, threshold=T)
        ref = oracle.dibr(img, oracle_params(oracle, **kw), want=ALL[:3] + ("depth",))
        assert_same(run_device(ctx, torch, img, ALL[:3] + ("depth",), **kw), ref, "T=%d" % T)


@pytest.mark.parametrize("P", [0, 1, 7, 16, 64, 255])
def test_gather_fig3_mode(ctx, torch, oracle, P):
    img = scenes.Scene(222, 19, seed=11, n_objects=8).frame(0)
    kw = dict(max_parallax=P, warp_mode=1)
    ref = oracle.dibr(img, oracle_params(oracle, **kw), want=ALL)
    assert_same(run_device(ctx, torch, img, ALL, **kw), ref, "gather P=%d" % P)


def test_zero_parallax_is_identity(ctx, torch):
    img = scenes.Scene(160, 90, seed=3).frame(0)
    got = run_device(ctx, torch, img, ("left", "right", "anaglyph"), max_parallax=0)
    for n in got:
        assert np.array_equal(got[n], img), n


def test_strided_and_misaligned_buffers(ctx, torch, oracle):
    H, W, P = 37, 101, 24
    img = scenes.Scene(W, H, seed=21).frame(0)
    ref = oracle.dibr(img, oracle_params(oracle, max_parallax=P), want=("anaglyph", "left", "depth"))
    p = gpu_params(("anaglyph", "left", "depth"), max_parallax=P)
    # input: row pitch 3W+13 and a base 1 byte past an allocation boundary
    big = torch.zeros(H * (3 * W + 13) + 1, dtype=torch.uint8, device="cuda")
    view = big[1:1 + H * (3 * W + 13)].view(H, 3 * W + 13)
    view[:, :3 * W] = torch.from_numpy(img.reshape(H, 3 * W)).cuda()
    # outputs: pitches 3W+5 and W+3, bases offset by 3 bytes
    ob = torch.zeros(H * (3 * W + 5) + 3, dtype=torch.uint8, device="cuda")
    lb = torch.zeros(H * (3 * W + 5) + 3, dtype=torch.uint8, device="cuda")
    db = torch.zeros(H * (W + 3) + 3, dtype=torch.uint8, device="cuda")
    img_s = D.dibr_image(view.data_ptr(), W, H, 3 * W + 13, 1)
    out_s = D.dibr_outputs()
    out_s.anaglyph, out_s.left, out_s.depth = ob.data_ptr() + 3, lb.data_ptr() + 3, db.data_ptr() + 3
    out_s.pitch, out_s.depth_pitch, out_s.on_device = 3 * W + 5, W + 3, 1
    ctx.check(D.dibr_synthesize_image(ctx.handle, img_s, p, out_s))
    rows = lambda buf, pitch, n: buf[3:3 + H * pitch].view(H, pitch)[:, :n].cpu().numpy()
    assert np.array_equal(rows(ob, 3 * W + 5, 3 * W).reshape(H, W, 3), ref["anaglyph"])
    assert np.array_equal(rows(lb, 3 * W + 5, 3 * W).reshape(H, W, 3), ref["left"])
    assert np.array_equal(rows(db, W + 3, W), ref["depth"])


def test_enqueue_then_synchronize_matches_blocking(ctx, torch):
    img = scenes.Scene(640, 360, seed=8).frame(0)
    want = ("anaglyph", "hsbs")
    a = run_device(ctx, torch, img, want, max_parallax=20)
    t = torch.from_numpy(img).cuda()
    outs = {n: torch.zeros((360, 640, 3), dtype=torch.uint8, device="cuda") for n in want}
    for _ in range(3):
        ctx.enqueue_image(t, gpu_params(want, max_parallax=20), outs)
    ctx.synchronize()
    for n in want:
        assert np.array_equal(outs[n].cpu().numpy(), a[n])


def test_xbf_depth_tolerance_and_exact_back_half(ctx, torch, oracle):
    img = scenes.config_scene(1)
    H, W, _ = img.shape
    kw = dict(max_parallax=16, depth_rule=2)
    got = run_device(ctx, torch, img, ALL, **kw)
    refD = oracle.depth(img, oracle_params(oracle, **kw))
    diff = np.abs(got["depth"].astype(int) - refD.astype(int))
    assert diff.max() <= 1
    assert (diff > 0).mean() <= 1e-4, (diff > 0).mean()
    # the integer back half, fed the GPU's own depth, is bit-exact
    back = oracle.from_depth(img, got["depth"], oracle_params(oracle, **kw), want=ALL[:4])
    assert_same({k: got[k] for k in ALL[:4]}, back, "xbf back half")


def test_xbf_4k_depth_tolerance(ctx, torch, oracle):
    img = scenes.config_scene(2)
    kw = dict(max_parallax=64, depth_rule=2)
    got = run_device(ctx, torch, img, ("depth",), **kw)["depth"]
    refD = oracle.depth(img, oracle_params(oracle, **kw))
    diff = np.abs(got.astype(int) - refD.astype(int))
    assert diff.max() <= 1
    assert (diff > 0).mean() <= 1e-4, (diff > 0).mean()


@pytest.mark.parametrize("radius,ss,sr", [(1, 0.8, 8.0), (2, 1.5, 16.0), (3, 2.0, 24.0), (5, 3.0, 30.0),
                                          (8, 4.0, 50.0)])
def test_xbf_parameters(ctx, torch, oracle, radius, ss, sr):
    img = scenes.Scene(300, 120, seed=31, texture="gauss8").frame(0)
    kw = dict(max_parallax=16, depth_rule=2, xbf_radius=radius, xbf_sigma_s=ss, xbf_sigma_r=sr)
    got = run_device(ctx, torch, img, ("depth", "left"), **kw)
    refD = oracle.depth(img, oracle_params(oracle, **kw))
    diff = np.abs(got["depth"].astype(int) - refD.astype(int))
    assert diff.max() <= 1 and (diff > 0).mean() <= 1e-4


def test_invalid_arguments_report_cleanly(ctx, torch):
    img = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    p = gpu_params(("anaglyph",))
    o = D.dibr_outputs()  # anaglyph pointer NULL
    o.pitch, o.on_device = 24, 1
    st = D.dibr_synthesize_image(ctx.handle, D.image_struct(img), p, o)
    assert st == D.DIBR_E_INVALID and "NULL" in D.dibr_last_error(ctx.handle)
    bad = D.dibr_image(img.data_ptr(), 8, 8, 23, 1)
    st = D.dibr_synthesize_image(ctx.handle, bad, p, D.outputs_struct({"anaglyph": img}))
    assert st == D.DIBR_E_INVALID
    # the context stays usable
    ctx.synthesize_image(img, p, {"anaglyph": torch.zeros_like(img)})


def test_batch_equals_single(ctx, torch):
    imgs, outs, singles = [], [], []
    for j, (W, H) in enumerate([(64, 48), (1280, 720), (50, 30), (1920, 1080)]):
        img = scenes.Scene(W, H, seed=40 + j).frame(0)
        P = scenes.batch_parallax(W) if W >= 1280 else 8
        singles.append(run_device(ctx, torch, img, ("anaglyph",), max_parallax=P)["anaglyph"])
        imgs.append(torch.from_numpy(img).cuda())
        outs.append({"anaglyph": torch.zeros_like(imgs[-1])})
    params = [gpu_params(("anaglyph",), max_parallax=(scenes.batch_parallax(t.shape[1]) if t.shape[1] >= 1280 else 8))
              for t in imgs]
    ctx.synthesize_batch(imgs, params, outs)
    for o, s in zip(outs, singles):
        assert np.array_equal(o["anaglyph"].cpu().numpy(), s)


def test_page_locked_host_outputs(ctx, torch, oracle):
    # outputs in page-locked host memory, both fills
    img = scenes.Scene(640, 360, seed=77, n_objects=10).frame(0)
    H, W, _ = img.shape
    want = ("anaglyph", "left", "right", "hsbs", "depth", "holes")
    outs = {n: torch.zeros((H, W) if n in D.MAP_OUTPUTS else (H, W, 3), dtype=torch.uint8).pin_memory()
            for n in want}
    for fill in (0, 1):
        p = D.make_params(max_parallax=24, outputs=want, hole_fill=fill, inpaint_block=16)
        for v in outs.values():
            v.fill_(3)
        ctx.synthesize_image(np.ascontiguousarray(img), p, {n: v.numpy() for n, v in outs.items()})
        ref = oracle.dibr(img, oracle.params(max_parallax=24, fill_mode=fill, inpaint_block=16), want=want)
        assert_same({n: v.numpy() for n, v in outs.items()}, ref, "pinned host fill=%d" % fill)


@pytest.mark.parametrize("W,H,P", [(1920, 1080, 48), (3840, 2160, 64), (1001, 2049, 24), (640, 512, 200)])
def test_host_buffers_row_bands(ctx, torch, oracle, W, H, P):
    # blocking calls with host input and outputs run as overlapping row bands
    img = scenes.Scene(W, H, seed=W + H, n_objects=20).frame(0)
    want = ("anaglyph", "left", "right", "depth", "holes") + (("hsbs",) if W % 2 == 0 else ())
    outs = {n: np.zeros((H, W) if n in D.MAP_OUTPUTS else (H, W, 3), np.uint8) for n in want}
    ctx.synthesize_image(np.ascontiguousarray(img), D.make_params(max_parallax=P, outputs=want), outs)
    ref = oracle.dibr(img, oracle.params(max_parallax=P), want=want)
    assert_same(outs, ref, "banded %dx%d" % (W, H))


@pytest.mark.parametrize("bands", [1, 2, 3, 5, 8])
def test_host_buffers_band_counts(ctx, torch, oracle, bands):
    # every band count of the blocking host-buffer path, down to bands of one or two rows
    # (the 2-row halos then span two bands)
    for W, H in [(333, 9), (640, 37)]:
        img = scenes.Scene(W, H, seed=W + bands, n_objects=8).frame(0)
        want = ("anaglyph", "left", "right", "depth")
        outs = {n: np.zeros((H, W) if n in D.MAP_OUTPUTS else (H, W, 3), np.uint8) for n in want}
        ctx.set_tuning(host_bands=bands)
        try:
            ctx.synthesize_image(np.ascontiguousarray(img), D.make_params(max_parallax=24, outputs=want), outs)
        finally:
            ctx.set_tuning(host_bands=0)
        ref = oracle.dibr(img, oracle.params(max_parallax=24), want=want)
        assert_same(outs, ref, "%d bands %dx%d" % (bands, W, H))


def test_xbf_back_to_back_frames(ctx, torch):
    # cross-bilateral frames on the context's own stream: a frame's cross-bilateral launch
    # may start beside the previous frame's band launch when their buffers are disjoint (the
    # depth scratch alternates between two halves); a frame reading the previous frame's
    # output may not.  Each frame must equal the same frame computed alone (the kernels are
    # deterministic).
    H, W, P = 360, 640, 32
    imgs = [scenes.Scene(W, H, seed=800 + k, n_objects=15).frame(0) for k in range(4)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    want = ("anaglyph", "left", "depth")
    p = gpu_params(want, max_parallax=P, depth_rule=2)
    pc = gpu_params(("anaglyph",), max_parallax=P, depth_rule=2)

    def alloc(names):
        return {n: torch.zeros((H, W) if n in D.MAP_OUTPUTS else (H, W, 3), dtype=torch.uint8, device="cuda")
                for n in names}

    alone = []
    for k in range(4):
        o = alloc(want)
        ctx.synthesize_image(ins[k], p, o)
        alone.append({n: v.cpu().numpy() for n, v in o.items()})
    outs = [alloc(want) for _ in range(4)]
    chained = alloc(("anaglyph",))
    torch.cuda.synchronize()
    lib = D.load()
    for rep in range(3):
        for k in range(4):
            assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k]), p, D.outputs_struct(outs[k])) == 0
        # reads the left view frame 3 just wrote
        assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(outs[3]["left"]), pc, D.outputs_struct(chained)) == 0
    ctx.synchronize()
    for k in range(4):
        assert_same({n: v.cpu().numpy() for n, v in outs[k].items()}, alone[k], "frame %d" % k)
    c_alone = alloc(("anaglyph",))
    ctx.synthesize_image(outs[3]["left"], pc, c_alone)
    assert_same({"anaglyph": chained["anaglyph"].cpu().numpy()}, {"anaglyph": c_alone["anaglyph"].cpu().numpy()},
                "chained frame")


def test_mixed_mode_frames_back_to_back(ctx, torch):
    # row-fill, 2-D fill and cross-bilateral frames interleaved on the context's own stream:
    # each launch may start beside the previous frame's last one only when their buffers are
    # disjoint, whatever mode either frame had; every frame must equal the same frame computed
    # alone (the kernels are deterministic), also one that reads the previous frame's output
    H, W, P = 200, 480, 24
    imgs = [scenes.Scene(W, H, seed=950 + k, n_objects=12).frame(0) for k in range(6)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    want = ("anaglyph", "left")
    modes = [dict(), dict(hole_fill=1), dict(depth_rule=2), dict(hole_fill=1), dict(), dict(depth_rule=2)]
    ps = [D.make_params(max_parallax=P, depth_rule=m.get("depth_rule", 1), outputs=want,
                        hole_fill=m.get("hole_fill", 0), inpaint_block=16) for m in modes]

    def alloc():
        return {n: torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda") for n in want}

    alone = []
    for k in range(6):
        o = alloc()
        ctx.synthesize_image(ins[k], ps[k], o)
        alone.append({n: v.cpu().numpy() for n, v in o.items()})
    outs = [alloc() for _ in range(6)]
    chained = alloc()
    torch.cuda.synchronize()
    lib = D.load()
    for rep in range(3):
        for k in range(6):
            assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k]), ps[k], D.outputs_struct(outs[k])) == 0
        # a cross-bilateral frame reading the left view the last frame wrote
        assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(outs[5]["left"]), ps[2], D.outputs_struct(chained)) == 0
    ctx.synchronize()
    for k in range(6):
        assert_same({n: v.cpu().numpy() for n, v in outs[k].items()}, alone[k], "frame %d (%s)" % (k, modes[k]))
    c_alone = alloc()
    ctx.synthesize_image(outs[5]["left"], ps[2], c_alone)
    assert_same({n: v.cpu().numpy() for n, v in chained.items()}, {n: v.cpu().numpy() for n, v in c_alone.items()},
                "chained frame")


def test_back_to_back_frames_overlap_only_when_independent(ctx, torch, oracle):
    # consecutive asynchronous frames on the context's own stream: disjoint buffers may
    # overlap on the GPU, a frame reading the previous frame's output must not
    H, W, P = 720, 1280, 32
    imgs = [scenes.Scene(W, H, seed=500 + k, n_objects=15).frame(0) for k in range(4)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [{"anaglyph": torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda"),
             "left": torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")} for _ in imgs]
    chained = {"anaglyph": torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")}
    p = gpu_params(("anaglyph", "left"), max_parallax=P)
    pc = gpu_params(("anaglyph",), max_parallax=P)
    torch.cuda.synchronize()
    lib = D.load()
    for rep in range(3):
        for k in range(4):
            assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k]), p, D.outputs_struct(outs[k])) == 0
        # reads the left view frame 3 just wrote
        assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(outs[3]["left"]), pc, D.outputs_struct(chained)) == 0
    ctx.synchronize()
    for k in range(4):
        ref = oracle.dibr(imgs[k], oracle_params(oracle, max_parallax=P), want=("anaglyph", "left"))
        assert_same({n: v.cpu().numpy() for n, v in outs[k].items()}, ref, "frame %d" % k)
    ref2 = oracle.dibr(outs[3]["left"].cpu().numpy(), oracle_params(oracle, max_parallax=P), want=("anaglyph",))
    assert_same({"anaglyph": chained["anaglyph"].cpu().numpy()}, ref2, "chained frame")


@pytest.mark.parametrize("fif", [0, 3])
def test_4k_frames_side_by_side(ctx, torch, oracle, fif):
    # a dozen independent 4K frames enqueued back to back: from the second on, each is
    # enqueued behind queued work and runs beside its neighbours in a share of the SM
    # slots (taller row bands); every frame keeps its own outputs
    imgs = [scenes.config_scene(2), scenes.config_scene(3)]
    H, W = imgs[0].shape[:2]
    prm = oracle_params(oracle, max_parallax=64)
    refs = [oracle.dibr_parallel(im, prm, want=("anaglyph", "left", "right")) for im in imgs]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [{n: torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda") for n in ("anaglyph", "left", "right")}
            for _ in range(12)]
    p = gpu_params(("anaglyph", "left", "right"), max_parallax=64)
    ctx.set_tuning(frames_in_flight=fif)
    try:
        torch.cuda.synchronize()
        lib = D.load()
        for k in range(12):
            assert lib.dibr_enqueue_image(ctx.handle, D.image_struct(ins[k % 2]), p, D.outputs_struct(outs[k])) == 0
        ctx.synchronize()
    finally:
        ctx.set_tuning(frames_in_flight=0)
    for k in range(12):
        assert_same({n: v.cpu().numpy() for n, v in outs[k].items()}, refs[k % 2], "frame %d" % k)


@pytest.mark.parametrize("W,H", [(2000, 1300), (1008, 2000), (3840, 2160), (2048, 1216)])
@pytest.mark.parametrize("outputs", [("anaglyph", "left", "right"), ("anaglyph",)])
def test_fixed_set_instances_in_tall_bands(ctx, torch, oracle, W, H, outputs):
    # 16-byte aligned device rows (3W a multiple of 16) and one CTA per SM: bands of 8 or
    # more rows, so the stereo / anaglyph instances that keep the vertical filter's state in
    # tensor memory run (including rows whose last warp is partial)
    img = scenes.Scene(W, H, seed=700 + W + H, n_objects=25).frame(0)
    P = max(2, int(round(0.025 * W)))
    ref = oracle.dibr_parallel(img, oracle_params(oracle, max_parallax=P), want=outputs)
    ctx.set_tuning(ctas_per_sm=1)
    try:
        got = run_device(ctx, torch, img, outputs, max_parallax=P)
    finally:
        ctx.set_tuning(ctas_per_sm=0)
    assert_same(got, ref, "%dx%d" % (W, H))
