"""Batched launches and the serving loop against the CPU oracle (GPU).

A batch of images of any sizes must give, image by image, exactly the oracle's output
(and so exactly the single-image path's).  Frames served on concurrent streams must give
exactly what each frame gives alone.
"""
import ctypes as C
import time

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


@pytest.fixture()
def ctx(torch):
    c = D.Context(device=0)
    yield c
    c.close()


def gparams(kw, outputs):
    return D.make_params(depth_rule=kw.get("depth_rule", 1), disparity_rule=kw.get("disparity_rule", 0),
                         warp_mode=kw.get("warp_mode", 0), max_parallax=kw.get("max_parallax", 16),
                         threshold=kw.get("threshold", 150), outputs=outputs)


def oparams(O, kw):
    return O.params(depth_rule=kw.get("depth_rule", 1), disparity_rule=kw.get("disparity_rule", 0),
                    warp_mode=kw.get("warp_mode", 0), max_parallax=kw.get("max_parallax", 16),
                    threshold=kw.get("threshold", 150))


def check(got, ref, what):
    for n in ref:
        g = got[n].cpu().numpy() if hasattr(got[n], "cpu") else got[n]
        if not np.array_equal(g, ref[n]):
            bad = np.argwhere(g != ref[n])
            raise AssertionError("%s %s: %d bytes differ, first %s" % (what, n, len(bad), bad[0].tolist()))


CASES = [
    ((64, 48), dict(max_parallax=8), ALL),
    ((333, 41), dict(max_parallax=40, depth_rule=0), ("anaglyph", "left", "right", "depth")),   # odd width
    ((1280, 720), dict(max_parallax=32), ("anaglyph",)),
    ((50, 30), dict(max_parallax=6, warp_mode=1), ALL),
    ((1920, 1080), dict(max_parallax=48, disparity_rule=1), ("left", "right")),
    ((17, 9), dict(max_parallax=64), ("anaglyph", "left", "right", "depth")),                   # W < P
    ((2560, 1440), dict(max_parallax=64, depth_rule=2), ("anaglyph", "depth")),
    ((640, 480), dict(max_parallax=16, threshold=60), ALL),
]


def make_case(torch, j, size, kw, want, device=True):
    W, H = size
    img = scenes.Scene(W, H, seed=500 + j, n_objects=10).frame(0)
    if device:
        i = torch.from_numpy(img).cuda()
        outs = {n: torch.zeros((H, W) if n == "depth" else (H, W, 3), dtype=torch.uint8, device="cuda") for n in want}
    else:
        i = img
        outs = {n: np.zeros((H, W) if n == "depth" else (H, W, 3), np.uint8) for n in want}
    return img, i, outs


@pytest.mark.parametrize("device", [True, False])
def test_batch_mixed_sizes_rules_outputs(ctx, torch, oracle, device):
    imgs, ins, outs, prms = [], [], [], []
    for j, (size, kw, want) in enumerate(CASES):
        img, i, o = make_case(torch, j, size, kw, want, device)
        imgs.append(img); ins.append(i); outs.append(o); prms.append(gparams(kw, want))
    ctx.synthesize_batch(ins, prms, outs)
    for j, (size, kw, want) in enumerate(CASES):
        ref = oracle.dibr(imgs[j], oparams(oracle, kw), want=want)
        if kw.get("depth_rule") == 2:
            got_d = outs[j]["depth"].cpu().numpy() if device else outs[j]["depth"]
            refd = ref["depth"]
            diff = np.abs(got_d.astype(int) - refd.astype(int))
            assert diff.max() <= 1 and (diff > 0).mean() <= 1e-4
            back = oracle.from_depth(imgs[j], got_d, oparams(oracle, kw), want=("anaglyph",))
            check({"anaglyph": outs[j]["anaglyph"]}, back, "xbf image %d" % j)
        else:
            check(outs[j], ref, "image %d %s" % (j, size))


@pytest.mark.parametrize("tuning", [dict(rows_per_unit=1), dict(rows_per_unit=7, ring_slots=4),
                                    dict(rows_per_unit=64, ctas_per_sm=1, ring_slots=8)])
def test_batch_tuning_does_not_change_results(ctx, torch, oracle, tuning):
    ctx.set_tuning(**tuning)
    sizes = [(1920, 1080), (96, 70), (1280, 720), (400, 31)]
    imgs, ins, outs = [], [], []
    for j, (W, H) in enumerate(sizes):
        img = scenes.Scene(W, H, seed=700 + j, n_objects=12).frame(0)
        imgs.append(img)
        ins.append(torch.from_numpy(img).cuda())
        outs.append({"anaglyph": torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")})
    ctx.synthesize_batch(ins, gparams(dict(max_parallax=30), ("anaglyph",)), outs)
    for j in range(len(sizes)):
        ref = oracle.dibr(imgs[j], oparams(oracle, dict(max_parallax=30)), want=("anaglyph",))
        check(outs[j], ref, "tuned batch image %d" % j)


def test_batch_workload4_classes_sampled_rows(ctx, torch, oracle):
    # one image of each size class of the batched workload (720p .. 8K), P = 2.5% of W,
    # checked on sampled rows (first, last, band edges, random)
    imgs, ins, outs, prms = [], [], [], []
    for j, (W, H) in enumerate(scenes.BATCH_CLASSES):
        img = scenes.Scene(W, H, seed=900 + j, n_objects=40).frame(0)
        imgs.append(img)
        ins.append(torch.from_numpy(img).cuda())
        outs.append({"anaglyph": torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")})
        prms.append(gparams(dict(max_parallax=scenes.batch_parallax(W)), ("anaglyph",)))
    ctx.enqueue_batch(ins, prms, outs)
    ctx.synchronize()
    rng = np.random.default_rng(4)
    for j, (W, H) in enumerate(scenes.BATCH_CLASSES):
        got = outs[j]["anaglyph"].cpu().numpy()
        rows = sorted(set([0, 1, H - 1, H - 2, 31, 32, 33] + rng.integers(0, H, 6).tolist()))
        p = oparams(oracle, dict(max_parallax=scenes.batch_parallax(W)))
        for y in rows:
            ref = oracle.dibr_rows(imgs[j], p, y, y + 1, want=("anaglyph",))["anaglyph"][y]
            assert np.array_equal(got[y], ref), (W, H, y)


def test_tuning_api_validates(ctx):
    t = ctx.get_tuning()
    assert t == dict(ring_slots=0, ctas_per_sm=0, load_mode=0, l2_prefetch=0, rows_per_unit=0, host_bands=0,
                     frames_in_flight=0)
    for bad in [dict(load_mode=6), dict(ring_slots=9), dict(ring_slots=1), dict(l2_prefetch=3), dict(rows_per_unit=-1),
                dict(host_bands=9), dict(host_bands=-1), dict(frames_in_flight=17), dict(frames_in_flight=-1)]:
        with pytest.raises(D.DibrError):
            ctx.set_tuning(**bad)


@pytest.mark.parametrize("load_mode", [1, 2, 3, 4, 5])
def test_load_modes_give_same_results(ctx, torch, oracle, load_mode):
    ctx.set_tuning(load_mode=load_mode, l2_prefetch=1 + (load_mode % 2))
    for (W, H) in [(3840, 64), (1000, 20), (1280, 40)]:
        img = scenes.Scene(W, H, seed=W, n_objects=8).frame(0)
        t = torch.from_numpy(img).cuda()
        o = {"anaglyph": torch.zeros_like(t), "left": torch.zeros_like(t)}
        ctx.synthesize_image(t, gparams(dict(max_parallax=64), ("anaglyph", "left")), o)
        check(o, oracle.dibr(img, oparams(oracle, dict(max_parallax=64)), want=("anaglyph", "left")), "mode %d" % load_mode)


# ------------------------------------------------------------------------- serving
def serve_all(ctx, frames, timeout_s=60.0):
    """Submit (sid, seq, img, outs) tuples in order; return completions by (sid, seq)."""
    got = {}
    pending = list(frames)
    deadline = time.time() + timeout_s
    while (pending or len(got) < len(frames)) and time.time() < deadline:
        while pending:
            sid, seq, img, outs = pending[0]
            st = ctx.submit_frame(sid, seq, img, outs)
            if st == D.DIBR_E_BUSY:
                break
            assert st == D.DIBR_OK, st
            pending.pop(0)
        for c in ctx.poll(64, 2000):
            got[(c.stream_id, c.seq)] = c
    return got


def test_serving_mixed_streams_equal_alone(ctx, torch, oracle):
    specs = [((320, 180), dict(max_parallax=16), ("anaglyph", "left")),
             ((640, 360), dict(max_parallax=24, depth_rule=0), ("right", "depth")),
             ((200, 150), dict(max_parallax=12, warp_mode=1), ("anaglyph", "hsbs"))]
    sids, frames, refs = [], [], {}
    for k, (size, kw, want) in enumerate(specs):
        sids.append(ctx.open_stream(size[0], size[1], gparams(kw, want)))
    scs = [scenes.stream_scene(k, s[0][0], s[0][1]) for k, s in enumerate(specs)]
    for f in range(6):
        for k, (size, kw, want) in enumerate(specs):
            W, H = size
            img = scs[k].frame(f)
            outs = {n: np.zeros((H, W) if n == "depth" else (H, W, 3), np.uint8) for n in want}
            frames.append((sids[k], f, img, outs))
            refs[(sids[k], f)] = (oracle.dibr(img, oparams(oracle, kw), want=want), outs)
    got = serve_all(ctx, frames)
    assert len(got) == len(frames)
    for key, c in got.items():
        assert c.status == D.DIBR_OK and c.t_done_ns >= c.t_submit_ns
        ref, outs = refs[key]
        check(outs, ref, "served frame %s" % (key,))
    for s in sids:
        ctx.close_stream(s)


def test_serving_admission_close_and_poll(torch):
    p = gparams({}, ("anaglyph",))
    per_stream = 3 * 2 * (640 * 3) * 480  # 3 slots x (input + anaglyph)
    with D.Context(device=0, mem_budget_bytes=int(per_stream * 1.5), max_streams=2) as c:
        a = c.open_stream(640, 480, p)
        with pytest.raises(D.DibrError) as e:
            c.open_stream(640, 480, p)  # over the memory budget
        assert e.value.status == D.DIBR_E_BUSY
        b = c.open_stream(64, 48, p)
        with pytest.raises(D.DibrError) as e:
            c.open_stream(32, 32, p)  # over the stream limit
        assert e.value.status == D.DIBR_E_BUSY
        assert c.poll(8, 1000) == []  # nothing submitted: not ready
        img = np.zeros((48, 64, 3), np.uint8)
        out = {"anaglyph": np.zeros_like(img)}
        assert c.submit_frame(b, 7, img, out) == D.DIBR_OK
        c.close_stream(b)  # closes with a frame in flight: it still completes
        assert c.submit_frame(b, 8, img, out) == D.DIBR_E_CLOSED
        comps = []
        t0 = time.time()
        while not comps and time.time() - t0 < 30:
            comps = c.poll(8, 100000)
        assert len(comps) == 1 and comps[0].seq == 7 and comps[0].status == D.DIBR_OK
        wrong = np.zeros((10, 10, 3), np.uint8)
        assert c.submit_frame(a, 1, wrong, {"anaglyph": np.zeros_like(wrong)}) == D.DIBR_E_INVALID
        c.close_stream(a)
        c.open_stream(640, 480, p)  # budget freed by the close


def test_video_workload3_frames_streamed(ctx, torch, oracle):
    # 4K moving scene streamed from pinned host memory, anaglyph, P = 64
    sc = scenes.Scene(3840, 2160, 2009_09501 + 3, 40, "gauss8", moving=True)
    p = gparams(dict(max_parallax=64), ("anaglyph",))
    sid = ctx.open_stream(3840, 2160, p)
    frames, refs = [], {}
    for f in range(3):
        img = torch.from_numpy(sc.frame(f)).pin_memory()
        out = torch.zeros((2160, 3840, 3), dtype=torch.uint8).pin_memory()
        frames.append((sid, f, img.numpy(), {"anaglyph": out.numpy()}))
        refs[f] = (oracle.dibr(img.numpy(), oparams(oracle, dict(max_parallax=64)), want=("anaglyph",)), out)
    got = serve_all(ctx, frames)
    assert len(got) == 3
    for f in range(3):
        check({"anaglyph": refs[f][1].numpy()}, refs[f][0], "video frame %d" % f)
    ctx.close_stream(sid)


def test_serving_workload5_streams_sample(ctx, torch, oracle):
    # 4 x 1080p + 4 x 4K streams, two frames each, results equal to the oracle's
    p = gparams(dict(max_parallax=64), ("anaglyph",))
    sizes = [(1920, 1080)] * 4 + [(3840, 2160)] * 4
    sids = [ctx.open_stream(W, H, p) for (W, H) in sizes]
    frames, refs = [], {}
    for f in range(2):
        for k, (W, H) in enumerate(sizes):
            img = scenes.stream_scene(k, W, H).frame(f)
            out = np.zeros((H, W, 3), np.uint8)
            frames.append((sids[k], f, img, {"anaglyph": out}))
            refs[(sids[k], f)] = (img, out)
    got = serve_all(ctx, frames, timeout_s=120)
    assert len(got) == len(frames)
    rng = np.random.default_rng(5)
    po = oparams(oracle, dict(max_parallax=64))
    for (sid, f), (img, out) in refs.items():
        H = img.shape[0]
        for y in sorted(set([0, H - 1] + rng.integers(0, H, 4).tolist())):
            ref = oracle.dibr_rows(img, po, y, y + 1, want=("anaglyph",))["anaglyph"][y]
            assert np.array_equal(out[y], ref), (sid, f, y)
    for s in sids:
        ctx.close_stream(s)


# ------------------------------------------------------------------------- autotuner
def test_autotuned_batches_equal_the_oracle_and_persist(torch, oracle, tmp_path):
    sizes = [(1920, 1080), (1920, 1080), (1280, 720), (3840, 2160), (333, 97), (1280, 720)]
    imgs, ins, prms = [], [], []
    for j, (W, H) in enumerate(sizes):
        img = scenes.Scene(W, H, seed=1500 + j, n_objects=16).frame(0)
        imgs.append(img)
        ins.append(torch.from_numpy(img).cuda())
        prms.append(gparams(dict(max_parallax=scenes.batch_parallax(W)), ("anaglyph", "left")))
    refs = [oracle.dibr_parallel(imgs[j], oparams(oracle, dict(max_parallax=scenes.batch_parallax(W))),
                                 want=("anaglyph", "left")) for j, (W, H) in enumerate(sizes)]
    mk = lambda: [{n: torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda") for n in ("anaglyph", "left")}
                  for (W, H) in sizes]
    path = str(tmp_path / "tuning.json")
    with D.Context(device=0) as c:
        outs = mk()
        plans = c.autotune_batch(ins, prms, outs, reps=1)
        classes = sorted({D.block_threads(W) for (W, H) in sizes})
        assert sorted(p["block_threads"] for p in plans) == classes
        for j in range(len(sizes)):  # the tuner's own runs leave the final results
            check(outs[j], refs[j], "tuner run image %d" % j)
        outs = mk()
        c.synthesize_batch(ins, prms, outs)
        for j in range(len(sizes)):
            check(outs[j], refs[j], "tuned batch image %d" % j)
        c.save_tuning(path)
    with D.Context(device=0) as c2:
        c2.load_tuning(path)
        outs = mk()
        c2.synthesize_batch(ins, prms, outs)
        for j in range(len(sizes)):
            check(outs[j], refs[j], "reloaded tuning image %d" % j)
        bad = tmp_path / "bad.json"
        bad.write_text('{"batch_classes": [{"block_threads": 33, "rows_per_unit": 1, "ctas_per_sm": 0, '
                       '"ring_slots": 0, "own_launch": 0}]}')
        with pytest.raises(D.DibrError):
            c2.load_tuning(str(bad))
