"""Failure reporting and recovery (GPU), without faulting or hanging the GPU.

- An allocation failure is made on the host: the context's allocator hook returns NULL.
  The call reports DIBR_E_NOMEM and the same context then succeeds.
- A bounded device-side wait is made to give up by setting the wait limit to 1 ns.  Waits
  that would have succeeded a few microseconds later then give up, the launch unwinds
  after its own copies in flight have landed, and the call reports DIBR_E_TIMEOUT.  With
  the default limit restored, the same context -- and a served stream -- succeed again.
- The same through the instances that keep the vertical filter's state in tensor memory
  (a band launch in tall bands, a persistent batched launch): the unwinding releases the
  tensor memory, and the context then produces exact frames.
- A slow consumer: frames submitted while nobody polls complete and wait in the
  completion queue; submissions beyond a stream's slots and queue are refused with
  DIBR_E_BUSY, never dropped.
"""
import time

import numpy as np
import pytest

from paper_2009_09501_gb300 import dibr as D
from paper_2009_09501_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    return T


def _frame(W, H, seed):
    return scenes.Scene(W, H, seed=seed, n_objects=12).frame(0)


def test_allocation_failure_reports_nomem_and_context_recovers(torch, oracle):
    allow = {"on": True, "calls": 0}

    def alloc(n):
        allow["calls"] += 1
        return torch.cuda.caching_allocator_alloc(n) if allow["on"] else 0

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    img = _frame(800, 600, 31)
    p = D.make_params(max_parallax=24, outputs=("anaglyph", "left"))
    ref = oracle.dibr(img, oracle.params(max_parallax=24), want=("anaglyph", "left"))
    with D.Context(device=0, alloc=alloc, free=free) as ctx:
        assert allow["calls"] >= 1  # the context's own status word came from the hook
        allow["on"] = False
        outs = {n: np.zeros_like(img) for n in ("anaglyph", "left")}
        with pytest.raises(D.DibrError) as e:
            ctx.synthesize_image(img, p, outs)  # host buffers: the staging buffers are new
        assert e.value.status == D.DIBR_E_NOMEM
        allow["on"] = True
        ctx.synthesize_image(img, p, outs)
        for n in outs:
            assert np.array_equal(outs[n], ref[n]), n


def test_wait_limit_reports_timeout_and_context_recovers(torch, oracle):
    # a 4K frame: every CTA waits many times (for its input rows, for the other warps),
    # so with a 1 ns limit some wait is never already complete when first tested
    img = scenes.config_scene(2)
    H, W = img.shape[:2]
    p = D.make_params(max_parallax=64, outputs=("anaglyph",))
    ref = oracle.dibr_parallel(img, oracle.params(max_parallax=64), want=("anaglyph",))
    t = torch.from_numpy(img).cuda()
    with D.Context(device=0) as ctx:
        for attempt in range(2):  # single image, then a batch, each failing then recovering
            ctx.set_wait_limit(1)
            out = {"anaglyph": torch.zeros_like(t)}
            with pytest.raises(D.DibrError) as e:
                if attempt == 0:
                    ctx.synthesize_image(t, p, out)
                else:
                    ctx.synthesize_batch([t, t], [p, p], [out, {"anaglyph": torch.zeros_like(t)}])
            assert e.value.status == D.DIBR_E_TIMEOUT
            ctx.set_wait_limit(0)
            out = {"anaglyph": torch.zeros_like(t)}
            if attempt == 0:
                ctx.synthesize_image(t, p, out)
            else:
                ctx.synthesize_batch([t], [p], [out])
            assert np.array_equal(out["anaglyph"].cpu().numpy(), ref["anaglyph"]), attempt


def _wait_completions(ctx, n, timeout_s=60):
    got, t0 = [], time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        got += ctx.poll(64, 100000)
    return got


def test_served_stream_recovers_after_a_reported_timeout(torch, oracle):
    img = scenes.config_scene(2)
    H, W = img.shape[:2]
    p = D.make_params(max_parallax=64, outputs=("anaglyph",))
    ref = oracle.dibr_parallel(img, oracle.params(max_parallax=64), want=("anaglyph",))
    with D.Context(device=0) as ctx:
        sid = ctx.open_stream(W, H, p)
        ctx.set_wait_limit(1)
        out = {"anaglyph": np.zeros_like(img)}
        assert ctx.submit_frame(sid, 1, img, out) == D.DIBR_OK
        (c,) = _wait_completions(ctx, 1)
        assert c.seq == 1 and c.status == D.DIBR_E_TIMEOUT
        ctx.set_wait_limit(0)
        outs = [{"anaglyph": np.zeros_like(img)} for _ in range(3)]
        for k, o in enumerate(outs):
            assert ctx.submit_frame(sid, 2 + k, img, o) == D.DIBR_OK
        comps = _wait_completions(ctx, 3)
        assert sorted(c.seq for c in comps) == [2, 3, 4]
        assert all(c.status == D.DIBR_OK for c in comps)  # the failure did not stick
        for o in outs:
            assert np.array_equal(o["anaglyph"], ref["anaglyph"])
        ctx.close_stream(sid)


def test_slow_consumer_frames_wait_in_the_completion_queue(torch, oracle):
    imgs = [_frame(640, 480, 40 + k) for k in range(2)]
    p = D.make_params(max_parallax=16, outputs=("anaglyph",))
    refs = [oracle.dibr(im, oracle.params(max_parallax=16), want=("anaglyph",))["anaglyph"] for im in imgs]
    with D.Context(device=0) as ctx:
        sids = [ctx.open_stream(640, 480, p) for _ in imgs]
        accepted, refused, outs = [], 0, {}
        for seq in range(60):  # far more than a stream's 3 slots + 16 queued frames at once
            k = seq % 2
            o = {"anaglyph": np.zeros_like(imgs[k])}
            st = ctx.submit_frame(sids[k], seq, imgs[k], o)
            if st == D.DIBR_OK:
                accepted.append(seq)
                outs[seq] = (k, o)
            else:
                assert st == D.DIBR_E_BUSY, st
                refused += 1
        time.sleep(1.0)  # nobody polls meanwhile
        comps = _wait_completions(ctx, len(accepted))
        assert sorted(c.seq for c in comps) == sorted(accepted)
        assert all(c.status == D.DIBR_OK for c in comps)
        for seq, (k, o) in outs.items():
            assert np.array_equal(o["anaglyph"], refs[k]), seq
        assert ctx.poll(8, 1000) == []  # nothing else completes
        for s in sids:
            ctx.close_stream(s)


def test_wait_limit_in_the_tensor_memory_instances(torch, oracle):
    # the fixed-set instances that keep the vertical filter's state in tensor memory: a band
    # launch in 14-row bands (one CTA per SM) and a persistent batched launch of 1080p frames;
    # a wait that gives up must unwind through the release of the tensor memory, and the
    # context must produce exact frames afterwards
    img4k = scenes.config_scene(2)
    p4k = D.make_params(max_parallax=64, outputs=("anaglyph",))
    ref4k = oracle.dibr_parallel(img4k, oracle.params(max_parallax=64), want=("anaglyph",))
    hd = [_frame(1920, 1080, 50 + k) for k in range(6)]
    phd = D.make_params(max_parallax=48, outputs=("anaglyph",))
    refhd = [oracle.dibr_parallel(im, oracle.params(max_parallax=48), want=("anaglyph",))["anaglyph"] for im in hd]
    t4k = torch.from_numpy(img4k).cuda()
    thd = [torch.from_numpy(im).cuda() for im in hd]
    with D.Context(device=0) as ctx:
        # one CTA per SM: 14-row bands for the 4K frame; 16-row work units: the 1080p frames
        # share the persistent batched launch instead of launches of their own
        ctx.set_tuning(ctas_per_sm=1, rows_per_unit=16)
        for attempt in range(2):
            ctx.set_wait_limit(1)
            with pytest.raises(D.DibrError) as e:
                ctx.synthesize_image(t4k, p4k, {"anaglyph": torch.zeros_like(t4k)})
            assert e.value.status == D.DIBR_E_TIMEOUT
            with pytest.raises(D.DibrError) as e:
                ctx.synthesize_batch(thd, [phd] * len(thd), [{"anaglyph": torch.zeros_like(t)} for t in thd])
            assert e.value.status == D.DIBR_E_TIMEOUT
            ctx.set_wait_limit(0)
            out = {"anaglyph": torch.zeros_like(t4k)}
            ctx.synthesize_image(t4k, p4k, out)
            assert np.array_equal(out["anaglyph"].cpu().numpy(), ref4k["anaglyph"]), attempt
            outs = [{"anaglyph": torch.zeros_like(t)} for t in thd]
            ctx.synthesize_batch(thd, [phd] * len(thd), outs)
            for k, o in enumerate(outs):
                assert np.array_equal(o["anaglyph"].cpu().numpy(), refhd[k]), (attempt, k)
