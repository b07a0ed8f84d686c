#!/usr/bin/env python
"""Benchmark of the fused DIBR pipeline on the 4K UHD still-image workload.

Workload: one 3840 x 2160 RGB uint8 frame (seeded synthetic scene, 40 objects, sigma-8
texture), maximum parallax 64 px, binomial depth smoothing, Fig. 3 shift rule, outputs
left + right views and the red-cyan anaglyph.  A step is one pass of the whole pipeline
over one frame: one launch of the fused kernel.  The steps are enqueued back to back on the
library's stream with rotating buffers, so consecutive frames run side by side (each on a
share of the SMs, in tall row bands); single launches on an idle GPU are timed apart.

Prints one JSON line (rank 0):
  value      frames/s over all ranks, inputs resident in HBM, CUDA events on the
             launching stream, rotating buffer sets larger than 2x L2;
  e2e        frames/s through the streaming entry points dibr_submit_frame / dibr_poll
             with pinned HOST input and outputs (every frame's H2D copy, kernels and D2H
             copies inside the timed region, three frames in flight), beside the blocking
             dibr_synthesize_image figure (blocking_call_value);
  roofline   the fused kernel's algorithmic bytes per launch / its mean launch time (the
             timed region's length / the launches in it) against the measured HBM copy
             bandwidth, with the DRAM bytes of one steady-state launch from the committed
             ncu summary;
  cpu_baseline  the CPU oracle on this host's cores (band-parallel over row bands), on a
             bounded sample of frames;
  clocks     SM clock samples taken by nvidia-smi during the timed region;
  config1, batch, inpaint2d, xbf, video, served
             the other workloads (640x480 anaglyph; 64 mixed 720p-8K images batched and one
             call per image; 4K with the 2-D block inpainting, and with the cross-bilateral
             depth, each with its bound; 4K video and 8 served streams through the serving
             loop, with latency percentiles); --quick leaves them out.
--impl reference times the CPU oracle alone on the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "4K stereo/anaglyph frames/s and HBM GB/s vs roofline; p50/p99 frame latency served"
UNIT = "frames/s"
W4K, H4K, P4K = 3840, 2160, 64
OUTPUTS = ("anaglyph", "left", "right")
ALG_BYTES = 3 * W4K * H4K * (1 + len(OUTPUTS))  # input once + each output once
CONFIG = {"workload": "4K UHD still: 3840x2160 RGB uint8, 40 objects, P=64, binomial depth, "
                      "Fig. 3 rule, outputs L+R+anaglyph",
          "width": W4K, "height": H4K, "max_parallax_px": P4K,
          "outputs": list(OUTPUTS), "depth_rule": "binom5", "disparity_rule": "paper",
          "warp_mode": "forward"}


def reduce_max(x, dist=None, device="cpu"):
    """Maximum of a float over all ranks (the value itself when running alone)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_per_rank, world, dist=None, device="cpu"):
    """Units processed by all ranks / the slowest rank's time (weak scaling)."""
    return world * units_per_rank / reduce_max(seconds_per_rank, dist, device)


BAND_SOURCES = ("dibr_band.cu", "dibr_internal.h", "dibr_ptx.cuh")
INPAINT_SOURCES = ("dibr_inpaint.cu", "dibr_internal.h", "dibr_ptx.cuh")
XBF_SOURCES = ("dibr_xbf.cu", "dibr_internal.h", "dibr_ptx.cuh")


def kernel_source_digest(files=BAND_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2009_09501_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_profile_value(name, key, files):
    """One figure ("- key: value" line) of a committed ncu summary under profiles/, or None
    when the kernel's sources changed since it was captured (the summary's
    kernel_source_digest)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernel_source_digest") != kernel_source_digest(files):
            return None, "stale (kernel changed since the capture)"
        return float(vals[key]), "ncu capture, profiles/" + name
    except Exception:
        return None, "no capture"


def load_traffic():
    """DRAM bytes per launch of the band kernel from the committed ncu summary."""
    return load_profile_value("band_kernel_4k_stereo.md", "dram_bytes_per_launch", BAND_SOURCES)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of one GPU every 20 ms, with host timestamps."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.samples = []
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.monotonic(), [v.strip() for v in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        note = "during timed region"
        if not inside:
            # timed region shorter than the sampling period: nearest samples around it
            near = sorted(self.samples, key=lambda ts: min(abs(ts[0] - t0), abs(ts[0] - t1)))[:3]
            inside = [s for _, s in near]
            note = "nearest samples (timed region shorter than the 20 ms sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = sorted(float(s[0]) for s in inside if s[0].replace(".", "").isdigit())
        smax = max((float(s[1]) for s in inside if s[1].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4)
                          if len(s) > 4 + i and s[4 + i].lower().startswith("active")})
        power = [float(s[2]) for s in inside if s[2].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(inside), "power_w_max": max(power) if power else None, "note": note}


def oracle_frames_per_s(img, seconds=12.0, max_frames=40, rows_per_task=None):
    """CPU oracle, band-parallel over all host cores (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    O.lib()
    H = img.shape[0]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    p = O.params(max_parallax=P4K)
    bands = max(cores, 1)
    step = rows_per_task or (H + bands - 1) // bands
    tasks = [(y, min(H, y + step)) for y in range(0, H, step)]
    with ThreadPoolExecutor(max_workers=cores) as ex:
        n = 0
        t0 = time.perf_counter()
        while True:
            list(ex.map(lambda yy: O.dibr_rows(img, p, yy[0], yy[1], want=OUTPUTS), tasks))
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds or n >= max_frames:
                break
    return n / el, cores, n, el


def oracle_single_core(img, seconds=6.0):
    from oracle import oracle as O
    p = O.params(max_parallax=P4K)
    n, t0 = 0, time.perf_counter()
    while True:
        O.dibr(img, p, want=OUTPUTS)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n / el, n, el


def run_reference(args):
    """The CPU oracle as the reference arm: K steps, each a bounded band of the frame."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    from paper_2009_09501_gb300 import scenes
    img = scenes.config_scene(2)
    O.lib()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    p = O.params(max_parallax=P4K)
    # calibrate: seconds per row with all cores busy
    rows = 16 * cores
    with ThreadPoolExecutor(max_workers=cores) as ex:
        def band(nrows):
            per = max(1, nrows // cores)
            tasks = [(y, min(nrows, y + per)) for y in range(0, nrows, per)]
            list(ex.map(lambda yy: O.dibr_rows(img, p, yy[0], yy[1], want=OUTPUTS), tasks))
        t0 = time.perf_counter()
        band(rows)
        per_row = (time.perf_counter() - t0) / rows
        budget = 90.0 / max(1, args.steps + args.warmup)
        nrows = int(max(cores, min(H4K, budget / max(per_row, 1e-9))))
        for _ in range(args.warmup):
            band(nrows)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            band(nrows)
        el = time.perf_counter() - t0
    value = args.steps * nrows / H4K / el
    sample = "%d of %d rows of the 4K frame per step, %d threads" % (nrows, H4K, cores)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def bench_config1(D, torch, ctx, stream, reps=2000):
    """Workload 1: one 640 x 480 frame (12 objects, uniform texture), P = 16, anaglyph.
    Small enough to stay in L2: bound by launch and per-row latency, reported in us and
    frames/s (back-to-back launches on the context's stream, four buffer sets)."""
    from paper_2009_09501_gb300 import scenes
    img = torch.from_numpy(scenes.config_scene(1)).cuda()
    sets = [(img.clone(), {"anaglyph": torch.empty_like(img)}) for _ in range(4)]
    p = D.make_params(max_parallax=16, outputs=("anaglyph",))
    torch.cuda.synchronize()
    # the C-ABI call with its argument structs built once (as the main workload's loop does):
    # at a few microseconds per frame, the binding's per-call marshalling would be the bound
    lib = D.load()
    keep = [(D.image_struct(i), D.outputs_struct(o)) for i, o in sets]
    args_c = [(D.C.byref(a), D.C.byref(b)) for a, b in keep]
    pref, h = D.C.byref(p), ctx.handle

    def step(k):
        a, b = args_c[k % 4]
        st = lib.dibr_enqueue_image(h, a, pref, b)
        if st != 0:
            raise D.DibrError(st, D.dibr_last_error(h))

    for k in range(20):
        step(k)
    ctx.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(reps):
        step(k)
    e1.record(stream)
    ctx.synchronize()
    us = e0.elapsed_time(e1) / reps * 1000.0
    single = []
    for k in range(50):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(k)
        b.record(stream)
        ctx.synchronize()
        single.append(a.elapsed_time(b) * 1000.0)
    return {"workload": "640x480 RGB uint8, 12 objects, uniform texture, P=16, anaglyph",
            "us_per_frame": us, "frames_per_s": 1e6 / us,
            "single_launch_us_p50": float(np.percentile(single, 50)), "launches": reps}


def _stream_frames(args):
    from paper_2009_09501_gb300 import scenes
    k, W, H, n = args
    sc = scenes.stream_scene(k, W, H)
    return [sc.frame(f) for f in range(n)]


def bench_batch(D, torch, ctx, stream, n=64):
    """Batched workload: n images drawn from the 720p..8K classes (P = 2.5 % of the width,
    anaglyph), one persistent launch vs one launch per image, frames/s on the device."""
    from paper_2009_09501_gb300 import scenes
    sizes = scenes.batch_sizes(n)
    pool = {wh: torch.from_numpy(img).cuda() for wh, img in scenes.batch_pool().items()}
    ins = [pool[wh] for wh in sizes]
    outs = [{"anaglyph": torch.empty_like(t)} for t in ins]
    prms = [D.make_params(max_parallax=scenes.batch_parallax(t.shape[1]), outputs=("anaglyph",)) for t in ins]
    pixels = sum(t.shape[0] * t.shape[1] for t in ins)
    torch.cuda.synchronize()

    def timed(fn, reps=5):
        fn()
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        ctx.synchronize()
        return e0.elapsed_time(e1) / reps / 1000.0

    # both arms through the C-ABI with their argument structs built once, so that neither
    # measures the binding's per-call marshalling
    lib = D.load()
    bargs = ctx._batch_args(ins, prms, outs)
    singles = [(D.image_struct(i), q, D.outputs_struct(o)) for i, q, o in zip(ins, prms, outs)]
    sargs = [(D.C.byref(a), D.C.byref(q), D.C.byref(b)) for a, q, b in singles]

    def batched(c):
        c.check(D.dibr_enqueue_batch(c.handle, *bargs))

    def per_image():
        for a, q, b in sargs:
            ctx.check(lib.dibr_enqueue_image(ctx.handle, a, q, b))

    t_batch = timed(lambda: batched(ctx))
    t_single = timed(per_image)
    # the library's autotuner on this batch, then the same batched call with its choices
    with D.Context(device=torch.cuda.current_device()) as tctx:
        plans = tctx.autotune_batch(ins, prms, outs, reps=2)
        tstream = torch.cuda.ExternalStream(D.dibr_stream(tctx.handle))

        def timed_t(fn, reps=5):
            fn()
            tctx.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(tstream)
            for _ in range(reps):
                fn()
            e1.record(tstream)
            tctx.synchronize()
            return e0.elapsed_time(e1) / reps / 1000.0

        t_tuned = timed_t(lambda: batched(tctx))
    return {"images": n, "megapixels": pixels / 1e6, "frames_per_s_batched": n / t_batch,
            "frames_per_s_batched_autotuned": n / t_tuned,
            "frames_per_s_per_image_launches": n / t_single, "speedup": t_single / t_batch,
            "speedup_autotuned": t_single / t_tuned,
            "gb_per_s_batched": pixels * 6 / t_batch / 1e9, "gb_per_s_batched_autotuned": pixels * 6 / t_tuned / 1e9,
            "autotuned_plans": plans, "sizes": "seeded mix of %s" % list(scenes.BATCH_CLASSES)}


def bench_inpaint(D, torch, ctx, stream, reps=200):
    """4K L + R + anaglyph, P = 64, with the 2-D block inpainting fill (Fig. 3, 32 x 32
    blocks) against the row fill on the same rotating buffer sets (more than 2x L2)."""
    from paper_2009_09501_gb300 import scenes
    img = torch.from_numpy(scenes.config_scene(2)).cuda()
    H, W = img.shape[:2]
    sets = []
    for _ in range(4):
        i = img.clone()
        sets.append((i, {n: torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for n in OUTPUTS}))
    torch.cuda.synchronize()
    res = {}
    # both arms with every band launch over all SMs (a frame with the 2-D fill never runs
    # beside the next one), so that the difference is the inpainting's own time
    fif = ctx.get_tuning()["frames_in_flight"]
    ctx.set_tuning(frames_in_flight=1)
    for name, fill in (("row_fill", D.DIBR_FILL_ROW), ("inpaint2d", D.DIBR_FILL_INPAINT2D)):
        p = D.make_params(max_parallax=P4K, outputs=OUTPUTS, hole_fill=fill, inpaint_block=32)
        for k in range(10):
            ctx.enqueue_image(sets[k % 4][0], p, sets[k % 4][1])
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            ctx.enqueue_image(sets[k % 4][0], p, sets[k % 4][1])
        e1.record(stream)
        ctx.synchronize()
        res[name] = e0.elapsed_time(e1) / reps * 1000.0
    ctx.set_tuning(frames_in_flight=fif)
    # Issue-slot bound: the inpainting is bound by the issue slots its step loop and visits
    # share (it moves 50 MB per frame: far from HBM).  Its warp instructions per 4K frame
    # (fixed for this workload and code) come from the committed ncu summary; the floor is
    # that count at every scheduler issuing one warp instruction per clock.
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    clock_hz = 2.07e9  # the maximum SM clock; the clocks sampled in the timed region bound it
    peak = 4 * props.multi_processor_count * clock_hz  # warp instructions per second
    insts, src = load_profile_value("inpaint_kernel_4k.md", "warp_instructions_per_launch", INPAINT_SOURCES)
    over = res["inpaint2d"] - res["row_fill"]
    roof = {"bound": "issue", "unit": "warp instructions/s", "peak": peak,
            "peak_source": "4 schedulers x SMs x 2.07 GHz (derived)", "instructions_per_frame": insts,
            "instructions_source": src,
            "floor_us": insts / peak * 1e6 if insts else None,
            "achieved": insts / (over * 1e-6) if insts and over > 0 else None,
            "frac": insts / (over * 1e-6) / peak if insts and over > 0 else None,
            "note": "kernel time taken as the frame time with the 2-D fill minus the frame time with the row fill"}
    return {"workload": "3840x2160, P=64, L+R+anaglyph, 2-D block inpainting (32x32 blocks) after the row fill",
            "frames_per_s": 1e6 / res["inpaint2d"], "us_per_frame": res["inpaint2d"],
            "row_fill_us_per_frame": res["row_fill"], "inpaint_overhead_us": over,
            "launches_per_frame": 3, "roofline": roof}


def bench_xbf(D, torch, ctx, stream, reps=200):
    """4K L + R + anaglyph, P = 64, with the cross-bilateral depth (radius 2, sigma_s 1.5,
    sigma_r 16) against the binomial depth on the same rotating buffer sets.  The
    cross-bilateral kernel is bound by the SMs' exp2 rate: 25 exp2 per interior pixel."""
    from paper_2009_09501_gb300 import scenes
    img = torch.from_numpy(scenes.config_scene(2)).cuda()
    H, W = img.shape[:2]
    sets = [(img.clone(), {n: torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for n in OUTPUTS})
            for _ in range(4)]
    torch.cuda.synchronize()
    res = {}
    # both arms with every band launch over all SMs (a frame whose band launch reads the
    # cross-bilateral depth never runs beside the next one)
    fif = ctx.get_tuning()["frames_in_flight"]
    ctx.set_tuning(frames_in_flight=1)
    for name, rule in (("binom5", D.DIBR_DEPTH_LUMA_BINOM5), ("xbf", D.DIBR_DEPTH_LUMA_XBF)):
        p = D.make_params(max_parallax=P4K, outputs=OUTPUTS, depth_rule=rule)
        for k in range(10):
            ctx.enqueue_image(sets[k % 4][0], p, sets[k % 4][1])
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            ctx.enqueue_image(sets[k % 4][0], p, sets[k % 4][1])
        e1.record(stream)
        ctx.synchronize()
        res[name] = e0.elapsed_time(e1) / reps * 1000.0
    ctx.set_tuning(frames_in_flight=fif)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    taps = sum(min(y + 2, H - 1) - max(y - 2, 0) + 1 for y in range(H)) * \
        sum(min(x + 2, W - 1) - max(x - 2, 0) + 1 for x in range(W))
    xbf_us = res["xbf"] - res["binom5"] + 0.0
    clock_hz = 2.07e9  # the maximum SM clock; the clocks sampled in the timed region bound it
    peak = 16 * props.multi_processor_count * clock_hz  # exp2 results per second (16 per SM per clock)
    # the bound that holds: instruction issue (warp instructions per 4K frame, fixed for this
    # workload and code, from the committed ncu summary; one per clock per scheduler)
    ipeak = 4 * props.multi_processor_count * clock_hz
    insts, isrc = load_profile_value("xbf_kernel_4k.md", "warp_instructions_per_launch", XBF_SOURCES)
    issue = {"bound": "issue", "unit": "warp instructions/s", "peak": ipeak,
             "peak_source": "4 schedulers x SMs x 2.07 GHz (derived)", "instructions_per_frame": insts,
             "instructions_source": isrc,
             "thread_instructions_per_tap": insts * 32 / taps if insts else None,
             "floor_us": insts / ipeak * 1e6 if insts else None,
             "achieved": insts / (xbf_us * 1e-6) if insts and xbf_us > 0 else None,
             "frac": insts / (xbf_us * 1e-6) / ipeak if insts and xbf_us > 0 else None}
    return {"workload": "3840x2160, P=64, L+R+anaglyph, cross-bilateral depth r=2",
            "frames_per_s": 1e6 / res["xbf"], "us_per_frame": res["xbf"],
            "binom5_us_per_frame": res["binom5"], "xbf_kernel_us_est": xbf_us,
            "roofline": {"bound": "alu", "unit": "exp2/s", "exp2_per_frame": taps,
                         "achieved": taps / (xbf_us * 1e-6) if xbf_us > 0 else None, "peak": peak,
                         "frac": taps / (xbf_us * 1e-6) / peak if xbf_us > 0 else None,
                         "peak_source": "16 exp2/clock/SM x SMs x 2.07 GHz (derived)",
                         "note": "kernel time estimated as the frame time with this depth rule minus the binomial one"},
            "issue_roofline": issue}


def bench_video(D, torch, ctx, frames=300):
    """4K video streamed from pinned host memory through one serving stream (H2D, kernel
    and D2H overlapped across frames), anaglyph, P = 64."""
    from paper_2009_09501_gb300 import scenes
    sc = scenes.Scene(3840, 2160, 2009_09501 + 3, 40, "gauss8", moving=True)
    pool = [torch.from_numpy(sc.frame(k)).pin_memory() for k in range(2)]
    outs = [torch.empty((2160, 3840, 3), dtype=torch.uint8).pin_memory() for _ in range(4)]
    p = D.make_params(max_parallax=P4K, outputs=("anaglyph",))
    with D.Context(device=torch.cuda.current_device()) as c:
        sid = c.open_stream(3840, 2160, p)
        lat, done, k = [], 0, 0
        t0 = time.perf_counter()
        while done < frames:
            while k < frames and k - done < 4:
                st = c.submit_frame(sid, k, pool[k % 2].numpy(), {"anaglyph": outs[k % 4].numpy()})
                if st != D.DIBR_OK:
                    break
                k += 1
            for comp in c.poll(16, 100000):
                assert comp.status == D.DIBR_OK
                lat.append((comp.t_done_ns - comp.t_submit_ns) / 1e6)
                done += 1
        el = time.perf_counter() - t0
        c.close_stream(sid)
    fb = 3840 * 2160 * 3
    return {"frames": frames, "frames_per_s": frames / el, "host_link_gb_per_s": 2 * fb * frames / el / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}


def bench_served(D, torch, seconds, frames_per_stream=8, pool_frames=None):
    """Serving: 4 x 1080p and 4 x 4K moving-object streams, Poisson arrivals at 30 fps per
    stream, anaglyph, P = 2.5 % of the width; per-frame latency submit -> outputs in host
    memory.  Each stream cycles through its first frames_per_stream frames."""
    from paper_2009_09501_gb300 import scenes
    sizes = [(1920, 1080)] * 4 + [(3840, 2160)] * 4
    rng = np.random.default_rng(2009_09501 + 5)
    seqs = pool_frames
    frames = [[torch.from_numpy(f).pin_memory() for f in seq] for seq in seqs]
    with D.Context(device=torch.cuda.current_device()) as c:
        sids = [c.open_stream(W, H, D.make_params(max_parallax=scenes.batch_parallax(W), outputs=("anaglyph",)))
                for (W, H) in sizes]
        outs = [[torch.empty_like(frames[k][0]).pin_memory() for _ in range(20)] for k in range(len(sizes))]
        events = []
        for k in range(len(sizes)):
            t = 0.0
            while True:
                t += rng.exponential(1.0 / 30.0)
                if t >= seconds:
                    break
                events.append((t, k))
        events.sort()
        lat = {k: [] for k in range(len(sizes))}
        refused, n_sub, seq = 0, 0, [0] * len(sizes)
        t0 = time.perf_counter()
        i = 0
        while i < len(events) or sum(len(v) for v in lat.values()) < n_sub:
            now = time.perf_counter() - t0
            while i < len(events) and events[i][0] <= now:
                k = events[i][1]
                o = outs[k][seq[k] % 20]
                src = frames[k][seq[k] % len(frames[k])]
                st = c.submit_frame(sids[k], seq[k], src.numpy(), {"anaglyph": o.numpy()})
                if st == D.DIBR_OK:
                    n_sub += 1
                else:
                    refused += 1
                seq[k] += 1
                i += 1
            for comp in c.poll(64, 500):
                k = sids.index(comp.stream_id)
                lat[k].append((comp.t_done_ns - comp.t_submit_ns) / 1e6)
            if now > seconds + 30:
                break
        el = time.perf_counter() - t0
        for s_ in sids:
            c.close_stream(s_)
    all_l = [x for v in lat.values() for x in v]
    l4k = [x for k in range(4, 8) for x in lat[k]]
    return {"streams": "4 x 1920x1080 + 4 x 3840x2160 @ 30 fps Poisson, moving-object scenes", "seconds": seconds,
            "frames_per_stream_cycled": frames_per_stream,
            "frames": len(all_l), "frames_per_s": len(all_l) / el, "refused": refused,
            "p50_ms": float(np.percentile(all_l, 50)), "p99_ms": float(np.percentile(all_l, 99)),
            "p99_ms_4k": float(np.percentile(l4k, 99)) if l4k else None}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2009_09501_gb300 import dibr as D
    from paper_2009_09501_gb300 import scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    img = scenes.config_scene(2)
    H, W = img.shape[:2]
    # the context's own stream (the library's default): events are recorded on it, and no
    # other work is enqueued there, so consecutive frames with disjoint buffers may overlap
    ctx = D.Context(device=local)
    stream = torch.cuda.ExternalStream(D.dibr_stream(ctx.handle), device=torch.device("cuda", local))
    p = D.make_params(max_parallax=P4K, outputs=OUTPUTS)

    # rotate buffer sets so that every step reads and writes HBM, not L2
    l2 = torch.cuda.get_device_properties(local).L2_cache_size if hasattr(
        torch.cuda.get_device_properties(local), "L2_cache_size") else 128 << 20
    set_bytes = ALG_BYTES
    nsets = max(2, int(np.ceil(2.0 * l2 / set_bytes)) + 1)
    src = torch.from_numpy(img).cuda()
    sets = []
    for _ in range(nsets):
        i = src.clone()
        o = {n: torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for n in OUTPUTS}
        sets.append((D.image_struct(i), D.outputs_struct(o), i, o))
    torch.cuda.synchronize()  # the buffers (made on torch's stream) exist before the library's stream uses them
    lib = D.load()
    enqueue = lib.dibr_enqueue_image
    h = ctx.handle
    pref = D.C.byref(p)
    args_c = [(D.C.byref(s[0]), D.C.byref(s[1])) for s in sets]

    def step(k):
        a, b = args_c[k % nsets]
        st = enqueue(h, a, pref, b)
        if st != 0:
            raise D.DibrError(st, D.dibr_last_error(h))

    for k in range(args.warmup):
        step(k)
    ctx.synchronize()

    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
    sampler.start()
    time.sleep(0.3)
    K = args.steps
    # events only around the timed region: back-to-back launches then overlap one launch's
    # set-up with the previous one's end (programmatic dependent launch); an event between
    # two launches would serialise them
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.monotonic()
    e_start.record(stream)
    for k in range(K):
        step(k)
    e_end.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.monotonic()
    if dist:
        dist.barrier()
    time.sleep(0.1)
    sampler.stop()
    ctx.synchronize()
    total_ms = e_start.elapsed_time(e_end)
    mean_launch_ms = total_ms / K  # average launch duration over the timed region
    # latency of single launches on an idle GPU, each bracketed by its own events (outside
    # the timed region; a launch on an idle stream spreads over every SM)
    n_single = min(K, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_single)]
    for k in range(n_single):
        ctx.synchronize()
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    ctx.synchronize()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    value = whole_job_rate(K, total_ms / 1000.0, world, dist, "cuda")
    total_ms = reduce_max(total_ms, dist, "cuda")

    # end to end through the public API with pinned host buffers
    host_in = torch.from_numpy(img).pin_memory()
    host_out = {n: torch.empty((H, W, 3), dtype=torch.uint8).pin_memory() for n in OUTPUTS}
    hi = D.image_struct(host_in.numpy())
    ho = D.outputs_struct({n: v.numpy() for n, v in host_out.items()})
    sync_fn = lib.dibr_synthesize_image
    for _ in range(3):
        ctx.check(sync_fn(h, D.C.byref(hi), pref, D.C.byref(ho)))
    n_e2e = max(5, min(K, 60))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ctx.check(sync_fn(h, D.C.byref(hi), pref, D.C.byref(ho)))
    e2e_s = time.perf_counter() - t0
    e2e_blocking = whole_job_rate(n_e2e, e2e_s, world, dist, "cuda")

    # end to end through the streaming entry points (dibr_submit_frame / dibr_poll), the
    # API for frame sequences: the H2D copy of one frame, the kernels of another and the
    # D2H copies of a third overlap; every frame still crosses the host link both ways
    sid = ctx.open_stream(W, H, p)
    host_outs = [{n: torch.empty((H, W, 3), dtype=torch.uint8).pin_memory().numpy() for n in OUTPUTS}
                 for _ in range(4)]
    hin = host_in.numpy()

    def stream_frames(n):
        done = k = 0
        while done < n:
            while k < n and k - done < 3:
                if ctx.submit_frame(sid, k, hin, host_outs[k % 4]) != D.DIBR_OK:
                    break
                k += 1
            for comp in ctx.poll(16, 100000):
                if comp.status != D.DIBR_OK:
                    raise D.DibrError(comp.status, "frame %d" % comp.seq)
                done += 1

    stream_frames(5)
    n_stream = max(20, min(K, 200))
    t0 = time.perf_counter()
    stream_frames(n_stream)
    stream_s = time.perf_counter() - t0
    ctx.close_stream(sid)
    e2e_value = whole_job_rate(n_stream, stream_s, world, dist, "cuda")

    extra = {}
    if world == 1 and not args.quick:
        extra["config1"] = bench_config1(D, torch, ctx, stream)
        extra["batch"] = bench_batch(D, torch, ctx, stream)
        extra["inpaint2d"] = bench_inpaint(D, torch, ctx, stream)
        extra["xbf"] = bench_xbf(D, torch, ctx, stream)
        extra["video"] = bench_video(D, torch, ctx)
        # the served streams' moving frames, drawn on the host's cores (a spawned pool) only
        # now, so that the 1.2 GB of them do not sit in host memory through the other sections
        import multiprocessing as mp
        sizes = [(1920, 1080)] * 4 + [(3840, 2160)] * 4
        with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
            served_frames = pool.map(_stream_frames, [(k, W, H, 8) for k, (W, H) in enumerate(sizes)])
        extra["served"] = bench_served(D, torch, args.served_seconds, pool_frames=served_frames)
        del served_frames
    if rank == 0:
        peak, peak_kind = load_peaks()
        traffic, traffic_src = load_traffic()
        achieved = ALG_BYTES / (mean_launch_ms / 1000.0) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": dict(CONFIG, l2_defeat="rotating %d buffer sets of %.1f MB (> 2x L2 of %.0f MB)"
                           % (nsets, set_bytes / 1e6, l2 / 1e6), parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                         "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                         "kernel": "band_kernel", "alg_bytes_per_launch": ALG_BYTES,
                         "mean_launch_us": mean_launch_ms * 1000.0,
                         "single_launch_p10_us": float(np.percentile(launch_ms, 10)) * 1000.0,
                         "single_launch_p90_us": float(np.percentile(launch_ms, 90)) * 1000.0},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * W * H,
                    "d2h_bytes_per_step": 3 * W * H * len(OUTPUTS), "steps": n_stream,
                    "api": "dibr_submit_frame/dibr_poll, pinned host input and outputs, 3 frames in flight",
                    "blocking_call_value": e2e_blocking, "blocking_call_steps": n_e2e,
                    "blocking_call_api": "dibr_synthesize_image, pinned host buffers, one frame at a time"},
            "gpu_launches": K,
            "clocks": sampler.summary(t_host0 - 0.02, t_host1 + 0.02),
        }
        out.update(extra)
        if world == 1 and not args.no_cpu_baseline:
            v, cores, n, el = oracle_frames_per_s(img)
            v1, n1, el1 = oracle_single_core(img)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": "%d full 4K frames in %.1f s, band-parallel over %d threads"
                                             % (n, el, cores),
                                   "single_core_value": v1,
                                   "single_core_sample": "%d frames in %.1f s on 1 thread" % (n1, el1)}
        print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the batch, video and served sections")
    ap.add_argument("--served-seconds", type=float, default=20.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
