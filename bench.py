#!/usr/bin/env python
"""Benchmark of the fused DIBR pipeline on the 4K UHD still-image workload.

Workload: one 3840 x 2160 RGB uint8 frame (seeded synthetic scene, 40 objects, sigma-8
texture), maximum parallax 64 px, binomial depth smoothing, Fig. 3 shift rule, outputs
left + right views and the red-cyan anaglyph.  A step is one pass of the whole pipeline
over one frame: one launch of the fused kernel.

Prints one JSON line (rank 0):
  value      frames/s over all ranks, inputs resident in HBM, CUDA events on the
             launching stream, rotating buffer sets larger than 2x L2;
  e2e        frames/s through dibr_synthesize_image with pinned HOST buffers (H2D of the
             input, kernel, D2H of the outputs inside the timed region);
  roofline   the fused kernel's algorithmic bytes per launch / its mean launch time
             against the measured HBM copy bandwidth;
  cpu_baseline  the CPU oracle on this host's cores (band-parallel over row bands), on a
             bounded sample of frames;
  clocks     SM clock samples taken by nvidia-smi during the timed region.
--impl reference times the CPU oracle alone on the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

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
    # a dedicated stream: the library runs on it and the CUDA events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = D.Context(device=local, stream=stream.cuda_stream)
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
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.monotonic()
    for k in range(K):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_host1 = time.monotonic()
    if dist:
        dist.barrier()
    time.sleep(0.1)
    sampler.stop()
    ctx.synchronize()
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    mean_launch_ms = float(np.mean(launch_ms))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * K / (total_ms / 1000.0)

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
    e2e_value = world * n_e2e / e2e_s
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = world * n_e2e / float(t.item())

    if rank == 0:
        peak, peak_kind = load_peaks()
        achieved = ALG_BYTES / (mean_launch_ms / 1000.0) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": dict(CONFIG, l2_defeat="rotating %d buffer sets of %.1f MB (> 2x L2 of %.0f MB)"
                           % (nsets, set_bytes / 1e6, l2 / 1e6), parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": args.traffic,
                         "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                         "kernel": "band_kernel", "alg_bytes_per_launch": ALG_BYTES,
                         "mean_launch_us": mean_launch_ms * 1000.0,
                         "p10_launch_us": float(np.percentile(launch_ms, 10)) * 1000.0,
                         "p90_launch_us": float(np.percentile(launch_ms, 90)) * 1000.0},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * W * H,
                    "d2h_bytes_per_step": 3 * W * H * len(OUTPUTS), "steps": n_e2e},
            "gpu_launches": K,
            "clocks": sampler.summary(t_host0 - 0.02, t_host1 + 0.02),
        }
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
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the fused kernel, if captured")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
