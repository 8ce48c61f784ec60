#!/usr/bin/env python
"""Benchmark of the SwinGS frame-t splatting hot path on B300.

Workload (one "step"): the sliding-window training step on 300k Gaussians
(SH degree 3, 300-frame lifespans, frames 145..154, 4 of 20 ring cameras per
frame = 40 views of 1352x1014): a 6,000-Gaussian slice update (Alg. 2; from
HBM in the timed step, streamed from pinned host memory in the end-to-end
one), the batched forward of all 40 views, the L1 loss, the reverse blend and
projection backward, and the Adam + SGLD noise + relocation step (Alg. 1).
Metric: Mpix/s of the fwd+bwd step (batched); the plain per-view path,
forward-only rates and the serving latency are reported beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank trains a replica on its own
window of views; gradients are summed across ranks with NCCL before the SGLD
step (data parallel), so per-GPU work is fixed as N grows (weak scaling).
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# Algorithmic FP32 operations per evaluated (pixel, Gaussian) pair, the
# roofline's numerator: the forward pass of Eq. 3 takes about 12 (offset,
# Mahalanobis form, G, alpha, the transmittance and colour updates) plus one
# ex2; its adjoint about 40 plus one ex2.
FLOP_PER_PAIR_FWD = 12
FLOP_PER_PAIR_BWD = 40
# The same counted per issued FP32 operation of this implementation (an FMA
# counts 2), reported beside. Per pair, with the terms common to a thread's
# column of pixels (dx, qb dx, qa dx dx + lo) shared by its 4 (forward) or 8
# (reverse) pixels: forward offset 1.25, Mahalanobis form 5, T(1 - alpha) and
# the T update 3, colour 7 = 16; reverse alpha recompute 5.6, T recovery 2,
# colour weights 7, E and D - E 6, colour-behind 2, alpha dL/dalpha 1,
# moments 5, the per-Gaussian sums and their reduction over the tile 1.5 = 30
# (the conic/centre/opacity chain rule runs once per Gaussian and tile).
OWN_FLOP_PER_PAIR_FWD = 16
OWN_FLOP_PER_PAIR_BWD = 30

# DRAM bytes (read + write) per launch from one ncu capture of the full-size
# window step, keyed by stage and launch shape, with a digest of the sources
# that define the kernel: a changed kernel reports no traffic until it is
# captured again.
TRAFFIC_CAPTURES = {
    ("blend_bwd", "16x16/b32/ppt8"): {
        "bytes": 1_233_212_928 + 16_238_080,
        "sources": ("csrc/k_blend.cu", "csrc/swgs_internal.cuh"),
        "digest": "7e9f810f1153d704",
    },
}


def source_digest(files) -> str:
    """Digest of the code of CUDA sources: comments dropped and whitespace
    collapsed, so that only a change of code retires a capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        src = (ROOT / "paper_2409_07759_b300" / f).read_text()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def captured_traffic(stage: str, shape: str):
    c = TRAFFIC_CAPTURES.get((stage, shape))
    if c is None:
        return None
    return c["bytes"] if source_digest(c["sources"]) == c["digest"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="swgs", choices=["swgs", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-config3", action="store_true")
    ap.add_argument("--views", type=int, default=4, help="cameras per frame")
    ap.add_argument("--frames", type=int, default=10)
    ap.add_argument("--tile", default="16x16", help="blend tile, WxH")
    ap.add_argument("--batch", type=int, default=64, help="Gaussians staged per block step")
    ap.add_argument("--ppt", type=int, default=4, help="forward blend pixels per thread")
    ap.add_argument("--bwd-ppt", type=int, default=8, help="reverse blend pixels per thread")
    ap.add_argument("--bwd-batch", type=int, default=32, help="reverse blend staging batch")
    ap.add_argument("--targets", default="u8", choices=["u8", "f32"],
                    help="target frames: 8-bit (k/255) or float32")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--viewers", type=int, default=64)
    ap.add_argument("--rate", type=float, default=30.0, help="requests/s per viewer")
    ap.add_argument("--serve-streams", type=int, default=3)
    ap.add_argument("--serve-slots", type=int, default=1,
                    help="batches each serving worker may have in flight")
    ap.add_argument("--hbm-budget-gb", type=float, default=24.0)
    ap.add_argument("--no-images", action="store_true",
                    help="write no rendered image (the step needs only the loss and its "
                         "gradient, which the forward computes in its epilogue)")
    ap.add_argument("--deferred-sizing", action="store_true",
                    help="training renders without host round trips (capacities learned)")
    ap.add_argument("--serve-deferred", action="store_true",
                    help="serving workers render without host round trips")
    ap.add_argument("--sweep-seconds", type=float, default=2.5,
                    help="seconds per rate of the serving sweep (0: no sweep)")
    return ap.parse_args()


def config3_leg(args):
    """Config 3: batched multi-view forward of 1M Gaussians (~20% active) to 32
    Fibonacci-sphere cameras (8 x 640x480, 16 x 1280x720, 8 x 1920x1080) in one
    batched call with the autotuned launch shape, against the plain per-view path."""
    import torch
    from paper_2409_07759_b300 import api, autotune, synth
    sc, views = synth.config3()
    st = api.GaussianState.from_scene(sc)
    best = autotune.autotune(st, views, mode="fwd", reps=2, cache=None)
    r = api.Renderer(**best)
    mpix = sum(v.width * v.height for v in views) / 1e6

    def timed(batched, reps):
        r.render(st, views, batched=batched)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            r.render(st, views, batched=batched)
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    bms, pms = timed(True, 5), timed(False, 3)
    r.close()
    return {"mpix": mpix, "views": len(views), "gaussians": sc.n,
            "batched_ms": bms, "batched_mpix_s": mpix / (bms / 1e3),
            "plain_ms": pms, "plain_mpix_s": mpix / (pms / 1e3), "batched_over_plain": pms / bms,
            "autotuned": dict(best, tile="%dx%d" % tuple(best["tile"]))}


def mature_leg(state, swin=50, reps=20):
    """Alg. 1 mature(st) on the window scene laid out as gs (300k slots, swin
    50: 6,000-slot slices) + the ring of matured rows, snapshot to pinned host
    memory (stream.write): the per-frame maturation once the first window's
    full snapshot has been taken. Times each call (it synchronises once to read
    the count) with CUDA events and host time."""
    import torch
    from paper_2409_07759_b300 import api
    num_gs = state.n - state.n % swin
    gs = state.rows(0, num_gs)
    buf = api.GaussianState.with_matured_ring(
        api.GaussianState(*[t.clone() for t in (gs.means, gs.log_scales, gs.quats,
                                                 gs.opacity_logits, gs.sh, gs.start,
                                                 gs.expire, gs.birth, gs.frozen)],
                          sh_degree=gs.sh_degree))
    r = api.Renderer()
    buf.start.zero_()
    buf.birth.zero_()
    buf.expire[:num_gs] = swin
    snap = api.GaussianState(*[torch.empty_like(getattr(buf, k)[:num_gs]) for k in
                               api.PARAM_NAMES + ("start", "expire", "birth", "frozen")],
                             sh_degree=buf.sh_degree).pin_host()
    r.schedule_expire(buf, num_gs, swin)
    head = 0
    n0, head = r.mature(buf, num_gs, 1, swin, head, snapshot=snap)   # the first window
    times, ns = [], []
    for st in range(2, 2 + reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record()
        n, head = r.mature(buf, num_gs, st, swin, head, snapshot=snap)
        b.record()
        b.synchronize()
        times.append((a.elapsed_time(b), 1e3 * (time.perf_counter() - t0)))
        ns.append(n)
    r.close()
    row = sum(getattr(buf, k)[:1].numel() * getattr(buf, k).element_size() for k in
              api.PARAM_NAMES + ("start", "expire", "birth", "frozen"))
    dev_ms = statistics.median(t[0] for t in times)
    n = int(statistics.median(ns))
    # per maturation: lifespans of every gs slot read (4 B) + n rows read, written to
    # the ring and to the staging snapshot, 12 B of lifespans rewritten; n rows D2H
    moved = 4 * num_gs + 3 * n * row + 12 * n
    return {"num_gs": num_gs, "swin_size": swin, "first_window_rows": n0,
            "rows_per_frame": n, "row_bytes": row, "ms_per_frame": dev_ms,
            "host_ms_per_frame": statistics.median(t[1] for t in times),
            "device_bytes": moved, "d2h_bytes": n * row,
            "achieved_gbs": moved / (dev_ms / 1e3) / 1e9}


def codec_leg(state, views, slice_size=6000, fracs=(1.0, 0.8, 0.6, 0.4, 0.2)):
    """Table 6 codec + Sec. 5.5 tail drop on the window scene: encode/decode
    time of one 6,000-row slice (pinned host packets, as a client receives
    them), and the rate-distortion of keeping a fraction of every slice (the
    Fig. 10-12 sweep: 100/80/60/40/20%), as packet bytes per update and PSNR of
    the decoded scene's render against the unquantised render (4 views)."""
    import torch
    from paper_2409_07759_b300 import api
    r = api.Renderer()
    n = state.n - state.n % slice_size
    sl = state.rows(0, slice_size)
    host = torch.empty(api.Renderer.slice_packet_bytes(slice_size, slice_size),
                       dtype=torch.uint8).pin_memory()
    dst = api.GaussianState(*[t.clone() for t in (state.means, state.log_scales, state.quats,
                                                   state.opacity_logits, state.sh, state.start,
                                                   state.expire, state.birth, state.frozen)],
                            sh_degree=state.sh_degree)
    enc, dec = [], []
    for _ in range(20):
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        pkt = r.slice_encode(sl, slice_size, out=host)
        b.record()
        r.slice_decode(pkt, dst, 0)
        c.record()
        c.synchronize()
        enc.append(a.elapsed_time(b))
        dec.append(b.elapsed_time(c))
    # slices share one lifespan (Sec. 4.2.1): a copy of the scene active over
    # the rendered frames
    base = api.GaussianState(*[t.clone() for t in (state.means, state.log_scales, state.quats,
                                                    state.opacity_logits, state.sh, state.start,
                                                    state.expire, state.birth, state.frozen)],
                             sh_degree=state.sh_degree)
    base.start.zero_()
    base.birth.zero_()
    base.expire.fill_(1000)
    state = base
    vs = views[:4]
    ref, _ = r.render(state, vs)
    curve = []
    for f in fracs:
        keep = int(round(f * slice_size))
        q = api.GaussianState(*[t.clone() for t in (state.means, state.log_scales, state.quats,
                                                     state.opacity_logits, state.sh,
                                                     state.start, state.expire, state.birth,
                                                     state.frozen)], sh_degree=state.sh_degree)
        nbytes = 0
        for first in range(0, n, slice_size):
            p = r.slice_encode(state.rows(first, first + slice_size), slice_size, keep)
            nbytes = p.numel()
            r.slice_decode(p, q, first)
        img, _ = r.render(q, vs)
        mse = sum(float(((x - y) ** 2).mean()) for x, y in zip(img, ref)) / len(vs)
        curve.append({"keep_fraction": f, "packet_bytes_per_slice": nbytes,
                      "psnr_db": 10.0 * math.log10(1.0 / max(mse, 1e-20))})
    r.close()
    raw_row = 4 * (3 + 3 + 4 + 1 + state.sh.shape[1] * 3)
    return {"slice_rows": slice_size, "encode_ms": statistics.median(enc),
            "decode_ms": statistics.median(dec),
            "packet_bytes": api.Renderer.slice_packet_bytes(slice_size, slice_size),
            "raw_bytes": slice_size * raw_row, "bytes_per_gaussian": 29,
            "rate_distortion": curve,
            "note": "PSNR of the decoded synthetic scene against its unquantised render "
                    "(DC-only SH and fp16/uint8 codes); not a dataset PSNR"}


def memory_leg(lengths=(10, 100, 1000), num_gs=300_000, swin=5):
    """Table 3 in spirit: peak device memory of Alg. 1 main (ClipTrainer) over
    clips of 10, 100 and 1000 frames -- 300k Gaussians (swin 5: 60k-row slices),
    one 676x507 view per frame, one step per window, the stream to pinned host.
    The state (gs, matured ring, Adam moments, snapshot and packet buffers) is
    allocated once; the renderer's scratch follows the largest step's tile-key
    count, reported beside the peak. Two modes: "train" (Adam on the random
    8-bit targets, which resizes the Gaussians as the clip goes on, so the key
    count drifts) and "stationary" (Adam off: the noise, relocation,
    maturation and streaming still run, the scene's footprint stays put)."""
    import torch
    from paper_2409_07759_b300 import api, synth
    from paper_2409_07759_b300.window import ClipTrainer
    w, h = 676, 507
    sc, _, _ = synth.config2(width=w, height=h, n=num_gs, n_frames=1, per_frame=1)
    ring = synth.ring_cameras(20, 4.0, w, h)

    def window(st, ed):
        views, targets = [], []
        g = torch.Generator(device="cuda")
        for f in range(st, ed):
            v = ring[f % 20]
            views.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
            g.manual_seed(f)
            targets.append(torch.randint(0, 256, (3, h, w), dtype=torch.uint8, device="cuda",
                                         generator=g))
        return views, targets

    modes = {}
    for mode, params in (("train", None), ("stationary", dict(adam=0))):
        modes[mode] = _memory_clips(lengths, sc, swin, window, params)
    return {"num_gs": num_gs, "swin_size": swin, "view": f"{w}x{h}", "modes": modes}


def _memory_clips(lengths, sc, swin, window, params):
    import torch
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300.window import ClipTrainer
    out = {}
    for T in lengths:
        r = api.Renderer()
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        # the stream goes out as Table 6 packets (as a server would send it)
        sent = [0, 0]

        def sink(st, n, pkt):
            sent[0] += n
            sent[1] += pkt.numel()
        ct = ClipTrainer(r, api.GaussianState.from_scene(sc), swin, window, iterations=1,
                         params=params, codec=True, sink=sink)
        t0 = time.perf_counter()
        ct.run(T)
        torch.cuda.synchronize()
        out[str(T)] = {"peak_bytes_over_base": int(torch.cuda.max_memory_allocated() - base),
                       "seconds": time.perf_counter() - t0,
                       "stream_rows": sent[0], "stream_bytes": sent[1],
                       # the renderer's scratch follows the largest step's tile keys
                       "max_tile_keys": ct.trainer.max_keys}
        r.close()
        del ct
        gc.collect()
        torch.cuda.empty_cache()
    return out


def serving_leg(args):
    """Config 4: 300k Gaussians in 50 slices of 6,000 (swin_size 50), one
    slice swapped per frame at 30 fps, Poisson viewers on orbits requesting the
    current frame at 640x480 / 1280x720 / 1920x1080 (1:2:1)."""
    import torch
    from paper_2409_07759_b300 import api, serving, synth
    swin, S = synth.SWIN_SIZE_SERVING, synth.SLICE_SIZE_SERVING
    scene = synth.config4_initial(S, swin, 3)
    st = api.GaussianState.from_scene(scene)
    pool = [api.GaussianState.from_scene(synth.config4_slice(f, S, swin, 3)).pin_host()
            for f in range(1, 9)]

    def provider(frame):
        h = pool[frame % len(pool)]
        h["start"].fill_(frame)
        h["expire"].fill_(frame + swin)
        h["birth"].fill_(frame)
        return h

    loop = serving.ServingLoop(st, swin, fps=30.0, n_streams=args.serve_streams, max_batch=16,
                               hbm_budget_bytes=args.hbm_budget_gb * 1e9,
                               slice_provider=provider, n_slots=args.serve_slots,
                               deferred_sizing=args.serve_deferred)
    loop.reserve(1920, 1080)
    warm = serving.make_requests(args.viewers, args.rate, 1.0, seed=40)
    loop.run(warm, 1.0)
    reqs = serving.make_requests(args.viewers, args.rate, args.serve_seconds, seed=41)
    stats = loop.run(reqs, args.serve_seconds)
    ser = serving.serial_rates(st, reqs, loop.frame, renderer=loop.renderers[0], n=40)
    loop.close()
    out = stats.as_dict()
    out.update(viewers=args.viewers, rate_hz_per_viewer=args.rate,
               resolutions="640x480:1280x720:1920x1080 = 1:2:1", gaussians=scene.n,
               swin_size=swin, slice_size=S, streams=args.serve_streams,
               hbm_budget_gb=args.hbm_budget_gb, serial=ser, slots=args.serve_slots,
               delivered="8-bit RGB [H,W,3] to pinned host memory",
               offered_mpix_s=sum(r.width * r.height for r in reqs) / 1e6 / args.serve_seconds,
               latency="arrival to image in pinned host memory (p50/p99_ms); to the end of "
                       "the render on the device (p50/p99_render_ms)")
    if args.sweep_seconds > 0:
        out["sweep"] = {
            "mix_1_2_1": serving_sweep(args, st, swin, provider, None, "1920x1080"),
            "all_1280x720": serving_sweep(args, st, swin, provider, [(1280, 720)], "1280x720"),
        }
    return out


def serving_sweep(args, st, swin, provider, resolutions, reserve_res):
    """Per-viewer request rate raised step by step (64 viewers, Poisson
    arrivals) until p99 passes 16 ms or the served rate falls behind the
    offered one; reports each rate and the highest one whose p99 (arrival to
    image in host memory) stays under 16 ms."""
    from paper_2409_07759_b300 import serving
    loop = serving.ServingLoop(st, swin, fps=30.0, n_streams=args.serve_streams, max_batch=16,
                               hbm_budget_bytes=args.hbm_budget_gb * 1e9,
                               slice_provider=provider, n_slots=args.serve_slots,
                               deferred_sizing=args.serve_deferred)
    w, h = (int(x) for x in reserve_res.split("x"))
    loop.reserve(w, h)
    rows, best, misses = [], None, 0
    for rate in (10, 20, 30, 45, 60, 90, 120, 160, 200, 250, 300, 400, 500):
        warm = serving.make_requests(args.viewers, rate, 0.5, seed=50 + rate,
                                     resolutions=resolutions)
        loop.run(warm, 0.5)
        reqs = serving.make_requests(args.viewers, rate, args.sweep_seconds, seed=60 + rate,
                                     resolutions=resolutions)
        stats = loop.run(reqs, args.sweep_seconds)
        offered = sum(r.width * r.height for r in reqs) / 1e6 / args.sweep_seconds
        rows.append({"rate_hz_per_viewer": rate, "requests_per_s": len(reqs) / args.sweep_seconds,
                     "p50_ms": stats.p50_ms, "p99_ms": stats.p99_ms,
                     "p99_render_ms": stats.p99_render_ms, "served_mpix_s": stats.mpix_per_s,
                     "offered_mpix_s": offered, "mean_batch": stats.mean_batch})
        ok = stats.p99_ms < 16.0 and stats.mpix_per_s >= 0.9 * offered
        if ok:
            best = rate
            misses = 0
        else:
            misses += 1
            if misses >= 2:
                break
    loop.close()
    return {"viewers": args.viewers, "seconds_per_rate": args.sweep_seconds, "rates": rows,
            "max_rate_p99_under_16ms": best,
            "max_served_mpix_s_p99_under_16ms": max(
                (r["served_mpix_s"] for r in rows if r["rate_hz_per_viewer"] == best),
                default=None)}


# ----------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in loaded for n, v in zip(names, r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


# -------------------------------------------------------------- FP32 peak --

def fp32_peak_leg(reps=10, warmup=3):
    """Measured FP32-pipe throughput: the library's probe (8 independent FMA
    chains per thread, 8 blocks of 256 threads per SM) as scalar FFMA and as
    packed FFMA2, timed with CUDA events on the launching stream, with the SM
    clock sampled meanwhile. Returns TFLOP/s of each form (an FMA counts 2)."""
    import ctypes
    import torch
    from paper_2409_07759_b300 import _abi
    lib = _abi.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * 8
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"blocks": blocks, "threads_per_block": 256, "chains_per_thread": 8}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for packed, name in ((0, "ffma"), (1, "ffma2")):
        iters = 32768
        fl = ctypes.c_double(0.0)
        for _ in range(warmup):
            st = lib.swgs_fp32_peak_launch(packed, blocks, iters, sink.data_ptr(),
                                           ctypes.byref(fl), ctypes.c_void_p(stream.cuda_stream))
            if st != 0:
                raise RuntimeError(f"swgs_fp32_peak_launch failed ({st})")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            lib.swgs_fp32_peak_launch(packed, blocks, iters, sink.data_ptr(), ctypes.byref(fl),
                                      ctypes.c_void_p(stream.cuda_stream))
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[name] = {"tflops": fl.value / (ms / 1e3) / 1e12, "ms_per_launch": ms,
                     "flop_per_launch": fl.value}
    clocks = sampler.stop()
    out["clocks"] = clocks
    out["tflops"] = max(out["ffma"]["tflops"], out["ffma2"]["tflops"])
    out["form"] = "ffma2" if out["ffma2"]["tflops"] >= out["ffma"]["tflops"] else "ffma"
    if clocks.get("sm_mhz"):
        # FLOP per SM per clock at the sampled median clock
        for k in ("ffma", "ffma2"):
            out[k]["flop_per_sm_clk"] = out[k]["tflops"] * 1e12 / (sms * clocks["sm_mhz"] * 1e6)
    return out


# ------------------------------------------------------------- CPU oracle --

def cpu_oracle_sample(scene, views, targets, budget_s=15.0, max_views=None, threads=None):
    """Time the FP64 oracle (tiled fwd + bwd of whole views) on the host cores
    (or on `threads` threads) until about budget_s of work; returns
    (mpix_per_s, cores, sample text)."""
    import numpy as np
    import oracle
    oracle.build()
    all_cores = oracle.num_threads()
    if threads:
        oracle.set_threads(threads)
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    pix = 0
    n = 0
    for v, tgt in zip(views, targets):
        ref = oracle.render(scene, v, mode="tiled", bands=None)
        _, dl = oracle.l1_loss_grad([ref["rgb"]], [tgt])
        oracle.render_bwd(scene, v, dl[0])
        pix += v.width * v.height
        n += 1
        if time.perf_counter() - t0 > budget_s or (max_views and n >= max_views):
            break
    dt = time.perf_counter() - t0
    if threads:
        oracle.set_threads(all_cores)
    return pix / dt / 1e6, cores, f"{n} of {len(views)} views, fwd+bwd (tiled FP64 oracle), {dt:.1f} s"


# -------------------------------------------------------------- workload --

def build_workload(args, rank=0):
    from paper_2409_07759_b300 import synth
    scene, views, targets = synth.config2(n_frames=args.frames, per_frame=args.views,
                                          forced_dead_fraction=0.01, rank=rank)
    return scene, views, targets


def arm_config(args, views, world=1):
    """The workload both arms report (the reference arm samples it on the host)."""
    mpix = sum(v.width * v.height for v in views) / 1e6
    return {"workload": "sliding-window step: 300k Gaussians SH3, frames 145-154 x "
                        f"{args.views} of 20 ring cameras = {len(views)} views of 1352x1014, "
                        "fwd+bwd + Adam/SGLD + relocation + 6k-slot slice update (from HBM; "
                        "from pinned host in e2e)",
            "mpix_per_step": mpix, "tile": args.tile, "batch": args.batch,
            "pixels_per_thread": args.ppt,
            "bwd_pixels_per_thread": args.bwd_ppt, "bwd_batch": args.bwd_batch,
            "targets": ("8-bit RGB frames (k/255)" if args.targets == "u8" else "float32 RGB"),
            "parallelism": f"dp{world}", "l2": "flushed (256 MB write) before each step",
            "sizing": ("deferred (no host round trip in a step)" if args.deferred_sizing
                       else "exact (two host round trips per batch)"),
            "images": ("not written (the L1 term and its gradient are computed in the "
                       "forward's epilogue)" if args.no_images else "written every step")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, views, targets = build_workload(args)
    rates = []
    t_all = 0.0
    sample = ""
    cores = 1
    for k in range(args.warmup + args.steps):
        v = [views[k % len(views)]]
        tg = [targets[k % len(views)]]
        t0 = time.perf_counter()
        rate, cores, sample = cpu_oracle_sample(scene, v, tg, budget_s=1e9, max_views=1)
        if k >= args.warmup:
            rates.append(rate)
            t_all += time.perf_counter() - t0
    value = statistics.mean(rates)
    line = {"metric": "Mpix/s fwd+bwd (sliding-window training step)", "value": value,
            "unit": "Mpix/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": arm_config(args, views),
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                             "sample": "one view per step: " + sample},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    from paper_2409_07759_b300 import api, build, synth
    from paper_2409_07759_b300.window import WindowTrainer
    build.build()

    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # the FP32 pipe's measured throughput (the blends' roofline denominator)
    fp32 = fp32_peak_leg()

    # weak scaling: every rank holds a replica of the scene and renders its own
    # 4 cameras per frame of the window (rank 0: the single-GPU workload)
    scene, views, targets = build_workload(args, rank=rank)
    mpix = sum(v.width * v.height for v in views) / 1e6
    state = api.GaussianState.from_scene(scene)
    if args.targets == "u8":  # 8-bit frames, the form video targets come in
        targets = [np.rint(t * 255.0).astype(np.uint8) for t in targets]
        oracle_targets = [t.astype(np.float32) * np.float32(1.0 / 255.0) for t in targets]
    else:
        oracle_targets = targets
    tgt_host = [torch.from_numpy(t).pin_memory() for t in targets]
    tgt_dev = [t.cuda() for t in tgt_host]
    tw, th = (int(x) for x in args.tile.split("x"))
    r = api.Renderer(tile=(tw, th), batch=args.batch, pixels_per_thread=args.ppt,
                     bwd_pixels_per_thread=args.bwd_ppt, bwd_batch=args.bwd_batch,
                     deferred_sizing=args.deferred_sizing)
    reducer = None
    if world > 1:
        # one all-reduce of the flat gradient buffer (weighted by view share)
        # before the optimiser/SGLD step; same seed on every replica
        from paper_2409_07759_b300 import dp
        reducer = dp.GradientReducer(len(views), dp.total_views(len(views), device="cuda"))
    tr = WindowTrainer(r, state, views, tgt_dev, seed=1234, reduce=reducer,
                       keep_images=not args.no_images)
    # the streamed slices: 6,000-slot slices of the initial state. The timed
    # step takes them resident in HBM (its inputs are on the device); the end
    # to end step streams them from pinned host memory.
    S = 6000
    n_slices = scene.n // S
    dev_slices, host_slices = [], []
    for s in range(n_slices):
        sub = api.GaussianState(*[getattr(state, k)[s * S:(s + 1) * S].clone() for k in
                                  ("means", "log_scales", "quats", "opacity_logits", "sh",
                                   "start", "expire", "birth", "frozen")], sh_degree=3)
        dev_slices.append(sub)
        host_slices.append(sub.pin_host())
    slice_bytes = sum(t.numel() * t.element_size() for t in host_slices[0].values())

    def upd(k):
        s = k % n_slices
        return (s * S, dev_slices[s])

    def upd_host(k):
        s = k % n_slices
        return (s * S, host_slices[s])

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    for k in range(args.warmup):
        tr.step(k, update=upd(k))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # ---- timed region: the batched fwd+bwd window step ----
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    r.profile(True)
    r.profile_read(reset=True)
    launches0 = api.Renderer.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record()
        tr.step(args.warmup + k, update=upd(args.warmup + k))
        ev[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    tr.settle()
    launches = api.Renderer.kernel_launches() - launches0
    prof = r.profile_read(reset=True)
    r.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps * mpix / (ms / 1e3)

    # pair counts of this workload (one untimed forward with the counting blend)
    rc = api.Renderer(tile=(tw, th), batch=args.batch, pixels_per_thread=args.ppt,
                      bwd_pixels_per_thread=args.bwd_ppt, bwd_batch=args.bwd_batch,
                      count_pairs=True)
    _, saved = rc.render(state, views, keep_saved=True)
    info = saved.info()
    from paper_2409_07759_b300 import _abi
    pairs_fwd = int(info.pairs)
    pairs_bwd = int(saved.export(_abi.EXPORT_LAST).astype(np.int64).sum())
    n_keys, n_rec = int(info.n_keys), int(info.n_records)
    n_sort_keys, n_supers = int(info.n_sort_keys), int(info.n_supers)
    saved.release()
    rc.close()

    extra = {}
    # ---- forward only, batched ----
    torch.cuda.synchronize()
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        fe[k][0].record()
        tr.step(0, render_only=True)
        fe[k][1].record()
    torch.cuda.synchronize()
    fwd_ms = sum(a.elapsed_time(b) for a, b in fe) / args.steps
    extra["fwd_batched_mpix_s"] = mpix / (fwd_ms / 1e3)
    extra["step_batched_ms"] = ms / args.steps

    # ---- plain per-view path (one view per launch sequence) ----
    if not args.no_plain and args.plain_steps > 0:
        tr.batched = False
        tr.step(0)
        torch.cuda.synchronize()
        pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.plain_steps)]
        for k in range(args.plain_steps):
            flush.fill_(float(k))
            pe[k][0].record()
            tr.step(10_000 + k, update=upd(k))
            pe[k][1].record()
        torch.cuda.synchronize()
        pms = sum(a.elapsed_time(b) for a, b in pe) / args.plain_steps
        for k in range(args.plain_steps):
            flush.fill_(float(k))
            pe[k][0].record()
            tr.step(0, render_only=True)
            pe[k][1].record()
        torch.cuda.synchronize()
        pfms = sum(a.elapsed_time(b) for a, b in pe) / args.plain_steps
        tr.batched = True
        extra["plain_mpix_s"] = mpix / (pms / 1e3)
        extra["fwd_plain_mpix_s"] = mpix / (pfms / 1e3)
        extra["batched_over_plain"] = (ms / args.steps) and (pms / (ms / args.steps))

    # ---- end to end through the public API with host buffers ----
    # Every step's targets and slice are copied from pinned host memory (on a
    # side stream, issued once the step before has been issued, so the copies
    # overlap its blends; the slice lands in a device staging buffer that the
    # step writes into the slot buffer), and its loss is copied back to pinned
    # host memory and read by the host once the next step has been issued (so
    # the device does not wait for the host between steps).
    h2d = sum(t.numel() * t.element_size() for t in tgt_host) + slice_bytes
    loss_host = [torch.zeros(1, dtype=torch.float32).pin_memory() for _ in range(2)]
    loss_ev = [torch.cuda.Event(), torch.cuda.Event()]
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr.prefetch_targets(tgt_host, upd_host(0))
    for k in range(args.steps):
        loss = tr.step(20_000 + k, prefetched=True)
        loss_host[k % 2].copy_(loss, non_blocking=True)
        loss_ev[k % 2].record()
        if k + 1 < args.steps:
            tr.prefetch_targets(tgt_host, upd_host(k + 1))
        if k > 0:  # the previous step's loss, on the host
            loss_ev[(k - 1) % 2].synchronize()
            losses.append(float(loss_host[(k - 1) % 2].item()))
    loss_ev[(args.steps - 1) % 2].synchronize()
    losses.append(float(loss_host[(args.steps - 1) % 2].item()))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * args.steps * mpix / e2e_s, "unit": "Mpix/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4}

    # ---- roofline of the dominant kernel ----
    steps = args.steps
    alu_peak = fp32["tflops"]
    # the list sort orders (super tile, record) keys: ceil(bits / 9) digit passes
    sort_passes = math.ceil(math.ceil(math.log2(max(2, n_supers))) / 9)
    stage_cost = {
        "blend_fwd": ("alu", FLOP_PER_PAIR_FWD * pairs_fwd / 1e12, "TFLOP/s"),
        "blend_bwd": ("alu", FLOP_PER_PAIR_BWD * pairs_bwd / 1e12, "TFLOP/s"),
        # per digit pass: read + write key and value (16 B); once: the digit
        # counts' read of the keys (4 B)
        "tile_sort": ("hbm", (16.0 * sort_passes + 4.0) * n_sort_keys / 1e9, "GB/s"),
        "depth_sort": ("hbm", (16.0 * 4 + 4.0) * n_rec / 1e9, "GB/s"),
        # super keys written, record rectangles and row runs read
        "emit": ("hbm", (8.0 * n_sort_keys + 80.0 * n_rec) / 1e9, "GB/s"),
        # super ranges (4 B/key), count pass (4 B/key), write pass (8 B/key
        # read, 4 B per tile-list entry written)
        "ranges": ("hbm", (16.0 * n_sort_keys + 4.0 * n_keys) / 1e9, "GB/s"),
        "preprocess": ("hbm", (236.0 * n_rec / args.views + 64.0 * n_rec) / 1e9, "GB/s"),
        "preprocess_bwd": ("hbm", (236.0 * 2 * n_rec / args.views + 48.0 * n_rec) / 1e9, "GB/s"),
    }
    stages = {}
    for name, (tot_ms, calls) in prof.items():
        if calls == 0:
            continue
        per = tot_ms / steps
        s = {"ms_per_step": per, "share": tot_ms / ms if ms else None}
        if name in stage_cost:
            bound, amount, unit = stage_cost[name]
            ach = amount / (per / 1e3)
            peak = alu_peak if bound == "alu" else hbm_peak
            s.update(bound=bound, achieved=ach, unit=unit, frac=ach / peak)
        stages[name] = s
    dom = max(stages, key=lambda n: stages[n]["ms_per_step"])
    d = stages[dom]
    if dom == "blend_bwd":
        shape = f"{args.tile}/b{args.bwd_batch}/ppt{args.bwd_ppt}"
    else:
        shape = f"{args.tile}/b{args.batch}/ppt{args.ppt}"
    traffic = captured_traffic(dom, shape)
    if "bound" in d:
        roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"],
                "peak": alu_peak if d["bound"] == "alu" else hbm_peak, "unit": d["unit"],
                "frac": d["frac"], "traffic": traffic,
                "peak_source": (f"measured: FP32 probe ({fp32['form']}, "
                                f"{fp32['blocks']} blocks x 256 threads, CUDA events)"
                                if d["bound"] == "alu" else f"{hbm_src} copy bandwidth")}
        if d["bound"] == "alu":
            own = OWN_FLOP_PER_PAIR_BWD if dom == "blend_bwd" else OWN_FLOP_PER_PAIR_FWD
            roof["flop_per_pair"] = (FLOP_PER_PAIR_BWD if dom == "blend_bwd"
                                     else FLOP_PER_PAIR_FWD)
            roof["own_count"] = {"flop_per_pair": own, "achieved": d["achieved"] * own /
                                 roof["flop_per_pair"],
                                 "frac": d["frac"] * own / roof["flop_per_pair"]}
    else:
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None}
    extra["fp32_peak"] = fp32

    if not args.no_serving:
        torch.cuda.synchronize()
        extra["mature"] = mature_leg(state)
        torch.cuda.synchronize()
        # the codec on the scene as generated (training moves opacities toward 0)
        extra["codec"] = codec_leg(api.GaussianState.from_scene(scene), views)
        torch.cuda.synchronize()
        extra["memory_invariance"] = memory_leg()
        torch.cuda.synchronize()
        extra["serving"] = serving_leg(args)
    if not args.no_config3:
        torch.cuda.synchronize()
        extra["config3_batched_fwd"] = config3_leg(args)

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_sample(scene, views, oracle_targets, budget_s=15.0)
        cpu = {"value": rate, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
               "sample": sample}
        # the plain single-threaded oracle on one view of the same workload
        rate1, cores1, sample1 = cpu_oracle_sample(scene, views, oracle_targets, budget_s=1.0,
                                                   max_views=1, threads=1)
        cpu["single_thread"] = {"value": rate1, "unit": "Mpix/s", "cores": cores1,
                                "sample": sample1}

    if rank == 0:
        line = {
            "metric": "Mpix/s fwd+bwd (sliding-window training step)",
            "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene shaped like DyNeRF multi-view clips)",
            "config": arm_config(args, views, world),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "pairs_fwd": pairs_fwd, "pairs_bwd": pairs_bwd, "keys": n_keys, "records": n_rec,
            "sort_keys": n_sort_keys, "super_tiles": n_supers,
            "stages": stages,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    r.close()


if __name__ == "__main__":
    main()
