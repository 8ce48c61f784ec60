"""Continuous-batching playback server over a resident sliding-window model
(Alg. 2: render_thread renders the current frame continuously while
update_thread swaps in one slice per frame at the video frame rate).

Many viewers send render requests (pose, resolution) for the current frame.
Requests that arrive while others are on the GPU are admitted as soon as a
worker stream frees up and the HBM budget allows, and are rendered together in
one batched call; several worker streams keep batches overlapping on the
device. The slot buffer stays on the GPU; each video frame, the slice
(frame mod swin_size) is overwritten from pinned host memory on its own stream
(Alg. 2 update_thread). CUDA events order every slice update after the
renders already submitted (they read the old slice) and before the renders
submitted later (they see the new one).

Everything here is host-side scheduling; all GPU work is libswgs calls.
"""
from __future__ import annotations

import gc
import math
import sys
import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import api, synth

RESOLUTIONS = [(640, 480), (1280, 720), (1280, 720), (1920, 1080)]  # 1:2:1


@dataclass
class Request:
    rid: int
    viewer: int
    arrival: float            # seconds from the start of the run
    width: int
    height: int
    R: np.ndarray
    t: np.ndarray
    frame: int = -1           # assigned when the request is submitted
    submit: float = -1.0
    done: float = -1.0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def orbit_pose(axis: np.ndarray, phase: float, speed: float, t: float, radius: float = 4.0):
    """Camera on a great circle of the radius-`radius` sphere, looking at the origin."""
    axis = axis / np.linalg.norm(axis)
    ref = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(axis, ref)
    u /= np.linalg.norm(u)
    w = np.cross(axis, u)
    a = phase + speed * t
    eye = radius * (math.cos(a) * u + math.sin(a) * w)
    return synth.look_at(eye)


def make_requests(n_viewers: int, rate_hz: float, duration_s: float, seed: int = 4,
                  resolutions=None) -> List[Request]:
    """Poisson arrivals (rate_hz per viewer) of viewers orbiting the scene."""
    rng = np.random.default_rng(seed)
    res = resolutions or RESOLUTIONS
    reqs = []
    for v in range(n_viewers):
        axis = rng.normal(size=3)
        phase, speed = rng.uniform(0, 2 * math.pi), rng.uniform(0.2, 1.0)
        w, h = res[v % len(res)]
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            R, tt = orbit_pose(axis, phase, speed, t)
            reqs.append(Request(0, v, t, w, h, R, tt))
            t += rng.exponential(1.0 / rate_hz)
    reqs.sort(key=lambda r: r.arrival)
    for i, r in enumerate(reqs):
        r.rid = i
    return reqs


@dataclass
class ServeStats:
    n: int
    p50_ms: float
    p99_ms: float
    mean_ms: float
    mpix_per_s: float
    batches: int
    mean_batch: float
    updates: int
    wall_s: float
    latencies_ms: np.ndarray = field(repr=False, default=None)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms", None)
        return d


class ServingLoop:
    """Continuous batching over `n_streams` worker streams (one libswgs context
    each) plus one update stream."""

    def __init__(self, state: api.GaussianState, swin_size: int, fps: float = 30.0,
                 n_streams: int = 2, max_batch: int = 16, hbm_budget_bytes: float = 16e9,
                 slice_provider=None, tile=(16, 16), batch=64, pixels_per_thread=4,
                 first_frame: int = 0):
        self.state = state
        self.swin = swin_size
        self.fps = fps
        self.max_batch = max_batch
        self.budget = hbm_budget_bytes
        self.slice_provider = slice_provider
        self.frame = first_frame
        self.renderers = [api.Renderer(tile=tile, batch=batch,
                                       pixels_per_thread=pixels_per_thread)
                          for _ in range(n_streams)]
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.upd_renderer = api.Renderer()
        self.upd_stream = torch.cuda.Stream()
        self.submit_lock = threading.Lock()
        self.last_render_ev = [None] * n_streams
        self.update_ev: Optional[torch.cuda.Event] = None
        # bytes per pixel of one request's device footprint (image, final T,
        # last index, sort keys), refined from the key counts observed
        self.bytes_per_px = 12 + 8 + 16 * 8.0
        self.rec_bytes = 96.0 * state.n
        self.out_pool: List[List[torch.Tensor]] = []   # filled by reserve()
        self.pool_px = 0

    # -- memory model for admission ---------------------------------------------
    def request_bytes(self, r: Request) -> float:
        return self.bytes_per_px * r.width * r.height + self.rec_bytes

    def reserve(self, width: int, height: int):
        """Grow every worker's scratch to the largest batch the admission rule
        lets through at width x height (max_batch requests within the HBM
        budget), so that no device allocation happens while serving: a batch
        larger than any seen before would otherwise grow the scratch mid-run
        and stall every request queued behind it."""
        R, t = orbit_pose(np.array([0.0, 0.0, 1.0]), 0.0, 0.0, 0.0)
        probe = Request(rid=-1, viewer=-1, arrival=0.0, width=width, height=height, R=R, t=t)
        n, used = 0, 0.0
        while n < self.max_batch and (n == 0 or used + self.request_bytes(probe) <= self.budget):
            used += self.request_bytes(probe)
            n += 1
        fx, fy, cx, cy = synth.intrinsics_for(width, height)
        views = [synth.View(width, height, fx, fy, cx, cy, probe.R, probe.t, self.frame)] * n
        self.out_pool = []
        self.pool_px = width * height
        for w, s in enumerate(self.streams):
            with torch.cuda.stream(s):
                # the worker's output images: max_batch planar buffers of this size
                self.out_pool.append([torch.empty(3 * self.pool_px, dtype=torch.float32,
                                                  device="cuda") for _ in range(self.max_batch)])
                self.renderers[w].render(self.state, views, stream=s)
            s.synchronize()

    # -- Alg. 2 update_thread ---------------------------------------------------
    def apply_update(self, frame: int):
        """Swap in the slice of `frame` and make it the current frame. Renders
        already submitted read the old slice; renders submitted later wait for
        the copy."""
        host = self.slice_provider(frame)
        first, count = api.slice_range(frame, self.swin, self.state.n)
        with self.submit_lock:
            for ev in self.last_render_ev:
                if ev is not None:
                    self.upd_stream.wait_event(ev)
            self.upd_renderer.frame_update(self.state, first, host, src_on_host=True,
                                           stream=self.upd_stream)
            ev = torch.cuda.Event()
            ev.record(self.upd_stream)
            self.update_ev = ev
            self.frame = frame

    # -- one batch on one worker stream -----------------------------------------
    def render_batch(self, w: int, reqs: List[Request], t0: float):
        """Render `reqs` together on worker stream w at the current frame."""
        s = self.streams[w]
        pool = self.out_pool[w] if self.out_pool else None
        if pool is not None and len(reqs) <= len(pool) and \
                all(r.width * r.height <= self.pool_px for r in reqs):
            # views of the worker's reserved buffers: no allocation while serving
            outs = [pool[i][:3 * r.width * r.height].view(3, r.height, r.width)
                    for i, r in enumerate(reqs)]
        else:
            with torch.cuda.stream(s):
                outs = [torch.empty((3, r.height, r.width), dtype=torch.float32, device="cuda")
                        for r in reqs]
        with self.submit_lock:
            frame = self.frame
            views = []
            for r in reqs:
                fx, fy, cx, cy = synth.intrinsics_for(r.width, r.height)
                views.append(synth.View(r.width, r.height, fx, fy, cx, cy, r.R, r.t, frame))
            if self.update_ev is not None:
                s.wait_event(self.update_ev)
            now = time.perf_counter() - t0
            for r in reqs:
                r.frame, r.submit = frame, now
            _, saved = self.renderers[w].render(self.state, views, out=outs, keep_saved=True,
                                                stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            self.last_render_ev[w] = ev
        info = saved.info()
        saved.release()
        px = sum(r.width * r.height for r in reqs)
        if px:
            kpp = info.n_keys / px
            self.bytes_per_px = 0.8 * self.bytes_per_px + 0.2 * (20 + 16 * kpp)
        ev.synchronize()
        done = time.perf_counter() - t0
        for r in reqs:
            r.done = done
        return outs

    def run(self, requests: List[Request], duration_s: float, keep_images=False):
        """Serve `requests` (arrival times relative to the start) in real time
        for duration_s seconds of arrivals, then drain. Returns ServeStats.
        Python's cyclic garbage collector is held off while serving (a full
        collection of a large heap pauses every thread for tens of ms) and the
        interpreter's thread switch interval is shortened; both are restored
        afterwards."""
        gc_on = gc.isenabled()
        gc.collect()
        gc.disable()
        # the workers and the arrival loop share the GIL: hand it over every
        # 0.5 ms instead of every 5 ms while serving
        switch = sys.getswitchinterval()
        sys.setswitchinterval(min(switch, 0.0005))
        try:
            return self._run(requests, duration_s, keep_images)
        finally:
            sys.setswitchinterval(switch)
            if gc_on:
                gc.enable()

    def _run(self, requests: List[Request], duration_s: float, keep_images=False):
        pending = deque()
        todo = deque(requests)
        lock = threading.Lock()
        stop = threading.Event()
        free = [True] * len(self.streams)
        cond = threading.Condition(lock)
        batches = []
        images = {}
        t0 = time.perf_counter()
        n_updates = [0]

        def worker(w):
            while True:
                with cond:
                    while not stop.is_set() and not pending:
                        cond.wait(0.0005)
                    if stop.is_set() and not pending:
                        return
                    batch, used = [], 0.0
                    while pending and len(batch) < self.max_batch:
                        need = self.request_bytes(pending[0])
                        if batch and used + need > self.budget:
                            break
                        used += need
                        batch.append(pending.popleft())
                    free[w] = False
                outs = self.render_batch(w, batch, t0)
                if keep_images:
                    for r, o in zip(batch, outs):
                        images[r.rid] = o.clone() if self.out_pool else o
                with cond:
                    batches.append(len(batch))
                    free[w] = True
                    cond.notify_all()

        threads = [threading.Thread(target=worker, args=(w,), daemon=True)
                   for w in range(len(self.streams))]
        for th in threads:
            th.start()
        next_frame_t = 1.0 / self.fps
        while True:
            now = time.perf_counter() - t0
            if now >= next_frame_t and now < duration_s:
                self.apply_update(self.frame + 1)
                n_updates[0] += 1
                next_frame_t += 1.0 / self.fps
            moved = False
            with cond:
                while todo and todo[0].arrival <= now:
                    pending.append(todo.popleft())
                    moved = True
                if moved:
                    cond.notify_all()
                finished = not todo and not pending and all(free)
            if finished and now >= duration_s:
                break
            time.sleep(0.0002)
        stop.set()
        with cond:
            cond.notify_all()
        for th in threads:
            th.join()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lat = np.array([r.latency * 1e3 for r in requests if r.done >= 0])
        px = sum(r.width * r.height for r in requests if r.done >= 0)
        stats = ServeStats(n=len(lat), p50_ms=float(np.percentile(lat, 50)),
                           p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
                           mpix_per_s=px / 1e6 / wall, batches=len(batches),
                           mean_batch=float(np.mean(batches)) if batches else 0.0,
                           updates=n_updates[0], wall_s=wall, latencies_ms=lat)
        return (stats, images) if keep_images else stats

    def close(self):
        for r in self.renderers:
            r.close()
        self.upd_renderer.close()


def serial_rates(state: api.GaussianState, requests: List[Request], frame: int,
                 renderer: Optional[api.Renderer] = None, n: int = 50):
    """The plain method: one request per render call, one at a time (device time
    per request, median) -- the baseline the batched server is compared with."""
    r = renderer or api.Renderer()
    times, px = [], 0
    for q in requests[:n]:
        fx, fy, cx, cy = synth.intrinsics_for(q.width, q.height)
        v = synth.View(q.width, q.height, fx, fy, cx, cy, q.R, q.t, frame)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r.render(state, [v], batched=False)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
        px += q.width * q.height
    if renderer is None:
        r.close()
    ms = float(np.median(times))
    return {"median_ms_per_request": ms, "mpix_per_s": px / 1e6 / (sum(times) / 1e3)}
