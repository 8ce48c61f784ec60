"""Continuous-batching playback server over a resident sliding-window model
(Alg. 2: render_thread renders the current frame continuously while
update_thread swaps in one slice per frame at the video frame rate).

Many viewers send render requests (pose, resolution) for the current frame.
Requests that arrive while others are on the GPU are admitted as soon as a
worker stream frees up and the device memory they need fits in the HBM budget
next to the batches already in flight (one byte counter over all workers),
and are rendered together in one batched call; several worker streams keep
batches overlapping on the device. Each image is delivered to pinned host
memory, and a request's latency runs from its arrival to the end of that
copy. The slot buffer stays on the GPU; each video frame, the slice
(frame mod swin_size) is overwritten from pinned host memory on its own stream
(Alg. 2 update_thread). CUDA events order every slice update after the
renders already submitted (they read the old slice) and before the renders
submitted later (they see the new one).

Everything here is host-side scheduling; all GPU work is libswgs calls.
"""
from __future__ import annotations

import gc
import math
import queue
import sys
import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import _abi, api, synth

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
    rendered: float = -1.0    # the batch's render finished on the device
    done: float = -1.0        # the image is in host memory

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


class _SharedLock:
    """Shared holders (batch submissions, which may wait for their own stream
    while the library sizes a batch) or one exclusive holder (a slice update);
    a waiting exclusive request lets no new shared holder in."""

    def __init__(self):
        self._c = threading.Condition()
        self._shared = 0
        self._excl = False
        self._excl_waiting = 0

    def acquire_shared(self):
        with self._c:
            while self._excl or self._excl_waiting:
                self._c.wait()
            self._shared += 1

    def release_shared(self):
        with self._c:
            self._shared -= 1
            if self._shared == 0:
                self._c.notify_all()

    def acquire_exclusive(self):
        with self._c:
            self._excl_waiting += 1
            while self._excl or self._shared:
                self._c.wait()
            self._excl_waiting -= 1
            self._excl = True

    def release_exclusive(self):
        with self._c:
            self._excl = False
            self._c.notify_all()


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
    p50_render_ms: float = 0.0     # arrival -> render finished (before delivery)
    p99_render_ms: float = 0.0
    inflight_hwm_bytes: float = 0.0  # largest admitted in-flight bytes
    budget_bytes: float = 0.0
    rerenders: int = 0             # batches rendered again (deferred sizing overflow)
    latencies_ms: np.ndarray = field(repr=False, default=None)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms", None)
        return d


@dataclass
class _Submitted:
    """A batch on the device: its host images (filled by the delivery copies),
    the events after its render and after its delivery, and its sizes."""
    reqs: List[Request]
    hosts: List[torch.Tensor]
    ev_render: torch.cuda.Event
    ev_copy: torch.cuda.Event
    saved: object             # the forward's saved state, released by finish()
    px: int
    w: int = 0
    slot: int = 0
    info: object = None       # its sizes, read by finish()


class ServingLoop:
    """Continuous batching over `n_streams` worker streams (one libswgs context
    each, with its own delivery stream) plus one update stream.

    A worker admits a batch, submits its render and the copies of its images
    to pinned host memory, and goes on to admit the next batch; a completion
    thread per worker waits for each batch's events, stamps its requests and
    releases its bytes. Each worker has n_slots output slots: with two, one
    batch can render while the previous one is being delivered. Images are
    delivered as 8-bit RGB (the display format), a quarter of the float
    image's bytes."""

    def __init__(self, state: api.GaussianState, swin_size: int, fps: float = 30.0,
                 n_streams: int = 2, max_batch: int = 16, hbm_budget_bytes: float = 16e9,
                 slice_provider=None, tile=(16, 16), batch=64, pixels_per_thread=4,
                 first_frame: int = 0, n_slots: int = 1, deferred_sizing: bool = False):
        self.state = state
        self.n_slots = n_slots   # batches a worker may have in flight
        self.swin = swin_size
        self.fps = fps
        self.max_batch = max_batch
        self.budget = hbm_budget_bytes
        self.slice_provider = slice_provider
        self.frame = first_frame
        # deferred sizing: after a worker's first batch its renders never
        # wait for the device; each batch's status is read once it is delivered
        self.renderers = [api.Renderer(tile=tile, batch=batch,
                                       pixels_per_thread=pixels_per_thread,
                                       deferred_sizing=deferred_sizing)
                          for _ in range(n_streams)]
        self.rerenders = 0
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.copy_streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.upd_renderer = api.Renderer()
        self.upd_stream = torch.cuda.Stream()
        # submissions hold it shared (they run concurrently, each on its own
        # context and stream), a slice update exclusively: a render reads
        # either the old slice or the new one, never a mix
        self.submit_lock = _SharedLock()
        self.last_render_ev = [None] * n_streams
        self.update_ev: Optional[torch.cuda.Event] = None
        # Device bytes of one request: view_bytes (its records: one per active
        # Gaussian) + px_bytes per pixel (tile keys, tile lists and ranges, T,
        # last). Both are re-measured from every batch's reported sizes
        # (swgs_saved_info.device_bytes / record_bytes); these first values are
        # replaced by reserve()'s probe.
        self.view_bytes = 152.0 * state.n
        self.px_bytes = 8.0 + 20.0 * 4.0
        self.inflight = 0.0      # admitted bytes of the batches on the device
        self.inflight_hwm = 0.0
        # filled by reserve(): per worker and slot, max_batch 8-bit output
        # images on the device and their pinned host delivery buffers
        self.out_pool: List[List[List[torch.Tensor]]] = []
        self.host_pool: List[List[torch.Tensor]] = []
        self.pool_px = 0

    # -- memory model for admission ---------------------------------------------
    def request_bytes(self, r: Request) -> float:
        return self.view_bytes + self.px_bytes * r.width * r.height

    def _measure(self, info, px: int):
        """Re-estimate the per-view and per-pixel bytes from a batch's sizes."""
        if info.n_views <= 0 or px <= 0:
            return
        vb = info.record_bytes / info.n_views
        pb = (info.device_bytes - info.record_bytes) / px
        self.view_bytes = 0.7 * self.view_bytes + 0.3 * vb
        self.px_bytes = 0.7 * self.px_bytes + 0.3 * pb

    def reserve(self, width: int, height: int):
        """Grow every worker's scratch to the largest batch the admission rule
        lets through at width x height (max_batch requests within the HBM
        budget), give each worker its output images and pinned host delivery
        buffers, and measure the per-request bytes from a probe, so that no
        allocation happens while serving: a batch larger than any seen before
        would otherwise grow the scratch mid-run and stall every request queued
        behind it."""
        R, t = orbit_pose(np.array([0.0, 0.0, 1.0]), 0.0, 0.0, 0.0)
        probe = Request(rid=-1, viewer=-1, arrival=0.0, width=width, height=height, R=R, t=t)
        fx, fy, cx, cy = synth.intrinsics_for(width, height)
        view = synth.View(width, height, fx, fy, cx, cy, probe.R, probe.t, self.frame)
        # measure one request first, then size the batch the budget admits
        _, saved = self.renderers[0].render(self.state, [view], keep_saved=True,
                                            stream=self.streams[0])
        info = saved.info()
        self.view_bytes = float(info.record_bytes)
        self.px_bytes = (info.device_bytes - info.record_bytes) / (width * height)
        saved.release()
        self.streams[0].synchronize()
        n, used = 0, 0.0
        while n < self.max_batch and (n == 0 or used + self.request_bytes(probe) <= self.budget):
            used += self.request_bytes(probe)
            n += 1
        views = [view] * n
        self.out_pool, self.host_pool = [], []
        self.pool_px = width * height
        for w, s in enumerate(self.streams):
            with torch.cuda.stream(s):
                self.out_pool.append([[torch.empty(3 * self.pool_px, dtype=torch.uint8,
                                                   device="cuda")
                                       for _ in range(self.max_batch)]
                                      for _ in range(self.n_slots)])
                self.renderers[w].render_rgb8(self.state, views, stream=s)
            self.host_pool.append([torch.empty((self.max_batch, 3 * self.pool_px),
                                               dtype=torch.uint8).pin_memory()
                                   for _ in range(self.n_slots)])
            s.synchronize()

    # -- Alg. 2 update_thread ---------------------------------------------------
    def apply_update(self, frame: int):
        """Swap in the slice of `frame` and make it the current frame. Renders
        already submitted read the old slice; renders submitted later wait for
        the copy."""
        host = self.slice_provider(frame)
        first, count = api.slice_range(frame, self.swin, self.state.n)
        self.submit_lock.acquire_exclusive()
        try:
            for ev in self.last_render_ev:
                if ev is not None:
                    self.upd_stream.wait_event(ev)
            self.upd_renderer.frame_update(self.state, first, host, src_on_host=True,
                                           stream=self.upd_stream)
            ev = torch.cuda.Event()
            ev.record(self.upd_stream)
            self.update_ev = ev
            self.frame = frame
        finally:
            self.submit_lock.release_exclusive()

    # -- one batch on one worker stream -----------------------------------------
    def submit_batch(self, w: int, reqs: List[Request], t0: float, slot: int = 0) -> _Submitted:
        """Submit the render of `reqs` together on worker stream w at the
        current frame into output slot `slot`, and the copies of the images to
        pinned host memory on the worker's delivery stream; returns without
        waiting for either."""
        s = self.streams[w]
        pool = self.out_pool[w][slot] if self.out_pool else None
        pooled = pool is not None and len(reqs) <= len(pool) and \
            all(r.width * r.height <= self.pool_px for r in reqs)
        if pooled:
            # views of the worker's reserved buffers: no allocation while serving
            outs = [pool[i][:3 * r.width * r.height].view(r.height, r.width, 3)
                    for i, r in enumerate(reqs)]
            hosts = [self.host_pool[w][slot][i][:3 * r.width * r.height]
                     .view(r.height, r.width, 3) for i, r in enumerate(reqs)]
        else:
            with torch.cuda.stream(s):
                outs = [torch.empty((r.height, r.width, 3), dtype=torch.uint8, device="cuda")
                        for r in reqs]
            hosts = [torch.empty((r.height, r.width, 3), dtype=torch.uint8).pin_memory()
                     for r in reqs]
        self.submit_lock.acquire_shared()
        try:
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
            _, saved = self.renderers[w].render_rgb8(self.state, views, out=outs,
                                                     keep_saved=True, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            self.last_render_ev[w] = ev
        finally:
            self.submit_lock.release_shared()
        # delivery on the worker's copy stream, after the render
        cs = self.copy_streams[w]
        cs.wait_event(ev)
        with torch.cuda.stream(cs):
            for h, o in zip(hosts, outs):
                h.copy_(o, non_blocking=True)
            dev = torch.cuda.Event()
            dev.record(cs)
        if not pooled:
            # the unpooled images must outlive the copies
            for o in outs:
                o.record_stream(cs)
        return _Submitted(reqs, hosts, ev, dev, saved, sum(r.width * r.height for r in reqs),
                          w, slot)

    def finish(self, b: _Submitted, t0: float):
        """Wait for a submitted batch: stamp its requests when the render ends
        and when its images are in host memory. A batch that outgrew the
        deferred capacities (rare: the first batches of new sizes) rendered
        background; it is rendered and delivered again, and its requests are
        stamped when that copy is done."""
        b.ev_render.synchronize()
        rendered = time.perf_counter() - t0
        b.ev_copy.synchronize()
        st = b.saved.status(wait=True)
        if st == _abi.SWGS_EDEVICE:
            b.saved.release()
            self.rerenders += 1
            again = self.submit_batch(b.w, b.reqs, t0, b.slot)
            self.finish(again, t0)
            b.info, b.hosts = again.info, again.hosts
            return
        if st != _abi.SWGS_OK:
            raise _abi.SwgsError(st, "serving batch failed on the device")
        b.info = b.saved.info()
        b.saved.release()
        done = time.perf_counter() - t0
        for r in b.reqs:
            r.rendered = rendered
            r.done = done

    def render_batch(self, w: int, reqs: List[Request], t0: float, slot: int = 0):
        """Render and deliver `reqs` on worker w and wait for them; returns
        (host images: uint8 [H,W,3], batch sizes, pixels)."""
        b = self.submit_batch(w, reqs, t0, slot)
        self.finish(b, t0)
        return b.hosts, b.info, b.px

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
        self.inflight, self.inflight_hwm = 0.0, 0.0
        rerenders0 = self.rerenders
        pending = deque()
        todo = deque(requests)
        lock = threading.Lock()
        stop = threading.Event()
        cond = threading.Condition(lock)
        on_device = [0]   # batches submitted and not yet delivered
        batches = []
        images = {}
        t0 = time.perf_counter()
        n_updates = [0]

        def admit():
            """Take the longest run of pending requests (at most max_batch) whose
            bytes fit in the budget next to the batches in flight; a request
            that alone exceeds the budget is admitted only onto an idle device.
            Called with the lock held; returns (batch, bytes)."""
            batch, used = [], 0.0
            while pending and len(batch) < self.max_batch:
                need = self.request_bytes(pending[0])
                if self.inflight + used + need > self.budget and \
                        (batch or self.inflight > 0.0):
                    break
                used += need
                batch.append(pending.popleft())
            return batch, used

        def completer(q, slots):
            while True:
                item = q.get()
                if item is None:
                    return
                b, used = item
                self.finish(b, t0)
                if keep_images:
                    for r, o in zip(b.reqs, b.hosts):
                        images[r.rid] = o.clone()
                with cond:
                    self.inflight -= used
                    self._measure(b.info, b.px)
                    batches.append(len(b.reqs))
                    on_device[0] -= 1
                    cond.notify_all()
                slots.release()

        def worker(w):
            q = queue.Queue()
            slots = threading.Semaphore(self.n_slots)
            done_th = threading.Thread(target=completer, args=(q, slots), daemon=True)
            done_th.start()
            slot = 0
            while True:
                slots.acquire()
                with cond:
                    while True:
                        if stop.is_set() and not pending:
                            q.put(None)
                            done_th.join()
                            return
                        batch, used = admit() if pending else ([], 0.0)
                        if batch:
                            break
                        cond.wait(0.0005)
                    self.inflight += used
                    self.inflight_hwm = max(self.inflight_hwm, self.inflight)
                    on_device[0] += 1
                q.put((self.submit_batch(w, batch, t0, slot), used))
                slot = (slot + 1) % self.n_slots

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
                finished = not todo and not pending and on_device[0] == 0
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
        rlat = np.array([(r.rendered - r.arrival) * 1e3 for r in requests if r.done >= 0])
        px = sum(r.width * r.height for r in requests if r.done >= 0)
        stats = ServeStats(n=len(lat), p50_ms=float(np.percentile(lat, 50)),
                           p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
                           mpix_per_s=px / 1e6 / wall, batches=len(batches),
                           mean_batch=float(np.mean(batches)) if batches else 0.0,
                           updates=n_updates[0], wall_s=wall,
                           p50_render_ms=float(np.percentile(rlat, 50)),
                           p99_render_ms=float(np.percentile(rlat, 99)),
                           inflight_hwm_bytes=float(self.inflight_hwm),
                           budget_bytes=float(self.budget),
                           rerenders=self.rerenders - rerenders0, latencies_ms=lat)
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
        r.render_rgb8(state, [v], batched=False)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
        px += q.width * q.height
    if renderer is None:
        r.close()
    ms = float(np.median(times))
    return {"median_ms_per_request": ms, "mpix_per_s": px / 1e6 / (sum(times) / 1e3)}
