"""The inner step of Alg. 1 (train_swin) over a whole sliding window at once:
every (frame, camera) view of the window is rendered forward and backward in
one batched pass, then the optimiser / SGLD noise / relocation step runs on
the Gaussians active in the window's frames. A per-frame slice replacement
(Alg. 2 update_thread) can be streamed in from pinned host memory first.

Every stage is one call into libswgs on the current torch stream.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import _abi, api

DEFAULT_SGLD = dict(lr_means=1.6e-4, lr_log_scales=5e-3, lr_quats=1e-3, lr_logits=5e-2,
                    lr_sh_dc=2.5e-3, lr_sh_rest=2.5e-3 / 20.0, beta1=0.9, beta2=0.999, eps=1e-15,
                    noise_lr=5e4, noise_k=100.0, noise_t=0.005, adam=1, relocate=1, max_n=51,
                    # Alg. 1 reg(): the regulariser weights of Sec. 8.1
                    opacity_reg=2e-2, scale_reg=1e-2,
                    # Sec. 4.5.1 means-gradient scale (1 = off); ClipTrainer sets the window
                    mean_grad_decay=1.0, window_start=0, swin_size=0,
                    # the optimiser step leaves the gradients zero for the next
                    # backward (no separate clearing pass)
                    clear_grads=1)


def _flat_views(n: int, K: int, device="cuda"):
    """One flat zero-filled buffer viewed as the five parameter-shaped arrays
    (one memset clears all of them)."""
    sizes = [n * 3, n * 3, n * 4, n, n * K * 3]
    flat = torch.zeros(sum(sizes), dtype=torch.float32, device=device)
    parts = torch.split(flat, sizes)
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]
    return flat, [p.view(s) for p, s in zip(parts, shapes)]


# the arrays of a streamed slice (GaussianState.pin_host's keys), in the
# GaussianState constructor's order
_SLICE_FIELDS = api.PARAM_NAMES + ("start", "expire", "birth", "frozen")


class WindowTrainer:
    """Holds the state, gradients, Adam moments and per-view buffers of one
    window and runs training steps on it."""

    def __init__(self, renderer: api.Renderer, state: api.GaussianState, views: Sequence,
                 targets: Sequence[torch.Tensor], params: Optional[dict] = None, seed: int = 0,
                 batched: bool = True, bg=(0.0, 0.0, 0.0), reduce=None,
                 keep_images: bool = True):
        self.r = renderer
        self.state = state
        self.views = list(views)
        self.targets = list(targets)
        self.frames = sorted({int(v.frame) for v in self.views})
        self.params = dict(DEFAULT_SGLD)
        if params:
            self.params.update(params)
        self.seed = seed
        self.batched = batched
        self.bg = bg
        # data parallel: called as reduce(flat_grads, loss) between the backward
        # and the optimiser step (see dp.GradientReducer)
        self.reduce = reduce
        K = (state.sh_degree + 1) ** 2
        self._gflat, g = _flat_views(state.n, K)
        self.grads = api.GaussianGrads(*g, state.sh_degree)
        self._mflat, m = _flat_views(state.n, K)
        self._vflat, v = _flat_views(state.n, K)
        names = ("means", "log_scales", "quats", "opacity_logits", "sh")
        self.adam = {}
        for k, a, b in zip(names, m, v):
            self.adam["m_" + k] = a
            self.adam["v_" + k] = b
        # the rendered images of the last step (keep_images = False: the L1 term
        # is fused into the forward, so a step needs no image written)
        self.keep_images = keep_images
        self.images = None
        if keep_images:
            self._alloc_images()
        # host-input pipeline: two target buffers, the back one filled on a side
        # stream while a step reads the front one
        self._bufs = None
        self._front = 0
        self._copy_stream = None
        self._copied = None      # event: the back buffer is filled
        self._released = None    # per buffer: the last step reading it has ended
        self._stage_bufs = [None, None]  # per buffer: device staging slice
        self._staged = [None, None]      # per buffer: (first slot, staged slice)
        self.dl = [torch.empty((3, vw.height, vw.width), dtype=torch.float32, device="cuda")
                   for vw in self.views]
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        # largest number of tile keys of any step so far (sizes the scratch)
        self.max_keys = 0
        self._rows = None  # data parallel: the eligible rows' exchange buffers
        # deferred sizing: the last step's forward, checked at the next step
        self._pending = None
        self.reruns = 0

    def set_window(self, views: Sequence, targets: Sequence[torch.Tensor]):
        """Move the trainer to another window's views and targets (buffers are
        reallocated only where a view's size changes)."""
        views = list(views)
        if len(views) != len(self.views) or any(
                (a.width, a.height) != (b.width, b.height) for a, b in zip(views, self.views)):
            self.dl = [torch.empty((3, v.height, v.width), dtype=torch.float32, device="cuda")
                       for v in views]
            self.images = None
            self._bufs = None
        self.views = views
        if self.keep_images and self.images is None:
            self._alloc_images()
        self.targets = list(targets)
        self.frames = sorted({int(v.frame) for v in views})

    def prefetch_targets(self, host_targets: Sequence[torch.Tensor], host_update=None):
        """Start copying the next step's targets from pinned host memory into a
        back buffer on a side stream, so that the copy overlaps the step in
        flight; the next step(..., prefetched=True) waits for it and uses it.
        host_update = (first_slot, pinned host dict): that step's slice is
        copied alongside into a device staging slice, which the step then
        writes into the slot buffer on the device."""
        if self._bufs is None:
            self._bufs = [self.targets, [torch.empty_like(t) for t in self.targets]]
            self._front = 0
            self._copy_stream = torch.cuda.Stream()
            self._copied = torch.cuda.Event()
            self._released = [torch.cuda.Event(), torch.cuda.Event()]
            for e in self._released:
                e.record()
        back = 1 - self._front
        with torch.cuda.stream(self._copy_stream):
            self._copy_stream.wait_event(self._released[back])
            for d, h in zip(self._bufs[back], host_targets):
                d.copy_(h, non_blocking=True)
            self._staged[back] = None
            if host_update is not None:
                first, host = host_update
                n = int(host["means"].shape[0])
                st = self._stage_bufs[back]
                if st is None or st.n != n:
                    st = api.GaussianState(*[torch.empty_like(host[k], device="cuda")
                                             for k in _SLICE_FIELDS],
                                           sh_degree=self.state.sh_degree)
                    self._stage_bufs[back] = st
                for k in _SLICE_FIELDS:
                    getattr(st, k).copy_(host[k], non_blocking=True)
                self._staged[back] = (int(first), st)
            self._copied.record(self._copy_stream)

    def settle(self):
        """With a deferred-sizing renderer: check the last step's forward (this
        waits until it has finished on the device, which the next step's
        launches do not need). A step whose batch outgrew the capacities
        changed nothing (its optimiser step was gated); it runs again now that
        the capacities have grown."""
        p, self._pending = self._pending, None
        if p is None:
            return
        saved, args = p
        st = saved.status(wait=True)
        self.max_keys = max(self.max_keys, int(saved.info().n_keys))
        saved.release()
        if st == _abi.SWGS_EDEVICE:
            self.reruns += 1
            self.step(*args)
            self.settle()
        elif st != _abi.SWGS_OK:
            raise _abi.SwgsError(st, "window step failed on the device")

    def _alloc_images(self):
        self.images = [torch.empty((3, vw.height, vw.width), dtype=torch.float32, device="cuda")
                       for vw in self.views]

    def step(self, step: int, update: Optional[tuple] = None, render_only: bool = False,
             prefetched: bool = False):
        """One training step. update = (first_slot, src) overwrites a slice
        before rendering: src a pinned host dict (GaussianState.pin_host, the
        form a streamed slice arrives in) or a GaussianState on the device;
        prefetched = True takes the targets (and the slice, if one was staged)
        from the last prefetch_targets call. Returns the (device) loss tensor."""
        self.settle()
        if prefetched:
            torch.cuda.current_stream().wait_event(self._copied)
            self._front = 1 - self._front
            self.targets = self._bufs[self._front]
            if self._staged[self._front] is not None:
                update = self._staged[self._front]
        if update is not None:
            first, src = update
            self.r.frame_update(self.state, first, src,
                                src_on_host=not isinstance(src, api.GaussianState))
        if render_only:
            if self.images is None:
                self._alloc_images()
            self.r.render(self.state, self.views, bg=self.bg, batched=self.batched,
                          out=self.images)
            return None
        # forward with the L1 term fused into the blend's epilogue
        _, _, _, saved = self.r.render_l1(self.state, self.views, self.targets, bg=self.bg,
                                          batched=self.batched,
                                          out=self.images if self.keep_images else False,
                                          dL_out=self.dl, loss_out=self.loss)
        if not self.params.get("clear_grads", 0):
            # the last step kept its gradients: clear them for this backward
            self._gflat.zero_()
        reg = None
        if self.params.get("opacity_reg", 0.0) or self.params.get("scale_reg", 0.0):
            reg = dict(opacity_reg=self.params["opacity_reg"],
                       scale_reg=self.params["scale_reg"])
        self.r.backward(self.state, saved, self.dl, self.grads, reg=reg, loss=self.loss)
        if self.r.cfg.deferred_sizing:
            # its counts are still on the device: check it at the next step
            self._pending = (saved, (step, update, False, False))
        else:
            self.max_keys = max(self.max_keys, int(saved.info().n_keys))
            saved.release()
        if self.reduce is not None:
            if self._rows is None:
                from . import dp
                self._rows = dp.RowExchange(self.r, self.state, self.grads, self.frames)
            self._rows.frames = self.frames
            self.reduce(self._gflat, self.loss, rows=self._rows)
        self.r.sgld_step(self.state, self.frames, self.params, self.seed, step,
                         grads=self.grads, adam=self.adam)
        if self._bufs is not None:
            self._released[self._front].record()
        return self.loss


class ClipTrainer:
    """Alg. 1 main over a clip: the first window [0, swin_size) trained from the
    initial Gaussians, schedule_expire, then for every window start st: mature
    (st) -- whose snapshot is the stream that Alg. 2 clients read -- and the
    window [st, st + swin_size) trained.

    The buffer holds gs in slots [0, num_gs) and the ring of matured rows in
    [num_gs, 2 num_gs) (GaussianState.with_matured_ring), so every render sees
    gs and matured together and only gs is optimised (the ring is frozen).
    Each iteration is one batched step over every view of the window's frames
    (the paper samples one frame per iteration).

    window(st, ed) -> (views, targets): the training views of frames [st, ed)
    and their target images (device tensors, float32 or uint8).
    Each maturation's rows go to sink(st, n, data): with codec = False, data is
    a dict of host tensors of the n rows as they were (stream.write); with
    codec = True, host uint8 packets of the slice codec (Table 6), one per
    slice of num_gs / swin_size rows (`keep` gives the Sec. 5.5 tail drop as a
    fraction of each slice's rows). The default sink
    appends (st, n, data) to self.stream. The snapshot and packet buffers are
    allocated once, so memory does not grow with the clip.
    """

    def __init__(self, renderer: api.Renderer, gs: api.GaussianState, swin_size: int,
                 window, iterations: int = 1, params: Optional[dict] = None, seed: int = 0,
                 codec: bool = False, keep: float = 1.0, sink=None):
        self.r = renderer
        self.num_gs = gs.n
        if self.num_gs % swin_size:
            raise ValueError("num_gs must be a multiple of swin_size")
        self.swin = swin_size
        self.buf = api.GaussianState.with_matured_ring(gs)
        self.window = window
        self.iterations = iterations
        self.head = 0
        self.step_count = 0
        views, targets = window(0, swin_size)
        self.trainer = WindowTrainer(renderer, self.buf, views, targets, params=params, seed=seed)
        self.codec = codec
        self.keep = keep
        self.stream = []   # [(st, n, data)] with the default sink
        self.sink = sink   # None: append to self.stream (no self-reference, no cycle)
        self._snap = api.GaussianState(
            *[torch.empty_like(getattr(self.buf, k)[:self.num_gs]) for k in
              api.PARAM_NAMES + ("start", "expire", "birth", "frozen")],
            sh_degree=self.buf.sh_degree)
        self._packet = None
        if codec:
            n = api.Renderer.slice_packet_bytes(self.num_gs, self.num_gs) + 16
            self._packet = torch.empty(n, dtype=torch.uint8).pin_memory()

    def _train(self, st: int):
        views, targets = self.window(st, st + self.swin)
        self.trainer.set_window(views, targets)
        self.trainer.params.update(window_start=st, swin_size=self.swin)
        loss = None
        for _ in range(self.iterations):
            loss = self.trainer.step(self.step_count)
            self.step_count += 1
        return loss

    def mature(self, st: int):
        n, self.head = self.r.mature(self.buf, self.num_gs, st, self.swin, self.head,
                                     snapshot=self._snap)
        if n == 0:
            self._emit(st, 0, None)
            return 0
        if self.codec:
            # one packet per slice (a slice's rows share their lifespan, Sec.
            # 4.2.1): the first full snapshot gives swin_size of them
            S = self.num_gs // self.swin
            for c0 in range(0, n, S):
                m = min(S, n - c0)
                keep = max(0, min(m, int(round(self.keep * m))))
                pkt = self.r.slice_encode(self._snap.rows(c0, c0 + m), m, keep, out=self._packet)
                torch.cuda.current_stream().synchronize()
                self._emit(st, m, pkt.clone())
        else:
            rows = {k: getattr(self._snap, k)[:n].cpu() for k in
                    api.PARAM_NAMES + ("start", "expire", "birth", "frozen")}
            self._emit(st, n, rows)
        return n

    def _emit(self, st, n, data):
        if self.sink is None:
            self.stream.append((st, n, data))
        else:
            self.sink(st, n, data)

    def run(self, total_frames: int, start: int = 0, stop: Optional[int] = None):
        """Alg. 1 main (the initial Gaussians are the caller's gs) over the
        window starts [start, stop) of a clip of total_frames frames (start 0:
        the first window; a later start continues a run restored with
        load_state_dict; stop defaults to the end, where the last maturation
        runs). Returns the loss of the last step."""
        stop = total_frames if stop is None else min(stop, total_frames)
        loss = None
        if start == 0 and stop > 0:
            # main: birth = start = 0, expire = swin_size for every gs slot
            g = self.buf.rows(0, self.num_gs)
            g.birth.zero_()
            g.start.zero_()
            g.expire.fill_(self.swin)
            loss = self._train(0)
            self.r.schedule_expire(self.buf, self.num_gs, self.swin)
            start = 1
            self.next_start = 1
        for st in range(start, stop):
            self.mature(st)
            loss = self._train(st)
            self.next_start = st + 1
        if stop == total_frames and getattr(self, "next_start", 0) == total_frames:
            self.mature(total_frames)
            self.next_start = total_frames + 1
        return loss

    def state_dict(self) -> dict:
        """Everything a resumed run needs: the buffer (gs and matured ring),
        the Adam moments, the ring head, the step counter, the seed and the
        next window start (random draws are counter-based, nothing else)."""
        arrays = {k: getattr(self.buf, k) for k in
                  api.PARAM_NAMES + ("start", "expire", "birth", "frozen")}
        arrays.update({"adam_" + k: v for k, v in self.trainer.adam.items()})
        scalars = dict(num_gs=self.num_gs, swin_size=self.swin, head=self.head,
                       step_count=self.step_count, seed=self.trainer.seed,
                       sh_degree=self.buf.sh_degree, next_start=getattr(self, "next_start", 0))
        return {"arrays": arrays, "scalars": scalars}

    def load_state_dict(self, sd: dict):
        a, sc = sd["arrays"], sd["scalars"]
        if sc["num_gs"] != self.num_gs or sc["swin_size"] != self.swin:
            raise ValueError("checkpoint of another num_gs / swin_size")
        for k in api.PARAM_NAMES + ("start", "expire", "birth", "frozen"):
            getattr(self.buf, k).copy_(a[k])
        for k, v in self.trainer.adam.items():
            v.copy_(a["adam_" + k])
        self.head = int(sc["head"])
        self.step_count = int(sc["step_count"])
        self.trainer.seed = int(sc["seed"])
        self.next_start = int(sc["next_start"])

    def save(self, path):
        from . import checkpoint
        sd = self.state_dict()
        checkpoint.save(path, sd["arrays"], sd["scalars"])

    def load(self, path):
        from . import checkpoint
        arrays, scalars = checkpoint.load(path)
        self.load_state_dict({"arrays": arrays, "scalars": scalars})
