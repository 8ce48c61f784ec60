"""Torch-facing API over libswgs. PyTorch provides device memory, streams and
autograd plumbing; every step of the splatting path runs in the library's
CUDA kernels (this module marshals pointers and sizes only).

Main entry points:
  GaussianState      -- the slot buffer (Sec. 4.2 gs/matured, Alg. 2 buffer)
  Renderer           -- one library context: render / backward / L1 /
                        SGLD step / frame update / active ids
  render(...)        -- differentiable render (torch.autograd.Function)
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import SwgsError

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class GaussianState:
    """Slot-major Gaussian state on the GPU (float32 attributes, int32
    lifespans, uint8 frozen flags)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, start, expire, birth=None,
                 frozen=None, sh_degree: Optional[int] = None):
        self.means = means
        self.log_scales = log_scales
        self.quats = quats
        self.opacity_logits = opacity_logits
        self.sh = sh
        self.start = start
        self.expire = expire
        self.birth = birth if birth is not None else start.clone()
        self.frozen = frozen if frozen is not None else torch.zeros_like(start, dtype=torch.uint8)
        K = sh.shape[1]
        self.sh_degree = int(round(K ** 0.5)) - 1 if sh_degree is None else sh_degree
        self._check()

    def _check(self):
        n = self.n
        assert self.means.shape == (n, 3) and self.log_scales.shape == (n, 3)
        assert self.quats.shape == (n, 4) and self.opacity_logits.shape == (n,)
        assert self.sh.shape == (n, (self.sh_degree + 1) ** 2, 3)
        for t in (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh):
            assert t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()
        for t in (self.start, self.expire, self.birth):
            assert t.dtype == torch.int32 and t.is_cuda and t.is_contiguous()
        assert self.frozen.dtype == torch.uint8 and self.frozen.is_contiguous()

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianState":
        f = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return GaussianState(f(scene.means, torch.float32), f(scene.log_scales, torch.float32),
                             f(scene.quats, torch.float32), f(scene.opacity_logits, torch.float32),
                             f(scene.sh, torch.float32), f(scene.start, torch.int32),
                             f(scene.expire, torch.int32), f(scene.birth, torch.int32),
                             f(scene.frozen, torch.uint8), scene.sh_degree)

    def params(self):
        return [getattr(self, k) for k in PARAM_NAMES]

    def with_params(self, params) -> "GaussianState":
        s = GaussianState.__new__(GaussianState)
        s.__dict__.update(self.__dict__)
        for k, v in zip(PARAM_NAMES, params):
            setattr(s, k, v)
        return s

    def c_struct(self) -> _abi.SwgsGaussians:
        return _abi.SwgsGaussians(self.means.data_ptr(), self.log_scales.data_ptr(),
                                  self.quats.data_ptr(), self.opacity_logits.data_ptr(),
                                  self.sh.data_ptr(), self.start.data_ptr(),
                                  self.expire.data_ptr(), self.birth.data_ptr(),
                                  self.frozen.data_ptr(), self.n, self.sh_degree)

    def zero_grads(self) -> "GaussianGrads":
        return GaussianGrads(*[torch.zeros_like(t) for t in self.params()], self.sh_degree)

    def pin_host(self) -> dict:
        """A pinned host copy of every array (the form a streamed slice arrives in)."""
        return {k: getattr(self, k).cpu().pin_memory() for k in
                PARAM_NAMES + ("start", "expire", "birth", "frozen")}

    def rows(self, lo: int, hi: int) -> "GaussianState":
        """Views of the slots [lo, hi) (no copy)."""
        return GaussianState(*[getattr(self, k)[lo:hi] for k in
                               PARAM_NAMES + ("start", "expire", "birth", "frozen")],
                             sh_degree=self.sh_degree)

    @staticmethod
    def with_matured_ring(gs: "GaussianState") -> "GaussianState":
        """The training buffer of Alg. 1: gs in slots [0, num_gs) followed by an
        empty ring of num_gs matured slots (frozen, empty lifespan start =
        expire = 0) that swgs_mature fills."""
        def cat(a, fill):
            return torch.cat([a, torch.full_like(a, fill)]).contiguous()
        return GaussianState(cat(gs.means, 0), cat(gs.log_scales, 0), cat(gs.quats, 0),
                             cat(gs.opacity_logits, 0), cat(gs.sh, 0), cat(gs.start, 0),
                             cat(gs.expire, 0), cat(gs.birth, 0),
                             torch.cat([torch.zeros_like(gs.frozen),
                                        torch.ones_like(gs.frozen)]).contiguous(),
                             sh_degree=gs.sh_degree)


@dataclass
class GaussianGrads:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    def c_struct(self) -> _abi.SwgsGaussians:
        return _abi.SwgsGaussians(self.means.data_ptr(), self.log_scales.data_ptr(),
                                  self.quats.data_ptr(), self.opacity_logits.data_ptr(),
                                  self.sh.data_ptr(), None, None, None, None,
                                  int(self.means.shape[0]), self.sh_degree)

    def zero_(self):
        for k in PARAM_NAMES:
            getattr(self, k).zero_()
        return self

    def as_dict(self):
        return {k: getattr(self, k) for k in PARAM_NAMES}


def make_view(v) -> _abi.SwgsView:
    """A swgs_view from any object with width, height, fx, fy, cx, cy, R, t, frame."""
    R = np.asarray(v.R, np.float32).reshape(9)
    t = np.asarray(v.t, np.float32).reshape(3)
    return _abi.SwgsView(int(v.width), int(v.height), float(v.fx), float(v.fy), float(v.cx),
                         float(v.cy), (C.c_float * 9)(*R.tolist()), (C.c_float * 3)(*t.tolist()),
                         int(v.frame))


def _views_array(views):
    arr = (_abi.SwgsView * len(views))()
    for i, v in enumerate(views):
        arr[i] = v if isinstance(v, _abi.SwgsView) else make_view(v)
    return arr


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class SavedState:
    """Handle to a forward's saved state; returned to the library's pool on
    release() or garbage collection."""

    def __init__(self, renderer: "Renderer", handle: C.c_void_p, views):
        self.renderer = renderer
        self.handle = handle
        self.views = views

    def release(self):
        if self.handle is not None and self.renderer.ctx is not None:
            _abi.load().swgs_saved_release(self.renderer.ctx, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def status(self, wait: bool = True) -> int:
        """The forward's outcome (see swgs_saved_status): _abi.SWGS_OK, SWGS_EDEVICE
        (a batch outgrew the deferred capacities: render again), SWGS_ETIMEOUT,
        or with wait=False SWGS_EPENDING if it has not arrived yet."""
        return int(_abi.load().swgs_saved_status(self.renderer.ctx, self.handle, int(bool(wait))))

    def info(self) -> _abi.SwgsSavedInfo:
        inf = _abi.SwgsSavedInfo()
        self.renderer._check(_abi.load().swgs_saved_query(self.renderer.ctx, self.handle,
                                                          C.byref(inf)))
        return inf

    def export(self, what: int) -> np.ndarray:
        """Copy one intermediate array to host numpy (see include/swgs.h)."""
        L = _abi.load()
        n = C.c_int64(0)
        self.renderer._check(L.swgs_saved_count(self.renderer.ctx, self.handle, what,
                                                C.byref(n)))
        shapes = {_abi.EXPORT_RECORD_RECT: (np.int32, 4), _abi.EXPORT_TILE_RANGES: (np.int32, 2),
                  _abi.EXPORT_GRAD2D: (np.float32, 12), _abi.EXPORT_RECORD_2D: (np.float32, 12),
                  _abi.EXPORT_RECORD_DEPTH: (np.float32, 1), _abi.EXPORT_FINAL_T: (np.float32, 1),
                  _abi.EXPORT_VIEW_TABLE: (np.int32, 6)}
        dt, w = shapes.get(what, (np.int32, 1))
        out = np.zeros((n.value, w) if w > 1 else (n.value,), dt)
        if n.value > 0:
            self.renderer._check(L.swgs_saved_export(
                self.renderer.ctx, self.handle, what, out.ctypes.data_as(C.c_void_p), out.nbytes,
                C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return out


class Renderer:
    """One libswgs context (tile shape, batch size, near plane). Scratch memory
    comes from torch's caching allocator through the library's callbacks."""

    def __init__(self, tile=(16, 16), batch=64, near_plane=0.2, blocks_per_sm=0,
                 count_pairs=False, pixels_per_thread=None, bwd_pixels_per_thread=None,
                 bwd_batch=32, use_torch_allocator=True, alloc_guard=None,
                 sort_single_pass=True, deferred_sizing=False):
        if pixels_per_thread is None:      # 8x8 tiles hold at most 2 pixels per thread
            pixels_per_thread = 2 if tuple(tile) == (8, 8) else 4
        if bwd_pixels_per_thread is None:
            bwd_pixels_per_thread = 2 if tuple(tile) == (8, 8) else 8
        L = _abi.load()
        cfg = _abi.SwgsConfig()
        L.swgs_default_config(C.byref(cfg))
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
        cfg.batch = int(batch)
        cfg.near_plane = float(near_plane)
        cfg.blocks_per_sm = int(blocks_per_sm)
        cfg.count_pairs = int(bool(count_pairs))
        cfg.pixels_per_thread = int(pixels_per_thread)
        cfg.bwd_pixels_per_thread = int(bwd_pixels_per_thread)
        cfg.bwd_batch = int(bwd_batch)
        cfg.sort_single_pass = int(bool(sort_single_pass))
        # True: after the first forward, no stream synchronisation; the caller
        # checks SavedState.status() (the trainer and the server do)
        cfg.deferred_sizing = int(bool(deferred_sizing))
        self.cfg = cfg
        self.alloc_guard = alloc_guard
        self.device = torch.cuda.current_device()
        if use_torch_allocator:
            dev = self.device

            def _alloc(user, nbytes, stream):
                # alloc_guard(nbytes) -> False refuses the allocation (a memory
                # budget, or an injected failure): the call returns SWGS_ENOMEM
                if self.alloc_guard is not None and not self.alloc_guard(int(nbytes)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
                except Exception:
                    return None

            def _free(user, ptr, nbytes, stream):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = _abi.ALLOC_FN(_alloc)
            self._free_cb = _abi.FREE_FN(_free)
        else:
            self._alloc_cb = _abi.ALLOC_FN()
            self._free_cb = _abi.FREE_FN()
        h = C.c_void_p()
        st = L.swgs_create(C.byref(cfg), self._alloc_cb, self._free_cb, None, C.byref(h))
        if st != 0:
            raise SwgsError(st, "swgs_create failed")
        self.ctx = h

    def close(self):
        if self.ctx is not None:
            torch.cuda.synchronize()
            _abi.load().swgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        if status != 0:
            msg = _abi.load().swgs_last_error(self.ctx)
            raise SwgsError(status, msg.decode() if msg else "")

    @staticmethod
    def _stream(stream=None):
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    # -- measurement -----------------------------------------------------------
    def profile(self, on: bool = True):
        self._check(_abi.load().swgs_profile_enable(self.ctx, int(bool(on))))

    def profile_read(self, reset: bool = True) -> dict:
        """Summed device milliseconds per stage since the last reset."""
        p = _abi.SwgsProfile()
        self._check(_abi.load().swgs_profile_read(self.ctx, C.byref(p), int(bool(reset))))
        return {n: (p.ms[i], int(p.calls[i])) for i, n in enumerate(_abi.STAGE_NAMES)}

    @staticmethod
    def kernel_launches() -> int:
        return int(_abi.load().swgs_kernel_launches())

    def selftest_sort_timeout(self, stream=None):
        """Run the radix sort's look-back timeout check (include/swgs.h): raises
        SwgsError (ETIMEOUT) when the bounded wait ran out, as it should."""
        self._check(_abi.load().swgs_selftest_sort_timeout(self.ctx, self._stream(stream)))

    # -- Sec. 4.2 / Alg. 2 filter ------------------------------------------------
    def active_ids(self, state: GaussianState, frame: int, stream=None) -> torch.Tensor:
        ids = torch.empty(max(1, state.n), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        self._check(_abi.load().swgs_active_ids(self.ctx, _ptr(state.start), _ptr(state.expire),
                                                state.n, int(frame), _ptr(ids), _ptr(cnt),
                                                self._stream(stream)))
        return ids[: int(cnt.item())]

    # -- Eq. 3 forward ---------------------------------------------------------
    def render(self, state: GaussianState, views: Sequence, bg=(0.0, 0.0, 0.0), batched=True,
               keep_saved=False, out=None, out_T=None, stream=None):
        """Render views (each at its own frame). Returns (images, saved) where
        images[v] is a [3,H,W] float32 tensor and saved a SavedState or None."""
        cviews = _views_array(views)
        if out is None:
            out = [torch.empty((3, v.height, v.width), dtype=torch.float32, device="cuda")
                   for v in cviews]
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        handle = C.c_void_p()
        g = state.c_struct()
        self._check(_abi.load().swgs_render_fwd(
            self.ctx, C.byref(g), len(cviews), cviews, bgv, _ptr_array(out),
            _ptr_array(out_T) if out_T is not None else None, int(bool(batched)),
            C.byref(handle) if keep_saved else None, self._stream(stream)))
        saved = SavedState(self, handle, cviews) if keep_saved else None
        return out, saved

    def render_rgb8(self, state: GaussianState, views: Sequence, bg=(0.0, 0.0, 0.0),
                    batched=True, keep_saved=False, out=None, out_T=None, stream=None):
        """Render views to 8-bit images: images[v] is a uint8 [H,W,3] tensor
        (round(255 clamp(c, 0, 1))). Returns (images, saved)."""
        cviews = _views_array(views)
        if out is None:
            out = [torch.empty((v.height, v.width, 3), dtype=torch.uint8, device="cuda")
                   for v in cviews]
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        handle = C.c_void_p()
        g = state.c_struct()
        self._check(_abi.load().swgs_render_fwd_rgb8(
            self.ctx, C.byref(g), len(cviews), cviews, bgv, _ptr_array(out),
            _ptr_array(out_T) if out_T is not None else None, int(bool(batched)),
            C.byref(handle) if keep_saved else None, self._stream(stream)))
        saved = SavedState(self, handle, cviews) if keep_saved else None
        return out, saved

    def render_l1(self, state: GaussianState, views: Sequence, targets, bg=(0.0, 0.0, 0.0),
                  batched=True, keep_saved=True, out=None, dL_out=None, loss_out=None,
                  stream=None):
        """Forward render fused with the L1 term: returns (images, dL/drgb, loss,
        saved). targets: float32 [3,H,W] per view, or uint8 [3,H,W] (8-bit
        frames, read as k * (1/255) in FP32). out=False writes no image (the
        loss and its gradient need none; images is then None)."""
        cviews = _views_array(views)
        dts = {t.dtype for t in targets}
        if len(dts) != 1 or dts.pop() not in (torch.float32, torch.uint8):
            raise ValueError("targets must all be float32 or all uint8")
        u8 = targets[0].dtype == torch.uint8
        for t, v in zip(targets, cviews):
            if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (3, v.height, v.width):
                raise ValueError("each target must be a contiguous CUDA [3, H, W] tensor")
        if out is None:
            out = [torch.empty((3, v.height, v.width), dtype=torch.float32, device="cuda")
                   for v in cviews]
        if dL_out is None:
            dL_out = [torch.empty((3, v.height, v.width), dtype=torch.float32, device="cuda")
                      for v in cviews]
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float32, device="cuda")
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        handle = C.c_void_p()
        g = state.c_struct()
        fn = _abi.load().swgs_render_fwd_l1_u8 if u8 else _abi.load().swgs_render_fwd_l1
        self._check(fn(
            self.ctx, C.byref(g), len(cviews), cviews, bgv,
            None if out is False else _ptr_array(out), None,
            _ptr_array(targets), _ptr_array(dL_out), _ptr(loss_out), int(bool(batched)),
            C.byref(handle) if keep_saved else None, self._stream(stream)))
        saved = SavedState(self, handle, cviews) if keep_saved else None
        return (None if out is False else out), dL_out, loss_out, saved

    def backward(self, state: GaussianState, saved: SavedState, dL_drgb, grads: GaussianGrads,
                 reg: Optional[dict] = None, loss: Optional[torch.Tensor] = None, stream=None):
        """Accumulate into grads the gradient of the render (and, with reg =
        dict(opacity_reg=..., scale_reg=...), of Alg. 1 reg(); its value is
        added to `loss` when given)."""
        for t in dL_drgb:
            assert t.is_contiguous() and t.dtype == torch.float32
        g = state.c_struct()
        gr = grads.c_struct()
        rp = None
        if reg is not None:
            rp = _abi.SwgsRegParams(float(reg.get("opacity_reg", 0.0)),
                                    float(reg.get("scale_reg", 0.0)),
                                    int(reg.get("n_views_total", 0)))
        self._check(_abi.load().swgs_render_bwd_reg(self.ctx, C.byref(g), saved.handle,
                                                    _ptr_array(dL_drgb), C.byref(gr),
                                                    C.byref(rp) if rp is not None else None,
                                                    _ptr(loss), self._stream(stream)))
        return grads

    # -- Alg. 1 loss_func (L1) -------------------------------------------------
    def loss_l1(self, views, rgbs, targets, dL_out=None, loss_out=None, stream=None):
        cviews = _views_array(views)
        if dL_out is None:
            dL_out = [torch.empty_like(r) for r in rgbs]
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float32, device="cuda")
        self._check(_abi.load().swgs_loss_l1(self.ctx, len(cviews), cviews, _ptr_array(rgbs),
                                             _ptr_array(targets), _ptr_array(dL_out),
                                             _ptr(loss_out), self._stream(stream)))
        return loss_out, dL_out

    # -- Alg. 1 noise / relocate -----------------------------------------------
    def sgld_step(self, state: GaussianState, frames, params: dict, seed: int, step: int,
                  grads: Optional[GaussianGrads] = None, adam: Optional[dict] = None,
                  targets: Optional[torch.Tensor] = None, count_relocated=False, stream=None):
        known = {f[0] for f in _abi.SwgsSgldParams._fields_}
        p = _abi.SwgsSgldParams(**{"mean_grad_decay": 1.0,
                                   **{k: v for k, v in params.items() if k in known}})
        fr = (C.c_int32 * max(1, len(frames)))(*[int(f) for f in frames])
        ad = None
        if adam is not None:
            ad = _abi.SwgsAdamState(*[adam[k].data_ptr() for k in (
                "m_means", "v_means", "m_log_scales", "v_log_scales", "m_quats", "v_quats",
                "m_opacity_logits", "v_opacity_logits", "m_sh", "v_sh")])
        nrel = C.c_int64(0)
        g = state.c_struct()
        gr = grads.c_struct() if grads is not None else None
        self._check(_abi.load().swgs_sgld_step(
            self.ctx, C.byref(g), C.byref(gr) if gr is not None else None,
            C.byref(ad) if ad is not None else None, fr, len(frames), C.byref(p), int(seed),
            int(step), _ptr(targets), C.byref(nrel) if count_relocated else None,
            self._stream(stream)))
        return int(nrel.value) if count_relocated else None

    # -- data-parallel gradient exchange -----------------------------------------
    def grad_pack(self, state: GaussianState, grads: GaussianGrads, frames, ids: torch.Tensor,
                  count: torch.Tensor, packed: torch.Tensor, scale: float = 1.0, stream=None):
        """Pack the gradient rows (times `scale`) of the slots eligible at
        `frames` (active at one of them, not frozen) into packed[:count] (rows
        of 11 + 3K floats), their slots into ids[:count] and their number into
        count (device int64)."""
        fr = (C.c_int32 * max(1, len(frames)))(*[int(f) for f in frames])
        g = state.c_struct()
        gr = grads.c_struct()
        self._check(_abi.load().swgs_grad_pack(self.ctx, C.byref(g), C.byref(gr), fr, len(frames),
                                               float(scale), _ptr(ids), _ptr(count), _ptr(packed),
                                               self._stream(stream)))

    def grad_unpack(self, grads: GaussianGrads, ids: torch.Tensor, count: torch.Tensor,
                    packed: torch.Tensor, stream=None):
        """Write packed row k back to slot ids[k] of grads, for k < count."""
        gr = grads.c_struct()
        self._check(_abi.load().swgs_grad_unpack(self.ctx, C.byref(gr), _ptr(ids), _ptr(count),
                                                 _ptr(packed), self._stream(stream)))

    # -- Alg. 2 update_thread ----------------------------------------------------
    def frame_update(self, dst: GaussianState, first: int, src, src_on_host: bool, stream=None):
        """Overwrite slots [first, first + n) of dst with src (a GaussianState on
        the device, or a dict of pinned host tensors from GaussianState.pin_host)."""
        if src_on_host:
            get = lambda k: src[k]
            n = int(src["means"].shape[0])
        else:
            get = lambda k: getattr(src, k)
            n = src.n
        s = _abi.SwgsGaussians(*[get(k).data_ptr() for k in
                                 PARAM_NAMES + ("start", "expire", "birth", "frozen")],
                               n, dst.sh_degree)
        d = dst.c_struct()
        self._check(_abi.load().swgs_frame_update(self.ctx, C.byref(d), int(first), n,
                                                  C.byref(s), int(bool(src_on_host)),
                                                  self._stream(stream)))

    # -- streamed-slice codec (Table 6, Sec. 5.5) ---------------------------------
    @staticmethod
    def slice_packet_bytes(count: int, keep: int) -> int:
        return int(_abi.load().swgs_slice_packet_bytes(int(count), int(keep)))

    def slice_encode(self, src: GaussianState, count: int, keep: Optional[int] = None,
                     out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Encode rows [0, count) of src; keep < count drops the lowest-opacity
        Gaussians. out: a uint8 tensor (device, or pinned host) of at least
        slice_packet_bytes(count, keep) bytes; allocated on the device if None.
        Returns the packet (a view of out)."""
        keep = count if keep is None else int(keep)
        nbytes = self.slice_packet_bytes(count, keep)
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        used = C.c_size_t(0)
        g = src.c_struct()
        self._check(_abi.load().swgs_slice_encode(self.ctx, C.byref(g), int(count), keep,
                                                  out.data_ptr(), out.numel(),
                                                  int(not out.is_cuda), C.byref(used),
                                                  self._stream(stream)))
        return out[:used.value]

    def slice_decode(self, packet: torch.Tensor, dst: GaussianState, first: int, stream=None):
        """Decode a packet (device or pinned host uint8 tensor) into the slots
        [first, first + count) of dst."""
        d = dst.c_struct()
        self._check(_abi.load().swgs_slice_decode(self.ctx, packet.data_ptr(), packet.numel(),
                                                  int(not packet.is_cuda), C.byref(d),
                                                  int(first), self._stream(stream)))

    # -- Alg. 1 mature / schedule_expire ---------------------------------------
    def schedule_expire(self, buf: GaussianState, num_gs: int, swin_size: int, stream=None):
        """Stagger the gs expiries after the first window (slice k: expire k,
        slice 0: swin_size). buf: GaussianState.with_matured_ring layout."""
        b = buf.c_struct()
        self._check(_abi.load().swgs_schedule_expire(self.ctx, C.byref(b), int(num_gs),
                                                     int(swin_size), self._stream(stream)))

    def mature(self, buf: GaussianState, num_gs: int, st: int, swin_size: int, head: int,
               snapshot=None, stream=None):
        """Alg. 1 mature(st) on buf (GaussianState.with_matured_ring layout).
        snapshot: None, a GaussianState of >= num_gs rows (device), or a dict of
        pinned host tensors of >= num_gs rows (GaussianState.pin_host form); its
        first n rows receive the matured rows as they were (stream.write).
        Returns (n, new ring head)."""
        b = buf.c_struct()
        h = C.c_int64(int(head))
        n = C.c_int64(0)
        snap, on_host = None, 0
        if isinstance(snapshot, dict):
            snap = _host_struct(snapshot, int(snapshot["means"].shape[0]), buf.sh_degree)
            on_host = 1
        elif snapshot is not None:
            snap = snapshot.c_struct()
        self._check(_abi.load().swgs_mature(self.ctx, C.byref(b), int(num_gs), int(st),
                                            int(swin_size), C.byref(h),
                                            C.byref(snap) if snap is not None else None,
                                            on_host, C.byref(n), self._stream(stream)))
        return n.value, h.value


def _host_struct(d: dict, n: int, sh_degree: int) -> _abi.SwgsGaussians:
    return _abi.SwgsGaussians(*[d[k].data_ptr() for k in
                                PARAM_NAMES + ("start", "expire", "birth", "frozen")],
                              n, sh_degree)


def slice_range(target_frame: int, swin_size: int, num_gs: int):
    """Alg. 2: the slot range [first, first + count) that target_frame's update
    overwrites."""
    first, count = C.c_int64(0), C.c_int64(0)
    st = _abi.load().swgs_slice_range(int(target_frame), int(swin_size), int(num_gs),
                                      C.byref(first), C.byref(count))
    if st != 0:
        raise SwgsError(st, "bad slice arguments")
    return first.value, count.value


class _RenderFn(torch.autograd.Function):
    """Differentiable render: forward saves the final transmittance and the
    last-contributor index (inside the library's saved state) so that the
    backward recomputes the blend in reverse instead of storing it."""

    @staticmethod
    def forward(ctx, renderer, state, views, bg, batched, *params):
        st = state.with_params([p.detach() for p in params])
        imgs, saved = renderer.render(st, views, bg=bg, batched=batched, keep_saved=True)
        ctx.renderer, ctx.state, ctx.saved = renderer, st, saved
        ctx.shapes = [tuple(i.shape) for i in imgs]
        return tuple(imgs)

    @staticmethod
    def backward(ctx, *grad_imgs):
        dl = [torch.zeros(s, dtype=torch.float32, device="cuda") if g is None else g.contiguous()
              for g, s in zip(grad_imgs, ctx.shapes)]
        grads = ctx.state.zero_grads()
        ctx.renderer.backward(ctx.state, ctx.saved, dl, grads)
        ctx.saved.release()
        return (None, None, None, None, None) + tuple(getattr(grads, k) for k in PARAM_NAMES)


def render(renderer: Renderer, state: GaussianState, views, bg=(0.0, 0.0, 0.0), batched=True,
           params=None):
    """Differentiable render of `views`; gradients flow to `params` (defaults to
    the state's own attribute tensors)."""
    ps = state.params() if params is None else list(params)
    return _RenderFn.apply(renderer, state, views, tuple(bg), batched, *ps)
