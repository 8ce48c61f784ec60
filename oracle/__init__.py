"""FP64 CPU oracle for the SwinGS frame-t splatting hot path (arXiv 2409.07759).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only users. The product path never imports this
package; the CUDA library and this oracle share no code.

The arithmetic lives in ``swgs_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module marshals numpy arrays through ctypes and
adds two steps that are plain array bookkeeping:

* ``frame_update`` -- the slice replacement of Alg. 2 (update_thread);
* ``schedule_expire`` and ``mature`` -- the maturation of Alg. 1 (mature);
* ``reg_loss_grad`` -- the opacity and scale regularisers of Alg. 1 reg() (Sec. 4.4);
* ``mean_grad_scale`` -- the per-Gaussian gradient scale on the means (Sec. 4.5.1);
* ``slice_encode`` / ``slice_decode`` -- the Table 6 attribute quantisation of a
  streamed slice and the Sec. 5.5 tail drop of its lowest-opacity Gaussians;
* ``l1_loss_grad`` -- the L1 photometric term of Alg. 1 (loss_func) and its
  gradient.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "swgs_oracle.c"
_LIB_PATH = _HERE / "liboracle.so"

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=c11", "-Wall"]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (seconds)."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(".so.tmp%d" % os.getpid())
        subprocess.run(["gcc", *CFLAGS, "-o", str(tmp), str(_SRC), "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


# --------------------------------------------------------------------------
# ctypes mirrors of the oracle's structures
# --------------------------------------------------------------------------

class OrView(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3), ("frame", C.c_int32)]


class OrScene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p), ("start", C.c_void_p),
                ("expire", C.c_void_p), ("frozen", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32)]


class OrKm(C.Structure):
    _fields_ = [("u", C.c_float), ("v", C.c_float), ("z", C.c_float), ("a", C.c_float),
                ("b", C.c_float), ("c", C.c_float), ("det", C.c_float),
                ("lambda1", C.c_float), ("radius", C.c_float), ("culled", C.c_int32),
                ("tx0", C.c_int32), ("tx1", C.c_int32), ("ty0", C.c_int32),
                ("ty1", C.c_int32), ("tiles", C.c_int32), ("A", C.c_float), ("B", C.c_float),
                ("C", C.c_float)]


KM_DTYPE = np.dtype([("u", "<f4"), ("v", "<f4"), ("z", "<f4"), ("a", "<f4"), ("b", "<f4"),
                     ("c", "<f4"), ("det", "<f4"), ("lambda1", "<f4"), ("radius", "<f4"),
                     ("culled", "<i4"), ("tx0", "<i4"), ("tx1", "<i4"), ("ty0", "<i4"),
                     ("ty1", "<i4"), ("tiles", "<i4"), ("A", "<f4"), ("B", "<f4"),
                     ("C", "<f4")])
assert KM_DTYPE.itemsize == C.sizeof(OrKm)


class OrBands(C.Structure):
    _fields_ = [("m", C.c_double), ("alpha", C.c_double), ("t_stop", C.c_double),
                ("clamp", C.c_double), ("guard", C.c_double), ("colour", C.c_double)]


class OrGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p)]


class OrSgldParams(C.Structure):
    _fields_ = [("lr_means", C.c_float), ("lr_log_scales", C.c_float), ("lr_quats", C.c_float),
                ("lr_logits", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("noise_lr", C.c_float), ("noise_k", C.c_float), ("noise_t", C.c_float),
                ("adam", C.c_int32), ("relocate", C.c_int32), ("max_n", C.c_int32)]


class OrState(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p), ("start", C.c_void_p),
                ("expire", C.c_void_p), ("frozen", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32)]


class OrAdam(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("m_means", "v_means", "m_log_scales", "v_log_scales", "m_quats", "v_quats",
                 "m_logits", "v_logits", "m_sh", "v_sh")]


class OrFGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        P = C.POINTER
        _lib.or_active_ids.restype = C.c_int64
        _lib.or_active_ids.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
        _lib.or_keymode.restype = None
        _lib.or_keymode.argtypes = [P(OrScene), P(OrView), C.c_int64, C.c_int32, C.c_int32,
                                    C.c_float, C.c_void_p]
        _lib.or_render.restype = C.c_int
        _lib.or_render.argtypes = [P(OrScene), P(OrView), C.c_void_p, C.c_int32, C.c_int32,
                                   C.c_float, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.or_render_pixels.restype = C.c_int
        _lib.or_render_pixels.argtypes = [P(OrScene), P(OrView), C.c_void_p, C.c_float,
                                          C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.or_render_variants.restype = C.c_int
        _lib.or_render_variants.argtypes = [P(OrScene), P(OrView), C.c_void_p, C.c_int32,
                                            C.c_int32, C.c_float, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
        _lib.or_view_lists.restype = C.c_int64
        _lib.or_view_lists.argtypes = [P(OrScene), P(OrView), C.c_int32, C.c_int32, C.c_float,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]
        _lib.or_render_bwd.restype = C.c_int
        _lib.or_render_bwd.argtypes = [P(OrScene), P(OrView), C.c_void_p, C.c_int32, C.c_int32,
                                       C.c_float, C.c_void_p, C.c_void_p, P(OrGrads),
                                       C.c_void_p, C.c_void_p]
        _lib.or_project.restype = None
        _lib.or_project.argtypes = [P(OrScene), P(OrView), C.c_int64, C.c_void_p]
        _lib.or_sh_basis.restype = None
        _lib.or_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, C.c_void_p]
        _lib.or_philox4x64.restype = None
        _lib.or_philox4x64.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.or_normal3.restype = None
        _lib.or_normal3.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p]
        _lib.or_reloc_weight.restype = C.c_uint64
        _lib.or_reloc_weight.argtypes = [C.c_float]
        _lib.or_reloc_values.restype = None
        _lib.or_reloc_values.argtypes = [C.c_double, C.c_int, P(C.c_double), P(C.c_double)]
        _lib.or_sgld_step.restype = C.c_int64
        _lib.or_sgld_step.argtypes = [P(OrState), P(OrFGrads), P(OrAdam), C.c_void_p, C.c_int32,
                                      P(OrSgldParams), C.c_uint64, C.c_uint64, C.c_void_p]
        _lib.or_opacity_u8.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        _lib.or_set_threads.argtypes = [C.c_int]
        _lib.or_set_threads.restype = None
        _lib.or_num_threads.restype = C.c_int
        _lib.or_record_tiles.restype = C.c_int32
        _lib.or_record_tiles.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_void_p]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _SceneRef:
    """Keeps contiguous copies alive while the C code reads them."""

    def __init__(self, scene):
        self.arrays = dict(
            means=_c(scene.means, np.float32), log_scales=_c(scene.log_scales, np.float32),
            quats=_c(scene.quats, np.float32), logits=_c(scene.opacity_logits, np.float32),
            sh=_c(scene.sh, np.float32), start=_c(scene.start, np.int32),
            expire=_c(scene.expire, np.int32), frozen=_c(scene.frozen, np.uint8))
        a = self.arrays
        self.s = OrScene(_p(a["means"]).value, _p(a["log_scales"]).value, _p(a["quats"]).value,
                         _p(a["logits"]).value, _p(a["sh"]).value, _p(a["start"]).value,
                         _p(a["expire"]).value, _p(a["frozen"]).value, scene.n,
                         scene.sh_degree)


def make_view(v) -> OrView:
    R = np.asarray(v.R, np.float32).reshape(9)
    t = np.asarray(v.t, np.float32).reshape(3)
    return OrView(int(v.width), int(v.height), float(v.fx), float(v.fy), float(v.cx),
                  float(v.cy), (C.c_float * 9)(*R.tolist()), (C.c_float * 3)(*t.tolist()),
                  int(v.frame))


DEFAULT_BANDS = dict(m=2e-4, alpha=2e-4, t_stop=2e-3, clamp=2e-4, guard=1e-4, colour=1e-5)


def _bands(b):
    if b is None:
        return None
    d = dict(DEFAULT_BANDS)
    d.update(b)
    return OrBands(**d)


# --------------------------------------------------------------------------
# Public API
# --------------------------------------------------------------------------

def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    """Number of host threads the oracle's parallel loops use from now on."""
    lib().or_set_threads(int(n))


def active_ids(start, expire, frame: int) -> np.ndarray:
    """Slots with start <= frame < expire, ascending (Sec. 4.2)."""
    start = _c(start, np.int32)
    expire = _c(expire, np.int32)
    out = np.empty(max(1, start.shape[0]), np.int32)
    k = lib().or_active_ids(_p(start), _p(expire), start.shape[0], int(frame), _p(out))
    return out[:k].copy()


def keymode(scene, view, slots, tile_w=16, tile_h=16, near=0.2) -> np.ndarray:
    """FP32 key-mode records (culling, 2D covariance, radius, tile rectangle)."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    slots = np.asarray(slots, np.int64)
    out = np.zeros(len(slots), KM_DTYPE)
    rec = OrKm()
    L = lib()
    for i, s in enumerate(slots):
        L.or_keymode(C.byref(ref.s), C.byref(vw), int(s), tile_w, tile_h, near, C.byref(rec))
        out[i] = tuple(getattr(rec, f[0]) for f in OrKm._fields_)
    return out


def record_tiles(km_row, view, tile_w=16, tile_h=16) -> np.ndarray:
    """Tile ids (row-major in the view) that one key-mode record covers."""
    rec = np.array([km_row], KM_DTYPE)
    ntx = (view.width + tile_w - 1) // tile_w
    out = np.zeros(max(1, int(km_row["tiles"])), np.int32)
    n = lib().or_record_tiles(_p(rec), ntx, tile_w, tile_h, _p(out))
    return out[:n].copy()


def view_lists(scene, view, tile_w=16, tile_h=16, near=0.2, with_lists=True):
    """Active ids, key-mode records and the per-tile depth-sorted slot lists of
    one view. Returns (ids, km, n_keys, tile_off, tile_slot)."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    L = lib()
    n_keys = C.c_int64(0)
    ids = np.empty(max(1, scene.n), np.int32)
    km = np.zeros(max(1, scene.n), KM_DTYPE)
    n = L.or_view_lists(C.byref(ref.s), C.byref(vw), tile_w, tile_h, near, _p(ids), _p(km),
                        C.byref(n_keys), None, None)
    ids, km = ids[:n].copy(), km[:n].copy()
    if not with_lists:
        return ids, km, int(n_keys.value), None, None
    ntx = (view.width + tile_w - 1) // tile_w
    nty = (view.height + tile_h - 1) // tile_h
    tile_off = np.zeros(ntx * nty + 1, np.int64)
    tile_slot = np.zeros(max(1, n_keys.value), np.int32)
    L.or_view_lists(C.byref(ref.s), C.byref(vw), tile_w, tile_h, near, None, None,
                    C.byref(n_keys), _p(tile_off), _p(tile_slot))
    return ids, km, int(n_keys.value), tile_off, tile_slot[: n_keys.value].copy()


def render(scene, view, bg=(0.0, 0.0, 0.0), tile_w=16, tile_h=16, near=0.2, mode="tiled",
           bands=None):
    """FP64 render of one view (Eq. 3). mode: 'brute' or 'tiled'."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    H, W = view.height, view.width
    bgv = np.asarray(bg, np.float64)
    rgb = np.zeros((3, H, W), np.float64)
    T = np.zeros((H, W), np.float64)
    last_slot = np.zeros((H, W), np.int32)
    last_pos = np.zeros((H, W), np.int32)
    flags = np.zeros((H, W), np.uint8)
    b = _bands(bands if bands is not None else {})
    rc = lib().or_render(C.byref(ref.s), C.byref(vw), _p(bgv), tile_w, tile_h, near,
                         0 if mode == "brute" else 1, C.byref(b), _p(rgb), _p(T),
                         _p(last_slot), _p(last_pos), _p(flags))
    if rc != 0:
        raise MemoryError("oracle render failed")
    return dict(rgb=rgb, T=T, last_slot=last_slot, last_pos=last_pos, flags=flags)


def render_variants(scene, view, px, py, bands, bg=(0.0, 0.0, 0.0), tile_w=16, tile_h=16,
                    near=0.2, max_per=256):
    """Every valid (rgb, T, last) of selected pixels (tiled walk) when the
    per-pair tests of Eq. 3 may be decided either way at pairs whose FP64 test
    value lies within `bands` of its threshold. Returns a list, per pixel, of
    (rgb[v,3], T[v], last[v]) arrays, or None for a pixel with more than
    max_per results."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    n = px.shape[0]
    bgv = np.asarray(bg, np.float64)
    out = np.zeros((max(1, n), max_per, 4), np.float64)
    last = np.zeros((max(1, n), max_per), np.int32)
    cnt = np.zeros(max(1, n), np.int32)
    b = _bands(bands)
    rc = lib().or_render_variants(C.byref(ref.s), C.byref(vw), _p(bgv), tile_w, tile_h, near,
                                  C.byref(b), n, _p(px), _p(py), max_per, _p(out), _p(last),
                                  _p(cnt))
    if rc != 0:
        raise MemoryError("oracle variants failed")
    res = []
    for k in range(n):
        c = int(cnt[k])
        res.append(None if c < 0 else (out[k, :c, :3].copy(), out[k, :c, 3].copy(),
                                       last[k, :c].copy()))
    return res


def render_pixels(scene, view, px, py, bg=(0.0, 0.0, 0.0), near=0.2, bands=None):
    """Brute-force FP64 render of selected pixels."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    n = px.shape[0]
    bgv = np.asarray(bg, np.float64)
    rgb = np.zeros((n, 3), np.float64)
    T = np.zeros(n, np.float64)
    last_slot = np.zeros(n, np.int32)
    flags = np.zeros(n, np.uint8)
    b = _bands(bands if bands is not None else {})
    lib().or_render_pixels(C.byref(ref.s), C.byref(vw), _p(bgv), near, C.byref(b), n, _p(px),
                           _p(py), _p(rgb), _p(T), _p(last_slot), _p(flags))
    return dict(rgb=rgb, T=T, last_slot=last_slot, flags=flags)


def zero_grads(scene):
    K = (scene.sh_degree + 1) ** 2
    n = scene.n
    return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)))


def render_bwd(scene, view, dLdC, bg=(0.0, 0.0, 0.0), tile_w=16, tile_h=16, near=0.2,
               bands=None, grads=None):
    """FP64 analytic backward of one tiled view for dL/dC ([3,H,W]); grads of
    non-frozen slots are accumulated into `grads` (FP64 dict). Returns
    (grads, grad2d [n_active,9], rec_flags [n_active], ids)."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    if grads is None:
        grads = zero_grads(scene)
    for k in grads:
        assert grads[k].dtype == np.float64 and grads[k].flags.c_contiguous
    G = OrGrads(_p(grads["means"]).value, _p(grads["log_scales"]).value,
                _p(grads["quats"]).value, _p(grads["opacity_logits"]).value,
                _p(grads["sh"]).value)
    ids = active_ids(scene.start, scene.expire, view.frame)
    g2 = np.zeros((max(1, len(ids)), 9), np.float64)
    rf = np.zeros(max(1, len(ids)), np.uint8)
    d = _c(dLdC, np.float64)
    bgv = np.asarray(bg, np.float64)
    b = _bands(bands if bands is not None else {})
    rc = lib().or_render_bwd(C.byref(ref.s), C.byref(vw), _p(bgv), tile_w, tile_h, near, _p(d),
                             C.byref(b), C.byref(G), _p(g2), _p(rf))
    if rc != 0:
        raise MemoryError("oracle backward failed")
    return grads, g2[: len(ids)], rf[: len(ids)], ids


def project(scene, view, slot):
    """FP64 (u, v, A, B, C, opacity, r, g, b, depth) of one Gaussian in one view."""
    ref = _SceneRef(scene)
    vw = make_view(view)
    out = np.zeros(10, np.float64)
    lib().or_project(C.byref(ref.s), C.byref(vw), int(slot), _p(out))
    return out


def sh_basis(dirs) -> np.ndarray:
    """Real SH basis (16 functions, degrees 0..3) at unit directions [n,3]."""
    dirs = np.asarray(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((dirs.shape[0], 16), np.float64)
    L = lib()
    for i, (x, y, z) in enumerate(dirs):
        L.or_sh_basis(float(x), float(y), float(z), _p(out[i]))
    return out


def philox4x64(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, np.uint64).reshape(4).copy()
    k = np.asarray(key, np.uint64).reshape(2).copy()
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64(_p(c), _p(k), _p(out))
    return out


def normal3(seed: int, step: int, slot: int) -> np.ndarray:
    out = np.zeros(3, np.float64)
    lib().or_normal3(seed, step, slot, _p(out))
    return out


def reloc_weight(logit: float) -> int:
    return int(lib().or_reloc_weight(float(logit)))


def reloc_values(o: float, n: int):
    on, ratio = C.c_double(0), C.c_double(0)
    lib().or_reloc_values(float(o), int(n), C.byref(on), C.byref(ratio))
    return on.value, ratio.value


DEFAULT_SGLD = dict(lr_means=1.6e-4, lr_log_scales=5e-3, lr_quats=1e-3, lr_logits=5e-2,
                    lr_sh_dc=2.5e-3, lr_sh_rest=2.5e-3 / 20.0, beta1=0.9, beta2=0.999,
                    eps=1e-15, noise_lr=5e4, noise_k=100.0, noise_t=0.005, adam=0,
                    relocate=1, max_n=51)


def sgld_step(scene, grads, adam, frames, params=None, seed=0, step=0):
    """One Adam (optional) + SGLD noise (+ relocation) step on a copy of
    `scene`. grads: dict of float32 arrays (same keys as zero_grads) or None;
    adam: dict with m_*/v_* float32 arrays or None. Returns (scene, adam,
    n_dead, targets)."""
    p = dict(DEFAULT_SGLD)
    if params:
        p.update(params)
    s = scene.copy()
    st_arr = dict(means=_c(s.means, np.float32), log_scales=_c(s.log_scales, np.float32),
                  quats=_c(s.quats, np.float32), logits=_c(s.opacity_logits, np.float32),
                  sh=_c(s.sh, np.float32), start=_c(s.start, np.int32),
                  expire=_c(s.expire, np.int32), frozen=_c(s.frozen, np.uint8))
    st = OrState(*[_p(st_arr[k]).value for k in ("means", "log_scales", "quats", "logits", "sh",
                                                  "start", "expire", "frozen")],
                 s.n, s.sh_degree)
    if grads is None:
        grads = {k: np.zeros_like(v, dtype=np.float32) for k, v in zero_grads(scene).items()}
    g_arr = {k: _c(grads[k], np.float32) for k in ("means", "log_scales", "quats",
                                                    "opacity_logits", "sh")}
    fg = OrFGrads(_p(g_arr["means"]).value, _p(g_arr["log_scales"]).value,
                  _p(g_arr["quats"]).value, _p(g_arr["opacity_logits"]).value,
                  _p(g_arr["sh"]).value)
    if adam is None:
        adam = {f"{mv}_{k}": np.zeros_like(v, dtype=np.float32)
                for k, v in zero_grads(scene).items() for mv in ("m", "v")}
    a_arr = {k: _c(v, np.float32) for k, v in adam.items()}
    ad = OrAdam(*[_p(a_arr[k]).value for k in (
        "m_means", "v_means", "m_log_scales", "v_log_scales", "m_quats", "v_quats",
        "m_opacity_logits", "v_opacity_logits", "m_sh", "v_sh")])
    fr = _c(frames, np.int32)
    targets = np.full(max(1, s.n), -1, np.int32)
    n_dead = lib().or_sgld_step(C.byref(st), C.byref(fg), C.byref(ad), _p(fr), len(fr),
                                C.byref(OrSgldParams(**p)), int(seed), int(step), _p(targets))
    s.means, s.log_scales, s.quats = st_arr["means"], st_arr["log_scales"], st_arr["quats"]
    s.opacity_logits, s.sh = st_arr["logits"], st_arr["sh"]
    return s, a_arr, int(n_dead), targets[: s.n]


def l1_loss_grad(rgbs, targets):
    """Alg. 1 loss_func (L1 term): mean over views of mean |C - target| over
    3*H*W, and dL/dC = sign(C - target) / (3*H*W*V) with sign(0) = 0."""
    V = len(rgbs)
    loss = 0.0
    grads = []
    for c, t in zip(rgbs, targets):
        d = np.asarray(c, np.float64) - np.asarray(t, np.float64)
        n = d.size
        loss += np.abs(d).sum() / n / V
        grads.append(np.sign(d) / (n * V))
    return loss, grads


def slice_range(target_frame: int, swin_size: int, num_gs: int):
    """Alg. 2: slice = target_frame mod swin_size, slots [slice*S, (slice+1)*S)
    with S = num_gs / swin_size."""
    slice_size = num_gs // swin_size
    s = target_frame % swin_size
    return s * slice_size, (s + 1) * slice_size


def frame_update(buffer, update, target_frame: int, swin_size: int):
    """Alg. 2 update_thread: overwrite the slice of `buffer` (a Scene) that
    target_frame maps to with `update` (a Scene of slice_size Gaussians),
    lifespans included. Returns a new Scene."""
    out = buffer.copy()
    lo, hi = slice_range(target_frame, swin_size, buffer.n)
    assert hi - lo == update.n
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire",
              "birth", "frozen"):
        getattr(out, k)[lo:hi] = getattr(update, k)
    return out


_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire", "birth",
           "frozen")


def _rows(scene, idx):
    """The rows idx of a scene, as a new object of the same type."""
    d = {k: getattr(scene, k)[idx].copy() for k in _FIELDS}
    return type(scene)(sh_degree=scene.sh_degree, **d)


def _concat(a, b):
    d = {k: np.concatenate([getattr(a, k), getattr(b, k)]) for k in _FIELDS}
    return type(a)(sh_degree=a.sh_degree, **d)


def schedule_expire(gs, swin_size: int):
    """Alg. 1 schedule_expire, which the paper does not define (reading): after
    the first window [0, swin_size) the gs slots split into swin_size equal
    slices (Sec. 4.2.1) and slice k gets expire = k for k >= 1, slice 0 expire =
    swin_size. Expiries then fall on distinct frames modulo swin_size, so one
    slice matures per frame, and a slice's next version (birth = its expire) is
    inserted by Alg. 2 at buffer slice birth mod swin_size = k, the slice whose
    data just expired. Returns a new scene."""
    out = gs.copy()
    slice_size = gs.n // swin_size
    for k in range(swin_size):
        out.expire[k * slice_size:(k + 1) * slice_size] = k if k >= 1 else swin_size
    return out


def mature(gs, matured, st: int, swin_size: int, num_gs: int):
    """Alg. 1 mature(st), in the algorithm's order:
    mature_idx = the gs slots with start < st (ascending);
    the stream receives gs[mature_idx] as they are (stream.write);
    matured += those rows (marked frozen: no longer optimised), then only the
    last num_gs rows are kept;
    gs[mature_idx]: birth = expire, start = expire, expire = start + swin_size.
    gs: scene of the optimisable Gaussians; matured: scene of the matured rows,
    oldest first (may be empty). Returns (gs', matured', snapshot, mature_idx)."""
    idx = np.nonzero(gs.start < st)[0]
    snap = _rows(gs, idx)
    grown = _rows(snap, np.arange(snap.n))
    grown.frozen[:] = 1
    m2 = grown if matured is None or matured.n == 0 else _concat(matured, grown)
    if m2.n > num_gs:
        m2 = _rows(m2, np.arange(m2.n - num_gs, m2.n))
    g2 = gs.copy()
    g2.birth[idx] = gs.expire[idx]
    g2.start[idx] = gs.expire[idx]
    g2.expire[idx] = g2.start[idx] + swin_size
    return g2, m2, snap, idx


def reg_loss_grad(scene, view_frames, opacity_reg: float, scale_reg: float):
    """Alg. 1 reg(active_gs) with the regularisers of [14] (Sec. 4.4; weights
    opacity_reg = 2e-2, scale_reg = 1e-2 in Sec. 8.1), for a batch whose loss is
    the mean over its views (view v renders frame view_frames[v]):
        reg_v = opacity_reg * mean_{i active at f_v} sigmoid(logit_i)
              + scale_reg * mean_{i active at f_v, c} exp(log_scale_ic),
    loss = mean_v reg_v. Active includes frozen (matured) Gaussians, which
    receive no gradient. Returns (loss, grads) with grads of the logits and
    log-scales (FP64; the other attributes get none)."""
    V = len(view_frames)
    logit = scene.opacity_logits.astype(np.float64)
    ls = scene.log_scales.astype(np.float64)
    sig = 1.0 / (1.0 + np.exp(-logit))
    sc = np.exp(ls)
    g_logit = np.zeros_like(logit)
    g_ls = np.zeros_like(ls)
    loss = 0.0
    live = scene.frozen == 0
    for f in view_frames:
        act = (scene.start <= f) & (f < scene.expire)
        n = int(act.sum())
        if n == 0:
            continue
        loss += (opacity_reg * sig[act].mean() + scale_reg * sc[act].mean()) / V
        m = act & live
        g_logit[m] += opacity_reg * sig[m] * (1.0 - sig[m]) / (n * V)
        g_ls[m] += scale_reg * sc[m] / (3 * n * V)
    return loss, {"opacity_logits": g_logit, "log_scales": g_ls}


def mean_grad_scale(start, window_start: int, swin_size: int, decay: float):
    """Sec. 4.5.1, whose formula the paper does not give (reading): the gradient
    of a Gaussian's means is scaled by decay^(k - 1), k = window_start - start +
    swin_size the number of windows [st, st + swin_size) that have trained its
    current lifespan [start, start + swin_size) so far (k >= 1)."""
    k = np.maximum(1, window_start - np.asarray(start, np.int64) + swin_size)
    return np.float64(decay) ** (k - 1).astype(np.float64)


def opacity_u8(logits) -> np.ndarray:
    """Table 6 opacity code k = rint(255 sigmoid(logit)) (FP32, key-mode exp)."""
    lg = _c(logits, np.float32)
    out = np.zeros(max(1, lg.size), np.uint8)
    lib().or_opacity_u8(_p(lg), lg.size, _p(out))
    return out[: lg.size].copy()


def slice_encode(rows, keep: int):
    """Table 6 quantisation of one slice (Sec. 5.6.2: means fp16, rotation
    uint8, scale fp16, opacity uint8, only the DC of the SH kept, at full
    precision) and the ABR tail drop of Sec. 5.5 (keep the `keep` Gaussians of
    highest opacity, ties by slot; the rest travel as nothing and are marked
    empty on decode). The slice's rows share one lifespan (Sec. 4.2.1), sent
    once. Returns the packet as a dict of arrays, kept rows in slot order.

    Codes: means and log-scales: float16 (round to nearest even); quaternion:
    q / |q| per component as rint((q_c + 1) * 127.5); opacity: opacity_u8; DC:
    float32."""
    S = rows.n
    keep = int(min(max(keep, 0), S))
    order = np.lexsort((np.arange(S), -rows.opacity_logits.astype(np.float64)))
    kept = np.sort(order[:keep]).astype(np.uint32)
    q = rows.quats[kept].astype(np.float32)
    nn = q[:, 0] * q[:, 0]
    nn = nn + q[:, 1] * q[:, 1]
    nn = nn + q[:, 2] * q[:, 2]
    nn = nn + q[:, 3] * q[:, 3]
    qn = q / np.sqrt(nn)[:, None]
    qk = np.clip(np.rint((qn + np.float32(1.0)) * np.float32(127.5)), 0, 255).astype(np.uint8)
    return dict(count=S, keep=keep, sh_degree=rows.sh_degree,
                birth=int(rows.birth[0]) if S else 0, start=int(rows.start[0]) if S else 0,
                expire=int(rows.expire[0]) if S else 0,
                index=kept, means=rows.means[kept].astype(np.float16),
                log_scales=rows.log_scales[kept].astype(np.float16), quats=qk,
                opacity=opacity_u8(rows.opacity_logits[kept]),
                dc=rows.sh[kept, 0, :].astype(np.float32))


def slice_decode(pkt, make):
    """Inverse of slice_encode into a full slice of pkt['count'] rows built by
    make(n, sh_degree) -> empty scene: kept rows get means and log-scales back
    to float32, q_c = k * (2/255) - 1, logit = ln(o / (1 - o)) with o =
    clamp(k, 0.5, 254.5) / 255, the DC and zero higher SH bands, the slice's
    lifespan and frozen = 1 (a streamed snapshot); dropped rows are left empty
    (start = expire: never active)."""
    S, K = pkt["count"], (pkt["sh_degree"] + 1) ** 2
    out = make(S, pkt["sh_degree"])
    out.start[:] = pkt["start"]
    out.expire[:] = pkt["start"]
    out.birth[:] = pkt["birth"]
    out.frozen[:] = 1
    i = pkt["index"].astype(np.int64)
    out.means[i] = pkt["means"].astype(np.float32)
    out.log_scales[i] = pkt["log_scales"].astype(np.float32)
    out.quats[i] = pkt["quats"].astype(np.float32) * np.float32(2.0 / 255.0) - np.float32(1.0)
    o = np.clip(pkt["opacity"].astype(np.float32), np.float32(0.5), np.float32(254.5)) \
        / np.float32(255.0)
    out.opacity_logits[i] = np.log(o / (np.float32(1.0) - o))
    out.sh[i] = 0.0
    out.sh[i, 0, :] = pkt["dc"]
    out.expire[i] = pkt["expire"]
    return out


def slice_packet_bytes(count: int, keep: int) -> int:
    """Payload bytes of a packet: 29 per kept Gaussian (6 + 6 + 4 + 1 + 12),
    plus a 4-byte slot index each when the tail drop removed any."""
    return keep * 29 + (4 * keep if keep < count else 0)
