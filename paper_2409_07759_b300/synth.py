"""Seeded synthetic inputs shaped like the multi-view dynamic captures SwinGS
trains and streams (Sec. 5.1: a ring of cameras around a scene, 300-frame clips,
Gaussians with [start, expire) lifespans; Sec. 4.2, Alg. 1 and Alg. 2).

This module only draws random numbers and places cameras. It contains none of
the splatting arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any of the method's code.

Everything is numpy, float32 for Gaussian attributes (the renderer's input
precision) and int32 for lifespans.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "View", "make_gaussians", "look_at", "ring_cameras",
    "fibonacci_cameras", "intrinsics_for", "config0", "config1", "config2",
    "config3", "config4_initial", "config4_slice", "tiny_scene",
    "sh_coeff_count",
]


def sh_coeff_count(degree: int) -> int:
    """Number of SH coefficients per colour channel for a degree (Sec. 8.1)."""
    return (degree + 1) * (degree + 1)


@dataclass
class Scene:
    """Slot-major (structure of arrays) Gaussian state.

    means[N,3], log_scales[N,3], quats[N,4] (w,x,y,z, unnormalised),
    opacity_logits[N], sh[N,K,3] (K = (degree+1)^2), start/expire/birth[N]
    (a slot is active at frame t iff start <= t < expire, Alg. 1 and 2),
    frozen[N] (1 = matured: rendered, never optimised; Alg. 1 'matured').
    """
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    start: np.ndarray
    expire: np.ndarray
    birth: np.ndarray
    frozen: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def copy(self) -> "Scene":
        return Scene(**{k: (v.copy() if isinstance(v, np.ndarray) else v)
                        for k, v in self.__dict__.items()})


@dataclass
class View:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    R (3x3, row-major) and t map world to camera: p_cam = R @ p_world + t.
    frame is the video frame whose active set this view renders.
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))
    frame: int = 0


def intrinsics_for(width: int, height: int):
    """Field of view of the 128x96, fx=100 camera kept at every resolution."""
    f = 100.0 * width / 128.0
    return f, f, width / 2.0, height / 2.0


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, -1.0, 0.0)):
    """World-to-camera (R, t) for a camera at `eye` looking at `target`.

    Rows of R are the camera's x (right), y (down) and z (forward) axes in world
    coordinates; `up` is the world direction that appears at the top of the image.
    """
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, dtype=np.float64)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-6:  # looking along `up`: pick another reference
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    return R, t


def ring_cameras(n: int, radius: float, width: int, height: int):
    """n cameras in the y=0 plane at angle 2*pi*k/n, looking at the origin."""
    fx, fy, cx, cy = intrinsics_for(width, height)
    views = []
    for k in range(n):
        a = 2.0 * math.pi * k / n
        R, t = look_at((radius * math.cos(a), 0.0, radius * math.sin(a)))
        views.append(View(width, height, fx, fy, cx, cy, R, t, 0))
    return views


def fibonacci_cameras(n: int, radius: float):
    """n camera positions on a Fibonacci sphere of the given radius."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for k in range(n):
        y = 1.0 - 2.0 * (k + 0.5) / n
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        a = golden * k
        out.append((radius * rr * math.cos(a), radius * y, radius * rr * math.sin(a)))
    return out


def make_gaussians(rng: np.random.Generator, n: int, sh_degree: int, *,
                   dc_low: float = 0.0, dc_high: float = 1.0,
                   rest_std: float = 0.1) -> dict:
    """Draw the attribute distributions used by every workload:
    means U[-1,1]^3, log-scales N(-3, 0.5), quaternions N(0,1)^4 normalised,
    opacity logits N(0,1), SH DC U[dc_low, dc_high], higher bands N(0, rest_std).
    """
    k = sh_coeff_count(sh_degree)
    means = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    log_scales = rng.normal(-3.0, 0.5, size=(n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    logits = rng.normal(0.0, 1.0, size=n).astype(np.float32)
    sh = np.empty((n, k, 3), dtype=np.float32)
    sh[:, 0, :] = rng.uniform(dc_low, dc_high, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, size=(n, k - 1, 3))
    return dict(means=means, log_scales=log_scales, quats=quats,
                opacity_logits=logits, sh=sh)


def _lifespans(rng, n, clip_frames, len_lo, len_hi):
    start = rng.integers(0, clip_frames, size=n).astype(np.int32)
    length = rng.integers(len_lo, len_hi + 1, size=n).astype(np.int32)
    return start, (start + length).astype(np.int32)


def _scene(attrs, sh_degree, start, expire, frozen=None, birth=None) -> Scene:
    n = attrs["means"].shape[0]
    return Scene(sh_degree=sh_degree, start=start, expire=expire,
                 birth=(start.copy() if birth is None else birth),
                 frozen=(np.zeros(n, np.uint8) if frozen is None else frozen),
                 **attrs)


def config0():
    """Plain forward: 4,096 Gaussians, SH degree 0, one 128x96 camera (fx=fy=100)
    at the origin looking down +z, means U[-1,1]^3 shifted 4 units ahead, every
    lifespan covering frame 0, 16x16 tiles. The DC coefficient is drawn from
    U[-sqrt(pi), sqrt(pi)], the range that the degree-0 band maps onto colours
    U[0, 1]."""
    rng = np.random.default_rng(0)
    s = math.sqrt(math.pi)
    attrs = make_gaussians(rng, 4096, 0, dc_low=-s, dc_high=s)
    attrs["means"][:, 2] += 4.0
    n = 4096
    scene = _scene(attrs, 0, np.zeros(n, np.int32), np.ones(n, np.int32))
    view = View(128, 96, 100.0, 100.0, 64.0, 48.0, np.eye(3, dtype=np.float32),
                np.zeros(3, np.float32), 0)
    return scene, [view]


def config1(width: int = 1352, height: int = 1014):
    """Single frame fwd+bwd: 100k Gaussians, SH degree 3, lifespans start
    U{0..299}, length U{10..60}; frame 150; one camera at (0,0,-4); an L1 target
    image U[0,1] (seed 1)."""
    rng = np.random.default_rng(1)
    n = 100_000
    attrs = make_gaussians(rng, n, 3)
    start, expire = _lifespans(rng, n, 300, 10, 60)
    scene = _scene(attrs, 3, start, expire)
    fx, fy, cx, cy = intrinsics_for(width, height)
    R, t = look_at((0.0, 0.0, -4.0))
    view = View(width, height, fx, fy, cx, cy, R, t, 150)
    target = rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)
    return scene, [view], [target]


def config2(width: int = 1352, height: int = 1014, n: int = 300_000,
            first_frame: int = 145, n_frames: int = 10, per_frame: int = 4,
            forced_dead_fraction: float = 0.0, rank: int = 0):
    """Sliding-window training step: 300k Gaussians, SH3, lifespans as config 1;
    20 ring cameras; frames 145..154 with 4 of the 20 cameras per frame drawn
    without replacement (seed 2) -> 40 views; targets U[0,1]; frozen = start <
    first_frame (the maturation rule of Alg. 1). `forced_dead_fraction` sets that
    fraction of logits to -8 so that relocation has work to do. `rank` > 0 keeps
    the scene and draws that rank's own cameras and targets (data-parallel
    weak scaling; rank 0 is the single-GPU workload)."""
    rng = np.random.default_rng(2)
    attrs = make_gaussians(rng, n, 3)
    start, expire = _lifespans(rng, n, 300, 10, 60)
    frozen = (start < first_frame).astype(np.uint8)
    if forced_dead_fraction > 0:
        k = int(round(forced_dead_fraction * n))
        idx = rng.choice(n, size=k, replace=False)
        attrs["opacity_logits"][idx] = -8.0
    scene = _scene(attrs, 3, start, expire, frozen=frozen)
    ring = ring_cameras(20, 4.0, width, height)
    if rank > 0:
        rng = np.random.default_rng([2, rank])
    views, targets = [], []
    for f in range(first_frame, first_frame + n_frames):
        for c in rng.choice(20, size=per_frame, replace=False):
            v = ring[int(c)]
            views.append(View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
    for v in views:
        targets.append(rng.uniform(0.0, 1.0, size=(3, v.height, v.width)).astype(np.float32))
    return scene, views, targets


CONFIG3_RESOLUTIONS = [(640, 480)] * 8 + [(1280, 720)] * 16 + [(1920, 1080)] * 8


def config3(n: int = 1_000_000, resolutions=None):
    """Batched multi-view forward: 1M Gaussians, SH3, start U{0..299}, length
    U{40..80}, frame 150 (about 20% active); 32 Fibonacci-sphere cameras at
    radius 4 with 8 x 640x480, 16 x 1280x720 and 8 x 1920x1080."""
    rng = np.random.default_rng(3)
    attrs = make_gaussians(rng, n, 3)
    start, expire = _lifespans(rng, n, 300, 40, 80)
    scene = _scene(attrs, 3, start, expire)
    res = CONFIG3_RESOLUTIONS if resolutions is None else resolutions
    views = []
    for pos, (w, h) in zip(fibonacci_cameras(len(res), 4.0), res):
        fx, fy, cx, cy = intrinsics_for(w, h)
        R, t = look_at(pos)
        views.append(View(w, h, fx, fy, cx, cy, R, t, 150))
    return scene, views


SWIN_SIZE_SERVING = 50
SLICE_SIZE_SERVING = 6_000


def config4_slice(frame: int, slice_size: int = SLICE_SIZE_SERVING,
                  swin_size: int = SWIN_SIZE_SERVING, sh_degree: int = 3) -> Scene:
    """The update a server streams for `frame` (Alg. 2): slice_size fresh
    Gaussians born at `frame`, living for swin_size frames (seed 4 + frame;
    slices born before frame 0 use the seed sequence [4, -frame])."""
    rng = np.random.default_rng(4 + frame if frame >= 0 else [4, -frame])
    attrs = make_gaussians(rng, slice_size, sh_degree)
    start = np.full(slice_size, frame, np.int32)
    return _scene(attrs, sh_degree, start, start + swin_size)


def config4_initial(slice_size: int = SLICE_SIZE_SERVING,
                    swin_size: int = SWIN_SIZE_SERVING, sh_degree: int = 3) -> Scene:
    """Slot buffer as a client holds it right after the frame-0 update: slice s
    holds the Gaussians born at the latest frame b <= 0 with b = s (mod
    swin_size), so every slot is active at frame 0."""
    parts = []
    for s in range(swin_size):
        b = s if s == 0 else s - swin_size
        parts.append(config4_slice(b, slice_size, swin_size, sh_degree))
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])
    return Scene(means=cat("means"), log_scales=cat("log_scales"), quats=cat("quats"),
                 opacity_logits=cat("opacity_logits"), sh=cat("sh"), start=cat("start"),
                 expire=cat("expire"), birth=cat("birth"), frozen=cat("frozen"),
                 sh_degree=sh_degree)


def tiny_scene(seed: int, n: int = 16, sh_degree: int = 1, width: int = 32,
               height: int = 24, depth: float = 4.0, log_scale_mean: float = -2.0,
               spread: float = 0.6):
    """A few Gaussians in front of a small camera, for brute-force and
    finite-difference checks."""
    rng = np.random.default_rng(seed)
    attrs = make_gaussians(rng, n, sh_degree)
    attrs["means"] *= spread
    attrs["means"][:, 2] += depth
    attrs["log_scales"] = rng.normal(log_scale_mean, 0.3, size=(n, 3)).astype(np.float32)
    scene = _scene(attrs, sh_degree, np.zeros(n, np.int32), np.ones(n, np.int32))
    fx, fy, cx, cy = intrinsics_for(width, height)
    view = View(width, height, fx, fy, cx, cy, np.eye(3, dtype=np.float32),
                np.zeros(3, np.float32), 0)
    return scene, view
