"""Launch-shape autotuner for the batched multi-view render.

Candidates: tile shape (8x8, 16x16, 32x8) x Gaussians staged per block step
(32, 64, 128, 256) x pixels per thread, for the forward blend (and, in
"fwdbwd" mode, the reverse blend). Each candidate is timed with CUDA events on
the workload given (after a warm-up render); the fastest is returned and
cached in a JSON file keyed by GPU name, workload signature (resolutions,
active count bucket) and mode, so later runs reuse it without timing.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path
from typing import Optional, Sequence

import torch

from . import api

TILES = [(8, 8), (16, 16), (32, 8)]
BATCHES = [32, 64, 128, 256]
FWD_PPT = {(8, 8): [1, 2], (16, 16): [1, 2, 4], (32, 8): [1, 2, 4]}
BWD_PPT = {(8, 8): [1, 2], (16, 16): [2, 4, 8], (32, 8): [2, 4, 8]}

DEFAULT_CACHE = Path(os.environ.get("SWGS_AUTOTUNE_CACHE",
                                    Path.home() / ".cache" / "swgs_autotune.json"))


def signature(state: api.GaussianState, views: Sequence, mode: str) -> str:
    res = sorted({(int(v.width), int(v.height)) for v in views})
    frames = sorted({int(v.frame) for v in views})
    n = state.n
    bucket = 2 ** int(round(math.log2(max(1, n))))
    dev = torch.cuda.get_device_name()
    return f"{dev}|{mode}|n~{bucket}|sh{state.sh_degree}|views{len(views)}|frames{len(frames)}|" + \
        ",".join(f"{w}x{h}" for w, h in res)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def candidates(mode: str):
    for tile in TILES:
        for batch in BATCHES:
            for ppt in FWD_PPT[tile]:
                if mode == "fwd":
                    yield dict(tile=tile, batch=batch, pixels_per_thread=ppt,
                               bwd_pixels_per_thread=min(ppt, 2) if tile == (8, 8) else 8,
                               bwd_batch=32)
                else:
                    for bppt in BWD_PPT[tile]:
                        for bbatch in (32, 64, 128):
                            yield dict(tile=tile, batch=batch, pixels_per_thread=ppt,
                                       bwd_pixels_per_thread=bppt, bwd_batch=bbatch)


def autotune(state: api.GaussianState, views: Sequence, mode: str = "fwd", reps: int = 3,
             cache: Optional[Path] = DEFAULT_CACHE, shortlist: Optional[list] = None,
             verbose: bool = False) -> dict:
    """Return the fastest launch shape for rendering `views` of `state`
    ("fwd": forward only; "fwdbwd": forward with the L1 term, backward)."""
    key = signature(state, views, mode)
    table = {}
    if cache is not None and Path(cache).exists():
        try:
            table = json.loads(Path(cache).read_text())
        except (OSError, ValueError):
            table = {}
        if key in table:
            c = dict(table[key]["config"])
            c["tile"] = tuple(c["tile"])
            return c
    cands = list(shortlist) if shortlist is not None else list(candidates(mode))
    targets = dl = grads = None
    if mode == "fwdbwd":
        targets = [torch.zeros((3, v.height, v.width), device="cuda") for v in views]
        grads = state.zero_grads()
    best, best_ms, results = None, float("inf"), []
    for c in cands:
        r = api.Renderer(**c)
        try:
            if mode == "fwd":
                def run():
                    r.render(state, views)
            else:
                def run():
                    _, d, _, saved = r.render_l1(state, views, targets)
                    r.backward(state, saved, d, grads)
                    saved.release()
            ms = _time(run, reps)
        finally:
            r.close()
        results.append((ms, c))
        if verbose:
            print(f"{ms:8.3f} ms  {c}")
        if ms < best_ms:
            best, best_ms = c, ms
    if cache is not None:
        table[key] = {"config": dict(best, tile=list(best["tile"])), "ms": best_ms}
        Path(cache).parent.mkdir(parents=True, exist_ok=True)
        tmp = Path(str(cache) + f".tmp{os.getpid()}")
        tmp.write_text(json.dumps(table, indent=1))
        os.replace(tmp, cache)
    return dict(best)
