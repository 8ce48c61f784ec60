"""Checkpoint / resume and injected failures on the device.

A clip (Alg. 1 main) interrupted after some windows, saved to a file, loaded
into a fresh trainer and continued ends bit-identical to an uninterrupted run
(Adam off: the gradient sums' atomic order would otherwise move Adam's first
step by +-lr; the SGLD noise and relocation draws are counter-based). An
allocation refused by the caller's allocator makes a call fail with ENOMEM and
leaves the context usable."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire", "birth",
          "frozen")


def _clip(swin=4, S=50):
    num_gs = swin * S
    sc, _, _ = synth.config2(width=64, height=48, n=num_gs, n_frames=1, per_frame=1,
                             forced_dead_fraction=0.05)
    ring = synth.ring_cameras(20, 4.0, 64, 48)

    def window(st, ed):
        views, targets = [], []
        g = torch.Generator(device="cuda")
        for f in range(st, ed):
            v = ring[(3 * f) % 20]
            views.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
            g.manual_seed(1000 + f)
            targets.append(torch.randint(0, 256, (3, 48, 64), dtype=torch.uint8, device="cuda",
                                         generator=g))
        return views, targets
    return sc, window, swin


def test_resume_is_bit_identical(tmp_path):
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300.window import ClipTrainer
    sc, window, swin = _clip()
    T = 11
    params = dict(adam=0)
    r = api.Renderer()
    full = ClipTrainer(r, api.GaussianState.from_scene(sc), swin, window, iterations=2,
                       params=params, seed=9)
    full.run(T)
    first = ClipTrainer(r, api.GaussianState.from_scene(sc), swin, window, iterations=2,
                        params=params, seed=9)
    first.run(T, stop=6)
    first.save(tmp_path / "ckpt.bin")
    resumed = ClipTrainer(r, api.GaussianState.from_scene(synth.config2(
        width=64, height=48, n=full.num_gs, n_frames=1, per_frame=1)[0]), swin, window,
        iterations=2, params=params, seed=0)
    resumed.load(tmp_path / "ckpt.bin")
    assert resumed.next_start == 6
    resumed.run(T, start=resumed.next_start)
    torch.cuda.synchronize()
    for k in FIELDS:
        assert torch.equal(getattr(full.buf, k), getattr(resumed.buf, k)), k
    assert full.head == resumed.head and full.step_count == resumed.step_count
    s_full = [(st, n) for st, n, _ in full.stream]
    s_split = [(st, n) for st, n, _ in first.stream + resumed.stream]
    assert s_full == s_split
    for (a, b) in zip(full.stream, first.stream + resumed.stream):
        for k in FIELDS:
            assert torch.equal(a[2][k], b[2][k]), (a[0], k)
    r.close()


def test_refused_allocation_fails_cleanly():
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300._abi import SwgsError, STATUS_NAMES
    sc, views, _ = synth.config2(width=96, height=64, n=3000, n_frames=2, per_frame=2)
    allow = {"on": True}
    r = api.Renderer(alloc_guard=lambda nbytes: allow["on"])
    st = api.GaussianState.from_scene(sc)
    ref, _ = api.Renderer().render(st, views)
    allow["on"] = False
    r2 = api.Renderer(alloc_guard=lambda nbytes: allow["on"])
    with pytest.raises(SwgsError) as e:
        r2.render(st, views)
    assert "ENOMEM" in str(e.value)
    allow["on"] = True
    img, _ = r2.render(st, views)
    for a, b in zip(img, ref):
        assert torch.equal(a, b)
    r.close()
    r2.close()
