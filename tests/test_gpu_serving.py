"""GPU tests of the continuous-batching playback server (Alg. 2 with many
viewers): a request's image is the same alone and inside a mixed batch, every
request is served while slices are swapped in per frame, the slot buffer ends
equal to the Alg. 2 replay, and admission respects the HBM budget."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SWIN, SLICE = 10, 3000
RES = [(320, 240), (640, 360), (640, 360), (480, 270)]


def _pool(n=4):
    return [synth.config4_slice(1000 + i, SLICE, SWIN, 3) for i in range(n)]


def _provider(pool):
    from paper_2409_07759_b300 import api
    pinned = [api.GaussianState.from_scene(s).pin_host() for s in pool]

    def get(frame):
        h = pinned[frame % len(pinned)]
        h["start"].fill_(frame)
        h["expire"].fill_(frame + SWIN)
        h["birth"].fill_(frame)
        return h
    return get


def _loop(budget=16e9, n_streams=2, deferred=False):
    from paper_2409_07759_b300 import api, serving
    scene = synth.config4_initial(SLICE, SWIN, 3)
    st = api.GaussianState.from_scene(scene)
    pool = _pool()
    loop = serving.ServingLoop(st, SWIN, fps=30.0, n_streams=n_streams, max_batch=8,
                               hbm_budget_bytes=budget, slice_provider=_provider(pool),
                               deferred_sizing=deferred)
    return scene, st, pool, loop


def test_alone_equals_mixed_batch():
    """Continuous batching changes nothing in the result: each request's image
    is bit-identical alone and rendered together with other viewers'."""
    from paper_2409_07759_b300 import serving
    _, st, _, loop = _loop()
    reqs = serving.make_requests(6, 5.0, 2.0, seed=1, resolutions=RES)[:5]
    alone = [loop.render_batch(0, [r], 0.0)[0][0] for r in reqs]
    mixed = loop.render_batch(1, reqs, 0.0)[0]
    torch.cuda.synchronize()
    for a, b in zip(alone, mixed):
        assert torch.equal(a, b)
    loop.close()


@pytest.mark.parametrize("deferred", [False, True])
def test_run_serves_everything_and_swaps_slices(oracle_mod, deferred):
    """A short real-time run: every request completes, one slice is swapped in
    per video frame, and the slot buffer equals the Alg. 2 replay (with the
    workers' forwards sized exactly, and with deferred sizing)."""
    from paper_2409_07759_b300 import serving
    scene, st, pool, loop = _loop(deferred=deferred)
    reqs = serving.make_requests(8, 30.0, 1.5, seed=2, resolutions=RES)
    stats = loop.run(reqs, 1.5)
    assert stats.n == len(reqs) > 100
    assert all(r.done >= r.arrival for r in reqs)
    assert stats.updates >= 30 and stats.p99_ms >= stats.p50_ms > 0
    ref = scene
    for f in range(1, loop.frame + 1):
        upd = pool[f % len(pool)].copy()
        upd.start[:] = f
        upd.expire[:] = f + SWIN
        upd.birth[:] = f
        ref = oracle_mod.frame_update(ref, upd, f, SWIN)
    torch.cuda.synchronize()
    for k in ("means", "opacity_logits", "sh", "start", "expire"):
        np.testing.assert_array_equal(getattr(st, k).cpu().numpy(), getattr(ref, k))
    # requests see a frame at or after the one current at their arrival
    for r in reqs:
        assert r.frame >= int(r.arrival * 30.0) - 1
    loop.close()


def test_budget_limits_batches():
    """With a budget smaller than two requests, every batch holds one request
    (and only one batch is in flight at a time)."""
    from paper_2409_07759_b300 import serving
    _, st, _, loop = _loop(budget=1.0)
    reqs = serving.make_requests(8, 30.0, 0.5, seed=3, resolutions=RES)
    stats = loop.run(reqs, 0.5)
    assert stats.n == len(reqs) and stats.mean_batch == 1.0
    loop.close()


def test_budget_bounds_bytes_in_flight_across_workers():
    """A budget of about three requests and three worker streams under heavy
    load: the admitted bytes of the batches in flight together (one counter
    over all workers) never exceed the budget, and the budget binds."""
    from paper_2409_07759_b300 import serving
    _, st, _, loop = _loop(n_streams=3)
    loop.reserve(640, 360)
    one = loop.request_bytes(serving.make_requests(1, 5.0, 1.0, seed=9,
                                                   resolutions=[(640, 360)])[0])
    assert one > 152 * st.n * 0.9  # the measured size: about one record per Gaussian
    loop.budget = 3.2 * one
    reqs = serving.make_requests(16, 60.0, 0.6, seed=6, resolutions=RES)
    stats = loop.run(reqs, 0.6)
    assert stats.n == len(reqs)
    assert 2.0 * one < stats.inflight_hwm_bytes <= loop.budget, (stats, one)
    assert stats.mean_batch <= 3.0
    loop.close()


def test_reserved_buffers_give_the_same_images():
    """After reserve(), a worker renders into its reserved output buffers (no
    allocation while serving); the images equal the allocating path's, and a
    run that keeps its images gets copies, not the reused buffers."""
    from paper_2409_07759_b300 import serving
    _, st, _, loop = _loop()
    reqs = serving.make_requests(6, 5.0, 2.0, seed=1, resolutions=RES)[:5]
    before = [o.clone() for o in loop.render_batch(1, reqs, 0.0)[0]]
    loop.reserve(640, 360)
    after = loop.render_batch(1, reqs, 0.0)[0]
    # delivered into the worker's pinned host rows
    base = loop.host_pool[1][0].data_ptr()
    end = base + loop.host_pool[1][0].numel() * 4
    assert all(base <= o.data_ptr() < end and o.is_pinned() for o in after)
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    run = serving.make_requests(8, 30.0, 0.5, seed=5, resolutions=RES)
    stats, images = loop.run(run, 0.5, keep_images=True)
    assert stats.n == len(run) == len(images)
    assert all(not (base <= im.data_ptr() < end) for im in images.values())
    assert stats.p99_ms >= stats.p99_render_ms
    loop.close()
