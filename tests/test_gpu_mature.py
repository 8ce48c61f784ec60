"""Maturation of Alg. 1 on the device (swgs_mature, swgs_schedule_expire)
against the oracle, step by step over a clip: the matured count, the
snapshot rows (stream.write), the optimisable half of the buffer and the ring
of matured rows read oldest first from its head, all bit for bit."""
import gc

import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire", "birth",
          "frozen")


def _gs(num_gs, swin, seed=3):
    rng = np.random.default_rng(seed)
    attrs = synth.make_gaussians(rng, num_gs, 1)
    z = np.zeros(num_gs, np.int32)
    return synth._scene(attrs, 1, z.copy(), np.full(num_gs, swin, np.int32), birth=z.copy())


def _train_host(gs, st):
    g = gs.copy()
    g.means[:, 1] += np.float32(1.0)
    g.means[:, 2] = np.float32(st)
    return g


def _train_dev(buf, num_gs, st):
    buf.means[:num_gs, 1] += 1.0
    buf.means[:num_gs, 2] = float(st)


def _eq(dev, host, what):
    np.testing.assert_array_equal(dev.cpu().numpy(), host, err_msg=what)


@pytest.mark.parametrize("swin,S", [(5, 300), (4, 7)])
def test_maturation_matches_oracle(oracle_mod, swin, S):
    from paper_2409_07759_b300 import api
    num_gs = swin * S
    r = api.Renderer()
    g0 = _gs(num_gs, swin)
    host = _train_host(g0, 0)
    buf = api.GaussianState.with_matured_ring(api.GaussianState.from_scene(g0))
    _train_dev(buf, num_gs, 0)
    host = oracle_mod.schedule_expire(host, swin)
    r.schedule_expire(buf, num_gs, swin)
    _eq(buf.expire[:num_gs], host.expire, "schedule_expire")
    matured, head = None, 0
    dev_snap = api.GaussianState.from_scene(g0)             # num_gs rows on the device
    host_snap = api.GaussianState.from_scene(g0).pin_host()  # num_gs rows, pinned host
    for st in range(1, 4 * swin + 3):
        host, matured, snap, idx = oracle_mod.mature(host, matured, st, swin, num_gs)
        use_host = st % 2 == 0
        n, head = r.mature(buf, num_gs, st, swin, head,
                           snapshot=host_snap if use_host else dev_snap)
        torch.cuda.synchronize()
        assert n == len(idx), st
        for k in FIELDS:
            got = host_snap[k][:n].numpy() if use_host else getattr(dev_snap, k)[:n].cpu().numpy()
            np.testing.assert_array_equal(got, getattr(snap, k), err_msg=f"snapshot {k} st={st}")
            _eq(getattr(buf, k)[:num_gs], getattr(host, k), f"gs {k} st={st}")
        # the ring, oldest first from the head, is the matured list
        order = (head + np.arange(num_gs)) % num_gs + num_gs
        assert matured.n == num_gs
        for k in FIELDS:
            _eq(getattr(buf, k)[torch.from_numpy(order).cuda()], getattr(matured, k),
                f"ring {k} st={st}")
        host = _train_host(host, st)
        _train_dev(buf, num_gs, st)
    r.close()


def test_maturation_rejects_bad_buffers():
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300._abi import SwgsError
    r = api.Renderer()
    g = api.GaussianState.from_scene(_gs(20, 5))
    with pytest.raises(SwgsError):  # no room for the ring
        r.mature(g, 20, 1, 5, 0)
    buf = api.GaussianState.with_matured_ring(g)
    with pytest.raises(SwgsError):  # num_gs not a multiple of swin_size
        r.mature(buf, 20, 1, 3, 0)
    with pytest.raises(SwgsError):  # head outside the ring
        r.mature(buf, 20, 1, 5, 20)
    r.close()


def test_clip_trainer_streams_a_valid_alg2_sequence(oracle_mod):
    """Alg. 1 main on a short clip: the first snapshot holds all num_gs
    Gaussians, every later one one slice born at st - 1, and an Alg. 2 client
    fed the stream has exactly num_gs Gaussians covering every frame."""
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300.window import ClipTrainer
    swin, S, T = 5, 40, 9
    num_gs = swin * S
    sc, _, _ = synth.config2(width=64, height=48, n=num_gs, n_frames=1, per_frame=1)
    ring = synth.ring_cameras(20, 4.0, 64, 48)
    rng = np.random.default_rng(5)
    tg = {}

    def window(st, ed):
        views, targets = [], []
        for f in range(st, ed):
            for c in (f % 20, (f + 7) % 20):
                v = ring[c]
                views.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
                if (f, c) not in tg:
                    tg[(f, c)] = torch.from_numpy(
                        rng.integers(0, 256, size=(3, 48, 64), dtype=np.uint8)).cuda()
                targets.append(tg[(f, c)])
        return views, targets

    r = api.Renderer()
    gs = api.GaussianState.from_scene(sc)
    ct = ClipTrainer(r, gs, swin, window, iterations=2, seed=1)
    loss = ct.run(T)
    torch.cuda.synchronize()
    assert np.isfinite(float(loss.item()))
    assert [n for _, n, _ in ct.stream] == [num_gs] + [S] * (T - 1)
    for st, n, snap in ct.stream[1:]:
        assert set(snap["birth"][:n].tolist()) == {st - 1}
    assert bool((ct.buf.frozen[num_gs:] == 1).all()) and bool((ct.buf.frozen[:num_gs] == 0).all())
    # the codec stream decodes, on the device, into a client buffer that covers
    # every frame with num_gs Gaussians (Alg. 2 with Table 6 packets)
    ct2 = ClipTrainer(r, api.GaussianState.from_scene(sc), swin, window, iterations=1, seed=1,
                      codec=True)
    ct2.run(T)
    assert [n for _, n, _ in ct2.stream] == [S] * (swin + T - 1)
    client = api.GaussianState.from_scene(sc)
    for k in range(swin):  # Alg. 2 main: the first num_gs Gaussians
        r.slice_decode(ct2.stream[k][2], client, k * S)
    ev = {}
    for st, n, pkt in ct2.stream[swin:]:
        ev[st - 1] = pkt
    for f in range(T):
        if f in ev:
            first, _ = api.slice_range(f, swin, num_gs)
            r.slice_decode(ev[f], client, first)
        act = (client.start <= f) & (client.expire > f)
        assert int(act.sum()) == num_gs, f

    def scene_of(snap, n):
        d = {k: snap[k][:n].numpy().copy() for k in FIELDS}
        return synth.Scene(sh_degree=sc.sh_degree, **d)

    buffer = scene_of(ct.stream[0][2], num_gs)
    events = {int(snap["birth"][0]): scene_of(snap, n) for _, n, snap in ct.stream[1:]}
    for f in range(T):
        if f in events:
            buffer = oracle_mod.frame_update(buffer, events[f], f, swin)
        assert int(((buffer.start <= f) & (f < buffer.expire)).sum()) == num_gs, f
    r.close()


def test_training_memory_does_not_grow_with_clip_length():
    """Table 3 in spirit: the device memory of training a clip (Alg. 1 main)
    is the same for 10, 30 and 100 frames -- the buffer holds gs and the
    matured ring, the window's views are the only per-step inputs and the
    stream goes to pinned host memory."""
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300.window import ClipTrainer
    swin, S = 5, 60
    num_gs = swin * S
    sc, _, _ = synth.config2(width=64, height=48, n=num_gs, n_frames=1, per_frame=1)
    ring = synth.ring_cameras(20, 4.0, 64, 48)

    def window(st, ed):
        views, targets = [], []
        g = torch.Generator(device="cuda")
        for f in range(st, ed):
            v = ring[f % 20]
            views.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
            g.manual_seed(f)
            targets.append(torch.randint(0, 256, (3, 48, 64), dtype=torch.uint8, device="cuda",
                                         generator=g))
        return views, targets

    peaks = {}
    for T in (10, 30, 100):
        r = api.Renderer()
        ct = ClipTrainer(r, api.GaussianState.from_scene(sc), swin, window, iterations=1)
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        ct.run(T)
        torch.cuda.synchronize()
        peaks[T] = torch.cuda.max_memory_allocated() - base
        assert len(ct.stream) == T
        r.close()
        del ct
        gc.collect()
    assert peaks[10] > 0
    assert max(peaks.values()) <= 1.02 * min(peaks.values()), peaks
