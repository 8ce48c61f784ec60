"""Data-parallel host logic on CPU (gloo, world size 2).

The window's views are split across two ranks; each rank takes the FP64
oracle's L1 gradient of its own views, and the weighted all-reduce of
`dp.GradientReducer` must give the gradient (and loss) of the whole window
computed on one process. After the reduction both replicas take the same
SGLD/relocation step from the same seed and step, so their states are
bitwise equal. A rank that never joins makes the others' rendezvous fail
with an error instead of hanging."""
import datetime
import hashlib
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

from paper_2409_07759_b300 import dp, synth  # noqa: E402

GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _window():
    # two frames x two cameras of a small config-2-style window
    sc, views, targets = synth.config2(width=64, height=48, n=3000, n_frames=2, per_frame=2)
    return sc, views, targets


def _oracle_grads(oracle, sc, views, targets):
    rgbs = [oracle.render(sc, v)["rgb"] for v in views]
    loss, dl = oracle.l1_loss_grad(rgbs, targets)
    g = oracle.zero_grads(sc)
    for v, d in zip(views, dl):
        oracle.render_bwd(sc, v, d, grads=g)
    return loss, g


def _flat(g):
    return torch.from_numpy(np.concatenate([g[k].ravel() for k in GRAD_KEYS]))


def _unflat(flat, like):
    out, o = {}, 0
    for k in GRAD_KEYS:
        n = like[k].size
        out[k] = flat[o:o + n].numpy().reshape(like[k].shape)
        o += n
    return out


class _HostRows:
    """Host stand-in of dp.RowExchange for the CPU ranks: the gradient rows of
    the eligible slots (active at a frame of the window, not frozen) in the
    library's row layout (means 3, log_scales 3, quats 4, logit 1, sh 3K)."""

    def __init__(self, sc, g, frames):
        f = np.asarray(frames)
        act = ((sc.start[:, None] <= f[None, :]) & (f[None, :] < sc.expire[:, None])).any(1)
        self.ids = np.nonzero(act & (sc.frozen == 0))[0]
        self.g = g

    def pack(self, scale=1.0):
        rows = np.concatenate([self.g[k][self.ids].reshape(len(self.ids), -1) for k in GRAD_KEYS],
                              axis=1)
        return torch.from_numpy(rows * scale), len(self.ids)

    def unpack(self, packed, n):
        o = 0
        for k in GRAD_KEYS:
            w = int(np.prod(self.g[k].shape[1:]))
            self.g[k][self.ids] = packed[:n, o:o + w].numpy().reshape((n,) + self.g[k].shape[1:])
            o += w


def _worker(rank, world, port, result_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    import oracle
    sc, views, targets = _window()
    mine = dp.shard_views(len(views), rank, world)
    lv = [views[i] for i in mine]
    lt = [targets[i] for i in mine]
    loss, g = _oracle_grads(oracle, sc, lv, lt)
    flat = _flat(g)
    lt_loss = torch.tensor([loss], dtype=torch.float64)
    red = dp.GradientReducer(len(lv), dp.total_views(len(lv)))
    # the eligible rows' exchange: the same sums from far fewer floats
    frames = sorted({v.frame for v in views})
    g_rows = {k: v.copy() for k, v in g.items()}
    rows = _HostRows(sc, g_rows, frames)
    outside = np.setdiff1d(np.arange(sc.n), rows.ids)
    for k in GRAD_KEYS:  # nothing outside the eligible rows carries a gradient
        assert not np.any(g[k][outside]), k
    red(None, None, rows=rows)
    exchanged = red.last_exchanged
    red(flat, lt_loss)
    reduced = _unflat(flat, g)
    for k in GRAD_KEYS:
        np.testing.assert_allclose(g_rows[k], reduced[k], rtol=1e-13,
                                   atol=1e-15 * max(1e-30, np.abs(reduced[k]).max()))
    assert exchanged < flat.numel() / 2, (exchanged, flat.numel())
    # the replicas' optimiser step from the reduced gradients
    grads32 = {k: v.astype(np.float32) for k, v in reduced.items()}
    new, _, n_dead, tg = oracle.sgld_step(sc, grads32, None, [v.frame for v in views],
                                          dict(adam=1, relocate=1), seed=11, step=3)
    h = hashlib.sha256()
    for a in (new.means, new.log_scales, new.quats, new.opacity_logits, new.sh, tg):
        h.update(np.ascontiguousarray(a).tobytes())
    np.savez(os.path.join(result_dir, f"rank{rank}.npz"), loss=lt_loss.numpy(),
             digest=np.frombuffer(h.digest(), np.uint8), n_dead=n_dead,
             **{k: v for k, v in reduced.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_shard_views_partition():
    for world in range(1, 7):
        for n in (0, 1, 5, 40, 41):
            parts = [dp.shard_views(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        dp.shard_views(4, 2, 2)


def test_view_weight():
    assert dp.view_weight(20, 40) == 0.5
    assert dp.view_weight(3, 7) == 3 / 7
    for bad in ((-1, 4), (5, 4), (1, 0)):
        with pytest.raises(ValueError):
            dp.view_weight(*bad)


def test_rank_workloads_share_the_scene():
    a = synth.config2(width=32, height=24, n=500, n_frames=2, per_frame=2, rank=0)
    b = synth.config2(width=32, height=24, n=500, n_frames=2, per_frame=2, rank=1)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire",
              "frozen"):
        np.testing.assert_array_equal(getattr(a[0], k), getattr(b[0], k))
    assert [v.frame for v in a[1]] == [v.frame for v in b[1]]
    assert not all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))


def test_two_rank_gradient_allreduce_matches_whole_window(oracle_mod, tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    sc, views, targets = _window()
    loss, g = _oracle_grads(oracle_mod, sc, views, targets)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    for r in (r0, r1):
        assert abs(float(r["loss"][0]) - loss) <= 1e-12 * max(1.0, abs(loss))
        for k in GRAD_KEYS:
            np.testing.assert_allclose(r[k], g[k], rtol=1e-10,
                                       atol=1e-12 * max(1e-30, np.abs(g[k]).max()))
    assert np.abs(g["means"]).max() > 0
    # identical replicas after the optimiser / SGLD / relocation step
    np.testing.assert_array_equal(r0["digest"], r1["digest"])
    assert int(r0["n_dead"]) == int(r1["n_dead"])


def _lonely(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=3))
    except Exception:
        return
    raise AssertionError("rendezvous completed without the second rank")


def test_missing_rank_fails_the_rendezvous():
    # rank 1 of 2 never starts: rank 0's rendezvous must end with an error
    mp.spawn(_lonely, args=(2, _free_port()), nprocs=1, join=True)
