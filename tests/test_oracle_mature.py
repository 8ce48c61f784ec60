"""Pins of the oracle's maturation (Alg. 1 mature, schedule_expire) against
what the paper fixes: the worked example of Sec. 4.2.1 (slices of a 5-frame
window), one slice maturing per frame, the matured set keeping the last
num_gs rows, and the stream that maturation writes driving the client of
Alg. 2 (update_thread) to exactly the versions each frame needs."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth


def _gs(num_gs, swin, seed=0):
    """Alg. 1 main: num_gs random Gaussians, birth = start = 0, expire =
    swin_size. means[:, 0] carries the slot index, to follow copies."""
    rng = np.random.default_rng(seed)
    attrs = synth.make_gaussians(rng, num_gs, 1)
    attrs["means"][:, 0] = np.arange(num_gs, dtype=np.float32)
    z = np.zeros(num_gs, np.int32)
    return synth._scene(attrs, 1, z.copy(), np.full(num_gs, swin, np.int32), birth=z.copy())


def _train(gs, st):
    """Stand-in for train_swin: every version gets distinct parameters."""
    g = gs.copy()
    g.means[:, 1] += np.float32(1.0)
    g.means[:, 2] = np.float32(st)
    return g


def _run(oracle, num_gs, swin, last_st):
    gs = schedule_expire_first = None
    gs = _train(_gs(num_gs, swin), 0)
    gs = oracle.schedule_expire(gs, swin)
    matured, stream, idxs = None, [], []
    for st in range(1, last_st + 1):
        gs, matured, snap, idx = oracle.mature(gs, matured, st, swin, num_gs)
        stream.append(snap)
        idxs.append(idx)
        gs = _train(gs, st)
    return gs, matured, stream, idxs


def _slice_of(slot, num_gs, swin):
    return int(slot) // (num_gs // swin)


def test_schedule_expire_reading(oracle_mod):
    g = oracle_mod.schedule_expire(_gs(10, 5), 5)
    assert list(g.expire) == [5, 5, 1, 1, 2, 2, 3, 3, 4, 4]
    assert list(g.start) == [0] * 10


def test_sec_4_2_1_worked_example(oracle_mod):
    """Sec. 4.2.1 (Fig. 5, swin_size 5): training frame N+1 of the window
    [N, N+5) renders matured slices #0, #1, #4 and optimisable slices #2, #3;
    after that window slice #2 matures (no further chance to train frame N)."""
    swin, S = 5, 3
    num_gs = swin * S
    N = 12  # a window start at which slice #2 holds frame N
    gs, matured, stream, idxs = _run(oracle_mod, num_gs, swin, N)
    f = N + 1
    act_gs = {_slice_of(i, num_gs, swin) for i in range(num_gs)
              if gs.start[i] <= f < gs.expire[i]}
    act_ma = {_slice_of(matured.means[i, 0], num_gs, swin) for i in range(matured.n)
              if matured.start[i] <= f < matured.expire[i]}
    assert act_gs == {2, 3}
    assert act_ma == {0, 1, 4}
    _, _, _, idx = oracle_mod.mature(gs, matured, N + 1, swin, num_gs)
    assert {_slice_of(i, num_gs, swin) for i in idx} == {2}
    assert len(idx) == S


def test_one_slice_matures_per_frame(oracle_mod):
    swin, S = 4, 5
    num_gs = swin * S
    _, _, stream, idxs = _run(oracle_mod, num_gs, swin, 25)
    assert len(idxs[0]) == num_gs  # st = 1: the whole first window is snapshotted
    for st, idx in enumerate(idxs[1:], start=2):
        assert len(idx) == S
        assert {_slice_of(i, num_gs, swin) for i in idx} == {(st - 1) % swin}
        # the version streamed at st became active at its birth, st - 1
        assert set(stream[st - 1].birth.tolist()) == {st - 1}


def test_matured_keeps_the_last_num_gs(oracle_mod):
    swin, S = 4, 3
    num_gs = swin * S
    _, matured, stream, _ = _run(oracle_mod, num_gs, swin, 20)
    allrows = np.concatenate([s.means for s in stream])
    assert matured.n == num_gs
    np.testing.assert_array_equal(matured.means, allrows[-num_gs:])
    assert matured.frozen.all()


def test_stream_drives_the_alg2_client(oracle_mod):
    """Alg. 2: the client reads num_gs Gaussians, then inserts every later
    update at frame = its birth, into buffer slice birth mod swin_size. At
    every frame its active set must be the streamed versions covering it."""
    swin, S, T = 5, 4, 23
    num_gs = swin * S
    _, _, stream, _ = _run(oracle_mod, num_gs, swin, T)
    buffer = stream[0]
    assert buffer.n == num_gs
    events = {int(s.birth[0]): s for s in stream[1:]}
    allv = [s for s in stream]
    for f in range(0, T):
        if f in events:
            buffer = oracle_mod.frame_update(buffer, events[f], f, swin)
        got = sorted(map(tuple, buffer.means[(buffer.start <= f) & (f < buffer.expire)]))
        want = sorted(tuple(r) for s in allv for r, a, b in zip(s.means, s.start, s.expire)
                      if a <= f < b)
        assert got == want, f
        assert len(got) == num_gs
