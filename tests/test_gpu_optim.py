"""GPU parity of the steps after the backward pass (Alg. 1 noise and relocate,
the optimiser of [14]), of the L1 term, and of the per-frame slice update
(Alg. 2 update_thread), against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def R():
    assert torch.cuda.is_available()
    from paper_2409_07759_b300 import api
    r = api.Renderer()
    yield r
    r.close()


def _state(scene):
    from paper_2409_07759_b300 import api
    return api.GaussianState.from_scene(scene)


def _np(t):
    return t.detach().cpu().numpy()


def _scene(n=30000, dead=0.02, seed=7):
    sc, _, _ = synth.config2(width=64, height=48, n=n, n_frames=3, per_frame=1,
                             forced_dead_fraction=dead)
    rng = np.random.default_rng(seed)
    # most slots live through frames 145..147; 30% matured (frozen)
    sc.start = rng.integers(100, 150, n).astype(np.int32)
    sc.expire = (sc.start + 50).astype(np.int32)
    sc.frozen = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    grads = {k: rng.normal(0, 1e-3, size=getattr(sc, k).shape).astype(np.float32) for k in NAMES}
    adam = {}
    for k in NAMES:
        shape = getattr(sc, k).shape
        adam["m_" + k] = rng.normal(0, 1e-4, size=shape).astype(np.float32)
        adam["v_" + k] = rng.uniform(1e-8, 1e-6, size=shape).astype(np.float32)
    return sc, grads, adam


def _run_gpu(R, sc, grads, adam, frames, params, seed, step):
    from paper_2409_07759_b300 import api
    st = _state(sc)
    g = api.GaussianGrads(*[torch.from_numpy(grads[k]).cuda() for k in NAMES], sc.sh_degree)
    ad = {k: torch.from_numpy(v.copy()).cuda() for k, v in adam.items()}
    tg = torch.full((sc.n,), -5, dtype=torch.int32, device="cuda")
    nrel = R.sgld_step(st, frames, params, seed, step, grads=g, adam=ad, targets=tg,
                       count_relocated=True)
    return st, ad, _np(tg), nrel


BASE = dict(lr_means=1.6e-4, lr_log_scales=5e-3, lr_quats=1e-3, lr_logits=5e-2, lr_sh_dc=2.5e-3,
            lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15, noise_lr=5e4,
            noise_k=100.0, noise_t=0.005, adam=0, relocate=1, max_n=51)


def test_relocation_targets_bit_exact(R, oracle_mod):
    """Relocation sampling (integer CDF of floor(opacity 2^32), Philox draws)
    picks the same target for every dead slot as the oracle, the same number of
    dead slots, and the same relocated opacities and scales."""
    sc, grads, adam = _scene()
    frames = [145, 146, 147]
    st, ad, tg, nrel = _run_gpu(R, sc, grads, adam, frames, BASE, seed=11, step=3)
    ref, ref_adam, nd, tref = oracle_mod.sgld_step(sc, grads, adam, frames, BASE, seed=11, step=3)
    assert nrel == nd > 100
    np.testing.assert_array_equal(tg, tref)
    moved = tref >= 0
    touched = moved.copy()
    touched[tref[moved]] = True
    for k in ("opacity_logits", "log_scales"):
        np.testing.assert_allclose(_np(getattr(st, k))[touched], getattr(ref, k)[touched],
                                   rtol=2e-6, atol=2e-6)
    for k in ("quats", "sh"):
        np.testing.assert_array_equal(_np(getattr(st, k))[moved], getattr(ref, k)[moved])
    # moments of every touched slot are zeroed
    for k, v in ad.items():
        assert (_np(v)[touched] == 0).all()


def test_noise_matches_oracle(R, oracle_mod):
    """SGLD noise: mu += lr * noise_lr * sigmoid(-k(o - t)) Sigma eta with the
    same Philox draws; FP32 against FP64 within 1e-5 of the update scale."""
    sc, grads, adam = _scene(dead=0.0)
    sc.opacity_logits[:] = np.random.default_rng(3).normal(-5.3, 0.3, sc.n).astype(np.float32)
    p = dict(BASE, relocate=0)
    frames = [145, 146]
    st, _, _, _ = _run_gpu(R, sc, grads, adam, frames, p, seed=5, step=9)
    ref, _, _, _ = oracle_mod.sgld_step(sc, grads, adam, frames, p, seed=5, step=9)
    d_gpu = _np(st.means).astype(np.float64) - sc.means
    d_ref = ref.means.astype(np.float64) - sc.means
    scale = np.abs(d_ref).max()
    assert scale > 0
    assert np.abs(d_gpu - d_ref).max() <= 1e-5 * scale + 2e-7
    # untouched: frozen or inactive slots
    act = np.zeros(sc.n, bool)
    for f in frames:
        act |= (sc.start <= f) & (f < sc.expire)
    el = act & (sc.frozen == 0)
    np.testing.assert_array_equal(_np(st.means)[~el], sc.means[~el])


def test_adam_matches_oracle(R, oracle_mod):
    """Bias-corrected Adam on eligible slots (then noise) within FP32 rounding."""
    sc, grads, adam = _scene(dead=0.0)
    p = dict(BASE, adam=1, relocate=0, noise_lr=0.0)
    frames = [146]
    st, ad, _, _ = _run_gpu(R, sc, grads, adam, frames, p, seed=1, step=4)
    ref, ref_adam, _, _ = oracle_mod.sgld_step(sc, grads, adam, frames, p, seed=1, step=4)
    for k in NAMES:
        np.testing.assert_allclose(_np(getattr(st, k)), getattr(ref, k), rtol=1e-6, atol=1e-7)
    for k in ad:
        # beta1 m + (1 - beta1) g can cancel: compare at FP32 resolution of the
        # array's own scale
        ref_k = ref_adam[k]
        np.testing.assert_allclose(_np(ad[k]), ref_k, rtol=1e-5,
                                   atol=1e-6 * float(np.abs(ref_k).max()))


def test_full_step_valid(R, oracle_mod):
    """Adam + noise + relocation together: every relocated slot copies an
    alive, eligible target; the Gaussian count is unchanged; N coincident
    copies keep the target's opacity: 1 - (1 - o')^N = o."""
    sc, grads, adam = _scene()
    p = dict(BASE, adam=1)
    frames = [145, 146, 147]
    st, _, tg, nrel = _run_gpu(R, sc, grads, adam, frames, p, seed=2, step=0)
    assert nrel > 100 and st.n == sc.n
    act = np.zeros(sc.n, bool)
    for f in frames:
        act |= (sc.start <= f) & (f < sc.expire)
    el = act & (sc.frozen == 0)
    dead = np.nonzero(tg >= 0)[0]
    assert el[dead].all() and el[tg[dead]].all() and (tg[tg[dead]] == -1).all()
    counts = np.bincount(tg[dead], minlength=sc.n)
    o_new = 1 / (1 + np.exp(-_np(st.opacity_logits).astype(np.float64)))
    for j in np.unique(tg[dead])[:50]:
        N = min(counts[j] + 1, 51)
        on = o_new[j]
        o_before = 1 - (1 - on) ** N
        assert 0 < o_before < 1
        np.testing.assert_array_equal(_np(st.means)[dead[tg[dead] == j]],
                                      np.repeat(_np(st.means)[j][None], (tg[dead] == j).sum(), 0))


def test_l1_gradient_matches_oracle(R, oracle_mod):
    """L1 term on GPU images against the oracle's definition on the same
    (host) arrays: loss and every dL/dC element."""
    rng = np.random.default_rng(0)
    views = [synth.View(33, 17, 10, 10, 16, 8), synth.View(64, 48, 10, 10, 32, 24)]
    rgbs = [rng.uniform(size=(3, v.height, v.width)).astype(np.float32) for v in views]
    tgts = [rng.uniform(size=(3, v.height, v.width)).astype(np.float32) for v in views]
    tgts[0][1, 2, 3] = rgbs[0][1, 2, 3]
    loss, dls = R.loss_l1(views, [torch.from_numpy(x).cuda() for x in rgbs],
                          [torch.from_numpy(x).cuda() for x in tgts])
    ref_loss, ref_dl = oracle_mod.l1_loss_grad(rgbs, tgts)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    for a, b in zip(dls, ref_dl):
        np.testing.assert_allclose(_np(a), b, rtol=1e-6, atol=0)


@pytest.mark.parametrize("on_host", [True, False])
def test_frame_update_matches_alg2(R, oracle_mod, on_host):
    """Alg. 2 update_thread: the slice (target_frame mod swin_size) of the slot
    buffer is overwritten with the update, lifespans included; the rest stays."""
    from paper_2409_07759_b300 import api
    swin, S = 10, 500
    buf = synth.config4_initial(slice_size=S, swin_size=swin, sh_degree=3)
    st = _state(buf)
    ref = buf
    for f in range(1, 13):
        upd = synth.config4_slice(f, S, swin, 3)
        ust = _state(upd)
        first, count = api.slice_range(f, swin, buf.n)
        assert count == S
        R.frame_update(st, first, ust.pin_host() if on_host else ust, src_on_host=on_host)
        ref = oracle_mod.frame_update(ref, upd, f, swin)
        torch.cuda.synchronize()
        for k in NAMES + ("start", "expire", "birth", "frozen"):
            np.testing.assert_array_equal(_np(getattr(st, k)), getattr(ref, k))
        ids = _np(R.active_ids(st, f))
        np.testing.assert_array_equal(ids, np.arange(buf.n, dtype=np.int32))


# ------------------------------------------------- data-parallel exchange --

def test_grad_pack_unpack_eligible_rows(R):
    """swgs_grad_pack: the eligible slots (active at one of the frames, not
    frozen), ascending, and their gradient rows (means 3, log_scales 3, quats 4,
    logit 1, sh 3K) times the scale, bit for bit; swgs_grad_unpack writes the
    rows back to those slots only."""
    from paper_2409_07759_b300 import api
    sc, _, _ = _scene(n=20011)
    st = _state(sc)
    rng = np.random.default_rng(3)
    g = st.zero_grads()
    for k in NAMES:
        getattr(g, k).copy_(torch.from_numpy(
            rng.normal(size=tuple(getattr(g, k).shape)).astype(np.float32)))
    frames = [145, 147]
    f = np.asarray(frames)
    act = ((sc.start[:, None] <= f[None, :]) & (f[None, :] < sc.expire[:, None])).any(1)
    want_ids = np.nonzero(act & (sc.frozen == 0))[0]
    K = 16
    ids = torch.full((sc.n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    packed = torch.full((sc.n, 11 + 3 * K), float("nan"), dtype=torch.float32, device="cuda")
    R.grad_pack(st, g, frames, ids, cnt, packed, scale=0.25)
    n = int(cnt.item())
    assert n == len(want_ids) and 0 < n < sc.n
    np.testing.assert_array_equal(_np(ids[:n]), want_ids)
    host = {k: _np(getattr(g, k)) for k in NAMES}
    rows = np.concatenate([host[k][want_ids].reshape(n, -1) for k in NAMES], 1) * np.float32(0.25)
    np.testing.assert_array_equal(_np(packed[:n]), rows)
    g2 = st.zero_grads()
    R.grad_unpack(g2, ids, cnt, packed)
    for k in NAMES:
        a = _np(getattr(g2, k))
        np.testing.assert_array_equal(a[want_ids], host[k][want_ids] * np.float32(0.25))
        mask = np.ones(sc.n, bool)
        mask[want_ids] = False
        assert not np.any(a[mask])


def test_row_exchange_through_nccl():
    """One rank (NCCL): the eligible-row exchange of dp.GradientReducer leaves
    the backward's gradients scaled by the rank's view share, bit for bit
    (x 0.5 is exact), exchanging fewer than half the buffer's floats; and a
    window step with the reducer runs through it."""
    import datetime
    import os
    import socket
    import torch.distributed as dist
    from paper_2409_07759_b300 import api, dp
    from paper_2409_07759_b300.window import WindowTrainer
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(s.getsockname()[1])
    s.close()
    dist.init_process_group("nccl", rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=60))
    try:
        sc, views, targets = synth.config2(width=128, height=96, n=20000, n_frames=3,
                                           per_frame=2, forced_dead_fraction=0.01)
        tg = [torch.from_numpy(t).cuda() for t in targets]
        r = api.Renderer()
        st = api.GaussianState.from_scene(sc)
        grads = st.zero_grads()
        imgs, dls, loss, saved = r.render_l1(st, views, tg)
        r.backward(st, saved, dls, grads)
        saved.release()
        before = {k: _np(getattr(grads, k)).copy() for k in NAMES}
        frames = sorted({v.frame for v in views})
        red = dp.GradientReducer(1, 2)
        red(None, loss, rows=dp.RowExchange(r, st, grads, frames))
        for k in NAMES:
            np.testing.assert_array_equal(_np(getattr(grads, k)), before[k] * np.float32(0.5))
        assert 0 < red.last_exchanged < st.n * (11 + 48) // 2
        tr = WindowTrainer(r, st, views, tg, seed=5,
                           reduce=dp.GradientReducer(len(views), len(views)))
        assert torch.isfinite(tr.step(0)).all()
        torch.cuda.synchronize()
        r.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("adam_on", [1, 0])
def test_sgld_step_clears_gradients_it_reads(R, adam_on):
    """clear_grads = 1: with or without the Adam step, every gradient element of
    an eligible slot is zero after the step and the others are untouched. The
    parameters move exactly as with clear_grads = 0."""
    from paper_2409_07759_b300 import api
    sc, grads, adam = _scene(n=9001)
    frames = [145, 146]
    out = []
    for clear in (0, 1):
        st = _state(sc)
        g = api.GaussianGrads(*[torch.from_numpy(grads[k]).cuda() for k in NAMES], sc.sh_degree)
        ad = {k: torch.from_numpy(v.copy()).cuda() for k, v in adam.items()}
        R.sgld_step(st, frames, dict(adam=adam_on, relocate=1, lr_means=1e-3, noise_lr=5e4,
                                     noise_k=100.0, noise_t=0.005, beta1=0.9, beta2=0.999,
                                     eps=1e-15, lr_log_scales=5e-3, lr_quats=1e-3,
                                     lr_logits=5e-2, lr_sh_dc=2.5e-3, lr_sh_rest=1.25e-4,
                                     max_n=51, clear_grads=clear), 9, 4, grads=g, adam=ad)
        torch.cuda.synchronize()
        out.append((st, g))
    f = np.asarray(frames)
    elig = ((sc.start[:, None] <= f[None, :]) & (f[None, :] < sc.expire[:, None])).any(1) \
        & (sc.frozen == 0)
    for k in NAMES:
        assert torch.equal(getattr(out[0][0], k), getattr(out[1][0], k)), k
        kept, cleared = _np(getattr(out[0][1], k)), _np(getattr(out[1][1], k))
        np.testing.assert_array_equal(kept, grads[k])
        assert not np.any(cleared[elig])
        np.testing.assert_array_equal(cleared[~elig], grads[k][~elig])
