"""Alg. 1 reg() (opacity and scale regularisers, Sec. 4.4 / 8.1) in the
backward, and the means-gradient scale of Sec. 4.5.1 in the Adam step,
against the oracle."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _scene():
    rng = np.random.default_rng(21)
    n = 3000
    attrs = synth.make_gaussians(rng, n, 1)
    attrs["means"][:, 2] += 0.0
    start = rng.integers(0, 6, size=n).astype(np.int32)
    expire = (start + rng.integers(1, 5, size=n)).astype(np.int32)
    frozen = (rng.random(n) < 0.3).astype(np.uint8)
    return synth._scene(attrs, 1, start, expire, frozen=frozen)


def _views(frames, w=96, h=64):
    ring = synth.ring_cameras(20, 4.0, w, h)
    out = []
    for j, f in enumerate(frames):
        v = ring[(3 * j) % 20]
        out.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, f))
    return out


def test_regulariser_alone_matches_oracle(oracle_mod):
    from paper_2409_07759_b300 import api
    sc = _scene()
    views = _views([1, 1, 2, 4, 4, 4])
    r = api.Renderer()
    st = api.GaussianState.from_scene(sc)
    imgs, saved = r.render(st, views, keep_saved=True)
    dl = [torch.zeros_like(i) for i in imgs]
    grads = st.zero_grads()
    loss = torch.zeros(1, device="cuda")
    r.backward(st, saved, dl, grads, reg=dict(opacity_reg=2e-2, scale_reg=1e-2), loss=loss)
    saved.release()
    ref_loss, ref = oracle_mod.reg_loss_grad(sc, [v.frame for v in views], 2e-2, 1e-2)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    for k in ("opacity_logits", "log_scales"):
        np.testing.assert_allclose(getattr(grads, k).cpu().numpy(), ref[k], rtol=1e-4,
                                   atol=1e-6 * np.abs(ref[k]).max())
    for k in ("means", "quats", "sh"):
        assert float(getattr(grads, k).abs().max()) == 0.0
    r.close()


def test_regulariser_adds_to_the_render_gradient(oracle_mod):
    from paper_2409_07759_b300 import api
    sc = _scene()
    views = _views([2, 2, 3])
    r = api.Renderer()
    st = api.GaussianState.from_scene(sc)
    rng = np.random.default_rng(4)
    tg = [torch.from_numpy(rng.random((3, v.height, v.width), dtype=np.float32)).cuda()
          for v in views]
    _, dl, _, saved = r.render_l1(st, views, tg)
    g0 = st.zero_grads()
    r.backward(st, saved, dl, g0)
    g1 = st.zero_grads()
    r.backward(st, saved, dl, g1, reg=dict(opacity_reg=2e-2, scale_reg=1e-2))
    saved.release()
    _, ref = oracle_mod.reg_loss_grad(sc, [v.frame for v in views], 2e-2, 1e-2)
    for k in ("opacity_logits", "log_scales"):
        d = (getattr(g1, k) - getattr(g0, k)).cpu().numpy()
        scale = max(np.abs(ref[k]).max(), float(getattr(g0, k).abs().max()))
        np.testing.assert_allclose(d, ref[k], rtol=1e-3, atol=2e-5 * scale)
    for k in ("means", "quats", "sh"):
        torch.testing.assert_close(getattr(g1, k), getattr(g0, k), rtol=1e-5, atol=1e-7)
    r.close()


def test_mean_grad_decay_matches_oracle(oracle_mod):
    from paper_2409_07759_b300 import api
    n = 2000
    rng = np.random.default_rng(8)
    attrs = synth.make_gaussians(rng, n, 1)
    swin, st0 = 5, 10
    start = rng.integers(st0, st0 + swin, size=n).astype(np.int32)
    sc = synth._scene(attrs, 1, start, (start + swin).astype(np.int32))
    frames = list(range(st0, st0 + swin))
    p = dict(lr_means=1e-2, lr_log_scales=5e-3, lr_quats=1e-3, lr_logits=5e-2, lr_sh_dc=2.5e-3,
             lr_sh_rest=1.25e-4, beta1=0.9, beta2=0.999, eps=1e-15, noise_lr=5e4,
             noise_k=100.0, noise_t=0.005, adam=1, relocate=0, max_n=51)
    r = api.Renderer()
    st = api.GaussianState.from_scene(sc)
    K = (sc.sh_degree + 1) ** 2
    adam = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        adam["m_" + k] = torch.zeros_like(getattr(st, k))
        adam["v_" + k] = torch.zeros_like(getattr(st, k))
    host = sc.copy()
    hadam = None
    fac = oracle_mod.mean_grad_scale(sc.start, st0, swin, 0.5).astype(np.float32)
    for step in range(3):
        g = {k: rng.normal(0, 1e-3, size=getattr(sc, k).shape).astype(np.float32)
             for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        grads = api.GaussianGrads(*[torch.from_numpy(g[k]).cuda() for k in
                                    ("means", "log_scales", "quats", "opacity_logits", "sh")],
                                  sc.sh_degree)
        r.sgld_step(st, frames, dict(p, mean_grad_decay=0.5, window_start=st0, swin_size=swin),
                    7, step, grads=grads, adam=adam)
        gs = dict(g, means=(g["means"] * fac[:, None]).astype(np.float32))
        host, hadam, _, _ = oracle_mod.sgld_step(host, gs, hadam, frames, p, seed=7, step=step)
    got = st.means.cpu().numpy()
    np.testing.assert_allclose(got, host.means, rtol=0, atol=2e-6)
    np.testing.assert_allclose(adam["m_means"].cpu().numpy(), hadam["m_means"], rtol=1e-5,
                               atol=1e-9)
    r.close()
