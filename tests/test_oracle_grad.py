"""Finite-difference pins of the oracle's analytic backward (Alg. 1
loss.backward) and of the L1 term (Alg. 1 loss_func)."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

ATTRS = ("means", "log_scales", "quats", "opacity_logits", "sh")
# Bands wide enough that the FD steps below (1e-5 relative) never cross a
# threshold on an unflagged pixel.
WIDE = dict(m=2e-3, alpha=2e-3, t_stop=2e-3, clamp=2e-3, guard=1e-3, colour=1e-3)


def _fd_check(O, sc, view, seed=0, h_rel=1e-5, tol=1e-6, bg=(0.1, 0.0, 0.2)):
    r = O.render(sc, view, bg=bg, mode="tiled", bands=WIDE)
    flag = r["flags"] != 0
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(3, view.height, view.width))
    w[:, flag] = 0.0  # the loss only looks at pixels away from every threshold

    def L(s):
        return float((O.render(s, view, bg=bg, mode="tiled")["rgb"] * w).sum())

    g, _, rf, ids = O.render_bwd(sc, view, w, bg=bg, bands=WIDE)
    assert not (rf & 12).any(), "scene has a Gaussian near the guard band or colour clamp"
    for attr in ATTRS:
        A = getattr(sc, attr)
        fd = np.zeros(A.shape)
        for i in range(A.size):
            x = A.reshape(-1)[i]
            h = np.float32(h_rel * max(abs(float(x)), 0.1))
            s1, s2 = sc.copy(), sc.copy()
            getattr(s1, attr).reshape(-1)[i] = x + h
            getattr(s2, attr).reshape(-1)[i] = x - h
            hp = float(getattr(s1, attr).reshape(-1)[i]) - float(getattr(s2, attr).reshape(-1)[i])
            fd.reshape(-1)[i] = (L(s1) - L(s2)) / hp
        err = np.abs(g[attr] - fd).max() / max(np.abs(fd).max(), 1e-30)
        assert err < tol, (attr, err)
    return g


@pytest.mark.parametrize("seed,deg", [(3, 3), (8, 1), (13, 2)])
def test_fd_gradients_all_attributes(oracle_mod, seed, deg):
    """Analytic FP64 gradients of every attribute (means, log-scales, raw
    quaternions, opacity logits, SH up to degree 3) equal central differences."""
    sc, view = synth.tiny_scene(seed, n=10, sh_degree=deg, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.6, spread=0.5)
    view.fx = view.fy = 40.0
    sc.quats *= np.float32(1.7)  # unnormalised quaternions exercise the norm's chain rule
    _fd_check(oracle_mod, sc, view, seed=seed)


def test_fd_gradients_rotated_camera_guard_band(oracle_mod):
    """A camera off the axes, and Gaussians outside the image whose footprint
    reaches it (the clamped part of the Jacobian guard band)."""
    sc, view = synth.tiny_scene(21, n=8, sh_degree=1, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.4, spread=0.3)
    R, t = synth.look_at((1.0, 0.4, -2.5), target=(0.0, 0.0, 3.0))
    view.R, view.t = R, t
    view.fx = view.fy = 40.0
    # two Gaussians far to the side: x/z beyond 1.3 * tan(fov/2)
    p_cam = np.array([[2.2, 0.1, 3.0], [-0.3, -1.9, 2.6]])
    for k, pc in enumerate(p_cam):
        sc.means[k] = (R.T.astype(np.float64) @ (pc - t)).astype(np.float32)
        sc.log_scales[k] = np.log(np.float32([0.8, 0.6, 0.7]))
        sc.opacity_logits[k] = 2.5
    ref = oracle_mod.render(sc, view, mode="tiled")
    assert (ref["last_slot"] == 0).any() or (ref["last_slot"] == 1).any()
    _fd_check(oracle_mod, sc, view, seed=2)


def test_frozen_gaussians_get_no_gradient(oracle_mod):
    """Alg. 1: matured (frozen) Gaussians are rendered but receive no gradient."""
    sc, view = synth.tiny_scene(5, n=12, sh_degree=1, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.6, spread=0.5)
    view.fx = view.fy = 40.0
    w = np.random.default_rng(0).normal(size=(3, 32, 40))
    g_all, *_ = oracle_mod.render_bwd(sc, view, w)
    sc.frozen[::2] = 1
    g_fr, *_ = oracle_mod.render_bwd(sc, view, w)
    for a in ATTRS:
        assert (g_fr[a][::2] == 0).all()
        np.testing.assert_allclose(g_fr[a][1::2], g_all[a][1::2], rtol=1e-12, atol=1e-14)
        assert np.abs(g_all[a][::2]).max() > 0


def test_l1_gradient(oracle_mod):
    """L1 term: mean |C - target| over 3*H*W, averaged over views; its gradient
    is sign(C - target)/(3 H W V) with sign(0) = 0 (checked by differences)."""
    rng = np.random.default_rng(0)
    rgbs = [rng.uniform(size=(3, 4, 5)), rng.uniform(size=(3, 6, 2))]
    tgts = [rng.uniform(size=(3, 4, 5)), rng.uniform(size=(3, 6, 2))]
    tgts[0][0, 0, 0] = rgbs[0][0, 0, 0]
    loss, grads = oracle_mod.l1_loss_grad(rgbs, tgts)
    assert grads[0][0, 0, 0] == 0.0
    h = 1e-7
    for v in range(2):
        for idx in [(1, 2, 3), (2, 0, 1), (0, 3, 1)]:
            if idx[1] >= rgbs[v].shape[1] or idx[2] >= rgbs[v].shape[2]:
                continue
            rp = [r.copy() for r in rgbs]
            rp[v][idx] += h
            lp, _ = oracle_mod.l1_loss_grad(rp, tgts)
            assert (lp - loss) / h == pytest.approx(grads[v][idx], rel=1e-5)
