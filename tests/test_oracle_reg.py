"""Pins of the oracle's regulariser (Alg. 1 reg(), Sec. 4.4 / 8.1) and of the
means-gradient scale (Sec. 4.5.1): closed forms, central finite differences,
the exclusion of frozen Gaussians, and the scale's special cases."""
import numpy as np

from paper_2409_07759_b300 import synth


def _scene(n=40, seed=1):
    rng = np.random.default_rng(seed)
    attrs = synth.make_gaussians(rng, n, 1)
    start = rng.integers(0, 4, size=n).astype(np.int32)
    expire = (start + rng.integers(1, 4, size=n)).astype(np.int32)
    frozen = (rng.random(n) < 0.25).astype(np.uint8)
    return synth._scene(attrs, 1, start, expire, frozen=frozen)


def test_single_gaussian_closed_form(oracle_mod):
    sc = _scene(1)
    sc.start[:] = 0
    sc.expire[:] = 5
    sc.frozen[:] = 0
    sc.opacity_logits[:] = 0.3
    sc.log_scales[:] = [[-1.0, 0.0, 0.5]]
    loss, g = oracle_mod.reg_loss_grad(sc, [2], 0.02, 0.01)
    sig = 1 / (1 + np.exp(-np.float64(sc.opacity_logits[0])))
    s = np.exp(sc.log_scales[0].astype(np.float64))
    assert abs(loss - (0.02 * sig + 0.01 * s.mean())) < 1e-15
    assert abs(g["opacity_logits"][0] - 0.02 * sig * (1 - sig)) < 1e-15
    np.testing.assert_allclose(g["log_scales"][0], 0.01 * s / 3, rtol=1e-15)


def test_finite_differences(oracle_mod):
    sc = _scene()
    frames = [0, 1, 1, 3]
    _, g = oracle_mod.reg_loss_grad(sc, frames, 0.02, 0.01)
    live = np.nonzero(sc.frozen == 0)[0][:6]
    for i in live:
        for name, idx in (("opacity_logits", (i,)), ("log_scales", (i, 1))):
            # the arrays are float32: step by 64 ulps and divide by the stored step
            x = getattr(sc, name)[idx]
            xa = np.float32(x) + np.float32(64) * np.spacing(np.float32(x))
            xb = np.float32(x) - np.float32(64) * np.spacing(np.float32(x))
            a, b = sc.copy(), sc.copy()
            getattr(a, name)[idx] = xa
            getattr(b, name)[idx] = xb
            la, _ = oracle_mod.reg_loss_grad(a, frames, 0.02, 0.01)
            lb, _ = oracle_mod.reg_loss_grad(b, frames, 0.02, 0.01)
            fd = (la - lb) / (np.float64(xa) - np.float64(xb))
            assert abs(fd - g[name][idx]) <= 1e-4 * abs(g[name][idx]) + 1e-13, (name, i)


def test_frozen_get_no_gradient_but_count(oracle_mod):
    sc = _scene()
    _, g = oracle_mod.reg_loss_grad(sc, [1, 2], 0.02, 0.01)
    fz = sc.frozen == 1
    assert np.all(g["opacity_logits"][fz] == 0) and np.all(g["log_scales"][fz] == 0)
    # freezing a Gaussian leaves the loss unchanged (it still counts in the mean)
    sc2 = sc.copy()
    sc2.frozen[:] = 0
    la, _ = oracle_mod.reg_loss_grad(sc, [1, 2], 0.02, 0.01)
    lb, _ = oracle_mod.reg_loss_grad(sc2, [1, 2], 0.02, 0.01)
    assert la == lb


def test_mean_over_views(oracle_mod):
    sc = _scene()
    la, ga = oracle_mod.reg_loss_grad(sc, [1], 0.02, 0.01)
    lb, gb = oracle_mod.reg_loss_grad(sc, [1, 1, 1], 0.02, 0.01)
    assert abs(la - lb) < 1e-15
    np.testing.assert_allclose(ga["log_scales"], gb["log_scales"], rtol=1e-14)


def test_mean_grad_scale_cases(oracle_mod):
    start = np.array([10, 11, 12, 13, 14])
    # window [10, 15): the version starting at 14 has been trained in windows 10..14
    f = oracle_mod.mean_grad_scale(start, 10, 5, 0.5)
    np.testing.assert_array_equal(f, 0.5 ** np.array([4, 3, 2, 1, 0]))
    assert np.all(oracle_mod.mean_grad_scale(start, 10, 5, 1.0) == 1.0)
    # a version first trained in this window (start = st + swin - 1) is unscaled
    assert oracle_mod.mean_grad_scale([14], 10, 5, 0.3)[0] == 1.0
