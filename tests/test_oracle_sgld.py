"""Pins of the oracle's SH basis, counter RNG, optimiser step, SGLD noise and
relocation (Alg. 1 noise and relocate steps; Sec. 3.2, 4.4, 8.1; [14])."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import scipy.stats

from paper_2409_07759_b300 import synth


# ---------------------------------------------------------------- SH basis --

def test_sh_orthonormal_by_quadrature(oracle_mod):
    """Sec. 8.1 colour model: the 16 real SH functions of degrees 0..3 are
    orthonormal on the sphere (Gauss-Legendre x uniform-phi quadrature, exact
    for these polynomial degrees)."""
    xs, ws = np.polynomial.legendre.leggauss(16)
    nphi = 32
    dirs, wts = [], []
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            dirs.append((st * math.cos(ph), st * math.sin(ph), ct))
            wts.append(w * 2 * math.pi / nphi)
    Y = oracle_mod.sh_basis(np.array(dirs))
    G = (Y * np.array(wts)[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_real_harmonics(oracle_mod):
    """Each basis function equals (-1)^m times the standard real spherical
    harmonic built from scipy's complex Y_l^m (index l*l + l + m)."""
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle_mod.sh_basis(d)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                real = math.sqrt(2) * (-1) ** m * scipy.special.sph_harm_y(l, m, theta, phi).real
            elif m < 0:
                real = math.sqrt(2) * (-1) ** m * scipy.special.sph_harm_y(l, -m, theta, phi).imag
            else:
                real = scipy.special.sph_harm_y(l, 0, theta, phi).real
            np.testing.assert_allclose(Y[:, l * l + l + m], (-1) ** m * real, atol=1e-12)


# ------------------------------------------------------------------- RNG --

@pytest.mark.parametrize("key,ctr", [((5, 0), (0, 0, 0, 0)),
                                     ((0x123456789ABCDEF, 0xFEDCBA987), (7, 9, 11, 13)),
                                     ((2**64 - 1, 2**64 - 1), (2**64 - 1, 5, 2**64 - 1, 3))])
def test_philox_matches_numpy(oracle_mod, key, ctr):
    """Philox4x64-10 (Salmon et al. 2011) equals numpy's implementation;
    numpy advances its 256-bit counter by one before the first block."""
    kint = key[0] | (key[1] << 64)
    cint = sum(c << (64 * i) for i, c in enumerate(ctr))
    ref = np.random.Philox(key=kint, counter=cint).random_raw(4)
    nxt = (cint + 1) % 2**256
    mine = oracle_mod.philox4x64([(nxt >> (64 * i)) & (2**64 - 1) for i in range(4)], key)
    np.testing.assert_array_equal(ref, mine)


def test_box_muller_normals(oracle_mod):
    """The three noise draws per (seed, step, slot) are N(0,1), independent."""
    z = np.array([oracle_mod.normal3(11, 3, i) for i in range(20000)])
    for k in range(3):
        assert scipy.stats.kstest(z[:, k], "norm").pvalue > 1e-3
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 0.04


# ---------------------------------------------------------- optimiser/SGLD --

def _uniform_scene(n, logit, log_scale, quat, sh_degree=0):
    return synth.Scene(
        means=np.zeros((n, 3), np.float32),
        log_scales=np.tile(np.float32(log_scale), (n, 1)),
        quats=np.tile(np.float32(quat), (n, 1)),
        opacity_logits=np.full(n, logit, np.float32),
        sh=np.zeros((n, (sh_degree + 1) ** 2, 3), np.float32),
        start=np.zeros(n, np.int32), expire=np.ones(n, np.int32), birth=np.zeros(n, np.int32),
        frozen=np.zeros(n, np.uint8), sh_degree=sh_degree)


def test_sgld_noise_moments(oracle_mod):
    """Alg. 1 noise step as in [14]: mu += lr * noise_lr * sigmoid(-k(o - t)) *
    Sigma eta, eta ~ N(0, I). At o = t the gate is exactly 1/2, so the update has
    mean 0 and covariance (lr * noise_lr / 2)^2 Sigma^2."""
    n = 60000
    logit = math.log(0.005 / 0.995)
    ls = [-1.0, -1.5, -0.7]
    q = np.array([0.8, 0.3, -0.4, 0.2]); q /= np.linalg.norm(q)
    sc = _uniform_scene(n, logit, ls, q)
    p = dict(lr_means=1e-3, noise_lr=10.0, relocate=0, adam=0)
    out, _, _, _ = oracle_mod.sgld_step(sc, None, None, [0], p, seed=7, step=2)
    d = out.means.astype(np.float64)
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    gate = 1 / (1 + math.exp(100 * (o - 0.005)))
    w, x, y, z = (np.float32(q) / np.linalg.norm(np.float32(q))).astype(np.float64)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    S = np.diag(np.exp(np.float32(ls).astype(np.float64)))
    Sig = R @ S @ S @ R.T
    scale = 1e-3 * 10.0 * gate
    want = scale ** 2 * Sig @ Sig
    cov = np.cov(d.T)
    se = np.sqrt((want ** 2 + np.outer(np.diag(want), np.diag(want))) / n)
    assert np.all(np.abs(cov - want) <= 5 * se)
    assert np.all(np.abs(d.mean(0)) <= 5 * np.sqrt(np.diag(want) / n))
    assert gate == pytest.approx(0.5, abs=1e-5)


def test_sgld_only_touches_eligible(oracle_mod):
    """Noise and relocation act on gs[active_idx] only: frozen (matured) and
    inactive slots are left bit-for-bit unchanged."""
    sc, _ = synth.tiny_scene(1, n=400, sh_degree=1)
    rng = np.random.default_rng(0)
    sc.start = rng.integers(0, 6, sc.n).astype(np.int32)
    sc.expire = (sc.start + 2).astype(np.int32)
    sc.frozen = (rng.uniform(size=sc.n) < 0.3).astype(np.uint8)
    sc.opacity_logits[::7] = -8.0
    frames = [3, 4]
    out, _, n_dead, tg = oracle_mod.sgld_step(sc, None, None, frames, dict(relocate=1), seed=1,
                                              step=5)
    act = np.zeros(sc.n, bool)
    for f in frames:
        act |= (sc.start <= f) & (f < sc.expire)
    el = act & (sc.frozen == 0)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(getattr(out, k)[~el], getattr(sc, k)[~el])
    assert n_dead > 0
    assert np.all(el[tg >= 0]) and np.all(el[tg[tg >= 0]])


def test_adam_first_step_closed_form(oracle_mod):
    """Adam's first bias-corrected step moves each parameter by lr*g/(|g|+eps)."""
    sc, _ = synth.tiny_scene(2, n=50, sh_degree=1)
    rng = np.random.default_rng(1)
    grads = {k: rng.normal(size=getattr(sc, k).shape).astype(np.float32)
             for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    p = dict(adam=1, relocate=0, noise_lr=0.0)
    out, mom, _, _ = oracle_mod.sgld_step(sc, grads, None, [0], p, seed=0, step=0)
    lrs = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2)
    for k, lr in lrs.items():
        g = grads[k].astype(np.float64)
        want = getattr(sc, k).astype(np.float64) - lr * g / (np.abs(g) + 1e-15)
        np.testing.assert_allclose(getattr(out, k), want, rtol=1e-6, atol=1e-7)
    g = grads["sh"].astype(np.float64)
    lr = np.where(np.arange(4)[None, :, None] == 0, 2.5e-3, 2.5e-3 / 20)
    np.testing.assert_allclose(out.sh, sc.sh - lr * g / (np.abs(g) + 1e-15), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(mom["m_means"], 0.1 * grads["means"], rtol=1e-6)


# ------------------------------------------------------------- relocation --

@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 51])
def test_relocation_opacity_invariant(oracle_mod, n):
    """[14]'s relocation: N coincident copies of opacity o' composite to the
    original opacity, 1 - (1 - o')^N = o; N = 1 leaves the scale unchanged."""
    for o in (0.01, 0.2, 0.5, 0.9, 0.995):
        on, ratio = oracle_mod.reloc_values(o, n)
        assert 1 - (1 - on) ** n == pytest.approx(o, rel=1e-12)
        if n == 1:
            assert ratio == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5, 12])
def test_relocation_scale_preserves_footprint(oracle_mod, n):
    """The scale rule makes the composited 1D opacity profile of the N copies
    integrate to that of the original: int 1-(1-o' g_{s'})^N = int o g_s."""
    for o in (0.1, 0.6, 0.95):
        on, ratio = oracle_mod.reloc_values(o, n)
        s = 1.0
        lhs = scipy.integrate.quad(lambda x: 1 - (1 - on * math.exp(-0.5 * (x / (s * ratio)) ** 2))
                                   ** n, -60, 60, limit=400)[0]
        rhs = o * s * math.sqrt(2 * math.pi)
        assert lhs == pytest.approx(rhs, rel=1e-7)


def test_relocation_weight_is_exact_floor(oracle_mod):
    """The integer relocation weight is floor(sigmoid(logit) * 2^32), exactly,
    checked against 60-digit arithmetic."""
    import mpmath
    mpmath.mp.dps = 60
    rng = np.random.default_rng(0)
    for lg in np.concatenate([rng.normal(0, 3, 300), [-30.0, -5.0, 0.0, 5.0, 20.0]]).astype(np.float32):
        o = 1 / (1 + mpmath.exp(-mpmath.mpf(float(lg))))
        want = min(int(mpmath.floor(o * 2**32)), 2**32 - 1)
        assert oracle_mod.reloc_weight(float(lg)) == want


def test_relocation_sampling_proportional_to_opacity(oracle_mod):
    """Dead Gaussians (o <= 0.005) pick targets among alive ones with
    probability proportional to opacity (chi-square over 30k draws); every dead
    slot copies its target, and the Gaussian count is unchanged."""
    n_alive, n_dead = 6, 30000
    logits = np.concatenate([np.float32([-2.0, -0.5, 0.0, 0.7, 1.5, 3.0]),
                             np.full(n_dead, -8.0, np.float32)])
    sc = _uniform_scene(n_alive + n_dead, 0.0, [-2.0, -2.0, -2.0], [1, 0, 0, 0], sh_degree=1)
    sc.opacity_logits = logits
    sc.means = np.random.default_rng(0).normal(size=(sc.n, 3)).astype(np.float32)
    p = dict(noise_lr=0.0, relocate=1)
    out, _, nd, tg = oracle_mod.sgld_step(sc, None, None, [0], p, seed=3, step=1)
    assert nd == n_dead and out.n == sc.n
    counts = np.bincount(tg[tg >= 0], minlength=n_alive)[:n_alive]
    o = 1 / (1 + np.exp(-logits[:n_alive].astype(np.float64)))
    exp_counts = n_dead * o / o.sum()
    assert scipy.stats.chisquare(counts, exp_counts).pvalue > 1e-3
    dead = np.nonzero(tg >= 0)[0]
    np.testing.assert_array_equal(out.means[dead], sc.means[tg[dead]])
    # targets and their copies share the relocated opacity 1-(1-o)^(1/N)
    for j in range(n_alive):
        N = min(counts[j] + 1, 51)
        on, _ = oracle_mod.reloc_values(o[j], N)
        assert 1 / (1 + math.exp(-float(out.opacity_logits[j]))) == pytest.approx(on, rel=1e-5)
