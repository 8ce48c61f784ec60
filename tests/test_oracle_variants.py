"""Pins of the oracle's decision replay (render_variants): the set of valid
results of one pixel when the per-pair tests of Eq. 3 -- the 3-sigma support
m <= 9, alpha >= 1/255 and the transmittance stop T (1 - alpha) < 1e-4 -- are
decided either way near their thresholds. Checked against the plain walk,
closed forms of one and two Gaussians, and the stop rule's product form."""
import math

import numpy as np
import pytest

from paper_2409_07759_b300 import synth

from test_oracle_render import C0, _axis_scene

ZERO = dict(m=0.0, alpha=0.0, t_stop=0.0, clamp=0.0, guard=0.0, colour=0.0)


def _all_pixels(view):
    yy, xx = np.mgrid[0:view.height, 0:view.width]
    return xx.ravel(), yy.ravel()


@pytest.mark.parametrize("seed", [0, 3])
def test_zero_bands_give_the_plain_walk(oracle_mod, seed):
    """With no band, every pixel has exactly one result: the tiled render's."""
    sc, view = synth.tiny_scene(seed, n=64, sh_degree=1, width=48, height=40, depth=3.0,
                                log_scale_mean=-1.8, spread=0.8)
    view.fx = view.fy = 45.0
    ref = oracle_mod.render(sc, view, mode="tiled", bg=(0.1, 0.2, 0.3))
    px, py = _all_pixels(view)
    res = oracle_mod.render_variants(sc, view, px, py, ZERO, bg=(0.1, 0.2, 0.3))
    for k, r in enumerate(res):
        rgb, T, last = r
        assert len(T) == 1
        np.testing.assert_array_equal(rgb[0], ref["rgb"][:, py[k], px[k]])
        assert T[0] == ref["T"][py[k], px[k]]
        assert last[0] == ref["last_pos"][py[k], px[k]]


def test_fp64_result_is_always_a_variant(oracle_mod):
    """With wide bands the plain FP64 walk stays one of the results."""
    sc, view = synth.tiny_scene(5, n=96, sh_degree=2, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.6, spread=0.8)
    view.fx = view.fy = 40.0
    ref = oracle_mod.render(sc, view, mode="tiled")
    px, py = _all_pixels(view)
    wide = dict(m=3e-2, alpha=3e-2, t_stop=3e-1)
    res = oracle_mod.render_variants(sc, view, px, py, wide, max_per=4096)
    n_multi = 0
    for k, r in enumerate(res):
        assert r is not None
        rgb, T, last = r
        want = ref["rgb"][:, py[k], px[k]]
        hit = [i for i in range(len(T)) if np.array_equal(rgb[i], want)
               and T[i] == ref["T"][py[k], px[k]] and last[i] == ref["last_pos"][py[k], px[k]]]
        assert hit, k
        n_multi += len(T) > 1
    assert n_multi > 0  # the bands did branch somewhere


def _edge_scene(m_target):
    """One isotropic Gaussian on the axis, seen by a camera whose principal
    point is shifted so that pixel (20, 15)'s centre lies at Mahalanobis^2
    m_target from the projected centre (along x)."""
    z, ls, logit = 4.0, math.log(0.15), 2.0
    sc, view = _axis_scene([z], [ls], [logit], [[0.9, -0.4, 0.2]], width=41, height=31)
    sigma = math.exp(float(np.float32(ls)))
    var = (view.fx * sigma / z) ** 2 + 0.3
    dx = math.sqrt(m_target * var)
    view.cx = 20.5 - dx
    view.cy = 15.5
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    c = [max(0.0, C0 * float(np.float32(d)) + 0.5) for d in (0.9, -0.4, 0.2)]
    return sc, view, var, o, c


def test_support_edge_has_both_outcomes(oracle_mod):
    """A pixel at m = 9 (1 - 1e-6): inside by FP64, but within the support
    band, so 'skipped' (background, T = 1) is valid too; the inside result is
    c alpha + (1 - alpha) bg with alpha = o exp(-m/2) (closed form)."""
    sc, view, var, o, c = _edge_scene(9.0 * (1 - 1e-6))
    bg = (0.1, 0.2, 0.3)
    (rgb, T, last), = oracle_mod.render_variants(sc, view, [20], [15], dict(m=3e-5), bg=bg)
    assert sorted(T.tolist())[1] == 1.0 and len(T) == 2
    a = o * math.exp(-0.5 * 9.0 * (1 - 1e-6))
    i_in = int(np.argmin(T))
    assert T[i_in] == pytest.approx(1 - a, rel=1e-6)
    assert last[i_in] == 1 and last[1 - i_in] == 0
    for ch in range(3):
        assert rgb[i_in, ch] == pytest.approx(c[ch] * a + (1 - a) * bg[ch], rel=1e-5)
        assert rgb[1 - i_in, ch] == pytest.approx(bg[ch], rel=1e-12)
    # away from the edge: one result only
    sc, view, var, o, c = _edge_scene(8.0)
    (rgb, T, last), = oracle_mod.render_variants(sc, view, [20], [15], dict(m=3e-5), bg=bg)
    assert len(T) == 1 and last[0] == 1


def test_alpha_edge_has_both_outcomes(oracle_mod):
    """A pixel whose alpha is 1/255 (1 + 1e-7): both 'included' and 'skipped'."""
    z, ls, logit = 4.0, math.log(0.15), math.log(0.1 / 0.9)
    sc, view = _axis_scene([z], [ls], [logit], [[0.5, 0.5, 0.5]], width=41, height=31)
    sigma = math.exp(float(np.float32(ls)))
    var = (view.fx * sigma / z) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    m = -2.0 * math.log((1.0 / 255.0) * (1 + 1e-7) / o)
    assert m < 9.0
    view.cx = 20.5 - math.sqrt(m * var)
    view.cy = 15.5
    (rgb, T, last), = oracle_mod.render_variants(sc, view, [20], [15], dict(alpha=6e-5))
    assert sorted(last.tolist()) == [0, 1]
    assert max(T) == 1.0 and min(T) == pytest.approx(1 - (1.0 / 255.0), rel=1e-5)


def test_stop_edge_has_both_outcomes(oracle_mod):
    """Eleven centred Gaussians of alpha a with (1 - a)^11 = 1e-4 exactly
    (in FP64 up to rounding): stopping before the eleventh (T = (1 - a)^10,
    last = 10) and including it (T = (1 - a)^11, last = 11) are both valid."""
    n = 11
    a = 1.0 - 1e-4 ** (1.0 / 11.0)
    logit = math.log(a / (1 - a))
    sc, view = _axis_scene([2.0 + 0.1 * k for k in range(n)], [math.log(0.5)] * n, [logit] * n,
                           [[0.3, 0.3, 0.3]] * n, width=33, height=33)
    view.cx = view.cy = 16.5
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    (rgb, T, last), = oracle_mod.render_variants(sc, view, [16], [16], dict(t_stop=1e-3))
    got = sorted(zip(last.tolist(), T.tolist()))
    assert [g[0] for g in got] == [10, 11]
    assert got[0][1] == pytest.approx((1 - o) ** 10, rel=1e-12)
    assert got[1][1] == pytest.approx((1 - o) ** 11, rel=1e-12)
    # a planted stop band of zero leaves only the FP64 decision
    (rgb, T, last), = oracle_mod.render_variants(sc, view, [16], [16], dict(t_stop=0.0))
    assert len(T) == 1


def test_variant_cap_reports_overflow(oracle_mod):
    """More results than max_per: the pixel is reported as None, never cut short."""
    sc, view = synth.tiny_scene(5, n=96, sh_degree=2, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.6, spread=0.8)
    view.fx = view.fy = 40.0
    px, py = _all_pixels(view)
    res = oracle_mod.render_variants(sc, view, px, py, dict(m=0.5, alpha=0.5, t_stop=0.9),
                                     max_per=2)
    assert any(r is None for r in res)
