"""Pins of the FP64 oracle's forward path against closed forms, invariants and
brute force (no GPU). Each test names the passage it checks."""
import math

import numpy as np
import pytest

from paper_2409_07759_b300 import synth

C0 = 1.0 / (2.0 * math.sqrt(math.pi))  # degree-0 real SH constant


def _axis_scene(depths, log_sigmas, logits, dcs, width=33, height=31, f=40.0):
    """Isotropic Gaussians on the optical axis of a camera at the origin."""
    n = len(depths)
    sc = synth.Scene(
        means=np.array([[0.0, 0.0, z] for z in depths], np.float32),
        log_scales=np.array([[s, s, s] for s in log_sigmas], np.float32),
        quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
        opacity_logits=np.array(logits, np.float32),
        sh=np.array(dcs, np.float32).reshape(n, 1, 3),
        start=np.zeros(n, np.int32), expire=np.ones(n, np.int32),
        birth=np.zeros(n, np.int32), frozen=np.zeros(n, np.uint8), sh_degree=0)
    view = synth.View(width, height, f, f, width / 2.0, height / 2.0)
    return sc, view


def test_single_gaussian_closed_form(oracle_mod):
    """Eq. 1-3 for one isotropic Gaussian on the axis: the 2D covariance is
    (f sigma / z)^2 I + 0.3 I, alpha = min(0.99, o exp(-m/2)) inside the 3-sigma
    ellipse and above 1/255, and C = c alpha + (1 - alpha) bg."""
    z, ls, logit = 4.0, math.log(0.15), 0.7
    dc = [0.9, -0.4, 0.2]
    sc, view = _axis_scene([z], [ls], [logit], [dc])
    bg = (0.1, 0.2, 0.3)
    out = oracle_mod.render(sc, view, bg=bg, mode="brute")
    f = view.fx
    sigma = math.exp(float(np.float32(ls)))
    var = (f * sigma / z) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    c = [max(0.0, C0 * float(np.float32(d)) + 0.5) for d in dc]
    for j in range(view.height):
        for i in range(view.width):
            dx, dy = i + 0.5 - view.cx, j + 0.5 - view.cy
            m = (dx * dx + dy * dy) / var
            a = min(0.99, o * math.exp(-0.5 * m))
            inside = m <= 9.0 and a >= 1.0 / 255.0
            for ch in range(3):
                want = c[ch] * a + (1 - a) * bg[ch] if inside else bg[ch]
                assert out["rgb"][ch, j, i] == pytest.approx(want, rel=1e-12, abs=1e-14)
            assert out["T"][j, i] == pytest.approx(1 - a if inside else 1.0, rel=1e-12)
            assert out["last_slot"][j, i] == (0 if inside else -1)


def test_two_gaussian_compositing(oracle_mod):
    """Eq. 3 with two Gaussians in z order: C = c1 a1 + c2 a2 (1-a1) + (1-a1)(1-a2) bg,
    and the nearer one is composited first whatever the slot order."""
    sc, view = _axis_scene([5.0, 3.0], [math.log(0.3), math.log(0.2)], [0.3, -0.2],
                           [[0.5, 0.1, -0.3], [-0.2, 0.6, 0.4]])
    bg = (0.05, 0.1, 0.15)
    out = oracle_mod.render(sc, view, bg=bg, mode="brute")
    px, py = 14, 17
    dx, dy = px + 0.5 - view.cx, py + 0.5 - view.cy
    alphas, cols = [], []
    for k in (1, 0):  # slot 1 is nearer
        z = float(sc.means[k, 2])
        s = math.exp(float(sc.log_scales[k, 0]))
        var = (view.fx * s / z) ** 2 + 0.3
        o = 1 / (1 + math.exp(-float(sc.opacity_logits[k])))
        alphas.append(min(0.99, o * math.exp(-0.5 * (dx * dx + dy * dy) / var)))
        cols.append([max(0.0, C0 * float(d) + 0.5) for d in sc.sh[k, 0]])
    a1, a2 = alphas
    for ch in range(3):
        want = cols[0][ch] * a1 + cols[1][ch] * a2 * (1 - a1) + (1 - a1) * (1 - a2) * bg[ch]
        assert out["rgb"][ch, py, px] == pytest.approx(want, rel=1e-12)
    assert out["last_slot"][py, px] == 0


def test_transmittance_stop(oracle_mod):
    """Blending stops before a Gaussian that would take T below 1e-4: with
    twenty centred Gaussians of alpha ~0.6, ten are composited (0.4^10 > 1e-4 >
    0.4^11) and the final T is the product of their (1 - alpha)."""
    n = 20
    logit = math.log(0.6 / 0.4)
    sc, view = _axis_scene([2.0 + 0.1 * k for k in range(n)], [math.log(0.5)] * n, [logit] * n,
                           [[0.3, 0.3, 0.3]] * n, width=33, height=33)
    view.cx = view.cy = 16.5  # pixel (16,16) sits on every centre
    out = oracle_mod.render(sc, view, mode="brute")
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    assert out["last_slot"][16, 16] == 9
    assert out["T"][16, 16] == pytest.approx((1 - o) ** 10, rel=1e-12)
    tiled = oracle_mod.render(sc, view, mode="tiled")
    assert tiled["last_pos"][16, 16] == 10


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (32, 8)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiling_independence(oracle_mod, tile, seed):
    """The support rule (Mahalanobis^2 <= 9) and the tiles its 3-sigma ellipse covers make
    the per-tile render identical to the brute-force per-pixel walk over the
    whole depth-ordered active set, for every tile shape."""
    sc, view = synth.tiny_scene(seed, n=64, sh_degree=1, width=48, height=40, depth=3.0,
                                log_scale_mean=-1.8, spread=0.8)
    view.fx = view.fy = 45.0
    b = oracle_mod.render(sc, view, mode="brute")
    t = oracle_mod.render(sc, view, mode="tiled", tile_w=tile[0], tile_h=tile[1])
    np.testing.assert_array_equal(b["rgb"], t["rgb"])
    np.testing.assert_array_equal(b["T"], t["T"])
    np.testing.assert_array_equal(b["last_slot"], t["last_slot"])
    assert (b["T"] >= 1e-4).all() and (b["T"] <= 1.0).all()


def test_slot_permutation_invariance(oracle_mod):
    """Eq. 3 depends on z order only: permuting slots leaves the image unchanged."""
    sc, view = synth.tiny_scene(7, n=40, sh_degree=2, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.8, spread=0.8)
    view.fx = view.fy = 40.0
    perm = np.random.default_rng(1).permutation(sc.n)
    sp = sc.copy()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire",
              "birth", "frozen"):
        setattr(sp, k, getattr(sc, k)[perm].copy())
    a = oracle_mod.render(sc, view, mode="brute")
    b = oracle_mod.render(sp, view, mode="brute")
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    ls = b["last_slot"]
    mapped = np.where(ls >= 0, perm[np.maximum(ls, 0)], -1)
    np.testing.assert_array_equal(a["last_slot"], mapped)


def test_frame_scene_is_active_subset(oracle_mod):
    """Sec. 4.2 / Alg. 2: the scene at frame t is plain 3DGS over the Gaussians
    with start <= t < expire -- no temporal modulation of attributes."""
    sc, view = synth.tiny_scene(11, n=80, sh_degree=1, width=40, height=32, depth=3.0,
                                log_scale_mean=-1.8, spread=0.8)
    view.fx = view.fy = 40.0
    rng = np.random.default_rng(3)
    sc.start = rng.integers(0, 10, sc.n).astype(np.int32)
    sc.expire = (sc.start + rng.integers(1, 5, sc.n)).astype(np.int32)
    for t in (2, 5, 8):
        view.frame = t
        full = oracle_mod.render(sc, view, mode="brute")
        act = np.nonzero((sc.start <= t) & (t < sc.expire))[0]
        sub = sc.copy()
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "frozen"):
            setattr(sub, k, getattr(sc, k)[act].copy())
        sub.start = np.zeros(len(act), np.int32)
        sub.expire = np.ones(len(act), np.int32)
        sub.birth = np.zeros(len(act), np.int32)
        v0 = synth.View(view.width, view.height, view.fx, view.fy, view.cx, view.cy,
                        view.R, view.t, 0)
        ref = oracle_mod.render(sub, v0, mode="brute")
        np.testing.assert_array_equal(full["rgb"], ref["rgb"])


def test_active_ids_sliding_window(oracle_mod):
    """Alg. 2: after each per-frame slice update every slot of the client buffer
    is active, and the slice written for frame f is f mod swin_size."""
    swin, S = 6, 5
    buf = synth.config4_initial(slice_size=S, swin_size=swin, sh_degree=0)
    assert len(oracle_mod.active_ids(buf.start, buf.expire, 0)) == swin * S
    for f in range(1, 20):
        upd = synth.config4_slice(f, S, swin, 0)
        new = oracle_mod.frame_update(buf, upd, f, swin)
        lo, hi = oracle_mod.slice_range(f, swin, swin * S)
        changed = np.nonzero(np.any(new.means != buf.means, axis=1))[0]
        assert set(changed.tolist()) <= set(range(lo, hi))
        assert lo == (f % swin) * S
        assert (new.birth[lo:hi] == f).all()
        ids = oracle_mod.active_ids(new.start, new.expire, f)
        np.testing.assert_array_equal(ids, np.arange(swin * S, dtype=np.int32))
        # the slots that expire at f are exactly the replaced slice
        exp_before = np.nonzero(buf.expire == f)[0]
        np.testing.assert_array_equal(exp_before, np.arange(lo, hi))
        buf = new


def test_keymode_axis_covariance(oracle_mod):
    """Key mode (FP32) on the axis: the 2D covariance is (f sigma/z)^2 + 0.3 on the
    diagonal, 0 off it, the radius is ceil(3 sqrt(lambda_max)) and the polynomial exp
    of the log-scale is accurate to FP32 rounding."""
    for ls in (-4.0, -3.1, -2.2, -1.0, 0.3):
        sc, view = _axis_scene([3.7], [ls], [0.0], [[0, 0, 0]], width=64, height=48, f=60.0)
        km = oracle_mod.keymode(sc, view, [0])[0]
        s = math.exp(float(np.float32(ls)))
        var = (60.0 * s / float(np.float32(3.7))) ** 2 + 0.3
        assert km["a"] == pytest.approx(var, rel=2e-6)
        assert km["c"] == pytest.approx(var, rel=2e-6)
        assert abs(km["b"]) <= 1e-6 * var
        assert km["radius"] == math.ceil(3.0 * math.sqrt(km["lambda1"]))
        assert km["u"] == pytest.approx(32.0) and km["v"] == pytest.approx(24.0)


def test_keymode_quaternion_invariance(oracle_mod):
    """Eq. 2 uses R(q/|q|), quadratic in q: q, -q and 2q give identical FP32
    key-mode records (exact scalings)."""
    sc, view = synth.tiny_scene(4, n=30, sh_degree=0, width=64, height=48, depth=3.0,
                                log_scale_mean=-2.0, spread=0.9)
    base = oracle_mod.keymode(sc, view, np.arange(sc.n))
    for f in (-1.0, 2.0):
        s2 = sc.copy()
        s2.quats = (sc.quats * np.float32(f)).astype(np.float32)
        other = oracle_mod.keymode(s2, view, np.arange(sc.n))
        assert base.tobytes() == other.tobytes()


def test_keymode_matches_fp64_and_covers_support(oracle_mod):
    """The FP32 key mode agrees with the FP64 projection, and every pixel whose
    FP64 Mahalanobis^2 is <= 9 lies in a tile the key mode keeps."""
    sc, view = synth.tiny_scene(5, n=60, sh_degree=0, width=80, height=64, depth=3.0,
                                log_scale_mean=-2.0, spread=1.0)
    view.fx = view.fy = 70.0
    km = oracle_mod.keymode(sc, view, np.arange(sc.n), tile_w=16, tile_h=16)
    for i in range(sc.n):
        if km[i]["culled"]:
            continue
        u, v, A, B, Cc, *_ = oracle_mod.project(sc, view, i)
        assert km[i]["u"] == pytest.approx(u, rel=1e-5, abs=1e-4)
        assert km[i]["v"] == pytest.approx(v, rel=1e-5, abs=1e-4)
        det = km[i]["a"] * km[i]["c"] - km[i]["b"] ** 2
        assert km[i]["c"] / det == pytest.approx(A, rel=1e-4)
        assert km[i]["a"] / det == pytest.approx(Cc, rel=1e-4)
        ys, xs = np.mgrid[0:view.height, 0:view.width]
        dx, dy = xs + 0.5 - u, ys + 0.5 - v
        m = A * dx * dx + 2 * B * dx * dy + Cc * dy * dy
        inside = m <= 9.0
        tx, ty = xs // 16, ys // 16
        ntx, nty = 5, 4
        kept = np.zeros(ntx * nty, bool)
        kept[oracle_mod.record_tiles(km[i], view, 16, 16)] = True
        assert not np.any(inside & ~kept[ty * ntx + tx])
        assert km[i]["tiles"] == kept.sum() <= max(0, km[i]["tx1"] - km[i]["tx0"] + 1) * \
            max(0, km[i]["ty1"] - km[i]["ty0"] + 1)
        assert 0 <= km[i]["tx0"] and km[i]["tx1"] < ntx and km[i]["ty1"] < nty


def test_tile_coverage_is_the_support_minimum(oracle_mod):
    """A tile of the bounding rectangle is kept iff the minimum of the
    Mahalanobis form over the rectangle spanned by the tile's pixel centres is
    <= 9.009 (checked against scipy's box-constrained minimiser; the FP32 test
    may differ only within 1e-4 of the threshold)."""
    import scipy.optimize
    sc, view = synth.tiny_scene(6, n=40, sh_degree=0, width=96, height=80, depth=3.0,
                                log_scale_mean=-2.0, spread=1.0)
    view.fx = view.fy = 80.0
    km = oracle_mod.keymode(sc, view, np.arange(sc.n), tile_w=16, tile_h=16)
    ntx = 6
    checked = dropped = 0
    for i in range(sc.n):
        k = km[i]
        if k["culled"]:
            continue
        kept = set(oracle_mod.record_tiles(k, view, 16, 16).tolist())
        u, v, A, B, Cc = (float(k[f]) for f in ("u", "v", "A", "B", "C"))
        for ty in range(k["ty0"], k["ty1"] + 1):
            for tx in range(k["tx0"], k["tx1"] + 1):
                lo = np.array([tx * 16 + 0.5 - u, ty * 16 + 0.5 - v])
                hi = lo + 15.0
                f = lambda d: A * d[0] ** 2 + 2 * B * d[0] * d[1] + Cc * d[1] ** 2
                g = lambda d: np.array([2 * A * d[0] + 2 * B * d[1], 2 * B * d[0] + 2 * Cc * d[1]])
                x0 = np.clip(np.zeros(2), lo, hi)
                res = scipy.optimize.minimize(f, x0, jac=g, bounds=list(zip(lo, hi)),
                                              method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
                mmin = float(res.fun)
                if abs(mmin - 9.009) <= 9.009e-4:
                    continue
                assert ((ty * ntx + tx) in kept) == (mmin <= 9.009), (i, tx, ty, mmin)
                checked += 1
                dropped += (ty * ntx + tx) not in kept
    assert checked > 100 and dropped > 10


def test_near_plane_culls(oracle_mod):
    """Gaussians at or behind the near plane (z <= 0.2) are never rendered."""
    sc, view = _axis_scene([0.1, 0.2, -1.0, 0.25], [math.log(0.05)] * 4, [2.0] * 4,
                           [[0.1, 0.1, 0.1]] * 4)
    km = oracle_mod.keymode(sc, view, np.arange(4))
    assert list(km["culled"]) == [1, 1, 1, 0]


def test_sorted_lists_are_depth_then_slot(oracle_mod):
    """Per-tile lists hold exactly the Gaussians whose rectangle covers the tile,
    ordered by (depth bits, slot): the order Eq. 3 composites in, ties by slot."""
    sc, view = synth.tiny_scene(9, n=50, sh_degree=0, width=64, height=48, depth=3.0,
                                log_scale_mean=-2.0, spread=1.0)
    view.fx = view.fy = 60.0
    sc.means[10] = sc.means[11]  # an exact depth tie between slots 10 and 11
    ids, km, nk, off, slots = oracle_mod.view_lists(sc, view, 16, 16)
    assert nk == int(km["tiles"][km["culled"] == 0].sum())
    covers = [set(oracle_mod.record_tiles(km[i], view, 16, 16).tolist()) for i in range(len(ids))]
    for t in range(len(off) - 1):
        lst = slots[off[t]:off[t + 1]]
        want = [int(ids[i]) for i in range(len(ids)) if not km[i]["culled"] and t in covers[i]]
        assert sorted(lst.tolist()) == sorted(want)
        z = km["z"][np.searchsorted(ids, lst)]
        keys = list(zip(z.view(np.uint32).tolist(), lst.tolist()))
        assert keys == sorted(keys)


def _rect_min_m(A, B, Cc, lo, hi):
    """Exact minimum of m(d) = A dx^2 + 2 B dx dy + C dy^2 (positive definite)
    over the box lo <= d <= hi, in FP64: 0 when the box holds the centre,
    else the smallest of the four edges' 1D minima (each a clamped vertex)."""
    if lo[0] <= 0.0 <= hi[0] and lo[1] <= 0.0 <= hi[1]:
        return 0.0
    best = math.inf
    for dy in (lo[1], hi[1]):       # horizontal edges: minimise over dx
        dx = min(max(-B * dy / A, lo[0]), hi[0])
        best = min(best, A * dx * dx + 2 * B * dx * dy + Cc * dy * dy)
    for dx in (lo[0], hi[0]):       # vertical edges: minimise over dy
        dy = min(max(-B * dx / Cc, lo[1]), hi[1])
        best = min(best, A * dx * dx + 2 * B * dx * dy + Cc * dy * dy)
    return best


def _thin_scene(seed, n=60, width=112, height=96):
    """Needle-like Gaussians (one scale ~20-50x the others) at random
    orientations, plus round ones."""
    sc, view = synth.tiny_scene(seed, n=n, sh_degree=0, width=width, height=height, depth=3.0,
                                log_scale_mean=-2.0, spread=1.0)
    rng = np.random.default_rng(100 + seed)
    thin = rng.random(n) < 0.6
    ls = sc.log_scales.copy()
    ls[thin, 0] = rng.normal(-0.9, 0.3, thin.sum())
    ls[thin, 1] = rng.normal(-4.2, 0.3, thin.sum())
    ls[thin, 2] = rng.normal(-4.0, 0.3, thin.sum())
    sc.log_scales = ls.astype(np.float32)
    q = rng.normal(size=(n, 4))
    sc.quats = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    view.fx = view.fy = 90.0
    return sc, view


@pytest.mark.parametrize("seed,tile", [(0, (16, 16)), (1, (16, 16)), (2, (8, 8)),
                                       (3, (32, 8)), (4, (16, 16))])
def test_tile_coverage_exact_minimum_thin_gaussians(oracle_mod, seed, tile):
    """Tile coverage, pinned a second way: for every record, a tile of its
    bounding rectangle is kept iff the exact FP64 minimum of m over the
    rectangle of the tile's pixel centres (closed form: centre or edge
    minimisers) is <= 9.009, up to 1e-5 relative (the FP32 row rule's
    rounding); and every pixel whose centre has m <= 9 lies in a kept tile
    (brute force over all pixels). Scenes of thin, rotated Gaussians."""
    tw, th = tile
    sc, view = _thin_scene(seed)
    km = oracle_mod.keymode(sc, view, np.arange(sc.n), tile_w=tw, tile_h=th)
    ntx = (view.width + tw - 1) // tw
    yy, xx = np.mgrid[0:view.height, 0:view.width]
    checked = dropped = near = 0
    for i in range(sc.n):
        k = km[i]
        if k["culled"]:
            continue
        kept = set(oracle_mod.record_tiles(k, view, tw, th).tolist())
        u, v, A, B, Cc = (float(k[f]) for f in ("u", "v", "A", "B", "C"))
        for ty in range(k["ty0"], k["ty1"] + 1):
            for tx in range(k["tx0"], k["tx1"] + 1):
                lo = (tx * tw + 0.5 - u, ty * th + 0.5 - v)
                hi = (lo[0] + tw - 1, lo[1] + th - 1)
                mmin = _rect_min_m(A, B, Cc, lo, hi)
                if abs(mmin - 9.009) <= 9.009e-5:
                    near += 1
                    continue
                assert ((ty * ntx + tx) in kept) == (mmin <= 9.009), (i, tx, ty, mmin)
                checked += 1
                dropped += (ty * ntx + tx) not in kept
        # brute force over pixel centres: m <= 9 => the pixel's tile is kept
        dx, dy = xx + 0.5 - u, yy + 0.5 - v
        m = A * dx * dx + 2 * B * dx * dy + Cc * dy * dy
        for y, x in zip(*np.nonzero(m <= 9.0)):
            assert (y // th) * ntx + (x // tw) in kept, (i, x, y)
    assert checked > 200 and dropped > 20, (checked, dropped)
    assert near <= 0.01 * checked, near
