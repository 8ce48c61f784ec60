"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs. Discrete stages are compared bit for bit, pixels at
1e-4 max abs, gradients at 1e-3 relative."""
import math

import numpy as np
import pytest

from paper_2409_07759_b300 import synth

from gpu_helpers import BANDS, compare_grads, compare_image, gpu_lists, gpu_pixels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_07759_b300 import api
    r = api.Renderer()
    yield r
    r.close()


def _state(scene):
    from paper_2409_07759_b300 import api
    return api.GaussianState.from_scene(scene)


def _np(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------ compaction --

@pytest.mark.parametrize("frame", [0, 57, 150, 299, 400])
def test_active_ids_bit_exact(R, oracle_mod, frame):
    """Sec. 4.2 filter: the ascending active ids equal the oracle's."""
    sc, _, _ = synth.config1()
    st = _state(sc)
    ids = _np(R.active_ids(st, frame))
    ref = oracle_mod.active_ids(sc.start, sc.expire, frame)
    np.testing.assert_array_equal(ids, ref)


def test_active_ids_ragged_and_empty(R, oracle_mod):
    rng = np.random.default_rng(5)
    for n in (1, 1023, 1024, 1025, 4097):
        sc, _ = synth.tiny_scene(1, n=n, sh_degree=0)
        sc.start = rng.integers(0, 4, n).astype(np.int32)
        sc.expire = (sc.start + rng.integers(0, 3, n)).astype(np.int32)  # some empty spans
        st = _state(sc)
        for f in (0, 2, 9):
            np.testing.assert_array_equal(_np(R.active_ids(st, f)),
                                          oracle_mod.active_ids(sc.start, sc.expire, f))


# ------------------------------------------------------- records and keys --

def _check_records_and_lists(R, oracle_mod, sc, views, tile=(16, 16)):
    from paper_2409_07759_b300 import _abi
    st = _state(sc)
    _, saved = R.render(st, views, keep_saved=True)
    rslot = saved.export(_abi.EXPORT_RECORD_SLOT)
    rview = saved.export(_abi.EXPORT_RECORD_VIEW)
    rtiles = saved.export(_abi.EXPORT_RECORD_TILES)
    rrect = saved.export(_abi.EXPORT_RECORD_RECT)
    rdepth = saved.export(_abi.EXPORT_RECORD_DEPTH)
    total_keys = 0
    for vi, v in enumerate(views):
        ids, km, nk, off, slots = oracle_mod.view_lists(sc, v, tile[0], tile[1])
        m = rview == vi
        np.testing.assert_array_equal(rslot[m], ids)
        want_tiles = np.where(km["culled"] == 1, 0, km["tiles"])
        np.testing.assert_array_equal(rtiles[m], want_tiles)
        live = (km["culled"] == 0)
        np.testing.assert_array_equal(rrect[m][live & (want_tiles > 0)],
                                      np.stack([km["tx0"], km["tx1"], km["ty0"], km["ty1"]], 1)
                                      [live & (want_tiles > 0)])
        np.testing.assert_array_equal(rdepth[m][live].view(np.uint32),
                                      km["z"][live].view(np.uint32))
        goff, gslots = gpu_lists(saved, vi)
        np.testing.assert_array_equal(goff, off)
        np.testing.assert_array_equal(gslots, slots)
        total_keys += nk
    assert saved.info().n_keys == total_keys
    saved.release()
    return total_keys


def test_config0_records_keys_order_bit_exact(R, oracle_mod):
    """Active ids, tile counts, tile rectangles, depth keys and the per-tile
    sorted order of config 0 equal the oracle bit for bit."""
    sc, views = synth.config0()
    assert _check_records_and_lists(R, oracle_mod, sc, views) > 0


def test_config1_records_keys_order_bit_exact(R, oracle_mod):
    """Same at the full config-1 size (100k Gaussians, 1352x1014, SH3)."""
    sc, views, _ = synth.config1()
    assert _check_records_and_lists(R, oracle_mod, sc, views) > 100_000


def test_mixed_resolution_batch_lists_bit_exact(R, oracle_mod):
    """One batch of four resolutions (96x72, 320x240, 640x480, 1280x720) of
    one scene: a batch of few super tiles, whose tile-list expansion cuts each
    view's super tiles into its own number of parts (more for the smaller
    views, whose super tiles hold longer lists). Every view's records, per-tile
    lists and their depth order equal the oracle's bit for bit."""
    sc, v0 = synth.tiny_scene(21, n=30_000, sh_degree=1, width=96, height=72, depth=4.0,
                              log_scale_mean=-3.2, spread=1.2)
    views = []
    for w, h in ((96, 72), (320, 240), (640, 480), (1280, 720)):
        fx, fy, cx, cy = synth.intrinsics_for(w, h)
        views.append(synth.View(w, h, fx, fy, cx, cy, v0.R, v0.t, 0))
    assert _check_records_and_lists(R, oracle_mod, sc, views) > 30_000


def test_depth_ties_follow_slot_order(R, oracle_mod):
    sc, view = synth.tiny_scene(9, n=300, sh_degree=0, width=64, height=48, depth=3.0,
                                log_scale_mean=-2.0, spread=1.0)
    view.fx = view.fy = 60.0
    sc.means[100:140] = sc.means[100]  # 40 Gaussians at one depth
    _check_records_and_lists(R, oracle_mod, sc, [view])


# ---------------------------------------------------------------- pixels --

def _render_and_compare(R, oracle_mod, sc, views, bg=(0.0, 0.0, 0.0), tile=(16, 16)):
    from paper_2409_07759_b300 import _abi
    st = _state(sc)
    imgs, saved = R.render(st, views, bg=bg, keep_saved=True)
    reps = []
    for vi, v in enumerate(views):
        ref = oracle_mod.render(sc, v, bg=bg, tile_w=tile[0], tile_h=tile[1], mode="tiled",
                                bands=BANDS)
        T = gpu_pixels(saved, vi, _abi.EXPORT_FINAL_T)
        last = gpu_pixels(saved, vi, _abi.EXPORT_LAST)
        reps.append(compare_image(_np(imgs[vi]), T, last, ref,
                                  replay=(sc, v, tile[0], tile[1], bg)))
    saved.release()
    return reps


def test_config0_pixels(R, oracle_mod):
    """Config 0 image within 1e-4 of the FP64 oracle (flagged pixels reported)."""
    sc, views = synth.config0()
    rep = _render_and_compare(R, oracle_mod, sc, views)
    print(rep)


def test_config0_background_and_ragged(R, oracle_mod):
    """A non-black background and an image size that is not a multiple of the
    tile (ragged last row and column of tiles)."""
    sc, views = synth.config0()
    v = views[0]
    v2 = synth.View(131, 97, v.fx, v.fy, 65.5, 48.5, v.R, v.t, 0)
    _render_and_compare(R, oracle_mod, sc, [v2], bg=(0.2, 0.5, 0.9))


@pytest.mark.parametrize("tile,batch,ppt", [((8, 8), 32, 1), ((8, 8), 256, 2),
                                            ((16, 16), 64, 1), ((16, 16), 128, 4),
                                            ((32, 8), 128, 2), ((32, 8), 256, 4)])
def test_tile_shapes_and_batches(oracle_mod, tile, batch, ppt):
    """Every tile shape, staging batch size and pixels-per-thread choice gives
    the oracle's image."""
    from paper_2409_07759_b300 import api
    r = api.Renderer(tile=tile, batch=batch, pixels_per_thread=ppt,
                     bwd_pixels_per_thread=ppt, bwd_batch=batch)
    sc, views = synth.config0()
    _check_records_and_lists(r, oracle_mod, sc, views, tile=tile)
    _render_and_compare(r, oracle_mod, sc, views, tile=tile)
    r.close()


def test_config1_pixels_full(R, oracle_mod):
    """Full config-1 frame (1352x1014, SH3, 100k Gaussians at frame 150)."""
    sc, views, _ = synth.config1()
    rep = _render_and_compare(R, oracle_mod, sc, views)
    print(rep)


def test_empty_and_offscreen(R, oracle_mod):
    """No active Gaussian, and every Gaussian behind the camera: background."""
    sc, views = synth.config0()
    v = views[0]
    empty = synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, 5)
    st = _state(sc)
    imgs, _ = R.render(st, [empty], bg=(0.3, 0.1, 0.7))
    want = np.broadcast_to(np.array([0.3, 0.1, 0.7], np.float32)[:, None, None], (3, 96, 128))
    np.testing.assert_array_equal(_np(imgs[0]), want)
    behind = synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R,
                        np.array([0, 0, -10], np.float32), 0)
    imgs, _ = R.render(st, [behind])
    assert np.abs(_np(imgs[0])).max() == 0.0


def test_batched_equals_plain(R, oracle_mod):
    """The batched launch and the plain per-view path give identical images."""
    sc, views, _ = synth.config2(width=160, height=120, n=20000, n_frames=3, per_frame=2)
    st = _state(sc)
    a, _ = R.render(st, views, batched=True)
    b, _ = R.render(st, views, batched=False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(_np(x), _np(y))


def test_multiview_multiframe_pixels(R, oracle_mod):
    """Views at different frames in one batched call (several frame groups,
    interleaved in the call order)."""
    sc, views, _ = synth.config2(width=200, height=150, n=30000, n_frames=3, per_frame=2)
    views = [views[0], views[2], views[1], views[4], views[3], views[5]]
    _render_and_compare(R, oracle_mod, sc, views)


# -------------------------------------------------------------- backward --

def _grads_vs_oracle(R, oracle_mod, sc, views, dLs, bg=(0.0, 0.0, 0.0), gpu_dLs=None):
    """GPU backward with gpu_dLs (device tensors, default: dLs) against the
    oracle's backward with dLs (host arrays that never come from the GPU)."""
    from paper_2409_07759_b300 import api
    st = _state(sc)
    imgs, saved = R.render(st, views, bg=bg, keep_saved=True)
    grads = st.zero_grads()
    if gpu_dLs is None:
        gpu_dLs = [torch.from_numpy(np.asarray(d, np.float32)).cuda() for d in dLs]
    R.backward(st, saved, gpu_dLs, grads)
    saved.release()
    ref = oracle_mod.zero_grads(sc)
    for v, d in zip(views, dLs):
        oracle_mod.render_bwd(sc, v, np.asarray(d, np.float32).astype(np.float64), bg=bg,
                              grads=ref, bands=BANDS)
    gpu = {k: _np(getattr(grads, k)) for k in api.PARAM_NAMES}
    return compare_grads(gpu, ref)


@pytest.mark.parametrize("ppt,tile", [(1, (16, 16)), (2, (16, 16)), (4, (16, 16)),
                                      (8, (16, 16)), (8, (32, 8)), (2, (8, 8))])
def test_backward_small_scene(oracle_mod, ppt, tile):
    """Gradients of every attribute (SH3) against the FP64 adjoint, for each
    pixels-per-thread variant of the reverse blend."""
    from paper_2409_07759_b300 import api
    r = api.Renderer(tile=tile, bwd_pixels_per_thread=ppt, pixels_per_thread=min(ppt, 2))
    sc, view = synth.tiny_scene(3, n=200, sh_degree=3, width=96, height=72, depth=3.0,
                                log_scale_mean=-2.2, spread=0.9)
    view.fx = view.fy = 90.0
    d = np.random.default_rng(0).normal(size=(3, 72, 96))
    print(_grads_vs_oracle(r, oracle_mod, sc, [view], [d], bg=(0.1, 0.2, 0.3)))
    r.close()


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_sh_degrees_pixels_and_gradients(oracle_mod, deg):
    """SH degrees 0-2: 3K coefficients per Gaussian of 3, 12 and 27 floats, so the
    projection and its backward read them as float4 rows (12) and as scalars
    (3, 27, not multiples of 4). Pixels and the gradients of every attribute
    against the FP64 oracle."""
    from paper_2409_07759_b300 import api
    r = api.Renderer()
    sc, view = synth.tiny_scene(3 + deg, n=200, sh_degree=deg, width=96, height=72, depth=3.0,
                                log_scale_mean=-2.2, spread=0.9)
    view.fx = view.fy = 90.0
    _render_and_compare(r, oracle_mod, sc, [view], bg=(0.1, 0.2, 0.3))
    d = np.random.default_rng(40 + deg).normal(size=(3, 72, 96))
    print(_grads_vs_oracle(r, oracle_mod, sc, [view], [d], bg=(0.1, 0.2, 0.3)))
    r.close()


def test_backward_config1_l1(R, oracle_mod):
    """Config 1 full size: L1 loss against the seeded target, gradients of all
    attributes of the 100k Gaussians."""
    sc, views, targets = synth.config1()
    st = _state(sc)
    imgs, _ = R.render(st, views)
    loss, dls = R.loss_l1(views, imgs, [torch.from_numpy(t).cuda() for t in targets])
    ref_img = oracle_mod.render(sc, views[0], mode="tiled")["rgb"]
    ref_loss, ref_dl = oracle_mod.l1_loss_grad([ref_img], targets)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    # each side differentiates its own L1: the signs differ only where the two
    # images straddle the target within rounding
    flips = int((np.sign(_np(dls[0])) != np.sign(ref_dl[0])).sum())
    assert flips <= 1e-4 * ref_dl[0].size, flips
    print(flips, _grads_vs_oracle(R, oracle_mod, sc, views, ref_dl, gpu_dLs=dls))


def test_backward_multiview_frozen(R, oracle_mod):
    """Several views and frames summed into one gradient; frozen slots get none."""
    sc, views, _ = synth.config2(width=160, height=120, n=20000, n_frames=3, per_frame=2)
    rng = np.random.default_rng(1)
    dls = [rng.normal(size=(3, v.height, v.width)) for v in views]
    print(_grads_vs_oracle(R, oracle_mod, sc, views, dls))


def test_autograd_function(R, oracle_mod):
    """torch.autograd through the library's forward and backward."""
    from paper_2409_07759_b300 import api
    sc, view = synth.tiny_scene(4, n=150, sh_degree=1, width=64, height=48, depth=3.0,
                                log_scale_mean=-2.0, spread=0.8)
    view.fx = view.fy = 60.0
    st = _state(sc)
    params = [p.clone().requires_grad_(True) for p in st.params()]
    (img,) = api.render(R, st, [view], params=params)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    ref = oracle_mod.zero_grads(sc)
    oracle_mod.render_bwd(sc, view, _np(w).astype(np.float64), grads=ref, bands=BANDS)
    compare_grads({k: _np(p.grad) for k, p in zip(api.PARAM_NAMES, params)}, ref)


def test_fused_forward_l1_u8_targets(R):
    """8-bit targets give the same image, dL/dC and loss as the float
    targets k * (1/255) (FP32 product, as the kernel reads them)."""
    sc, views, targets = synth.config1()
    st = _state(sc)
    rng = np.random.default_rng(11)
    t8 = [rng.integers(0, 256, size=t.shape, dtype=np.uint8) for t in targets]
    tu = [torch.from_numpy(t).cuda() for t in t8]
    inv = torch.tensor(1.0 / 255.0, dtype=torch.float32, device="cuda")
    tf = [t.float() * inv for t in tu]
    ia, da, la, sa = R.render_l1(st, views, tu)
    ib, db, lb, sb = R.render_l1(st, views, tf)
    sa.release()
    sb.release()
    for x, y in zip(ia + da, ib + db):
        assert torch.equal(x, y)
    assert float(la.item()) == pytest.approx(float(lb.item()), rel=1e-5)
    with pytest.raises(ValueError):
        R.render_l1(st, views, [tu[0].float().double()])


def test_fused_forward_l1(R, oracle_mod):
    """The forward with the L1 term fused into the blend gives the same image
    and gradient as the separate loss pass, and the oracle's loss."""
    sc, views, targets = synth.config1()
    st = _state(sc)
    tg = [torch.from_numpy(t).cuda() for t in targets]
    imgs, dl, loss, saved = R.render_l1(st, views, tg)
    saved.release()
    imgs2, _ = R.render(st, views)
    loss2, dl2 = R.loss_l1(views, imgs2, tg)
    assert torch.equal(imgs[0], imgs2[0]) and torch.equal(dl[0], dl2[0])
    # both losses are FP32 sums of ~4e4 warp partials added atomically in no
    # fixed order: relative spread ~sqrt(n) * 6e-8, so 1e-5 (as against FP64)
    assert float(loss.item()) == pytest.approx(float(loss2.item()), rel=1e-5)
    ref_img = oracle_mod.render(sc, views[0], mode="tiled")["rgb"]
    ref_loss, _ = oracle_mod.l1_loss_grad([ref_img], targets)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_backward_sh_degrees(oracle_mod, deg):
    """Gradients of every attribute for SH degrees 0-2 (degree 3 above)."""
    from paper_2409_07759_b300 import api
    r = api.Renderer()
    sc, view = synth.tiny_scene(5 + deg, n=180, sh_degree=deg, width=80, height=64, depth=3.0,
                                log_scale_mean=-2.2, spread=0.9)
    view.fx = view.fy = 80.0
    d = np.random.default_rng(deg).normal(size=(3, 64, 80))
    print(_grads_vs_oracle(r, oracle_mod, sc, [view], [d], bg=(0.2, 0.1, 0.0)))
    r.close()


def test_batches_split_by_super_tiles():
    """A batched call whose views hold more than 2^16 super tiles (8x8 tiles:
    32x32-pixel super tiles; 33 views of 1920x1080 need 67,320) runs in
    several batches and gives exactly the images of the plain path."""
    from paper_2409_07759_b300 import api
    sc, _, _ = synth.config2(width=64, height=48, n=20000, n_frames=1, per_frame=1)
    ring = synth.ring_cameras(20, 4.0, 1920, 1080)
    views = []
    for j in range(33):
        v = ring[j % 20]
        views.append(synth.View(v.width, v.height, v.fx, v.fy, v.cx, v.cy, v.R, v.t, 150))
    r = api.Renderer(tile=(8, 8), pixels_per_thread=2)
    st = _state(sc)
    a, saved = r.render(st, views, batched=True, keep_saved=True)
    assert saved.info().n_batches == 2
    saved.release()
    b, _ = r.render(st, views, batched=False)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    r.close()


def test_view_beyond_the_super_tile_limit_is_rejected():
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300._abi import SwgsError
    sc, _ = synth.tiny_scene(1, n=10, sh_degree=0)
    # 8x8 tiles, 32-pixel super tiles: 8224 x 8224 pixels hold 257^2 > 2^16
    v = synth.View(8224, 8224, 8000.0, 8000.0, 4112.0, 4112.0, np.eye(3, dtype=np.float32),
                   np.zeros(3, np.float32), 0)
    r = api.Renderer(tile=(8, 8), pixels_per_thread=2)
    with pytest.raises(SwgsError):
        r.render(_state(sc), [v])
    r.close()


@pytest.mark.parametrize("ppt", [2, 8])
def test_backward_high_opacity_clamp(oracle_mod, ppt):
    """A third of the Gaussians above the 0.99 alpha clamp (opacity 0.9975):
    the blends' clamp branch gives the oracle's image and gradients (where
    the clamp holds, dalpha/dm is zero), next to the unclamped Gaussians."""
    from paper_2409_07759_b300 import api
    r = api.Renderer(bwd_pixels_per_thread=ppt, pixels_per_thread=min(ppt, 4))
    sc, view = synth.tiny_scene(5, n=200, sh_degree=1, width=96, height=72, depth=3.0,
                                log_scale_mean=-2.2, spread=0.9)
    view.fx = view.fy = 90.0
    high = np.random.default_rng(6).random(sc.n) < 1 / 3
    sc.opacity_logits[high] = 6.0
    assert (1 / (1 + np.exp(-sc.opacity_logits)) > 0.99).sum() >= 40
    _render_and_compare(r, oracle_mod, sc, [view])
    d = np.random.default_rng(2).normal(size=(3, 72, 96))
    print(_grads_vs_oracle(r, oracle_mod, sc, [view], [d], bg=(0.1, 0.2, 0.3)))
    r.close()


def test_sort_forms_agree():
    """The single-pass digit passes and the three-kernel passes give the same
    depth order, per-tile lists and images (bit for bit), over several views."""
    from paper_2409_07759_b300 import api, _abi
    sc, views, _ = synth.config2(width=320, height=240, n=60000, n_frames=3, per_frame=2)
    st = _state(sc)
    out = {}
    for single in (True, False):
        r = api.Renderer(sort_single_pass=single)
        imgs, saved = r.render(st, views, keep_saved=True)
        torch.cuda.synchronize()
        out[single] = ([_np(i) for i in imgs],
                       saved.export(_abi.EXPORT_SORTED_SLOT), saved.export(_abi.EXPORT_TILE_RANGES),
                       saved.export(_abi.EXPORT_RECORD_DEPTH), saved.export(_abi.EXPORT_LAST))
        saved.release()
        r.close()
    a, b = out[True], out[False]
    assert a[1].size > 10000
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)


def _edge_scene():
    """Small, thin, rotated Gaussians spread over a 128x96 view (supports a
    few pixels across), a sixth of them above the 0.99 clamp."""
    sc, view = synth.tiny_scene(11, n=3000, sh_degree=1, width=128, height=96, depth=3.0,
                                log_scale_mean=-3.6, spread=1.0)
    rng = np.random.default_rng(12)
    sc.log_scales[:, 0] += rng.uniform(-0.2, 1.6, size=sc.n).astype(np.float32)
    sc.opacity_logits[rng.random(sc.n) < 1 / 6] = 6.0
    view.fx = view.fy = 110.0
    return sc, view


@pytest.mark.parametrize("tile,ppts", [((16, 16), (1, 2, 4)), ((32, 8), (1, 2, 4))])
def test_forward_forms_agree(oracle_mod, tile, ppts):
    """Every pixels-per-thread form of the forward blend gives the same image,
    final transmittance and last-contributor index, bit for bit: the packed
    FP32x2 forms (2 and 4 pixels a thread, negated staging, the clamp branch)
    against the scalar form (1 pixel a thread), on thin rotated Gaussians and
    a window-step scene."""
    from paper_2409_07759_b300 import api, _abi
    scenes = [_edge_scene()]
    sc2, views2, _ = synth.config2(width=200, height=150, n=30000, n_frames=2, per_frame=2)
    scenes.append((sc2, views2))
    for sc, views in scenes:
        views = views if isinstance(views, list) else [views]
        st = _state(sc)
        out = []
        for ppt in ppts:
            r = api.Renderer(tile=tile, batch=64, pixels_per_thread=ppt)
            imgs, saved = r.render(st, views, bg=(0.2, 0.3, 0.4), keep_saved=True)
            torch.cuda.synchronize()
            out.append(([_np(i) for i in imgs], saved.export(_abi.EXPORT_FINAL_T),
                        saved.export(_abi.EXPORT_LAST)))
            saved.release()
            r.close()
        assert out[0][2].max() > 0
        for o in out[1:]:
            for x, y in zip(out[0][0], o[0]):
                np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(out[0][1], o[1])
            np.testing.assert_array_equal(out[0][2], o[2])
    sc, view = scenes[0]
    r = api.Renderer(tile=tile, pixels_per_thread=4)
    _render_and_compare(r, oracle_mod, sc, [view], tile=tile)
    r.close()


def test_backward_forms_agree_on_covered_tiles():
    """Every pixels-per-thread form of the reverse blend gives the same
    gradients (to 1e-5 of each attribute's largest magnitude: the forms sum
    in different orders) on a scene where a third of the tiles are fully
    covered, so that the packed forms run their body for Gaussians in front
    of every pixel's last contributor. The scalar form (1 pixel a thread) has no such body,
    no paired warp reductions and reduces with shared-memory atomics."""
    from paper_2409_07759_b300 import api, _abi
    sc, views, _ = synth.config2(width=256, height=192, n=60000, n_frames=1, per_frame=2)
    st = _state(sc)
    rng = np.random.default_rng(9)
    dls = [torch.from_numpy(rng.normal(size=(3, v.height, v.width)).astype(np.float32)).cuda()
           for v in views]
    grads = {}
    covered = None
    for ppt in (1, 2, 4, 8):
        r = api.Renderer(bwd_pixels_per_thread=ppt, pixels_per_thread=min(ppt, 4))
        imgs, saved = r.render(st, views, keep_saved=True)
        if covered is None:
            last = saved.export(_abi.EXPORT_LAST).reshape(len(views), 192, 256)
            t = last.reshape(len(views), 12, 16, 16, 16).min(axis=(2, 4))
            covered = float((t > 0).mean())
        g = st.zero_grads()
        r.backward(st, saved, dls, g)
        torch.cuda.synchronize()
        grads[ppt] = {k: _np(getattr(g, k)).copy() for k in api.PARAM_NAMES}
        saved.release()
        r.close()
    assert covered > 0.25, covered  # 38% of the tiles: the object fills the middle
    for ppt in (2, 4, 8):
        for k in api.PARAM_NAMES:
            a, b = grads[1][k], grads[ppt][k]
            scale = max(float(np.abs(a).max()), 1e-30)
            assert float(np.abs(a - b).max()) <= 1e-5 * scale, (ppt, k)


def test_rgb8_images_are_the_quantised_float_images(R):
    """swgs_render_fwd_rgb8 writes round(255 clamp(c, 0, 1)) of the float
    render's channels, interleaved [H,W,3], bit for bit (ragged sizes, a
    background, several views and frames in one batch)."""
    sc, views, _ = synth.config2(width=203, height=117, n=20000, n_frames=2, per_frame=2)
    st = _state(sc)
    bg = (0.1, 0.7, 1.3)  # a channel above 1 exercises the clamp
    f32, _ = R.render(st, views, bg=bg)
    u8, saved = R.render_rgb8(st, views, bg=bg, keep_saved=True)
    for a, b in zip(f32, u8):
        want = np.rint(np.clip(_np(a), 0.0, 1.0).astype(np.float32) * np.float32(255.0))
        np.testing.assert_array_equal(_np(b), want.transpose(1, 2, 0).astype(np.uint8))
    assert saved.info().n_views == len(views)
    saved.release()
