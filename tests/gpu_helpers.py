"""Shared helpers of the GPU parity tests (comparison of the CUDA path, called
through the C ABI, with the FP64 oracle on the same seeded inputs)."""
import numpy as np

# Parity tolerances of the FP32 path against the FP64 oracle: pixels 1e-4 max
# abs, gradients 1e-3 relative.
PIX_TOL = 1e-4
GRAD_REL_TOL = 1e-3
# Near-discontinuity bands (relative) within which FP32 and FP64 may decide a
# threshold differently. A pixel touched by such a pair is flagged: it leaves
# the plain 1e-4 comparison and is instead checked against every valid result
# the oracle's decision replay gives for it (check_flagged), and the flagged
# count is asserted to stay small. From FP32 error: m is off by at most ~1e-5
# relative (conic conditioning), alpha by ~m/2 of that (<= 4.5e-5), the
# running T by ~1e-4.
BANDS = dict(m=3e-5, alpha=6e-5, t_stop=5e-4, clamp=6e-5, guard=1e-4, colour=1e-5)


def view_table(saved):
    from paper_2409_07759_b300 import _abi
    return saved.export(_abi.EXPORT_VIEW_TABLE)


def gpu_lists(saved, view_index):
    """Per-tile slot lists of one view from the GPU's saved state, as
    (tile_off, tile_slot) in the oracle's CSR layout."""
    from paper_2409_07759_b300 import _abi
    tab = view_table(saved)
    row = tab[tab[:, 0] == view_index][0]
    _, tile_base, _, _, ntx, nty = row
    ranges = saved.export(_abi.EXPORT_TILE_RANGES)
    slots = saved.export(_abi.EXPORT_SORTED_SLOT)
    nt = ntx * nty
    off = [0]
    out = []
    for t in range(nt):
        b, e = ranges[tile_base + t]
        out.append(slots[b:e])
        off.append(off[-1] + (e - b))
    return np.array(off, np.int64), (np.concatenate(out) if out else np.zeros(0, np.int32))


def gpu_pixels(saved, view_index, what):
    from paper_2409_07759_b300 import _abi
    tab = view_table(saved)
    row = tab[tab[:, 0] == view_index][0]
    v = saved.views[view_index]
    arr = saved.export(what)
    pb = row[2]
    return arr[pb:pb + v.width * v.height].reshape(v.height, v.width)


def compare_image(gpu_rgb, gpu_T, gpu_last, ref, max_flag_frac=0.02, replay=None):
    """Pixel parity. Unflagged pixels: rgb and T within 1e-4 of the FP64
    oracle and last equal. Flagged pixels (an FP64 pair within BANDS of a
    threshold, where FP32 may decide the test the other way): with `replay` =
    (scene, view, tile_w, tile_h, bg), the oracle replays each such pixel's
    walk with both outcomes at every near-threshold pair, and the GPU's rgb, T
    (within 1e-4) and last (exactly) must equal one of those valid results.
    Returns the error report."""
    flag = (ref["flags"] & 1) != 0
    ok = ~flag
    err_rgb = np.abs(gpu_rgb.astype(np.float64) - ref["rgb"])
    err_T = np.abs(gpu_T.astype(np.float64) - ref["T"])
    rep = dict(max_abs_rgb=float(err_rgb[:, ok].max(initial=0.0)),
               max_abs_T=float(err_T[ok].max(initial=0.0)),
               flagged=int(flag.sum()), pixels=int(flag.size),
               max_abs_rgb_flagged=float(err_rgb[:, flag].max(initial=0.0)),
               last_mismatch=int(((gpu_last != ref["last_pos"]) & ok).sum()))
    assert rep["flagged"] <= max_flag_frac * flag.size, rep
    assert rep["max_abs_rgb"] <= PIX_TOL, rep
    assert rep["max_abs_T"] <= PIX_TOL, rep
    assert rep["last_mismatch"] == 0, rep
    if replay is not None and rep["flagged"]:
        rep.update(check_flagged(gpu_rgb, gpu_T, gpu_last, flag, ref, *replay))
    return rep


def check_flagged(gpu_rgb, gpu_T, gpu_last, flag, ref, scene, view, tile_w, tile_h, bg):
    """Every flagged pixel's GPU result equals one of the oracle's valid
    results (decision replay) within 1e-4 (rgb, T) and exactly (last).
    Also counts the flagged pixels where the GPU took the other side of a
    near-threshold test than FP64 (its result is not the FP64 walk's)."""
    import oracle
    py, px = np.nonzero(flag)
    res = oracle.render_variants(scene, view, px, py, BANDS, bg=bg, tile_w=tile_w,
                                 tile_h=tile_h, max_per=4096)
    unverifiable, mismatched, other_side, worst = 0, [], 0, 0.0
    for k, r in enumerate(res):
        if r is None:
            unverifiable += 1
            continue
        rgb, T, last = r
        y, x = int(py[k]), int(px[k])
        g_rgb = gpu_rgb[:, y, x].astype(np.float64)
        g_T = float(gpu_T[y, x])
        g_last = int(gpu_last[y, x])
        d = np.maximum(np.abs(rgb - g_rgb[None, :]).max(1), np.abs(T - g_T))
        d = np.where(last == g_last, d, np.inf)
        i = int(np.argmin(d))
        if not d[i] <= PIX_TOL:
            mismatched.append((x, y, float(d[i])))
            continue
        worst = max(worst, float(d[i]))
        d64 = max(float(np.abs(ref["rgb"][:, y, x] - g_rgb).max()), abs(ref["T"][y, x] - g_T))
        other_side += int(g_last != ref["last_pos"][y, x] or d64 > PIX_TOL)
    out = dict(flagged_unverifiable=unverifiable, flagged_mismatched=len(mismatched),
               flagged_max_abs=worst, flagged_other_side=other_side)
    assert unverifiable == 0 and not mismatched, (out, mismatched[:10])
    return out


def compare_grads(gpu: dict, ref: dict, tol=GRAD_REL_TOL):
    """Per attribute: ||d||_2 / ||g||_2 <= tol and max |d| <= tol * max |g|."""
    rep = {}
    for k, g in ref.items():
        a = gpu[k].astype(np.float64)
        d = a - g
        nrm = np.linalg.norm(g)
        rel = float(np.linalg.norm(d) / nrm) if nrm > 0 else float(np.linalg.norm(d))
        elem = float(np.abs(d).max() / max(np.abs(g).max(), 1e-30))
        rep[k] = (rel, elem)
    bad = {k: v for k, v in rep.items() if v[0] > tol or v[1] > tol}
    assert not bad, rep
    return rep
