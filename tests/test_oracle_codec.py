"""Pins of the oracle's slice codec (Table 6 quantisation, Sec. 5.6.2) and ABR
tail drop (Sec. 5.5): the packet size against the paper's per-frame update
size, the round-trip error bounds of each code, the opacity code against
FP64, and the tail drop against a brute-force ranking."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth


def _rows(n=500, seed=2, sh=3):
    rng = np.random.default_rng(seed)
    attrs = synth.make_gaussians(rng, n, sh)
    z = np.full(n, 7, np.int32)
    return synth._scene(attrs, sh, z.copy(), z + 5, birth=z.copy())


def _make(n, sh):
    K = (sh + 1) ** 2
    z = np.zeros(n, np.int32)
    return synth.Scene(means=np.zeros((n, 3), np.float32), log_scales=np.zeros((n, 3), np.float32),
                       quats=np.zeros((n, 4), np.float32), opacity_logits=np.zeros(n, np.float32),
                       sh=np.zeros((n, K, 3), np.float32), start=z.copy(), expire=z.copy(),
                       birth=z.copy(), frozen=np.zeros(n, np.uint8), sh_degree=sh)


def test_update_size_matches_table_2(oracle_mod):
    # Sec. 5.1 updates 40K Gaussians per frame; Table 2: 1.2 MB per frame quantised
    b = oracle_mod.slice_packet_bytes(40_000, 40_000)
    assert b == 40_000 * 29
    assert abs(b / 1e6 - 1.2) < 0.05


def test_round_trip_bounds(oracle_mod):
    r = _rows()
    pkt = oracle_mod.slice_encode(r, r.n)
    d = oracle_mod.slice_decode(pkt, _make)
    # float16: relative error <= 2^-11 in the normal range
    for k in ("means", "log_scales"):
        a, b = getattr(r, k).astype(np.float64), getattr(d, k).astype(np.float64)
        assert np.all(np.abs(a - b) <= 2.0 ** -11 * np.abs(a) + 1e-7)
    # rotation: each unit-quaternion component within half a code step (+ rounding)
    q = r.quats.astype(np.float64)
    qn = q / np.linalg.norm(q, axis=1, keepdims=True)
    assert np.all(np.abs(qn - d.quats) <= 1.0 / 255.0 + 1e-6)
    # opacity: decoded sigmoid within half a code step of the original
    o = 1 / (1 + np.exp(-r.opacity_logits.astype(np.float64)))
    od = 1 / (1 + np.exp(-d.opacity_logits.astype(np.float64)))
    assert np.all(np.abs(o - od) <= 0.5 / 255 + 1e-6)
    # DC kept at full precision, higher bands dropped, the slice's lifespan
    np.testing.assert_array_equal(d.sh[:, 0], r.sh[:, 0])
    assert np.all(d.sh[:, 1:] == 0)
    assert np.all((d.start == 7) & (d.expire == 12) & (d.birth == 7) & (d.frozen == 1))


def test_opacity_code_against_fp64(oracle_mod):
    rng = np.random.default_rng(9)
    lg = rng.normal(0, 3, size=20000).astype(np.float32)
    k = oracle_mod.opacity_u8(lg).astype(np.int64)
    t = 255.0 / (1.0 + np.exp(-lg.astype(np.float64)))
    near_half = np.abs(t - np.floor(t) - 0.5) < 1e-4
    exact = np.rint(t).astype(np.int64)
    assert np.all((k == exact) | near_half)
    assert np.mean(near_half) < 1e-3


def test_tail_drop_keeps_the_most_opaque(oracle_mod):
    r = _rows(n=300)
    r.opacity_logits[10] = r.opacity_logits[11]  # a tie, broken by slot
    for keep in (300, 240, 180, 60, 1, 0):
        pkt = oracle_mod.slice_encode(r, keep)
        idx = pkt["index"].astype(np.int64)
        assert len(idx) == keep and np.all(np.diff(idx) > 0)
        ranked = sorted(range(r.n), key=lambda i: (-float(r.opacity_logits[i]), i))
        assert set(idx.tolist()) == set(ranked[:keep])
        d = oracle_mod.slice_decode(pkt, _make)
        live = (d.start <= 7) & (7 < d.expire)
        assert int(live.sum()) == keep
        assert oracle_mod.slice_packet_bytes(300, keep) == keep * 29 + (4 * keep if keep < 300 else 0)
