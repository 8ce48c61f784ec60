"""The streamed-slice codec (Table 6 quantisation, Sec. 5.5 tail drop) on the
device against the oracle: every section of the packet bit for bit (device and
pinned-host output), and the decode into a slice of a larger buffer."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "start", "expire", "birth",
          "frozen")


def _rows(n, sh=3, seed=4):
    rng = np.random.default_rng(seed)
    attrs = synth.make_gaussians(rng, n, sh)
    attrs["opacity_logits"][: n // 10] = attrs["opacity_logits"][n // 10: 2 * (n // 10)]  # ties
    z = np.full(n, 40, np.int32)
    return synth._scene(attrs, sh, z.copy(), z + 50, birth=z.copy())


def _layout(count, keep):
    """The packet layout written down in the header (include/swgs.h)."""
    a16 = lambda x: (x + 15) & ~15
    o, L = 32, {}
    if keep < count:
        L["index"] = o
        o += a16(4 * keep)
    for name, size in (("means", 6), ("log_scales", 6), ("quats", 4), ("opacity", 1), ("dc", 12)):
        L[name] = o
        o += a16(size * keep)
    L["total"] = o
    return L


def _parse(buf, count, keep):
    b = buf.cpu().numpy().tobytes() if buf.is_cuda else buf.numpy().tobytes()
    L = _layout(count, keep)
    h = np.frombuffer(b[:32], np.int32)
    out = dict(header=h)
    if keep < count:
        out["index"] = np.frombuffer(b, np.uint32, keep, L["index"])
    out["means"] = np.frombuffer(b, np.float16, 3 * keep, L["means"]).reshape(keep, 3)
    out["log_scales"] = np.frombuffer(b, np.float16, 3 * keep, L["log_scales"]).reshape(keep, 3)
    out["quats"] = np.frombuffer(b, np.uint8, 4 * keep, L["quats"]).reshape(keep, 4)
    out["opacity"] = np.frombuffer(b, np.uint8, keep, L["opacity"])
    out["dc"] = np.frombuffer(b, np.float32, 3 * keep, L["dc"]).reshape(keep, 3)
    return out, L


@pytest.mark.parametrize("frac", [1.0, 0.8, 0.37, 0.0])
@pytest.mark.parametrize("to_host", [False, True])
def test_encode_matches_oracle(oracle_mod, frac, to_host):
    from paper_2409_07759_b300 import api
    n = 5000
    rows = _rows(n)
    keep = int(round(frac * n))
    r = api.Renderer()
    src = api.GaussianState.from_scene(rows)
    nbytes = api.Renderer.slice_packet_bytes(n, keep)
    assert nbytes == _layout(n, keep)["total"]
    out = torch.zeros(nbytes + 64, dtype=torch.uint8, device="cpu" if to_host else "cuda")
    if to_host:
        out = out.pin_memory()
    pkt = r.slice_encode(src, n, keep, out=out)
    torch.cuda.synchronize()
    assert pkt.numel() == nbytes
    got, _ = _parse(pkt, n, keep)
    ref = oracle_mod.slice_encode(rows, keep)
    h = got["header"]
    assert h[0] == 0x43574753 and h[1] == 1
    assert list(h[2:]) == [n, keep, 3, 40, 40, 90]
    if keep < n:
        np.testing.assert_array_equal(got["index"], ref["index"])
    for k in ("means", "log_scales"):
        np.testing.assert_array_equal(got[k].view(np.uint16), ref[k].view(np.uint16))
    for k in ("quats", "opacity", "dc"):
        np.testing.assert_array_equal(got[k], ref[k])
    r.close()


@pytest.mark.parametrize("keep", [4000, 1500])
def test_decode_matches_oracle(oracle_mod, keep):
    from paper_2409_07759_b300 import api
    n, first = 4000, 1200
    rows = _rows(n, seed=6)
    r = api.Renderer()
    pkt = r.slice_encode(api.GaussianState.from_scene(rows), n, keep)
    big = _rows(first + n + 300, seed=7)
    dst = api.GaussianState.from_scene(big)
    r.slice_decode(pkt, dst, first)
    host_pkt = pkt.cpu().pin_memory()
    dst2 = api.GaussianState.from_scene(big)
    r.slice_decode(host_pkt, dst2, first)
    torch.cuda.synchronize()

    def make(m, sh):
        K = (sh + 1) ** 2
        z = np.zeros(m, np.int32)
        return synth.Scene(means=np.zeros((m, 3), np.float32),
                           log_scales=np.zeros((m, 3), np.float32),
                           quats=np.zeros((m, 4), np.float32),
                           opacity_logits=np.zeros(m, np.float32),
                           sh=np.zeros((m, K, 3), np.float32), start=z.copy(), expire=z.copy(),
                           birth=z.copy(), frozen=np.zeros(m, np.uint8), sh_degree=sh)

    ref = oracle_mod.slice_decode(oracle_mod.slice_encode(rows, keep), make)
    for d in (dst, dst2):
        for k in FIELDS:
            a = getattr(d, k).cpu().numpy()
            np.testing.assert_array_equal(a[:first], getattr(big, k)[:first], err_msg=k)
            np.testing.assert_array_equal(a[first + n:], getattr(big, k)[first + n:], err_msg=k)
            if k == "opacity_logits":
                np.testing.assert_allclose(a[first:first + n], ref.opacity_logits, rtol=2e-6,
                                           atol=1e-6)
            else:
                np.testing.assert_array_equal(a[first:first + n], getattr(ref, k), err_msg=k)
    r.close()


def test_decode_rejects_bad_packets():
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300._abi import SwgsError
    r = api.Renderer()
    rows = _rows(100)
    pkt = r.slice_encode(api.GaussianState.from_scene(rows), 100, 60)
    dst = api.GaussianState.from_scene(_rows(200))
    with pytest.raises(SwgsError):          # truncated
        r.slice_decode(pkt[:-16], dst, 0)
    with pytest.raises(SwgsError):          # outside the buffer
        r.slice_decode(pkt, dst, 150)
    bad = pkt.clone()
    bad[0] = 0
    with pytest.raises(SwgsError):          # not a packet
        r.slice_decode(bad, dst, 0)
    r.close()
