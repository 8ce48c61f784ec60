"""Checkpoint file format (CPU): round trip of every supported dtype and the
scalars, and rejection of files that are not checkpoints or are cut short."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_07759_b300 import checkpoint  # noqa: E402


def test_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    arrays = {"a": torch.from_numpy(rng.normal(size=(7, 3)).astype(np.float32)),
              "b": torch.from_numpy(rng.integers(-5, 5, size=(11,)).astype(np.int32)),
              "c": torch.from_numpy(rng.integers(0, 255, size=(3, 5)).astype(np.uint8)),
              "d": torch.from_numpy(rng.integers(0, 2 ** 40, size=(2,)).astype(np.int64)),
              "empty": torch.zeros((0, 4), dtype=torch.float32)}
    sc = {"head": 3, "step_count": 17, "seed": 5, "name": "x"}
    p = tmp_path / "c.bin"
    checkpoint.save(p, arrays, sc)
    got, gsc = checkpoint.load(p, device="cpu")
    assert gsc == sc
    for k, v in arrays.items():
        assert got[k].dtype == v.dtype and got[k].shape == v.shape
        assert torch.equal(got[k], v)


def test_rejects_bad_files(tmp_path):
    p = tmp_path / "c.bin"
    checkpoint.save(p, {"a": torch.arange(100, dtype=torch.float32)}, {})
    data = p.read_bytes()
    (tmp_path / "bad.bin").write_bytes(b"NOTACKPT" + data[8:])
    with pytest.raises(checkpoint.CheckpointError):
        checkpoint.load(tmp_path / "bad.bin", device="cpu")
    (tmp_path / "cut.bin").write_bytes(data[:-40])
    with pytest.raises(checkpoint.CheckpointError):
        checkpoint.load(tmp_path / "cut.bin", device="cpu")
