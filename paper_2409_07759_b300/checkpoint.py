"""Checkpoint / resume of a training run as one flat binary file.

Layout: the 8-byte magic ``SWGSCKPT``, a little-endian uint32 format version, a
uint32 header length, a JSON header (name, dtype and shape of every array and
the scalars), then the arrays' raw bytes in header order, each starting on a
16-byte boundary. Nothing else is stored: the random draws of the SGLD noise
and of relocation come from Philox streams keyed by the seed with the slot
and step as counter, so a run resumed from the saved step draws exactly what
an uninterrupted run would have.
"""
from __future__ import annotations

import json
import struct
from pathlib import Path
from typing import Dict, Tuple

import numpy as np
import torch

MAGIC = b"SWGSCKPT"
VERSION = 1
_DTYPES = {torch.float32: "f4", torch.int32: "i4", torch.uint8: "u1", torch.int64: "i8"}
_TORCH = {v: k for k, v in _DTYPES.items()}


class CheckpointError(ValueError):
    pass


def save(path, arrays: Dict[str, torch.Tensor], scalars: Dict) -> None:
    """Write `arrays` (any device; copied to the host) and JSON-able `scalars`."""
    names = list(arrays)
    host = {}
    entries = []
    for n in names:
        t = arrays[n].detach()
        if t.dtype not in _DTYPES:
            raise CheckpointError(f"array {n}: unsupported dtype {t.dtype}")
        host[n] = t.contiguous().cpu().numpy()
        entries.append({"name": n, "dtype": _DTYPES[t.dtype], "shape": list(t.shape)})
    header = json.dumps({"arrays": entries, "scalars": scalars}).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<II", VERSION, len(header)))
        f.write(header)
        for n in names:
            pad = (-f.tell()) % 16
            f.write(b"\0" * pad)
            f.write(host[n].tobytes())


def load(path, device: str = "cuda") -> Tuple[Dict[str, torch.Tensor], Dict]:
    """Read a checkpoint; arrays are placed on `device`."""
    data = Path(path).read_bytes()
    if len(data) < 16 or data[:8] != MAGIC:
        raise CheckpointError("not a checkpoint file")
    version, hlen = struct.unpack("<II", data[8:16])
    if version != VERSION:
        raise CheckpointError(f"checkpoint format {version}, expected {VERSION}")
    if 16 + hlen > len(data):
        raise CheckpointError("truncated header")
    header = json.loads(data[16:16 + hlen])
    off = 16 + hlen
    out = {}
    for e in header["arrays"]:
        off += (-off) % 16
        dt = np.dtype(e["dtype"]).newbyteorder("<")
        n = int(np.prod(e["shape"])) if e["shape"] else 1
        end = off + n * dt.itemsize
        if end > len(data):
            raise CheckpointError(f"truncated array {e['name']}")
        a = np.frombuffer(data, dt, n, off).reshape(e["shape"]).copy()
        out[e["name"]] = torch.from_numpy(a).to(device)
        off = end
    return out, header["scalars"]
