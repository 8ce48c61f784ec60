"""The C-ABI library loads and exports every entry point include/swgs.h
declares (no GPU needed: nothing is called)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "swgs.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swgs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2409_07759_b300 import build, _abi
    build.build()
    lib = ctypes.CDLL(str(_abi.LIB_PATH))
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    bound = {p[0] for p in _abi.PROTOTYPES}
    assert set(names) <= bound, set(names) - bound


def test_slice_range_host_logic():
    """Alg. 2 slice arithmetic (host-only entry point)."""
    from paper_2409_07759_b300 import build, _abi
    build.build()
    L = _abi.load()
    first, count = ctypes.c_int64(), ctypes.c_int64()
    assert L.swgs_slice_range(123, 50, 300000, ctypes.byref(first), ctypes.byref(count)) == 0
    assert (first.value, count.value) == (23 * 6000, 6000)
    assert L.swgs_slice_range(1, 0, 10, ctypes.byref(first), ctypes.byref(count)) == 1
    assert L.swgs_slice_range(1, 3, 10, ctypes.byref(first), ctypes.byref(count)) == 1
