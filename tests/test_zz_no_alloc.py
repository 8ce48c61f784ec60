"""The allocation-free compaction entry point (swgs_active_ids_noalloc),
checked through the C ABI against the context-based swgs_active_ids.

It exists for callers that cannot let a library allocate device memory (their
memory belongs to one allocator or budget, or their threads cannot take
cudaMalloc's device-wide synchronisation). This file is collected last so that
a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lifespans(n, seed):
    rng = np.random.default_rng(seed)
    start = rng.integers(0, 300, n).astype(np.int32)
    expire = (start + rng.integers(10, 61, n)).astype(np.int32)
    return torch.from_numpy(start).cuda(), torch.from_numpy(expire).cuda()


def _ids_with_context(lib, ctx, start, expire, frame):
    n = start.numel()
    ids = torch.full((max(1, n),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = lib.swgs_active_ids(ctx, start.data_ptr(), expire.data_ptr(), n, frame, ids.data_ptr(),
                             cnt.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return ids, cnt


def _ids_noalloc(lib, start, expire, frame):
    n = start.numel()
    ids = torch.full((max(1, n),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = lib.swgs_active_ids_noalloc(start.data_ptr(), expire.data_ptr(), n, frame,
                                     ids.data_ptr(), cnt.data_ptr(),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return ids, cnt


def test_noalloc_matches_context_entry_point_twice():
    """Two calls in a row (different sizes and frames, the second smaller so
    that stale scratch from the first would show) give exactly the ids and
    count of swgs_active_ids."""
    from paper_2409_07759_b300 import _abi
    lib = _abi.load()
    ctx = C.c_void_p()
    assert lib.swgs_create(None, _abi.ALLOC_FN(), _abi.FREE_FN(), None, C.byref(ctx)) == 0
    try:
        for n, frame, seed in ((300_000, 150, 1), (70_001, 41, 2)):
            start, expire = _lifespans(n, seed)
            ids_a, cnt_a = _ids_with_context(lib, ctx, start, expire, frame)
            ids_b, cnt_b = _ids_noalloc(lib, start, expire, frame)
            torch.cuda.synchronize()
            k = int(cnt_a.item())
            assert k > 0 and int(cnt_b.item()) == k
            assert torch.equal(ids_a[:k], ids_b[:k])
    finally:
        lib.swgs_destroy(ctx)


def test_noalloc_rejects_oversize_and_handles_empty():
    from paper_2409_07759_b300 import _abi
    lib = _abi.load()
    start, expire = _lifespans(16, 3)
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    ids = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.swgs_active_ids_noalloc(start.data_ptr(), expire.data_ptr(),
                                       _abi.NOALLOC_MAX_SLOTS + 1, 0, ids.data_ptr(),
                                       cnt.data_ptr(), s) == _abi.SWGS_EINVAL
    assert lib.swgs_active_ids_noalloc(start.data_ptr(), expire.data_ptr(), 0, 0, ids.data_ptr(),
                                       cnt.data_ptr(), s) == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
