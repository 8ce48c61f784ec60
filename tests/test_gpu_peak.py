"""The FP32 throughput probe that the blends' roofline is taken against does
the work it claims: every chain ends where the recurrence a <- a*m + c says
(closed form in FP64), in both the scalar and the packed form."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("packed", [0, 1])
def test_fp32_probe_computes_its_chains(packed):
    from paper_2409_07759_b300 import _abi
    lib = _abi.load()
    blocks, iters, threads, chains = 3, 1000, 256, 8
    sink = torch.full((blocks * threads,), float("nan"), dtype=torch.float32, device="cuda")
    fl = C.c_double(0.0)
    st = lib.swgs_fp32_peak_launch(packed, blocks, iters, sink.data_ptr(), C.byref(fl),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert fl.value == blocks * threads * iters * chains * 2 * (2 if packed else 1)
    m, c = np.float64(np.float32(0.9999)), np.float64(np.float32(1e-4))
    mn = m ** iters
    fix = c * (1 - mn) / (1 - m)
    t = np.arange(blocks * threads)
    a0 = np.stack([np.float32(1e-3) * (t & 1023).astype(np.float32) + np.float32(k)
                   for k in range(chains)]).astype(np.float64)
    want = (mn * a0 + fix).sum(0)
    if packed:
        b0 = np.stack([np.float32(k) - np.float32(1e-3) * (t & 511).astype(np.float32)
                       for k in range(chains)]).astype(np.float64)
        want = want + (mn * b0 + fix).sum(0)
    got = sink.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=2e-4, atol=2e-4)


def test_fp32_probe_rejects_bad_arguments():
    from paper_2409_07759_b300 import _abi
    lib = _abi.load()
    fl = C.c_double(0.0)
    sink = torch.empty(256, dtype=torch.float32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.swgs_fp32_peak_launch(2, 1, 10, sink.data_ptr(), C.byref(fl), s) == 1
    assert lib.swgs_fp32_peak_launch(0, 0, 10, sink.data_ptr(), C.byref(fl), s) == 1
    assert lib.swgs_fp32_peak_launch(0, 1, 10, None, C.byref(fl), s) == 1
