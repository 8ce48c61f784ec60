"""Failure paths on the device, made without a fault: a bounded wait that runs
out returns a status the host reads, and the context stays usable."""
import numpy as np
import pytest

from paper_2409_07759_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_sort_lookback_timeout_is_reported():
    """The radix sort's look-back wait on a tile nobody publishes runs out at
    its iteration limit: ETIMEOUT, then the same context renders as before."""
    from paper_2409_07759_b300 import api
    from paper_2409_07759_b300._abi import SwgsError
    sc, views = synth.config0()
    st = api.GaussianState.from_scene(sc)
    r = api.Renderer()
    ref, _ = r.render(st, views)
    ref = [t.clone() for t in ref]
    with pytest.raises(SwgsError) as e:
        r.selftest_sort_timeout()
    assert "ETIMEOUT" in str(e.value)
    img, _ = r.render(st, views)
    for a, b in zip(img, ref):
        assert torch.equal(a, b)
    r.close()
