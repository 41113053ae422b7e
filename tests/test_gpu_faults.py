"""Failure detection without faulting the GPU.

- A bounded device wait runs out: a radix-sort tile waits on a look-back word
  that nothing publishes; the wait gives up after about a second, records
  CGA_ERR_TIMEOUT, and the device keeps working afterwards.
- Allocation failure is covered on the host (tests/test_alloc_failure.py)."""
import time

import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_11616_gb300 import build_ext, cga
    build_ext.build()
    cga.load()
    return cga


def test_lookback_wait_times_out_and_device_survives(cg, orc):
    t0 = time.perf_counter()
    observed = cg.selftest_wait_timeout()
    dt = time.perf_counter() - t0
    assert observed == cg.ERR_TIMEOUT
    assert dt < 10.0
    pts = synth.uniform_cube(20_000, seed=130)
    g = cg.grid_from_box([0, 0, 0], 1.0, 10)
    a = cg.cga_build(torch.from_numpy(pts).cuda(), g)
    o = orc.build(pts, orc.grid_from_box([0, 0, 0], 1.0, 10))
    d = a.download()
    assert np.array_equal(d["Z_index"], o.Z_index) and a.status() == cg.OK
