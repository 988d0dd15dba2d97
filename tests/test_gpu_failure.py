"""Failure detection without a GPU fault: the FP32 pair kernel's only wait (warps waiting for
the next tile of work units) is bounded.  A test hook makes the warp that should publish a new
tile publish nothing, so every other warp's wait runs out (about 2^20 short sleeps); the kernel
then returns, the job fails with STK_ETIMEOUT, and the same handle computes the next job
correctly."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stk():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1912_04753_gb300 import build as b

    b.build()
    import paper_1912_04753_gb300 as m

    m.load()
    return m


def test_bounded_wait_reports_timeout(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=5, n=3000)
    want = orc.k_function(w.x, w.y, w.t, w.box, w.s, w.tt)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        os.environ["STK_TEST_NEVER_PUBLISH"] = "1"
        try:
            with pytest.raises(stk.StkError) as e:
                p.run(w.s, w.tt, prec=stk.STK_PREC_FP32_GUARDED)
        finally:
            del os.environ["STK_TEST_NEVER_PUBLISH"]
        assert e.value.code == stk.STK_ETIMEOUT
        assert "bounded waits" in str(e.value)
        got = p.run(w.s, w.tt, prec=stk.STK_PREC_FP32_GUARDED)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], want["C"])
    rel = np.abs(got["K"] - want["K"]) / np.where(want["K"] == 0, 1.0, np.abs(want["K"]))
    assert rel.max() <= 1e-6
