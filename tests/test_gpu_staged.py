"""The filter variant that bulk-copies each row run of the filter arrays into shared memory
(1-D cp.async.bulk, double-buffered chunks on mbarriers; STK_FILTER_STAGED=1) evaluates the same
pairs with the same arithmetic as the default filter, which reads them through the L1 cache:
its grids must equal the default path's bit for bit, and the oracle's at the FP32-guarded bar."""
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


@pytest.mark.parametrize("case", ["csr", "thomas_long_rows"])
def test_staged_filter_equals_default(stk, orc, monkeypatch, case):
    from paper_1912_04753_gb300 import workloads as wl

    if case == "csr":
        w = wl.config_csr_small(seed=12, n=5000)
    else:  # dense clusters: row runs of many chunks
        w = wl.config_thomas(seed=13, n=60_000)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        monkeypatch.delenv("STK_FILTER_STAGED", raising=False)
        ref = p.run(w.s, w.tt, n_sims=3, seed=9, want_sims=True)
        monkeypatch.setenv("STK_FILTER_STAGED", "1")
        got = p.run(w.s, w.tt, n_sims=3, seed=9, want_sims=True)
        assert p.stats()["internal_errors"] == 0
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    if case == "csr":
        want = orc.k_function(w.x, w.y, w.t, w.box, w.s, w.tt)
        np.testing.assert_array_equal(got["C"], want["C"])
        rel = np.abs(got["K"] - want["K"]) / np.where(want["K"] == 0, 1, np.abs(want["K"]))
        assert rel.max() <= 1e-6
