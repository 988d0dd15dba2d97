"""Chunked / resumable envelope jobs: realizations first_sim.. of the counter-based generator
are the same whichever chunk computes them, so an interrupted job resumed from its saved
chunks equals the one-shot job bit for bit."""
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


def test_chunks_equal_the_whole_job(stk):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=2, n=3000)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        whole = p.run(w.s, w.tt, n_sims=10, seed=7, want_sims=True)
        part = p.run(w.s, w.tt, n_sims=3, seed=7, first_sim=5, want_sims=True)
    np.testing.assert_array_equal(part["K_sims"], whole["K_sims"][5:8])
    np.testing.assert_array_equal(part["C_sims"], whole["C_sims"][5:8])


@pytest.mark.parametrize("method", [0, 1])
def test_interrupted_job_resumes_exactly(stk, tmp_path, method):
    from paper_1912_04753_gb300 import checkpoint, workloads as wl

    w = wl.config_csr_small(seed=4, n=2500)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        whole = p.run(w.s, w.tt, n_sims=11, seed=3, want_sims=True, sim_method=method)
        d = str(tmp_path / "ck")
        assert checkpoint.envelope_resumable(p, w.s, w.tt, 11, 3, d, chunk=4, max_chunks=1,
                                             sim_method=method) is None  # "interrupted"
        got = checkpoint.envelope_resumable(p, w.s, w.tt, 11, 3, d, chunk=4, sim_method=method)
    for k in ("K", "C", "K_sims", "C_sims", "K_lo", "K_hi"):
        np.testing.assert_array_equal(got[k], whole[k], err_msg=k)
    for k in ("L_lo", "L_hi"):
        np.testing.assert_allclose(got[k], whole[k], rtol=1e-14, atol=1e-12)
