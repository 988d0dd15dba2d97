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


def test_resumable_directional_envelope_matches_oracle(stk, tmp_path):
    """A directional K (4 axial sectors, translation correction) run in chunks and resumed:
    the envelope and its L (with the sector factor of Eq. 4's directional form) come from the
    library and match the oracle's envelope at the FP32-guarded bar."""
    import oracle
    from paper_1912_04753_gb300 import checkpoint, workloads as wl

    oracle.build()
    w = wl.config_csr_small(seed=9, n=1200)
    n_sims, seed = 6, 17
    kw = dict(n_sectors=4, edge_mode=stk.STK_EDGE_TRANSLATION,
              prec=stk.STK_PREC_FP32_GUARDED)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        d = str(tmp_path / "ckd")
        assert checkpoint.envelope_resumable(p, w.s, w.tt, n_sims, seed, d, chunk=4,
                                             max_chunks=1, **kw) is None
        got = checkpoint.envelope_resumable(p, w.s, w.tt, n_sims, seed, d, chunk=4, **kw)
        whole = p.run(w.s, w.tt, n_sims=n_sims, seed=seed, **kw)
    ref = oracle.envelope_of(oracle.SIM_CSR, w.x, w.y, w.t, w.box, w.s, w.tt, n_sims, seed,
                             edge_mode=2, n_sec=4)
    s_col = np.asarray(w.s)[None, :, None]
    for k in ("K_lo", "K_hi"):
        r = np.abs(got[k] - ref[k]) / np.where(ref[k] == 0, 1.0, np.abs(ref[k]))
        assert r.max() <= 1e-6, (k, r.max())
        np.testing.assert_array_equal(got[k], whole[k])
    for k in ("L_lo", "L_hi"):
        a, b = got[k] + s_col, ref[k] + s_col  # sqrt(n_sec K / (2 pi t))
        r = np.abs(a - b) / np.where(b == 0, 1.0, np.abs(b))
        assert r.max() <= 1e-6, (k, r.max())
        np.testing.assert_allclose(got[k], whole[k], rtol=1e-14, atol=1e-12)
