"""Parity at the benchmark's full size and launch configuration (n = 2,000,000 POI mixture,
observed pattern + 99 CSR simulations in one batched job, FP32-guarded path).

The O(n^2) oracle cannot evaluate the whole job, so the check is split:
  * sampled outputs: the observed grids restricted to 96 random centres (sampled-centre mode,
    same launch as the benchmark) against the oracle on the same centres x all 2M points;
  * simulations: every realization's counts and sums must satisfy properties that hold at any
    size (monotone cumulative counts, S >= C, S <= 8 C, even counts: each unordered pair adds
    both orders), and three realizations must match the FP64 GPU path (counts exact, K within
    1e-6).
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.where(b == 0, 1.0, np.abs(b))


def test_full_size_job_sampled_centres_and_simulations(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_poi()
    rng = np.random.default_rng(77)
    mask = np.zeros(w.n, np.uint8)
    mask[rng.choice(w.n, 96, replace=False)] = 1
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        got = p.run(w.s, w.tt, n_sims=w.n_sims, seed=w.sim_seed, centre_mask=mask,
                    prec=stk.STK_PREC_FP32_GUARDED, want_sims=True)
        st = p.stats()
        assert st["internal_errors"] == 0
        ref = p.run(w.s, w.tt, n_sims=3, seed=w.sim_seed, prec=stk.STK_PREC_FP64,
                    exec_mode=stk.STK_EXEC_PLAIN, want_sims=True)
    cnt, wsum, _ = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=mask)
    C, S, K, L = orc.finalize(w.n, w.box, w.s, w.tt, cnt, wsum)
    np.testing.assert_array_equal(got["C"], C)
    assert _rel(got["S"], S).max() <= 1e-6
    assert _rel(got["K"], K).max() <= 1e-6
    Cs, Ks = got["C_sims"], got["K_sims"]
    assert (np.diff(Cs, axis=1) >= 0).all() and (np.diff(Cs, axis=2) >= 0).all()
    assert (Cs % 2 == 0).all()
    coef = (w.box[1] - w.box[0]) * (w.box[3] - w.box[2]) * (w.box[5] - w.box[4]) / (
        float(w.n) * (w.n - 1))
    Ss = Ks / coef
    assert (Ss >= Cs * (1 - 1e-9)).all() and (Ss <= 8 * Cs * (1 + 1e-9)).all()
    np.testing.assert_array_equal(Cs[:3], ref["C_sims"])
    assert _rel(Ks[:3], ref["K_sims"]).max() <= 1e-6
    # envelope = element-wise min / max of the realizations
    np.testing.assert_array_equal(got["K_lo"], Ks.min(axis=0))
    np.testing.assert_array_equal(got["K_hi"], Ks.max(axis=0))


def test_thomas_config_batched_fp64_equals_plain(stk, orc):
    # the Thomas configuration (n = 200,000, 99 simulations, FP64): one batched launch and one
    # launch per realization give the same grids bit for bit; sampled observed centres match
    # the oracle
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_thomas()
    rng = np.random.default_rng(5)
    mask = np.zeros(w.n, np.uint8)
    mask[rng.choice(w.n, 64, replace=False)] = 1
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        b = p.run(w.s, w.tt, n_sims=w.n_sims, seed=w.sim_seed, prec=stk.STK_PREC_FP64,
                  want_sims=True)
        q = p.run(w.s, w.tt, n_sims=w.n_sims, seed=w.sim_seed, prec=stk.STK_PREC_FP64,
                  exec_mode=stk.STK_EXEC_PLAIN, want_sims=True)
        m = p.run(w.s, w.tt, prec=stk.STK_PREC_FP64, centre_mask=mask)
        assert p.stats()["internal_errors"] == 0
    for k in b:
        np.testing.assert_array_equal(b[k], q[k], err_msg=k)
    cnt, wsum, _ = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=mask)
    C, S, K, L = orc.finalize(w.n, w.box, w.s, w.tt, cnt, wsum)
    np.testing.assert_array_equal(m["C"], C)
    assert _rel(m["K"], K).max() <= 1e-9


def test_large_config_in_waves(stk, orc):
    # n = 10^7 and 199 simulations do not fit at once: the job runs in waves; sampled observed
    # centres match the oracle and every realization satisfies the invariants
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_large()
    rng = np.random.default_rng(9)
    mask = np.zeros(w.n, np.uint8)
    mask[rng.choice(w.n, 48, replace=False)] = 1
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        got = p.run(w.s, w.tt, n_sims=w.n_sims, seed=w.sim_seed, centre_mask=mask,
                    want_sims=True)
        st = p.stats()
    assert st["internal_errors"] == 0 and st["realizations"] == 200
    assert st["waves"] >= 2
    cnt, wsum, _ = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=mask)
    C, S, K, L = orc.finalize(w.n, w.box, w.s, w.tt, cnt, wsum)
    np.testing.assert_array_equal(got["C"], C)
    assert _rel(got["K"], K).max() <= 1e-6
    Cs, Ks = got["C_sims"], got["K_sims"]
    assert (np.diff(Cs, axis=1) >= 0).all() and (np.diff(Cs, axis=2) >= 0).all()
    assert (Cs % 2 == 0).all()
    np.testing.assert_array_equal(got["K_lo"], Ks.min(axis=0))
    np.testing.assert_array_equal(got["K_hi"], Ks.max(axis=0))


def test_full_observed_grids_against_grid_oracle(stk, orc):
    # whole observed grids at full size: the benchmark's own job (2M points, observed + 99
    # simulations in one batched FP32-guarded launch) and the Thomas configuration in FP64,
    # against the grid-accelerated restatement of the oracle (all host cores)
    from paper_1912_04753_gb300 import workloads as wl

    for name, prec, tol, sims in (("thomas_n200k", stk.STK_PREC_FP64, 1e-9, 2),
                                  ("poi_n2M", stk.STK_PREC_FP32_GUARDED, 1e-6, 99)):
        w = wl.CONFIGS[name]()
        with stk.Pattern(w.x, w.y, w.t, w.box) as p:
            got = p.run(w.s, w.tt, n_sims=sims, seed=w.sim_seed, prec=prec)
            assert p.stats()["internal_errors"] == 0
        cnt, wsum, q = orc.pair_hist_grid(w.x, w.y, w.t, w.box, w.s, w.tt)
        C, S, K, L = orc.finalize(w.n, w.box, w.s, w.tt, cnt, wsum)
        assert q == C[-1, -1]
        np.testing.assert_array_equal(got["C"], C)
        assert _rel(got["S"], S).max() <= tol, name
        assert _rel(got["K"], K).max() <= tol, name
        assert _rel(got["L"] + w.s[:, None], L + w.s[:, None]).max() <= tol, name
