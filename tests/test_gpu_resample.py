"""Bootstrapping and random-permutation simulations (Section 3) on the device: realizations
bit-identical to the oracle's, and their K grids and envelopes within the parity bar (counts
exact; K relative 1e-9 in FP64, 1e-6 in FP32-guarded)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-9, 1: 1e-6}


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


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 4097, 300000])
def test_device_resampling_bit_exact(stk, orc, n):
    rng = np.random.default_rng(n)
    x, y, t = rng.uniform(0, 1e4, n), rng.uniform(-5e3, 5e3, n), np.floor(rng.uniform(0, 3e7, n))
    for seed, sim in ((0, 0), (2**40 + 9, 3), (77, 1234)):
        got = stk.stk_sim_resample(x, y, t, stk.STK_SIM_PERMUTATION, seed, sim)
        want = orc.permutation_points(x, y, t, seed, sim)
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)
        got = stk.stk_sim_resample(x, y, t, stk.STK_SIM_BOOTSTRAP, seed, sim)
        want = orc.bootstrap_points(x, y, t, seed, sim)
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_resampling_envelopes_match_oracle(stk, orc, method, prec):
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(40 + method)
    box = (0.0, 3000.0, 0.0, 2500.0, 0.0, 200.0)
    x, y, t = wl.thomas(2500, box, 15, 90.0, 6.0, rng)
    s, tt = wl.even_thresholds(240.0, 8), wl.even_thresholds(16.0, 6)
    sims, seed = 7, 91
    want = orc.envelope_of(method, x, y, t, box, s, tt, sims, seed)
    with stk.Pattern(x, y, t, box) as p:
        got = p.run(s, tt, n_sims=sims, seed=seed, prec=prec, sim_method=method,
                    want_sims=True)
        assert p.stats()["internal_errors"] == 0
        plain = p.run(s, tt, n_sims=sims, seed=seed, prec=prec, sim_method=method,
                      exec_mode=stk.STK_EXEC_PLAIN, want_sims=True)
    for k in range(sims):
        px, py, pt = orc.simulation_points(method, x, y, t, box, seed, k)
        ref = orc.k_function(px, py, pt, box, s, tt)
        np.testing.assert_array_equal(got["C_sims"][k], ref["C"])
        assert _rel(got["K_sims"][k], want["K_all"][k]).max() <= TOL[prec]
    for key in ("K_lo", "K_hi"):
        assert _rel(got[key], want[key]).max() <= TOL[prec]
    for key in got:  # batched and plain execution agree bit for bit
        np.testing.assert_array_equal(got[key], plain[key], err_msg=key)


def test_served_resampling_jobs_equal_alone(stk):
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(12)
    box = (0.0, 5000.0, 0.0, 5000.0, 0.0, 365.0)
    x, y, t = wl.thomas(30000, box, 60, 120.0, 8.0, rng)
    s, tt = wl.even_thresholds(300.0, 10), wl.even_thresholds(20.0, 7)
    jobs = [(stk.STK_SIM_PERMUTATION, 9, 1), (stk.STK_SIM_PERMUTATION, 4, 2),
            (stk.STK_SIM_BOOTSTRAP, 6, 3), (stk.STK_SIM_CSR, 5, 4)]
    with stk.Server(slots=2) as sv:
        d = sv.register(x, y, t, box)
        tks = [sv.submit(d, s, tt, n_sims=ns, seed=sd, sim_method=m, want_sims=True)
               for m, ns, sd in jobs]
        served = [sv.poll(tk)[0] for tk in tks]
    with stk.Pattern(x, y, t, box) as p:
        for (m, ns, sd), got in zip(jobs, served):
            alone = p.run(s, tt, n_sims=ns, seed=sd, sim_method=m, want_sims=True)
            for key in alone:
                np.testing.assert_array_equal(got[key], alone[key], err_msg=key)
