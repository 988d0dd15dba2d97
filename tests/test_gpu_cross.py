"""Bivariate (cross) space-time K on the device against the oracle: exact counts, K within
1e-9 (FP64) / 1e-6 (FP32), for both label orders and a label with itself, and per-realization
grids of CSR and permutation simulations (labels stay with the point index)."""
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


def _two_types(seed):
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(seed)
    box = (0.0, 3000.0, 0.0, 2500.0, 0.0, 200.0)
    x1, y1, t1 = wl.thomas(1800, box, 12, 80.0, 5.0, rng)   # clustered type 1
    x0, y0, t0 = wl.csr(1500, box, seed)                     # background type 0
    lab = np.r_[np.ones(1800, np.uint8), np.zeros(1500, np.uint8)]
    perm = rng.permutation(len(lab))
    x, y, t, lab = np.r_[x1, x0][perm], np.r_[y1, y0][perm], np.r_[t1, t0][perm], lab[perm]
    return x, y, t, lab, box


@pytest.mark.parametrize("ab", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_observed_cross_k(stk, orc, ab, prec):
    x, y, t, lab, box = _two_types(3)
    s, tt = np.linspace(30.0, 240.0, 8), np.linspace(4.0, 24.0, 6)
    want = orc.k_cross(x, y, t, lab, ab[0], ab[1], box, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        got = p.run(s, tt, prec=prec, labels=lab, cross=ab)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], want["C"])
    assert _rel(got["S"], want["S"]).max() <= TOL[prec]
    assert _rel(got["K"], want["K"]).max() <= TOL[prec]


@pytest.mark.parametrize("method", [0, 1])
def test_cross_k_simulations(stk, orc, method):
    x, y, t, lab, box = _two_types(5)
    s, tt = np.linspace(40.0, 200.0, 5), np.linspace(5.0, 25.0, 5)
    sims, seed = 4, 21
    with stk.Pattern(x, y, t, box) as p:
        got = p.run(s, tt, n_sims=sims, seed=seed, sim_method=method, labels=lab, cross=(1, 0),
                    want_sims=True)
        plain = p.run(s, tt, n_sims=sims, seed=seed, sim_method=method, labels=lab,
                      cross=(1, 0), want_sims=True, exec_mode=stk.STK_EXEC_PLAIN)
    Ks = []
    for k in range(sims):
        px, py, pt = orc.simulation_points(method, x, y, t, box, seed, k)
        ref = orc.k_cross(px, py, pt, lab, 1, 0, box, s, tt)
        np.testing.assert_array_equal(got["C_sims"][k], ref["C"])
        assert _rel(got["K_sims"][k], ref["K"]).max() <= TOL[1]
        Ks.append(ref["K"])
    assert _rel(got["K_lo"], np.min(Ks, axis=0)).max() <= TOL[1]
    assert _rel(got["K_hi"], np.max(Ks, axis=0)).max() <= TOL[1]
    for key in got:
        np.testing.assert_array_equal(got[key], plain[key], err_msg=key)


def test_cross_k_arguments(stk):
    x, y, t, lab, box = _two_types(7)
    s, tt = np.array([50.0]), np.array([5.0])
    with stk.Pattern(x, y, t, box) as p:
        for kw in (dict(labels=lab, cross=(1, 0), centre_mask=np.ones(len(x), np.uint8)),
                   dict(labels=lab, cross=(1, 0), n_sims=2, sim_method=stk.STK_SIM_BOOTSTRAP),
                   dict(labels=lab, cross=(1, 7))):
            with pytest.raises(stk.StkError) as e:
                p.run(s, tt, **kw)
            assert e.value.code == stk.STK_EINVAL
        # the handle stays usable
        assert p.run(s, tt)["C"][0, 0] >= 0
