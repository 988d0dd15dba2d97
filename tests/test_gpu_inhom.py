"""Inhomogeneous K (the variant Section 7 lists as future work) on the device against the
oracle: the intensity-weighted simulation bit for bit, observed grids and envelopes within the
parity bar (counts exact; S and K relative 1e-9 in FP64, 1e-6 in FP32-guarded), the reduction
to Eq. 2 for a constant intensity, sampled centres of the 200,000-point configuration, waves
and CUDA graphs, and the argument rules."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9
TOLP = {0: 1e-9, 1: 1e-6}  # by precision: STK_PREC_FP64, STK_PREC_FP32_GUARDED


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


BOX = (0.0, 2000.0, 0.0, 1500.0, 0.0, 365.0)


def _rho(shape=(4, 5, 6), seed=1, zero=False):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.2, 3.0, shape)
    r[..., 0] *= 4.0  # a strong gradient along x
    if zero:
        r[0, 0, 1] = 0.0
    return r


def _pattern(n, seed, rho=None):
    """Clustered points (a third jittered copies of CSR points), clipped to the box; with rho,
    points in cells with rho = 0 are dropped."""
    from paper_1912_04753_gb300 import workloads as wl

    x, y, t = wl.csr(n, BOX, seed)
    rng = np.random.default_rng(seed + 1)
    k = n // 3
    x = np.clip(np.r_[x, x[:k] + rng.normal(0, 20.0, k)], BOX[0], BOX[1])
    y = np.clip(np.r_[y, y[:k] + rng.normal(0, 20.0, k)], BOX[2], BOX[3])
    t = np.clip(np.r_[t, t[:k] + rng.normal(0, 3.0, k)], BOX[4], BOX[5])
    if rho is not None:
        import oracle

        lam = oracle.intensity_at(x, y, t, BOX, rho)
        keep = lam > 0
        x, y, t = x[keep], y[keep], t[keep]
    return x, y, t


S = np.linspace(30.0, 240.0, 7)
TT = np.linspace(4.0, 40.0, 5)


def test_inhom_simulation_bit_exact(stk, orc):
    for shape, n, seed, sim, zero in (((1, 1, 1), 3000, 5, 2, False), ((4, 5, 6), 1, 0, 0, True),
                                      ((4, 5, 6), 20000, 2**40 + 3, 7, True),
                                      ((3, 64, 64), 50000, 11, 1, False)):
        rho = _rho(shape, seed=n, zero=zero)
        got = stk.stk_sim_points_inhom(BOX, rho, n, seed, sim)
        want = orc.inhom_points(n, BOX, rho, seed, sim)
        for g, w in zip(got, want[:3]):
            np.testing.assert_array_equal(g, w)
    # one cell: exactly the CSR realization
    one = stk.stk_sim_points_inhom(BOX, np.full((1, 1, 1), 3.0), 4000, 9, 4)
    for g, w in zip(one, stk.stk_sim_points(BOX, 4000, 9, 4)):
        np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("edge", [0, 1])
@pytest.mark.parametrize("norm", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_observed_inhom_k(stk, orc, edge, norm, prec):
    rho = _rho(zero=True)
    x, y, t = _pattern(3000, 3, rho)
    lam = orc.intensity_at(x, y, t, BOX, rho)
    want = orc.k_function_inhom(x, y, t, BOX, S, TT, lam, edge_mode=edge, norm=norm)
    with stk.Pattern(x, y, t, BOX) as p:
        p.set_intensity(rho)
        got = p.k(S, TT, edge_mode=edge, norm=norm, prec=prec)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], want["C"])
    assert _rel(got["S"], want["S"]).max() <= TOLP[prec]
    assert _rel(got["K"], want["K"]).max() <= TOLP[prec]
    assert _rel(got["L"] + S[:, None], want["L"] + S[:, None]).max() <= TOLP[prec]


def test_constant_intensity_is_homogeneous(stk, orc):
    x, y, t = _pattern(4000, 8)
    with stk.Pattern(x, y, t, BOX) as p:
        hom = p.k(S, TT, prec=stk.STK_PREC_FP64)
        p.set_intensity(np.full((3, 7, 5), 0.25))
        inh = p.k(S, TT, prec=stk.STK_PREC_FP64)
        inh32 = p.k(S, TT)
        p.set_intensity(None)
        back = p.k(S, TT, prec=stk.STK_PREC_FP64)
    np.testing.assert_array_equal(inh["C"], hom["C"])
    assert _rel(inh["K"], hom["K"]).max() <= 1e-12
    np.testing.assert_array_equal(inh32["C"], hom["C"])
    assert _rel(inh32["K"], hom["K"]).max() <= 1e-6
    for key in ("C", "S", "K"):
        np.testing.assert_array_equal(back[key], hom[key])


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_inhom_envelope(stk, orc, method, prec):
    rho = _rho(seed=4)
    x, y, t = _pattern(2000, 21, rho)
    sims, seed = 4, 123
    want = orc.envelope_of(method, x, y, t, BOX, S, TT, sims, seed, rho=rho)
    with stk.Pattern(x, y, t, BOX) as p:
        p.set_intensity(rho)
        got = p.run(S, TT, n_sims=sims, seed=seed, sim_method=method, want_sims=True,
                    prec=prec)
        assert p.stats()["internal_errors"] == 0
    lam = orc.intensity_at(x, y, t, BOX, rho)
    obs = orc.k_function_inhom(x, y, t, BOX, S, TT, lam)
    tol = TOLP[prec]
    np.testing.assert_array_equal(got["C"], obs["C"])
    assert _rel(got["K"], obs["K"]).max() <= tol
    for k in range(sims):
        assert _rel(got["K_sims"][k], want["K_all"][k]).max() <= tol, k
    for key in ("K_lo", "K_hi"):
        assert _rel(got[key], want[key]).max() <= tol, key
    for key in ("L_lo", "L_hi"):
        assert _rel(got[key] + S[:, None], want[key] + S[:, None]).max() <= tol, key


def test_graph_replay_follows_the_intensity(stk, orc):
    # a small job is replayed from a CUDA graph; a new intensity must not reuse the old one
    x, y, t = _pattern(1500, 31)
    r1, r2 = _rho(seed=5), _rho(seed=6)
    with stk.Pattern(x, y, t, BOX) as p:
        out = []
        for rho in (r1, r1, r2, r1):
            p.set_intensity(rho)
            out.append(p.run(S, TT, n_sims=3, seed=9, want_sims=True))
    for a, rho in zip(out, (r1, r1, r2, r1)):
        want = orc.envelope_of(0, x, y, t, BOX, S, TT, 3, 9, rho=rho)
        for k in range(3):
            assert _rel(a["K_sims"][k], want["K_all"][k]).max() <= 1e-6  # FP32-guarded


def test_waves_equal_one_launch(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    x, y, t = wl.csr(60000, BOX, 77)
    rho = _rho(seed=8)
    with stk.Pattern(x, y, t, BOX) as p:
        p.set_intensity(rho)
        one = p.run(S, TT, n_sims=6, seed=4, want_sims=True)
        os.environ["STK_MEM_BUDGET_MB"] = "16"
        try:
            waves = p.run(S, TT, n_sims=6, seed=4, want_sims=True)
            assert p.stats()["waves"] > 1
        finally:
            del os.environ["STK_MEM_BUDGET_MB"]
        plain = p.run(S, TT, n_sims=6, seed=4, want_sims=True, exec_mode=stk.STK_EXEC_PLAIN)
    for other in (waves, plain):
        for key in ("C", "K", "C_sims", "K_sims", "K_lo", "K_hi"):
            np.testing.assert_array_equal(other[key], one[key])


@pytest.mark.slow
def test_thomas_inhom_sampled_centres(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_inhom()
    rho = w.meta["rho"]
    rng = np.random.default_rng(15)
    mask = np.zeros(w.n, np.uint8)
    mask[rng.choice(w.n, 48, replace=False)] = 1
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        p.set_intensity(rho)
        got = p.run(w.s, w.tt, n_sims=2, seed=w.sim_seed, centre_mask=mask, want_sims=True)
        assert p.stats()["internal_errors"] == 0
        got64 = p.run(w.s, w.tt, centre_mask=mask, prec=stk.STK_PREC_FP64)
    lam = orc.intensity_at(w.x, w.y, w.t, w.box, rho)
    want = orc.k_function_inhom(w.x, w.y, w.t, w.box, w.s, w.tt, lam, centre_mask=mask)
    for g, tol in ((got, 1e-6), (got64, TOL)):
        np.testing.assert_array_equal(g["C"], want["C"])
        assert _rel(g["S"], want["S"]).max() <= tol
        assert _rel(g["K"], want["K"]).max() <= tol
    # the simulations (intensity-weighted, no clustering): properties at any size, and the
    # expectation 2 pi s^2 t, which a 200,000-point realization meets to well under 3 % in
    # the cells with the most pairs
    Cs, Ks = got["C_sims"], got["K_sims"]
    assert (Cs % 2 == 0).all()
    assert (np.diff(Cs, axis=1) >= 0).all() and (np.diff(Cs, axis=2) >= 0).all()
    theory = 2 * np.pi * w.s[:, None] ** 2 * w.tt[None, :]
    big = np.s_[10:, 10:]
    assert (np.abs(Ks[:, 10:, 10:] / theory[big] - 1.0) < 0.03).all()


def test_inhom_arguments(stk, orc):
    rho = _rho(zero=True)
    x, y, t = _pattern(500, 41, rho)
    with stk.Pattern(x, y, t, BOX) as p:
        # a point in a cell with rho = 0
        bad = rho.copy()
        c = orc.intensity_cell(BOX, rho.shape, x[0], y[0], t[0])
        bad.reshape(-1)[c] = 0.0
        with pytest.raises(stk.StkError) as e:
            p.set_intensity(bad)
        assert e.value.code == stk.STK_EDOMAIN
        p.set_intensity(rho)
        with pytest.raises(stk.StkError) as e:  # permutations may land in rho = 0
            p.run(S, TT, n_sims=2, seed=1, sim_method=stk.STK_SIM_PERMUTATION)
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            p.run(S, TT, labels=np.zeros(len(x), np.uint8), cross=(0, 0))
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            p.set_polygon([0.0, 2000.0, 2000.0, 0.0], [0.0, 0.0, 1500.0, 1500.0])
        assert e.value.code == stk.STK_EINVAL
        p.set_intensity(None)
        p.set_polygon([0.0, 2000.0, 2000.0, 0.0], [0.0, 0.0, 1500.0, 1500.0])
        with pytest.raises(stk.StkError) as e:
            p.set_intensity(rho)
        assert e.value.code == stk.STK_EINVAL
