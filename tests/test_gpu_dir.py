"""Directional (sector) K with translation edge correction (the anisotropic analysis Section 7
lists as future work) on the device against the oracle: counts exact per sector in both
precisions, S and K within the parity bar (relative 1e-9 in FP64, 1e-6 in FP32-guarded), L of
a sector through L + s, envelopes over CSR and permutation simulations, the
translation-corrected K without sectors, waves = one launch, and the argument rules."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9
TOLP = {0: 1e-9, 1: 1e-6}  # by precision: STK_PREC_FP64, STK_PREC_FP32_GUARDED
BOX = (0.0, 2000.0, 0.0, 1500.0, 0.0, 365.0)
S = np.linspace(30.0, 240.0, 7)
TT = np.linspace(4.0, 40.0, 5)


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


def _pattern(n, seed, stretch=True):
    """Clusters stretched along one direction (an anisotropic pattern), plus CSR points and a
    few exact duplicates and axis-aligned offsets (sector boundaries at 0 and pi/2)."""
    from paper_1912_04753_gb300 import workloads as wl

    x, y, t = wl.csr(n, BOX, seed)
    rng = np.random.default_rng(seed + 1)
    k = n // 3
    sx, sy = (40.0, 8.0) if stretch else (20.0, 20.0)
    x = np.clip(np.r_[x, x[:k] + rng.normal(0, sx, k)], BOX[0], BOX[1])
    y = np.clip(np.r_[y, y[:k] + rng.normal(0, sy, k)], BOX[2], BOX[3])
    t = np.clip(np.r_[t, t[:k] + rng.normal(0, 3.0, k)], BOX[4], BOX[5])
    x[:20], y[:20] = x[20:40], y[20:40] + 7.0  # offsets straight along y
    x[40:60], y[40:60] = x[60:80] + 9.0, y[60:80]  # and along x
    x[80:90], y[80:90], t[80:90] = x[90:100], y[90:100], t[90:100]  # duplicates
    return np.clip(x, BOX[0], BOX[1]), np.clip(y, BOX[2], BOX[3]), t


@pytest.mark.parametrize("n_sec", [1, 2, 6])
@pytest.mark.parametrize("edge", [0, 2])
@pytest.mark.parametrize("norm", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_observed_directional_k(stk, orc, n_sec, edge, norm, prec):
    x, y, t = _pattern(3000, 5)
    want = orc.k_function_dir(x, y, t, BOX, S, TT, n_sec, edge_mode=edge, norm=norm)
    with stk.Pattern(x, y, t, BOX) as p:
        got = p.run(S, TT, edge_mode=edge, norm=norm, n_sectors=n_sec, prec=prec)
        assert p.stats()["internal_errors"] == 0
        assert p.stats()["qualifying_pairs"] == want["pairs"]
    if n_sec == 1:
        got = {k: v[None] for k, v in got.items()}
    np.testing.assert_array_equal(got["C"], want["C"])
    assert _rel(got["S"], want["S"]).max() <= TOLP[prec]
    assert _rel(got["K"], want["K"]).max() <= TOLP[prec]
    assert _rel(got["L"] + S[:, None], want["L"] + S[:, None]).max() <= TOLP[prec]


def test_directional_fp32_ties_and_boundaries(stk, orc):
    # dyadic points: many offsets exactly on sector boundaries of 4 sectors (axes and
    # diagonals) and at the thresholds; the FP32 path must leave each of them to FP64
    rng = np.random.default_rng(3)
    box = (0.0, 256.0, 0.0, 256.0, 0.0, 64.0)
    n = 2500
    x = rng.integers(0, 257, n) * 1.0
    y = rng.integers(0, 257, n) * 1.0
    t = rng.integers(0, 65, n) * 1.0
    s, tt = np.array([3.0, 5.0, 8.0, 13.0]), np.array([2.0, 4.0, 9.0])
    for n_sec in (4, 8):
        want = orc.k_function_dir(x, y, t, box, s, tt, n_sec, edge_mode=2)
        with stk.Pattern(x, y, t, box) as p:
            got = p.run(s, tt, edge_mode=2, n_sectors=n_sec, prec=stk.STK_PREC_FP32_GUARDED)
            st = p.stats()
        assert st["internal_errors"] == 0 and st["fp64_recomputed"] > 0
        np.testing.assert_array_equal(got["C"], want["C"])
        assert _rel(got["K"], want["K"]).max() <= 1e-6


def test_translation_k_equals_one_sector(stk, orc):
    # edge_mode TRANSLATION through stk_k (no sectors) is the single-sector estimator
    x, y, t = _pattern(2500, 9, stretch=False)
    want = orc.k_function_dir(x, y, t, BOX, S, TT, 1, edge_mode=2)
    with stk.Pattern(x, y, t, BOX) as p:
        got = p.k(S, TT, edge_mode=stk.STK_EDGE_TRANSLATION)
        got64 = p.k(S, TT, edge_mode=stk.STK_EDGE_TRANSLATION, prec=stk.STK_PREC_FP64)
    np.testing.assert_array_equal(got["C"], want["C"][0])
    assert _rel(got["K"], want["K"][0]).max() <= 1e-6
    np.testing.assert_array_equal(got64["C"], want["C"][0])
    assert _rel(got64["K"], want["K"][0]).max() <= TOL


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_directional_envelope(stk, orc, method, prec):
    x, y, t = _pattern(2000, 13)
    sims, seed, n_sec = 4, 77, 4
    want = orc.envelope_of(method, x, y, t, BOX, S, TT, sims, seed, edge_mode=2, n_sec=n_sec)
    with stk.Pattern(x, y, t, BOX) as p:
        got = p.run(S, TT, n_sims=sims, seed=seed, sim_method=method, want_sims=True,
                    edge_mode=stk.STK_EDGE_TRANSLATION, n_sectors=n_sec, prec=prec)
        assert p.stats()["internal_errors"] == 0
    assert got["K_sims"].shape == (sims, n_sec, len(S), len(TT))
    tol = TOLP[prec]
    for k in range(sims):
        assert _rel(got["K_sims"][k], want["K_all"][k]).max() <= tol, k
    for key in ("K_lo", "K_hi"):
        assert _rel(got[key], want[key]).max() <= tol, key
    for key in ("L_lo", "L_hi"):
        assert _rel(got[key] + S[:, None], want[key] + S[:, None]).max() <= tol, key


def test_directional_waves_equal_one_launch(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    x, y, t = wl.csr(60000, BOX, 3)
    kw = dict(n_sims=6, seed=2, want_sims=True, edge_mode=2, n_sectors=8)  # FP32-guarded
    with stk.Pattern(x, y, t, BOX) as p:
        one = p.run(S, TT, **kw)
        os.environ["STK_MEM_BUDGET_MB"] = "16"
        try:
            waves = p.run(S, TT, **kw)
            assert p.stats()["waves"] > 1
        finally:
            del os.environ["STK_MEM_BUDGET_MB"]
        plain = p.run(S, TT, exec_mode=stk.STK_EXEC_PLAIN, **kw)
    for other in (waves, plain):
        for key in ("C", "K", "C_sims", "K_sims", "K_lo", "K_hi", "L_lo"):
            np.testing.assert_array_equal(other[key], one[key])
    # under CSR each sector holds about 1 / n_sectors of the pairs
    share = one["C_sims"][:, :, -1, -1].sum(axis=0) / one["C_sims"][:, :, -1, -1].sum()
    assert np.abs(share - 1 / 8).max() < 0.01


def test_directional_arguments(stk, orc):
    x, y, t = _pattern(400, 21)
    with stk.Pattern(x, y, t, BOX) as p:
        for kw in (dict(n_sectors=4, edge_mode=stk.STK_EDGE_ISOTROPIC), dict(n_sectors=65),
                   dict(n_sectors=-1),
                   dict(n_sectors=2, edge_mode=2, labels=np.zeros(len(x), np.uint8))):
            with pytest.raises(stk.StkError) as e:
                p.run(S, TT, **kw)
            assert e.value.code == stk.STK_EINVAL, kw
        s10, t10 = np.linspace(20.0, 200.0, 10), np.linspace(2.0, 20.0, 10)
        with pytest.raises(stk.StkError) as e:  # 41 * 10 * 10 > 4096
            p.run(s10, t10, n_sectors=41, edge_mode=2)
        assert e.value.code == stk.STK_EINVAL
        assert p.run(s10, t10, n_sectors=40, edge_mode=2)["C"].shape == (40, 10, 10)
        with pytest.raises(stk.StkError) as e:  # t_max above half the period
            p.run(S, np.array([10.0, 190.0]), edge_mode=2)
        assert e.value.code == stk.STK_EINVAL
        p.set_intensity(np.ones((1, 2, 2)))
        with pytest.raises(stk.StkError) as e:
            p.run(S, TT, n_sectors=2, edge_mode=2)
        assert e.value.code == stk.STK_EINVAL
        p.set_intensity(None)
        ok = p.run(S, TT, n_sectors=2, edge_mode=2)
        assert ok["K"].shape == (2, len(S), len(TT))


def test_served_translation_k(stk, orc):
    # the serving loop takes the translation correction as a job parameter
    x, y, t = _pattern(1500, 17, stretch=False)
    with stk.Server(slots=2) as sv:
        d = sv.register(x, y, t, BOX)
        tk = sv.submit(d, S, TT, edge_mode=stk.STK_EDGE_TRANSLATION)
        iso = sv.submit(d, S, TT)
        got, _ = sv.poll(tk)
        got_iso, _ = sv.poll(iso)
    want = orc.k_function_dir(x, y, t, BOX, S, TT, 1, edge_mode=2)
    np.testing.assert_array_equal(got["C"], want["C"][0])
    assert _rel(got["K"], want["K"][0]).max() <= 1e-6
    # the isotropic job of the same batch is not merged with it
    want_iso = orc.k_function(x, y, t, BOX, S, TT)
    assert _rel(got_iso["K"], want_iso["K"]).max() <= 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_directional_sampled_centres(stk, orc, prec):
    # sampled-centre mode: only the masked centres count, each pair in its sector
    x, y, t = _pattern(6000, 29)
    rng = np.random.default_rng(8)
    mask = (rng.random(len(x)) < 0.05).astype(np.uint8)
    want = orc.k_function_dir(x, y, t, BOX, S, TT, 4, edge_mode=2, centre_mask=mask)
    with stk.Pattern(x, y, t, BOX) as p:
        got = p.run(S, TT, edge_mode=2, n_sectors=4, centre_mask=mask, prec=prec)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], want["C"])
    assert _rel(got["K"], want["K"]).max() <= TOLP[prec]


def test_served_directional_k(stk, orc):
    # sectors through the serving loop: jobs with different n_sectors are not merged
    x, y, t = _pattern(1500, 23, stretch=False)
    with stk.Server(slots=2) as sv:
        d = sv.register(x, y, t, BOX)
        t4 = sv.submit(d, S, TT, edge_mode=2, n_sectors=4, n_sims=2, seed=5)
        t1 = sv.submit(d, S, TT, edge_mode=2, n_sims=2, seed=5)
        g4, _ = sv.poll(t4)
        g1, _ = sv.poll(t1)
    want = orc.k_function_dir(x, y, t, BOX, S, TT, 4, edge_mode=2)
    assert g4["K"].shape == (4, len(S), len(TT)) and g4["K_lo"].shape == (4, len(S), len(TT))
    np.testing.assert_array_equal(g4["C"], want["C"])
    assert _rel(g4["K"], want["K"]).max() <= 1e-6
    np.testing.assert_array_equal(g4["C"].sum(axis=0), g1["C"])
