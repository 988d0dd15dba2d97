"""Pins for the oracle's inhomogeneous K (the variant Section 7 lists as future work).

Sources of truth: a hand-worked three-point example, the reduction to Eq. 2 when the intensity
is constant, exact invariance under scaling of the relative intensity, the exact reduction of
the intensity-weighted simulation to the CSR one on a single cell, the cell frequencies of the
simulation, and the expectation E[K_I(s,t)] = 2 pi s^2 t for points drawn independently with
density proportional to the intensity (derivation in the test's docstring).
"""
import math

import numpy as np
import pytest


def _rho_gradient():
    # [nit][niy][nix]: rises 10x along x and 3x along t, a step along y
    ix = np.arange(4)[None, None, :]
    iy = np.arange(2)[None, :, None]
    it = np.arange(3)[:, None, None]
    return (1.0 + 3.0 * ix) * (1.0 + it) * (1.0 + 0.5 * iy)


def test_hand_worked_three_points(orc):
    """Box [0,4]^3, two cells along x with rho = (1, 3), n = 3.

    V = 32 per cell, so sum rho V = 128, lambda_0 = 3/128 and lambda_1 = 9/128.  Only the pair
    of points 0 and 1 (distance 1, same time) is within s = 1.2; both circles lie inside the
    box (w = v = 1).  Sum over both orders: 2 * 128^2 / 27 = 32768 / 27.
    K_I = 3 / (2 * 64) * 32768 / 27 = 256 / 9; with norm 1, 32768 / (27 * 64) = 512 / 27;
    S = (32768 / 27) * (3 / 64)^2 = 8 / 3.
    """
    box = (0.0, 4.0, 0.0, 4.0, 0.0, 4.0)
    rho = np.array([1.0, 3.0]).reshape(1, 1, 2)
    x = np.array([1.5, 2.5, 1.5])
    y = np.array([2.0, 2.0, 3.5])
    t = np.array([2.0, 2.0, 2.0])
    lam = orc.intensity_at(x, y, t, box, rho)
    assert list(lam) == [3 / 128, 9 / 128, 3 / 128]
    s, tt = np.array([1.2]), np.array([1.0])
    for edge in (0, 1):
        r = orc.k_function_inhom(x, y, t, box, s, tt, lam, edge_mode=edge)
        assert r["C"][0, 0] == 2 and r["pairs"] == 2
        assert r["K"][0, 0] == pytest.approx(256 / 9, rel=1e-14)
        assert r["S"][0, 0] == pytest.approx(8 / 3, rel=1e-14)
        r1 = orc.k_function_inhom(x, y, t, box, s, tt, lam, edge_mode=edge, norm=1)
        assert r1["K"][0, 0] == pytest.approx(512 / 27, rel=1e-14)


def test_constant_intensity_is_eq2(orc):
    """rho constant on any grid: lambda = n / (A D) and K_I is the estimator of Eq. 2."""
    box = (0.0, 800.0, 0.0, 600.0, 0.0, 365.0)
    x, y, t = orc.csr_points(700, box, seed=5, sim=0)
    s = np.linspace(20.0, 150.0, 6)
    tt = np.linspace(5.0, 60.0, 5)
    rho = np.full((3, 5, 4), 2.5)
    lam = orc.intensity_at(x, y, t, box, rho)
    np.testing.assert_allclose(lam, 700 / (800 * 600 * 365), rtol=1e-14)
    for norm in (0, 1):
        for edge in (0, 1):
            a = orc.k_function_inhom(x, y, t, box, s, tt, lam, edge_mode=edge, norm=norm)
            b = orc.k_function(x, y, t, box, s, tt, edge_mode=edge, norm=norm)
            np.testing.assert_array_equal(a["C"], b["C"])
            np.testing.assert_allclose(a["K"], b["K"], rtol=1e-12)
            np.testing.assert_allclose(a["S"], b["S"], rtol=1e-12)
            np.testing.assert_allclose(a["L"] + s[:, None], b["L"] + s[:, None], rtol=1e-12)


def test_intensity_is_relative(orc):
    """Scaling rho by a power of two changes no bit of lambda (every step scales exactly)."""
    box = (0.0, 10.0, 0.0, 10.0, 0.0, 10.0)
    rho = _rho_gradient()
    for k in (-7, 3, 20):
        np.testing.assert_array_equal(orc.intensity_lambda(rho * 2.0**k, box, 321),
                                      orc.intensity_lambda(rho, box, 321))
    # and lambda integrates to n
    lam = orc.intensity_lambda(rho, box, 321)
    assert lam.sum() * 1000.0 / rho.size == pytest.approx(321, rel=1e-14)


def test_cell_lookup_edges(orc):
    box = (0.0, 4.0, -2.0, 2.0, 10.0, 14.0)
    shape = (2, 4, 4)  # nit, niy, nix
    assert orc.intensity_cell(box, shape, 0.0, -2.0, 10.0) == 0
    assert orc.intensity_cell(box, shape, 4.0, 2.0, 14.0) == 2 * 16 - 1  # closed upper faces
    assert orc.intensity_cell(box, shape, 1.0, -2.0, 10.0) == 1  # on an inner face: upper cell
    assert orc.intensity_cell(box, shape, np.nextafter(1.0, 0.0), -2.0, 10.0) == 0
    assert orc.intensity_cell(box, shape, 0.0, 0.0, 12.0) == (1 * 4 + 2) * 4


def test_single_cell_simulation_is_csr(orc):
    """With one intensity cell the intensity-weighted simulation is the CSR one, bit for bit."""
    box = (-3.0, 17.0, 1.0, 2.0, 0.0, 365.0)
    x, y, t, cell = orc.inhom_points(5000, box, np.full((1, 1, 1), 7.0), seed=99, sim=4)
    cx, cy, ctm = orc.csr_points(5000, box, seed=99, sim=4)
    np.testing.assert_array_equal(x, cx)
    np.testing.assert_array_equal(y, cy)
    np.testing.assert_array_equal(t, ctm)
    assert (cell == 0).all()


def test_simulation_follows_rho(orc):
    """Cell frequencies match rho / sum rho (5 binomial standard errors), cells with rho = 0
    get no point, and every point lies in the cell it was drawn in."""
    box = (0.0, 4.0, 0.0, 2.0, 0.0, 3.0)
    rho = _rho_gradient()
    rho[1, 0, 2] = 0.0
    n = 200_000
    x, y, t, cell = orc.inhom_points(n, box, rho, seed=7, sim=1)
    assert x.min() >= 0 and x.max() <= 4 and y.min() >= 0 and y.max() <= 2
    assert t.min() >= 0 and t.max() <= 3
    counts = np.bincount(cell, minlength=rho.size)
    p = rho.reshape(-1) / rho.sum()
    se = np.sqrt(n * p * (1 - p))
    assert np.all(np.abs(counts - n * p) <= 5 * se + 1e-9)
    assert counts[(1 * 2 + 0) * 4 + 2] == 0
    # the point lies in its cell: the lookup agrees (points on an inner face have probability
    # ~2^-50 per point)
    sub = slice(0, 3000)
    look = [orc.intensity_cell(box, rho.shape, a, b, c) for a, b, c in zip(x[sub], y[sub], t[sub])]
    np.testing.assert_array_equal(look, cell[sub])


def test_inhomogeneous_expectation_2pi_s2_t(orc):
    """E[K_I(s,t)] = 2 pi s^2 t for n points drawn independently with density f = rho / int rho.

    E sum_{i != j} g(p_i, p_j) = n(n-1) int int f(p) f(q) g(p, q).  With
    g = I w / (lambda(p) lambda(q)) and lambda = n f this is (n-1)/n int int I(p, q) w(p, q),
    the same integral as under CSR (A D 2 pi s^2 t, rho > 0 everywhere), so the factor
    n / ((n-1) A D) leaves 2 pi s^2 t.  The sample is drawn here with numpy (cell by rho, then
    uniform in the cell), independently of the oracle's own simulation.  The homogeneous
    estimator on the same sample, or intensities attached to the wrong points, miss by many
    standard errors (checked below), so the test has the power to see a wrong weight.
    """
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    rho = _rho_gradient()
    nit, niy, nix = rho.shape
    p = rho.reshape(-1) / rho.sum()
    lam_cell = orc.intensity_lambda(rho, box, 500)
    s = np.array([0.05, 0.1, 0.2, 0.25])
    tt = np.array([0.05, 0.15, 0.3, 0.5])
    n, R = 500, 300
    KI, KH, K1 = [], [], []
    for r in range(R):
        rng = np.random.default_rng(5000 + r)
        c = rng.choice(rho.size, size=n, p=p)
        ix, iy, it = c % nix, (c // nix) % niy, c // (nix * niy)
        x = (ix + rng.random(n)) / nix
        y = (iy + rng.random(n)) / niy
        t = (it + rng.random(n)) / nit
        lam = lam_cell[c]
        KI.append(orc.k_function_inhom(x, y, t, box, s, tt, lam)["K"])
        if r < 60:
            KH.append(orc.k_function(x, y, t, box, s, tt)["K"])
            # intensities attached to the wrong points (an index mistake)
            K1.append(orc.k_function_inhom(x, y, t, box, s, tt, rng.permutation(lam))["K"])
    theory = 2 * math.pi * s[:, None] ** 2 * tt[None, :]
    KI = np.array(KI)
    z = (KI.mean(axis=0) - theory) / (KI.std(axis=0, ddof=1) / math.sqrt(R))
    assert np.abs(z).max() < 4.0, z
    for bad in (np.array(KH), np.array(K1)):
        zb = (bad.mean(axis=0) - theory) / (bad.std(axis=0, ddof=1) / math.sqrt(len(bad)))
        assert np.abs(zb).max() > 10.0
