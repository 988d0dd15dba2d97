"""Pins for the oracle's directional (sector) K with translation edge correction, the
anisotropic analysis Section 7 lists as future work.

Sources of truth: sector assignment of hand-chosen offsets, the translation weight against
Monte Carlo overlap of the shifted window, the reduction to the oracle's Eq. 2 estimator for
one sector without edge correction, the exact partition of the pairs over sectors, exact
rotation symmetry on a square box, and the CSR expectation 2 pi s^2 t / n_sec of every sector
(derivation in the test's docstring).
"""
import math

import numpy as np
import pytest


def test_sector_of_hand_offsets(orc):
    deg = math.pi / 180
    for ang, n_sec, want in ((10, 4, 0), (80, 4, 1), (100, 4, 2), (170, 4, 3), (-10, 4, 3),
                             (190, 4, 0), (260, 4, 1), (44, 4, 0), (46, 4, 1), (91, 2, 1),
                             (89, 2, 0), (179, 8, 7), (23, 8, 1), (0, 6, 0), (180, 6, 0)):
        dx, dy = 3.0 * math.cos(ang * deg), 3.0 * math.sin(ang * deg)
        if ang in (0, 180):
            dx, dy = (3.0, 0.0) if ang == 0 else (-3.0, 0.0)
        assert orc.sector(dx, dy, n_sec) == want, (ang, n_sec)
        assert orc.sector(-dx, -dy, n_sec) == want  # both orders of a pair
    assert orc.sector(0.0, 0.0, 5) == 0
    assert all(orc.sector(1.0, 2.0, 1) == 0 for _ in range(3))


def test_translation_weight_is_inverse_overlap(orc):
    """W H / ((W - |dx|)(H - |dy|)) is |A| over the area of A intersected with A shifted by
    (dx, dy): checked by sampling the window; and the temporal factor D / (D - u)."""
    box = (0.0, 100.0, 0.0, 60.0, 0.0, 10.0)
    rng = np.random.default_rng(3)
    p = rng.uniform((0, 0), (100, 60), (400_000, 2))
    for dx, dy in ((20.0, 0.0), (-35.0, 12.5), (5.0, -29.0), (0.0, 0.0)):
        q = p + (dx, dy)
        frac = np.mean((q[:, 0] >= 0) & (q[:, 0] <= 100) & (q[:, 1] >= 0) & (q[:, 1] <= 60))
        w = orc.translation_weight(dx, dy, 0.0, box)
        assert abs(1.0 / w - frac) < 5 * math.sqrt(frac * (1 - frac) / len(p)) + 1e-12
    assert orc.translation_weight(0.0, 0.0, 4.0, box) == pytest.approx(10.0 / 6.0, rel=1e-15)
    assert orc.translation_weight(50.0, 30.0, 5.0, box) == pytest.approx(8.0, rel=1e-15)


def test_one_sector_no_correction_is_eq2(orc):
    box = (0.0, 500.0, 0.0, 400.0, 0.0, 100.0)
    x, y, t = orc.csr_points(600, box, seed=2, sim=0)
    s, tt = np.linspace(10, 120, 5), np.linspace(2, 30, 4)
    a = orc.k_function_dir(x, y, t, box, s, tt, 1, edge_mode=0)
    b = orc.k_function(x, y, t, box, s, tt, edge_mode=0)
    for key in ("C", "S", "K"):
        np.testing.assert_array_equal(a[key][0], b[key])
    np.testing.assert_allclose(a["L"][0], b["L"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n_sec", [2, 3, 8])
def test_sectors_partition_the_pairs(orc, n_sec):
    box = (0.0, 500.0, 0.0, 400.0, 0.0, 100.0)
    x, y, t = orc.csr_points(700, box, seed=4, sim=1)
    x[:50] = x[50:100]  # some coincident spatial positions
    y[:50] = y[50:100]
    s, tt = np.linspace(10, 150, 6), np.linspace(2, 40, 5)
    whole = orc.k_function_dir(x, y, t, box, s, tt, 1)
    parts = orc.k_function_dir(x, y, t, box, s, tt, n_sec)
    np.testing.assert_array_equal(parts["C"].sum(axis=0), whole["C"][0])
    np.testing.assert_allclose(parts["S"].sum(axis=0), whole["S"][0], rtol=1e-13)
    assert parts["pairs"] == whole["pairs"]


def test_rotation_maps_sectors(orc):
    """Rotating a square box by 90 degrees, (x, y) -> (L - y, x) (exact on dyadic points),
    moves an axis in sector k to sector k + n_sec / 2 (mod n_sec); the translation weight is
    unchanged, so counts map exactly and sums to rounding."""
    Lside = 1024.0
    box = (0.0, Lside, 0.0, Lside, 0.0, 64.0)
    rng = np.random.default_rng(9)
    x = rng.integers(0, 2**20, 900) * (Lside / 2**20)
    y = rng.integers(0, 2**20, 900) * (Lside / 2**20)
    t = rng.integers(0, 2**16, 900) * (64.0 / 2**16)
    s, tt = np.array([40.0, 90.0, 160.0]), np.array([4.0, 12.0])
    for n_sec in (4, 6):
        a = orc.k_function_dir(x, y, t, box, s, tt, n_sec)
        b = orc.k_function_dir(Lside - y, x, t, box, s, tt, n_sec)
        rolled_c = np.roll(a["C"], n_sec // 2, axis=0)
        np.testing.assert_array_equal(b["C"], rolled_c)
        np.testing.assert_allclose(b["S"], np.roll(a["S"], n_sec // 2, axis=0), rtol=1e-13)


def test_csr_expectation_per_sector(orc):
    """E[K_k(s, t)] = 2 pi s^2 t / n_sec under CSR in every sector.

    For the translation weight e(h) = |A| / |A intersected with A_h| (and D / (D - u) in time),
    E sum_{i != j} g(p_j - p_i) e(p_j - p_i) = n(n-1) / (A D)^2 * integral of g(h) e(h) times
    the measure of {p : p in A, p + h in A} = n(n-1) / (A D) * integral of g over offsets.  The
    offsets of sector k within distance s and lag t form two opposite circular sectors of angle
    pi / n_sec and radius s, times [-t, t]: area (pi / n_sec) s^2 times 2t.  Without the
    correction the mean misses by many standard errors (checked), so the test sees the weight."""
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    s = np.array([0.1, 0.2, 0.3])
    tt = np.array([0.1, 0.3, 0.5])
    n, R, n_sec = 400, 300, 4
    Ks, K0 = [], []
    for r in range(R):
        rng = np.random.default_rng(7000 + r)
        x, y, t = rng.random(n), rng.random(n), rng.random(n)
        Ks.append(orc.k_function_dir(x, y, t, box, s, tt, n_sec)["K"])
        if r < 80:
            K0.append(orc.k_function_dir(x, y, t, box, s, tt, n_sec, edge_mode=0)["K"])
    Ks = np.array(Ks)
    theory = 2 * math.pi * s[:, None] ** 2 * tt[None, :] / n_sec
    z = (Ks.mean(axis=0) - theory) / (Ks.std(axis=0, ddof=1) / math.sqrt(R))
    assert np.abs(z).max() < 4.0, z
    K0 = np.array(K0)
    z0 = (K0.mean(axis=0) - theory) / (K0.std(axis=0, ddof=1) / math.sqrt(len(K0)))
    assert np.abs(z0).max() > 10.0
