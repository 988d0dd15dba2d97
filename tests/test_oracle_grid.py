"""The grid-accelerated, multithreaded restatement of the oracle's pair histogram must give
the brute-force oracle's histograms on every input: identical counts and qualifying totals,
sums equal to rounding (1e-12).  Inputs: the small CSR configuration, clusters hugging the edges
and the start of the period, dyadic points with exact ties at the thresholds, points on the
box's faces, coincident points, thresholds as large as allowed (one cell) and tiny (many
cells), a centre mask, both edge modes, 1 to 8 threads."""
import numpy as np
import pytest


def _check(orc, x, y, t, box, s, tt, edge=1, mask=None, threads=(1, 3, 8)):
    c0, w0, q0 = orc.pair_hist(x, y, t, box, s, tt, edge_mode=edge, centre_mask=mask)
    for th in threads:
        c1, w1, q1 = orc.pair_hist_grid(x, y, t, box, s, tt, edge_mode=edge, centre_mask=mask,
                                        threads=th)
        np.testing.assert_array_equal(c1, c0)
        assert q1 == q0
        np.testing.assert_allclose(w1, w0, rtol=1e-12, atol=0)


def test_grid_matches_brute_force_csr(orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small()
    for edge in (0, 1):
        _check(orc, w.x, w.y, w.t, w.box, w.s, w.tt, edge=edge)


def test_grid_matches_brute_force_clusters_and_edges(orc):
    rng = np.random.default_rng(4)
    box = (0.0, 1000.0, 0.0, 800.0, 0.0, 365.0)
    k = 1500
    cx = np.r_[rng.uniform(0, 40, k // 2), rng.uniform(960, 1000, k // 2)]
    cy = np.r_[rng.uniform(0, 30, k // 2), rng.uniform(0, 800, k // 2)]
    ct = np.r_[rng.uniform(0, 5, k // 2), rng.uniform(0, 365, k // 2)]
    x = np.clip(np.r_[cx, rng.uniform(0, 1000, 700)], 0, 1000)
    y = np.clip(np.r_[cy, rng.uniform(0, 800, 700)], 0, 800)
    t = np.clip(np.r_[ct, rng.uniform(0, 365, 700)], 0, 365)
    x[:10], y[:10], t[:10] = 0.0, 0.0, 0.0  # coincident points at a corner
    x[10:20], y[10:20] = 1000.0, 800.0  # on the upper faces
    s, tt = np.array([5.0, 20.0, 60.0, 150.0]), np.array([1.0, 10.0, 40.0])
    mask = (rng.random(len(x)) < 0.3).astype(np.uint8)
    _check(orc, x, y, t, box, s, tt)
    _check(orc, x, y, t, box, s, tt, mask=mask)


def test_grid_matches_brute_force_dyadic_ties(orc):
    # coordinates on a 1/8 lattice and integer thresholds: many pairs exactly at d = s, u = t
    rng = np.random.default_rng(11)
    box = (0.0, 64.0, 0.0, 64.0, 0.0, 32.0)
    n = 1200
    x = rng.integers(0, 513, n) / 8.0
    y = rng.integers(0, 513, n) / 8.0
    t = rng.integers(0, 257, n) / 8.0
    s, tt = np.array([1.0, 2.0, 5.0, 13.0]), np.array([0.5, 1.0, 3.0])
    _check(orc, x, y, t, box, s, tt)


@pytest.mark.parametrize("smax,tmax", [(0.8, 0.4), (400.0, 180.0)])
def test_grid_extreme_cell_counts(orc, smax, tmax):
    from paper_1912_04753_gb300 import workloads as wl

    box = (0.0, 800.0, 0.0, 800.0, 0.0, 360.0)
    x, y, t = wl.csr(900, box, 2)
    x[:300], y[:300], t[:300] = x[300:600] + 0.3, y[300:600], t[300:600] + 0.1
    x = np.clip(x, 0, 800)
    t = np.clip(t, 0, 360)
    s, tt = np.linspace(smax / 4, smax, 4), np.linspace(tmax / 3, tmax, 3)
    _check(orc, x, y, t, box, s, tt, threads=(2, 5))
