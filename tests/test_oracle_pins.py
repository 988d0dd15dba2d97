"""Pins for the oracle: each test checks it against something other than itself.

Sources of truth: published known-answer vectors (Philox), hand-worked fixtures, textbook
closed forms of the isotropic weight (Section 3), brute-force angular sampling, exact rational
brute force on tiny dyadic inputs, invariances that hold exactly, and the CSTR expectation
E[K(s,t)] = 2 pi s^2 t (Section 3, Eq. 1) which holds exactly for the n(n-1)-normalised
isotropic estimator on a binomial CSR sample.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    lines = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                lines.append(ln)
    return lines


# ---------------------------------------------------------------------------- Philox / RNG


def test_philox_known_answers(orc):
    for ln in _read_golden("philox4x32_10_kat.txt"):
        lhs, rhs = ln.split("->")
        v = [int(w, 16) for w in lhs.split()]
        want = [int(w, 16) for w in rhs.split()]
        got = orc.philox4x32_10(v[:4], v[4:6])
        assert [int(g) for g in got] == want


def test_u01_range_and_resolution(orc):
    assert orc.u01(0, 0) == 0.0
    top = orc.u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0**-53
    # the low six bits of w1 and the low five of w0 are discarded
    assert orc.u01(0, 63) == 0.0
    assert orc.u01(0, 64) == 2.0**-53
    assert orc.u01(32, 0) == 2.0**-27  # (32 >> 5) * 2^26 * 2^-53


def test_csr_points_uniform_and_inside(orc):
    box = (-5.0, 7.0, 100.0, 103.0, 10.0, 375.0)
    x, y, t = orc.csr_points(20000, box, seed=12345, sim=3)
    for v, lo, hi in ((x, box[0], box[1]), (y, box[2], box[3]), (t, box[4], box[5])):
        assert v.min() >= lo and v.max() <= hi
        u = (v - lo) / (hi - lo)
        # mean 1/2, variance 1/12 of a uniform; 5 standard errors
        assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))
        assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / len(u))
    # streams and realizations differ; the same call repeats bit for bit
    x2, _, _ = orc.csr_points(20000, box, seed=12345, sim=4)
    assert not np.array_equal(x, x2)
    x3, y3, t3 = orc.csr_points(20000, box, seed=12345, sim=3)
    assert np.array_equal(x, x3) and np.array_equal(t, t3)


def test_csr_point_is_philox_draw(orc):
    """Point i of realization k is x0 + W * u01(philox((i, k, 0, 0), seed)) (stream 0 = x)."""
    box = (0.0, 10.0, 0.0, 20.0, 0.0, 30.0)
    seed = (7 << 32) | 99
    x, y, t = orc.csr_points(5, box, seed=seed, sim=2)
    for i in range(5):
        for stream, arr, lo, hi in ((0, x, 0.0, 10.0), (1, y, 0.0, 20.0), (2, t, 0.0, 30.0)):
            w = orc.philox4x32_10([i, 2, stream, 0], [99, 7])
            u = ((int(w[0]) >> 5) * 67108864 + (int(w[1]) >> 6)) / 2.0**53
            assert arr[i] == lo + (hi - lo) * u


# ---------------------------------------------------------------------------- weights


BOX = (0.0, 10.0, 0.0, 6.0, 0.0, 1.0)


def _angular_fraction(xi, yi, r, box, m=1 << 20):
    """Brute force: the share of m equally spaced points on the circle inside the box."""
    th = (np.arange(m) + 0.5) * (2 * np.pi / m)
    px = xi + r * np.cos(th)
    py = yi + r * np.sin(th)
    inside = (px >= box[0]) & (px <= box[1]) & (py >= box[2]) & (py <= box[3])
    return inside.mean()


def test_spatial_weight_interior_is_one(orc):
    assert orc.spatial_weight(5.0, 3.0, 2.0, BOX) == 1.0
    assert orc.spatial_weight(5.0, 3.0, 3.0, BOX) == 1.0  # tangent to top and bottom
    assert orc.spatial_weight(5.0, 3.0, 0.0, BOX) == 1.0


def test_spatial_weight_closed_forms(orc):
    # one edge at distance e < r: 1 - acos(e/r)/pi
    for e, r in ((1.0, 2.0), (0.0, 1.5), (1.9, 2.0), (0.25, 2.5)):
        got = orc.spatial_weight(e, 3.0, r, BOX)
        assert got == pytest.approx(1 - math.acos(e / r) / math.pi, abs=1e-15)
    # two adjacent edges, corner outside the circle: 1 - (a1 + a2)/pi
    e1, e2, r = 1.0, 1.2, 1.5
    assert e1 * e1 + e2 * e2 >= r * r
    got = orc.spatial_weight(e1, e2, r, BOX)
    want = 1 - (math.acos(e1 / r) + math.acos(e2 / r)) / math.pi
    assert got == pytest.approx(want, abs=1e-15)
    # corner inside the circle: the two outside arcs overlap by pi/2 beyond the corner
    e1, e2, r = 0.6, 0.8, 2.0
    assert e1 * e1 + e2 * e2 < r * r
    got = orc.spatial_weight(e1, e2, r, BOX)
    want = 1 - (math.acos(e1 / r) + math.acos(e2 / r) + math.pi / 2) / (2 * math.pi)
    assert got == pytest.approx(want, abs=1e-15)
    # a point exactly on a corner keeps a quarter circle, on an edge a half
    assert orc.spatial_weight(0.0, 0.0, 1.0, BOX) == pytest.approx(0.25, abs=1e-15)
    assert orc.spatial_weight(10.0, 6.0, 2.0, BOX) == pytest.approx(0.25, abs=1e-15)
    assert orc.spatial_weight(4.0, 0.0, 1.0, BOX) == pytest.approx(0.5, abs=1e-15)


@pytest.mark.parametrize(
    "xi,yi,r",
    [(1.0, 3.0, 2.0), (0.5, 0.7, 1.3), (9.3, 5.6, 2.2), (2.0, 1.0, 2.9), (5.0, 3.0, 3.5),
     (0.0, 3.0, 4.0), (9.99, 0.01, 0.5), (5.0, 0.2, 5.5), (3.0, 4.0, 1e-3)],
)
def test_spatial_weight_matches_angular_sampling(orc, xi, yi, r):
    # includes circles cut by two opposite edges (r > 3 in a box of height 6)
    got = orc.spatial_weight(xi, yi, r, BOX)
    assert got == pytest.approx(_angular_fraction(xi, yi, r, BOX), abs=2e-5)


def test_temporal_weight_cases(orc):
    assert orc.temporal_weight(0.5, 0.2, 0.0, 1.0) == 1.0
    assert orc.temporal_weight(0.5, 0.5, 0.0, 1.0) == 1.0  # both ends on the bounds
    assert orc.temporal_weight(0.0, 0.1, 0.0, 1.0) == 0.5  # centre at the start
    assert orc.temporal_weight(0.9, 0.2, 0.0, 1.0) == 0.5  # sticks out at the end
    assert orc.temporal_weight(0.5, 0.7, 0.0, 1.0) == 0.5  # sticks out on both sides
    assert orc.temporal_weight(0.0, 0.0, 0.0, 1.0) == 1.0  # u = 0 at the start


# ---------------------------------------------------------------------------- counts


def _hand_fixture():
    lines = _read_golden("hand_pairs.txt")
    pts, kv, it = [], {}, iter(lines)
    for ln in it:
        if ln == "points":
            for p in it:
                if p == "end":
                    break
                pts.append([float(v) for v in p.split()])
        else:
            key, *vals = ln.split()
            kv[key] = [float(v) for v in vals]
    P = np.array(pts)
    return P[:, 0], P[:, 1], P[:, 2], kv


def test_hand_fixture_counts_and_weights(orc):
    x, y, t, kv = _hand_fixture()
    box, s, tt = kv["box"], kv["s"], kv["t"]
    cnt, wsum, q = orc.pair_hist(x, y, t, box, s, tt, edge_mode=1)
    assert cnt.reshape(-1).tolist() == [int(v) for v in kv["cnt"]]
    assert q == sum(int(v) for v in kv["cnt"])
    W = 1.0 / (1.0 - math.acos(0.8) / math.pi)
    want = np.array(kv["wsum_unit_part"]) + np.array(kv["wsum_W_multiple"]) * W
    np.testing.assert_allclose(wsum.reshape(-1), want, rtol=1e-15)
    out = orc.k_function(x, y, t, box, s, tt, edge_mode=0, norm=0)
    assert out["C"].reshape(-1).tolist() == [int(v) for v in kv["cum_count"]]
    np.testing.assert_allclose(out["K"].reshape(-1),
                               kv["k_coef_n_nm1"][0] * np.array(kv["cum_count"]), rtol=1e-15)
    out2 = orc.k_function(x, y, t, box, s, tt, edge_mode=0, norm=1)
    np.testing.assert_allclose(out2["K"].reshape(-1),
                               kv["k_coef_n2"][0] * np.array(kv["cum_count"]), rtol=1e-15)


def _fraction_counts(P, s, tt):
    """Exact rational brute force of the cumulative counts over ordered pairs."""
    n = len(P)
    F = [[Fraction(v) for v in p] for p in P]
    S2 = [Fraction(v) ** 2 for v in s]
    T = [Fraction(v) for v in tt]
    C = np.zeros((len(s), len(tt)), np.int64)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d2 = (F[i][0] - F[j][0]) ** 2 + (F[i][1] - F[j][1]) ** 2
            u = abs(F[i][2] - F[j][2])
            for a in range(len(s)):
                for b in range(len(tt)):
                    if d2 <= S2[a] and u <= T[b]:
                        C[a, b] += 1
    return C


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_counts_match_exact_rational_bruteforce(orc, seed):
    # dyadic coordinates on a 1/8 grid: FP64 differences, squares and sums are exact, and
    # thresholds on the same grid create exact ties (Eq. 3 is inclusive)
    rng = np.random.default_rng(seed)
    n = 40
    P = rng.integers(0, 8 * 16, size=(n, 3)) / 8.0
    s = np.array([0.5, 1.0, 2.5, 4.0])
    tt = np.array([0.25, 1.0, 3.0])
    box = (0.0, 16.0, 0.0, 16.0, 0.0, 16.0)
    out = orc.k_function(P[:, 0], P[:, 1], P[:, 2], box, s, tt, edge_mode=1)
    np.testing.assert_array_equal(out["C"], _fraction_counts(P, s, tt))


def test_count_symmetry_and_monotonicity(orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=5, n=600)
    cnt, _, _ = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=1)
    assert (cnt % 2 == 0).all()  # (i,j) and (j,i) always share a bin
    out = orc.k_function(w.x, w.y, w.t, w.box, w.s, w.tt)
    C, S = out["C"], out["S"]
    assert (np.diff(C, axis=0) >= 0).all() and (np.diff(C, axis=1) >= 0).all()
    assert (S >= C).all()  # every weight 1/(omega v) is at least 1
    assert (S <= 8 * C + 1e-9).all()  # omega >= 1/4 and v >= 1/2 when s <= min(W,H)/2


def test_edge_mode_none_gives_counts(orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=6, n=500)
    out = orc.k_function(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=0)
    np.testing.assert_array_equal(out["S"], out["C"].astype(np.float64))


def test_exact_invariances(orc):
    # dyadic points in a square box: reflections and the x<->y swap change no FP64 value
    rng = np.random.default_rng(11)
    n = 300
    P = rng.integers(0, 64 * 256, size=(n, 3)) / 64.0
    box = (0.0, 256.0, 0.0, 256.0, 0.0, 256.0)
    s = np.array([8.0, 16.0, 32.0, 60.0])
    tt = np.array([4.0, 16.0, 50.0])
    base = orc.k_function(P[:, 0], P[:, 1], P[:, 2], box, s, tt)
    variants = [
        (256.0 - P[:, 0], P[:, 1], P[:, 2]),
        (P[:, 0], 256.0 - P[:, 1], P[:, 2]),
        (P[:, 1], P[:, 0], P[:, 2]),
        (P[:, 0], P[:, 1], 256.0 - P[:, 2]),
    ]
    for x, y, t in variants:
        o = orc.k_function(x, y, t, box, s, tt)
        np.testing.assert_array_equal(o["C"], base["C"])
        np.testing.assert_allclose(o["S"], base["S"], rtol=1e-13)


def test_sampled_centres_partition_the_sum(orc):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=7, n=400)
    cnt, wsum, q = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt)
    m = np.zeros(w.n, np.uint8)
    m[::3] = 1
    c1, w1, q1 = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=m)
    c2, w2, q2 = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=1 - m)
    np.testing.assert_array_equal(c1 + c2, cnt)
    assert q1 + q2 == q
    np.testing.assert_allclose(w1 + w2, wsum, rtol=1e-13)


# ---------------------------------------------------------------------------- CSTR expectation


def test_cstr_expectation_2pi_s2_t(orc):
    """E[K(s,t)] = 2 pi s^2 t under CSTR (Section 3) for the n(n-1) isotropic estimator.

    For a centre at p, the neighbours within distance s weighted by 1/omega integrate to
    pi s^2 exactly (the inside arc at radius rho is omega * 2 pi rho), and those within u <= t
    weighted by 1/v integrate to 2t whenever t <= D/2.  A wrong normalisation (n^2), an area
    instead of a circumference fraction, or a missing temporal weight all bias the mean by
    many standard errors at these sizes.
    """
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    s = np.array([0.05, 0.1, 0.15, 0.2, 0.25])
    tt = np.array([0.05, 0.1, 0.2, 0.35, 0.5])
    n, R = 500, 400
    Ks = []
    for r in range(R):
        rng = np.random.default_rng(1000 + r)
        x, y, t = rng.random(n), rng.random(n), rng.random(n)
        Ks.append(orc.k_function(x, y, t, box, s, tt)["K"])
    Ks = np.array(Ks)
    mean = Ks.mean(axis=0)
    se = Ks.std(axis=0, ddof=1) / math.sqrt(R)
    theory = 2 * math.pi * s[:, None] ** 2 * tt[None, :]
    z = (mean - theory) / se
    assert np.abs(z).max() < 4.0, z
    # Eq. 4: L of the mean K is ~0 under CSTR
    Lm = np.sqrt(mean / (2 * math.pi * tt[None, :])) - s[:, None]
    assert np.abs(Lm / s[:, None]).max() < 0.02
    # and the oracle's own L agrees with Eq. 4 applied to its K
    o = orc.k_function(x, y, t, box, s, tt)
    np.testing.assert_allclose(o["L"], np.sqrt(o["K"] / (2 * math.pi * tt[None, :])) - s[:, None],
                               rtol=0, atol=1e-14)


def test_envelope_is_min_max_of_simulations(orc):
    box = (0.0, 100.0, 0.0, 100.0, 0.0, 50.0)
    s = np.array([2.0, 5.0, 10.0])
    tt = np.array([1.0, 5.0])
    env = orc.envelope(300, box, s, tt, n_sims=7, seed=42, keep_all=True)
    Ka = env["K_all"]
    np.testing.assert_array_equal(env["K_lo"], Ka.min(axis=0))
    np.testing.assert_array_equal(env["K_hi"], Ka.max(axis=0))
    for k in (0, 6):
        x, y, t = orc.csr_points(300, box, 42, k)
        np.testing.assert_array_equal(orc.k_function(x, y, t, box, s, tt)["K"], Ka[k])
    assert (env["L_lo"] <= env["L_hi"]).all()


# ----------------------------------------------------------- bootstrap / permutation (Sec. 3)


@pytest.mark.parametrize("b", [2, 4, 6, 10])
def test_feistel_network_is_a_bijection(orc, b):
    for seed, sim in ((0, 0), (12345, 7), (2**63 + 5, 99)):
        out = sorted(orc.feistel(v, b, seed, sim) for v in range(1 << b))
        assert out == list(range(1 << b))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 1000, 4097])
def test_permutation_is_a_permutation(orc, n):
    assert orc.feistel_bits(n) % 2 == 0 and (1 << orc.feistel_bits(n)) >= n
    for sim in (0, 1, 2):
        p = [orc.permutation_index(n, 42, sim, i) for i in range(n)]
        assert sorted(p) == list(range(n))
    if n >= 17:  # distinct realizations differ
        assert [orc.permutation_index(n, 42, 0, i) for i in range(n)] != \
               [orc.permutation_index(n, 42, 1, i) for i in range(n)]


def test_permutation_exchanges_only_the_timestamps(orc):
    rng = np.random.default_rng(3)
    x, y, t = rng.uniform(0, 100, 300), rng.uniform(0, 50, 300), rng.uniform(0, 9, 300)
    px, py, pt = orc.permutation_points(x, y, t, 7, 4)
    np.testing.assert_array_equal(px, x)
    np.testing.assert_array_equal(py, y)
    np.testing.assert_array_equal(np.sort(pt), np.sort(t))
    assert not np.array_equal(pt, t)


def test_permutation_is_uniform_on_small_sets(orc):
    # all 6 orders of 3 points, and every (position, source) pair of 10 points, come out with
    # equal frequency (chi-square far inside a 1e-6 tail)
    import itertools

    sims = 6000
    orders = {p: 0 for p in itertools.permutations(range(3))}
    for k in range(sims):
        orders[tuple(orc.permutation_index(3, 11, k, i) for i in range(3))] += 1
    e = sims / 6
    chi2 = sum((c - e) ** 2 / e for c in orders.values())
    assert chi2 < 35.9, orders  # 5 dof
    sims = 3000
    cnt = np.zeros((10, 10))
    for k in range(sims):
        for i in range(10):
            cnt[i, orc.permutation_index(10, 5, k, i)] += 1
    e = sims / 10
    chi2 = ((cnt - e) ** 2 / e).sum()
    assert chi2 < 81 + 6 * math.sqrt(2 * 81)  # 81 dof


def test_permutation_keeps_spatial_pair_counts(orc):
    # exchanging timestamps leaves every spatial distance as it is: with a temporal threshold
    # that spans the whole period, the cumulative counts equal the observed ones
    rng = np.random.default_rng(8)
    box = (0.0, 400.0, 0.0, 300.0, 0.0, 50.0)
    x, y, t = rng.uniform(0, 400, 250), rng.uniform(0, 300, 250), rng.uniform(0, 50, 250)
    s, tt = np.array([20.0, 45.0, 90.0]), np.array([5.0, 50.0])
    obs = orc.k_function(x, y, t, box, s, tt)
    for sim in range(3):
        px, py, pt = orc.permutation_points(x, y, t, 99, sim)
        got = orc.k_function(px, py, pt, box, s, tt)
        np.testing.assert_array_equal(got["C"][:, -1], obs["C"][:, -1])


def test_bootstrap_draws_are_observed_points_uniformly(orc):
    rng = np.random.default_rng(4)
    n = 500
    x, y, t = rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    counts = np.zeros(n)
    sims = 200
    for k in range(sims):
        bx, by, bt = orc.bootstrap_points(x, y, t, 77, k)
        idx = np.array([orc.bootstrap_index(n, 77, k, i) for i in range(n)])
        assert idx.min() >= 0 and idx.max() < n
        np.testing.assert_array_equal(bx, x[idx])
        np.testing.assert_array_equal(by, y[idx])
        np.testing.assert_array_equal(bt, t[idx])
        counts += np.bincount(idx, minlength=n)
    e = sims
    chi2 = ((counts - e) ** 2 / e).sum()
    assert abs(chi2 - (n - 1)) < 6 * math.sqrt(2 * (n - 1))
    assert counts.min() > 0  # every point is drawn (expected 200 times each)
    assert orc.bootstrap_index(1, 3, 0, 0) == 0
    # three points: each index with probability 1/3 (5 binomial standard errors)
    draws = np.array([orc.bootstrap_index(3, 5, k, i) for k in range(400) for i in range(3)])
    freq = np.bincount(draws, minlength=3) / len(draws)
    assert np.all(np.abs(freq - 1 / 3) < 5 * math.sqrt((1 / 3) * (2 / 3) / len(draws)))


def test_bootstrap_duplicates_are_zero_distance_pairs(orc):
    # a realization that repeats a point pairs the copies at d = 0, u = 0, weight 1: the
    # first bin counts exactly the ordered pairs of copies of the same observed point
    rng = np.random.default_rng(6)
    box = (0.0, 1000.0, 0.0, 1000.0, 0.0, 100.0)
    n = 200
    x, y, t = rng.uniform(0, 1000, n), rng.uniform(0, 1000, n), rng.uniform(0, 100, n)
    bx, by, bt = orc.bootstrap_points(x, y, t, 5, 0)
    idx = np.array([orc.bootstrap_index(n, 5, 0, i) for i in range(n)])
    mult = np.bincount(idx, minlength=n)
    s, tt = np.array([1e-9, 10.0]), np.array([1e-9, 5.0])
    got = orc.k_function(bx, by, bt, box, s, tt)
    assert got["C"][0, 0] == int((mult * (mult - 1)).sum())
    assert got["S"][0, 0] == got["C"][0, 0]  # interior duplicates: weight exactly 1


# ---------------------------------------------------------------- polygon study areas


def _star(nv, r0, r1, cx, cy, seed):
    rng = np.random.default_rng(seed)
    th = np.sort(rng.uniform(0, 2 * np.pi, nv))
    rad = np.where(np.arange(nv) % 2 == 0, r0, r1) * rng.uniform(0.85, 1.0, nv)
    return cx + rad * np.cos(th), cy + rad * np.sin(th)


def test_polygon_area_and_orientation(orc):
    tri = ([0.0, 4.0, 0.0], [0.0, 0.0, 3.0])
    assert orc.polygon_area(*tri) == 6.0
    ell = ([0, 4, 4, 1, 1, 0], [0, 0, 1, 1, 3, 3])  # L shape: 4x1 + 1x2
    assert orc.polygon_area(*ell) == 6.0
    assert orc.polygon_area(ell[0][::-1], ell[1][::-1]) == 6.0


def test_point_in_polygon_closed(orc):
    ell = ([0, 4, 4, 1, 1, 0], [0, 0, 1, 1, 3, 3])
    assert orc.point_in_polygon(0.5, 2.5, *ell)
    assert not orc.point_in_polygon(2.0, 2.0, *ell)      # in the notch
    assert orc.point_in_polygon(4.0, 0.5, *ell)          # on an edge
    assert orc.point_in_polygon(1.0, 1.0, *ell)          # the reflex vertex
    assert orc.point_in_polygon(0.0, 3.0, *ell)          # a convex vertex
    assert not orc.point_in_polygon(4.0 + 1e-12, 0.5, *ell)


def test_rectangle_polygon_equals_box_weight(orc):
    # two independent constructions: arc union over the four edge half-planes (box) and
    # crossing angles with midpoint tests (polygon)
    rng = np.random.default_rng(2)
    box = (-3.0, 7.0, 1.0, 6.0, 0.0, 1.0)
    vx, vy = [-3.0, 7.0, 7.0, -3.0], [1.0, 1.0, 6.0, 6.0]
    for _ in range(400):
        x, y = rng.uniform(-3, 7), rng.uniform(1, 6)
        r = rng.uniform(0, 2.5)
        assert abs(orc.polygon_weight(x, y, r, vx, vy) - orc.spatial_weight(x, y, r, box)) < 1e-12


def test_polygon_weight_closed_forms(orc):
    sq = ([0.0, 2.0, 2.0, 0.0], [0.0, 0.0, 2.0, 2.0])
    assert orc.polygon_weight(1.0, 1.0, 0.9, *sq) == 1.0   # clear of the edges
    assert abs(orc.polygon_weight(0.0, 0.0, 1.0, *sq) - 0.25) < 1e-15  # at a corner
    assert abs(orc.polygon_weight(1.0, 0.0, 0.5, *sq) - 0.5) < 1e-15   # on an edge
    # at the reflex vertex of an L: three quarters of a small circle are inside
    ell = ([0, 4, 4, 1, 1, 0], [0, 0, 1, 1, 3, 3])
    assert abs(orc.polygon_weight(1.0, 1.0, 0.5, *ell) - 0.75) < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_polygon_weight_matches_angular_sampling(orc, seed):
    vx, vy = _star(24, 100.0, 55.0, 0.0, 0.0, seed)
    rng = np.random.default_rng(seed + 10)
    th = (np.arange(200000) + 0.5) * (2 * np.pi / 200000)
    for _ in range(4):
        while True:
            x, y = rng.uniform(-80, 80), rng.uniform(-80, 80)
            if orc.point_in_polygon(x, y, vx, vy):
                break
        r = rng.uniform(5, 60)
        # fraction of 200,000 evenly spaced points of the circle inside the polygon,
        # by a vectorised crossing-number test
        px, py = x + r * np.cos(th), y + r * np.sin(th)
        inside = np.zeros(px.shape, bool)
        for k in range(len(vx)):
            ax, ay, bx, by = vx[k], vy[k], vx[(k + 1) % len(vx)], vy[(k + 1) % len(vx)]
            straddle = (ay > py) != (by > py)
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = ax + (py - ay) * (bx - ax) / (by - ay)
            inside ^= straddle & (px < xc)
        assert abs(orc.polygon_weight(x, y, r, vx, vy) - inside.mean()) < 5e-5


def test_rectangle_polygon_gives_the_box_estimator(orc):
    rng = np.random.default_rng(5)
    box = (0.0, 300.0, 0.0, 200.0, 0.0, 30.0)
    x, y, t = rng.uniform(0, 300, 400), rng.uniform(0, 200, 400), rng.uniform(0, 30, 400)
    s, tt = np.array([10.0, 40.0, 90.0]), np.array([2.0, 7.0])
    a = orc.k_function(x, y, t, box, s, tt)
    b = orc.k_function_polygon(x, y, t, box, [0, 300, 300, 0], [0, 0, 200, 200], s, tt)
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_allclose(b["K"], a["K"], rtol=1e-12)


def test_csr_in_polygon_inside_and_uniform(orc):
    ell = ([0, 4, 4, 1, 1, 0], [0, 0, 1, 1, 3, 3])
    box = (0.0, 4.0, 0.0, 3.0, 10.0, 20.0)
    n = 60000
    x, y, t = orc.csr_polygon_points(n, box, *ell, 9, 2)
    assert all(orc.point_in_polygon(a, b, *ell) for a, b in zip(x[:2000], y[:2000]))
    assert ((x <= 1) | (y <= 1)).all()
    # the leg x <= 1, y > 1 holds 2 of the 6 area units
    frac = np.mean((x <= 1) & (y > 1))
    assert abs(frac - 2 / 6) < 6 * np.sqrt((1 / 3) * (2 / 3) / n)
    assert t.min() >= 10.0 and t.max() <= 20.0
    x2, y2, t2 = orc.csr_polygon_points(n, box, *ell, 9, 2)
    np.testing.assert_array_equal(x, x2)



# ------------------------------------------------------------------- bivariate (cross) K


def _two_types(seed, n=500):
    rng = np.random.default_rng(seed)
    box = (0.0, 500.0, 0.0, 400.0, 0.0, 60.0)
    x, y, t = rng.uniform(0, 500, n), rng.uniform(0, 400, n), rng.uniform(0, 60, n)
    lab = (rng.uniform(size=n) < 0.35).astype(np.uint8)
    return x, y, t, lab, box


def test_cross_k_same_label_is_the_subset_estimator(orc):
    x, y, t, lab, box = _two_types(1)
    s, tt = np.array([15.0, 40.0, 90.0]), np.array([3.0, 10.0])
    for a in (0, 1):
        sel = lab == a
        want = orc.k_function(x[sel], y[sel], t[sel], box, s, tt)
        got = orc.k_cross(x, y, t, lab, a, a, box, s, tt)
        np.testing.assert_array_equal(got["C"], want["C"])
        np.testing.assert_allclose(got["K"], want["K"], rtol=1e-13)


def test_cross_counts_partition_all_pairs_and_are_symmetric(orc):
    x, y, t, lab, box = _two_types(2)
    s, tt = np.array([20.0, 60.0]), np.array([5.0, 20.0])
    allc = orc.k_function(x, y, t, box, s, tt)["C"]
    c = {(a, b): orc.k_cross(x, y, t, lab, a, b, box, s, tt)["C"] for a in (0, 1)
         for b in (0, 1)}
    np.testing.assert_array_equal(sum(c.values()), allc)
    np.testing.assert_array_equal(c[(0, 1)], c[(1, 0)])
    none = orc.k_cross(x, y, t, lab, 0, 1, box, s, tt, edge_mode=0)
    np.testing.assert_array_equal(none["S"], none["C"].astype(float))


def test_point_in_polygon_at_vertex_heights(orc):
    # the ray towards +x passes exactly through vertices: a diamond and an L shape, answers by
    # inspection (a point is inside the diamond iff |x| + |y| <= 1)
    dia = ([0.0, 1.0, 0.0, -1.0], [-1.0, 0.0, 1.0, 0.0])
    for px, py in ((-0.5, 0.0), (0.25, 0.0), (0.0, 0.5), (-0.25, -0.5), (0.5, 0.25)):
        assert orc.point_in_polygon(px, py, *dia) == (abs(px) + abs(py) <= 1.0), (px, py)
    for px, py in ((-1.5, 0.0), (1.5, 0.0), (-2.0, 1.0), (-3.0, -1.0), (0.9, 0.5)):
        assert not orc.point_in_polygon(px, py, *dia), (px, py)
    ell = ([0, 4, 4, 1, 1, 0], [0, 0, 1, 1, 3, 3])
    assert orc.point_in_polygon(0.5, 1.0, *ell)        # at the height of the reflex vertex
    assert not orc.point_in_polygon(-1.0, 1.0, *ell)
    assert not orc.point_in_polygon(-1.0, 3.0, *ell)   # at the height of the top edge
    assert orc.point_in_polygon(0.5, 3.0, *ell)        # on the top edge (closed)


def test_cross_k_normalisations_recombine_to_the_univariate_sum(orc):
    """sum_{a != b} n_a n_b K_ab + sum_a n_a (n_a - 1) K_aa = n (n - 1) K: every ordered pair of
    the univariate sum belongs to exactly one label pair, and each K_ab is A D / (its
    denominator) times its part of the sum."""
    x, y, t, lab, box = _two_types(3)
    s, tt = np.array([20.0, 60.0]), np.array([5.0, 20.0])
    n = len(x)
    na = {a: int((lab == a).sum()) for a in (0, 1)}
    total = orc.k_function(x, y, t, box, s, tt)["K"] * n * (n - 1)
    acc = np.zeros_like(total)
    for a in (0, 1):
        for b in (0, 1):
            k = orc.k_cross(x, y, t, lab, a, b, box, s, tt)["K"]
            acc += k * (na[a] * na[b] if a != b else na[a] * (na[a] - 1))
    np.testing.assert_allclose(acc, total, rtol=1e-12)


def test_envelope_rank_under_csr(orc):
    """Section 3's Monte Carlo test: for CSR data and m CSR simulations the observed K exceeds
    the envelope's maximum with probability 1/(m+1), and falls below its minimum with the same
    probability (the m+1 patterns are exchangeable).  The observed patterns are drawn with
    numpy, independently of the oracle's generator, so a biased simulation fails this test."""
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    s, tt = np.array([0.1, 0.2]), np.array([0.2, 0.4])
    n, m, R = 150, 9, 300
    above = below = 0
    for r in range(R):
        rng = np.random.default_rng(9000 + r)
        x, y, t = rng.random(n), rng.random(n), rng.random(n)
        obs = orc.k_function(x, y, t, box, s, tt)["K"][1, 1]
        env = orc.envelope(n, box, s, tt, m, 500 + r)
        above += obs > env["K_hi"][1, 1]
        below += obs < env["K_lo"][1, 1]
    p = 1.0 / (m + 1)
    se = math.sqrt(p * (1 - p) / R)
    assert abs(above / R - p) < 4 * se, above
    assert abs(below / R - p) < 4 * se, below
