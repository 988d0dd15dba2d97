"""Property tests of the oracle on random small patterns (hypothesis): facts that hold for any
input and that a mistake in the pair loop, the bins, the weights or the cumulation breaks.
Points sit on a dyadic lattice, so reflections are exact and threshold ties occur."""
import numpy as np
import pytest

pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

BOX = (0.0, 64.0, 0.0, 32.0, 0.0, 16.0)


@st.composite
def patterns(draw):
    n = draw(st.integers(2, 40))
    ix = draw(st.lists(st.integers(0, 512), min_size=n, max_size=n))
    iy = draw(st.lists(st.integers(0, 256), min_size=n, max_size=n))
    it = draw(st.lists(st.integers(0, 128), min_size=n, max_size=n))
    x = np.array(ix, float) / 8.0
    y = np.array(iy, float) / 8.0
    t = np.array(it, float) / 8.0
    cs = draw(st.integers(1, 5))
    ct = draw(st.integers(1, 4))
    s = np.sort(np.array(draw(st.lists(st.integers(1, 128), min_size=cs, max_size=cs,
                                       unique=True)), float)) / 8.0
    tt = np.sort(np.array(draw(st.lists(st.integers(1, 64), min_size=ct, max_size=ct,
                                        unique=True)), float)) / 8.0
    return x, y, t, s, tt


@settings(max_examples=60, deadline=None)
@given(patterns())
def test_counts_weights_and_cumulation(orc, p):
    x, y, t, s, tt = p
    r = orc.k_function(x, y, t, BOX, s, tt)
    C, S = r["C"], r["S"]
    assert (C % 2 == 0).all()                       # each unordered pair counted twice
    assert (np.diff(C, axis=0) >= 0).all() and (np.diff(C, axis=1) >= 0).all()
    assert (S >= C - 1e-9).all() and (S <= 8 * C + 1e-9).all()   # 1 <= 1 / (w v) <= 8
    assert C[-1, -1] == r["pairs"]
    none = orc.k_function(x, y, t, BOX, s, tt, edge_mode=0)
    np.testing.assert_array_equal(none["C"], C)
    np.testing.assert_array_equal(none["S"], C.astype(float))


@settings(max_examples=40, deadline=None)
@given(patterns())
def test_exact_reflections(orc, p):
    x, y, t, s, tt = p
    base = orc.k_function(x, y, t, BOX, s, tt)
    for xr, yr, tr in ((64.0 - x, y, t), (x, 32.0 - y, t), (x, y, 16.0 - t)):
        r = orc.k_function(xr, yr, tr, BOX, s, tt)
        np.testing.assert_array_equal(r["C"], base["C"])
        np.testing.assert_allclose(r["S"], base["S"], rtol=1e-12)


@settings(max_examples=40, deadline=None)
@given(patterns(), st.integers(2, 7))
def test_variants_reduce_and_partition(orc, p, n_sec):
    x, y, t, s, tt = p
    base = orc.k_function(x, y, t, BOX, s, tt)
    # a constant intensity on any grid is Eq. 2
    lam = orc.intensity_at(x, y, t, BOX, np.full((2, 3, 2), 1.5))
    inh = orc.k_function_inhom(x, y, t, BOX, s, tt, lam)
    np.testing.assert_array_equal(inh["C"], base["C"])
    np.testing.assert_allclose(inh["K"], base["K"], rtol=1e-12)
    # sectors partition the pairs of the translation-corrected estimator
    one = orc.k_function_dir(x, y, t, BOX, s, tt, 1)
    parts = orc.k_function_dir(x, y, t, BOX, s, tt, n_sec)
    np.testing.assert_array_equal(parts["C"].sum(axis=0), one["C"][0])
    np.testing.assert_array_equal(one["C"][0], base["C"])
    # cross K over two labels recombines into the univariate sum
    lab = (np.arange(len(x)) % 2).astype(np.uint8)
    na = {a: int((lab == a).sum()) for a in (0, 1)}
    n = len(x)
    acc = np.zeros_like(base["K"])
    for a in (0, 1):
        for b in (0, 1):
            den = na[a] * na[b] if a != b else na[a] * (na[a] - 1)
            if den == 0:
                continue
            acc += orc.k_cross(x, y, t, lab, a, b, BOX, s, tt)["K"] * den
    np.testing.assert_allclose(acc, base["K"] * n * (n - 1), rtol=1e-12, atol=1e-9)
