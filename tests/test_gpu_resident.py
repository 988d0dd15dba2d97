"""The observed pattern's grid index stays resident on its handle between jobs: a job whose grid
and record constants equal the previous job's reuses the sorted arrays (no keys, sort or
scatter for the observed pattern) and gives exactly the grids a fresh handle gives; a job on
another grid, or after the study area changes, rebuilds it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("prec", [0, 1])
def test_resident_index_reused_and_exact(stk, monkeypatch, prec):
    from paper_1912_04753_gb300 import workloads as wl

    monkeypatch.setenv("STK_GRAPHS", "0")  # direct issue: the copies themselves are exercised
    w = wl.config_thomas(seed=8, n=25_000)
    s2, tt2 = w.s[: len(w.s) // 2], w.tt  # a smaller s_max: another grid
    with stk.Pattern(w.x, w.y, w.t, w.box) as fresh:
        want = fresh.run(w.s, w.tt, n_sims=4, seed=3, prec=prec, want_sims=True)
        want2 = fresh.run(s2, tt2, n_sims=2, seed=5, prec=prec)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        first = p.run(w.s, w.tt, n_sims=4, seed=3, prec=prec, want_sims=True)
        assert p.stats()["obs_index_reused"] == 0
        again = p.run(w.s, w.tt, n_sims=4, seed=3, prec=prec, want_sims=True)
        assert p.stats()["obs_index_reused"] == 1
        obs_only = p.run(w.s, w.tt, prec=prec)  # a wave of the observed pattern alone
        assert p.stats()["obs_index_reused"] == 1
        other = p.run(s2, tt2, n_sims=2, seed=5, prec=prec)
        assert p.stats()["obs_index_reused"] == 0
        vx, vy = np.array([0.0, 10_000.0, 10_000.0, 0.0]), np.array([0.0, 0.0, 10_000.0, 10_000.0])
        p.run(w.s, w.tt, prec=prec)
        p.set_polygon(vx, vy)  # the same square as a polygon: records change, index rebuilt
        p.run(w.s, w.tt, prec=prec)
        assert p.stats()["obs_index_reused"] == 0
    _same(first, want)
    _same(again, want)
    _same(other, want2)
    for k in ("K", "L", "S", "C"):
        np.testing.assert_array_equal(obs_only[k], want[k], err_msg=k)
