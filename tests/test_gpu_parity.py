"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: ordered-pair counts bit-exact in both precisions; K, raw sums (and L through K) within
relative 1e-9 (STK_PREC_FP64) or 1e-6 (STK_PREC_FP32_GUARDED) per grid cell, absolute where
the oracle's value is 0.  Inputs are seeded synthetic patterns from workloads.py.
"""
import math

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


@pytest.fixture(scope="module")
def wl():
    from paper_1912_04753_gb300 import workloads

    return workloads


def rel_err(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    den = np.where(want == 0, 1.0, np.abs(want))
    return np.abs(got - want) / den


def assert_grids(got, want, prec, what=""):
    np.testing.assert_array_equal(got["C"], want["C"], err_msg=f"counts {what}")
    tol = TOL[prec]
    for key in ("S", "K"):
        e = rel_err(got[key], want[key])
        assert e.max() <= tol, f"{what} {key} max rel err {e.max():.3e} > {tol}"
    # L + s = sqrt(K / (2 pi t)): relative tolerance on that
    s_col = None
    if "s" in want:
        s_col = want["s"][:, None]
    if s_col is not None:
        e = rel_err(got["L"] + s_col, want["L"] + s_col)
        assert e.max() <= tol, f"{what} L max rel err {e.max():.3e}"


def oracle_k(orc, x, y, t, box, s, tt, edge=1, norm=0):
    o = orc.k_function(x, y, t, box, s, tt, edge_mode=edge, norm=norm)
    o["s"] = np.asarray(s, np.float64)
    return o


# ------------------------------------------------------------------------------ generation


def test_device_csr_points_bit_exact(stk, orc):
    box = (-120.5, 880.25, 3.0, 1003.0, 10.0, 375.0)
    seed = (0xDEADBEEF << 32) | 12345
    for sim in (0, 1, 77):
        gx, gy, gt = stk.stk_sim_points(box, 3001, seed, sim)
        ox, oy, ot = orc.csr_points(3001, box, seed, sim)
        np.testing.assert_array_equal(gx, ox)
        np.testing.assert_array_equal(gy, oy)
        np.testing.assert_array_equal(gt, ot)


# ------------------------------------------------------------------------------ observed K


@pytest.mark.parametrize("prec", [0, 1])
def test_csr_small_config(stk, orc, wl, prec):
    w = wl.config_csr_small(seed=0)
    want = oracle_k(orc, w.x, w.y, w.t, w.box, w.s, w.tt)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        got = p.k(w.s, w.tt, prec=prec)
        assert_grids(got, want, prec, "csr n=2000")
        st = p.stats()
        assert st["qualifying_pairs"] == int(want["C"][-1, -1])
        assert st["internal_errors"] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_clustered_heavy_cells(stk, orc, wl, prec):
    # one tight cluster of 4000 points puts > 256 centres (several work items) and > 1024
    # neighbours (several staged chunks) into one cell, plus a Thomas background
    rng = np.random.default_rng(5)
    box = (0.0, 5000.0, 0.0, 4000.0, 0.0, 200.0)
    x1, y1, t1 = wl.thomas(3000, box, 12, 80.0, 5.0, rng)
    cx = np.clip(rng.normal(2500.0, 15.0, 4000), 0, 5000)
    cy = np.clip(rng.normal(10.0, 15.0, 4000), 0, 4000)  # hugs the bottom edge
    ct = np.clip(rng.normal(3.0, 2.0, 4000), 0, 200)  # hugs the start of the period
    x, y, t = np.r_[x1, cx], np.r_[y1, cy], np.r_[t1, ct]
    s = wl.even_thresholds(400.0, 12)
    tt = wl.even_thresholds(20.0, 9)
    want = oracle_k(orc, x, y, t, box, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        assert_grids(p.k(s, tt, prec=prec), want, prec, "clustered")


@pytest.mark.parametrize("prec", [0, 1])
def test_poi_shaped_integer_seconds(stk, orc, wl, prec):
    # POI mixture, timestamps floored to seconds and thresholds that are whole seconds: many
    # exact ties u == t_b, all of which FP32 must hand to FP64
    rng = np.random.default_rng(9)
    box = (0.0, 8000.0, 0.0, 8000.0, 0.0, 400 * wl.DAY)
    x, y, t = wl.poi_mixture(9000, box, 40, rng, sigma_s=120.0, sigma_t_s=4 * wl.DAY)
    s = wl.even_thresholds(640.0, 8)
    tt = np.array([86400.0 * b for b in range(1, 11)])
    want = oracle_k(orc, x, y, t, box, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        got = p.k(s, tt, prec=prec)
        assert_grids(got, want, prec, "poi seconds")


@pytest.mark.parametrize("prec", [0, 1])
def test_dyadic_exact_ties_and_boundary_points(stk, orc, prec):
    # coordinates on a 1/4 grid, thresholds on the same grid: d == s and u == t happen often;
    # points on edges and corners of the box (e = 0)
    rng = np.random.default_rng(17)
    n = 2500
    P = rng.integers(0, 4 * 64, size=(n, 3)) / 4.0
    P[:40, 0] = 0.0
    P[40:80, 1] = 64.0
    P[80:90, :2] = 0.0
    P[90:100, 2] = 64.0
    box = (0.0, 64.0, 0.0, 64.0, 0.0, 64.0)
    s = np.array([0.5, 1.0, 2.0, 2.25, 5.0, 8.0, 13.0])
    tt = np.array([0.25, 1.0, 3.0, 4.0, 9.5])
    want = oracle_k(orc, P[:, 0], P[:, 1], P[:, 2], box, s, tt)
    with stk.Pattern(P[:, 0], P[:, 1], P[:, 2], box) as p:
        assert_grids(p.k(s, tt, prec=prec), want, prec, "dyadic ties")


@pytest.mark.parametrize("prec", [0, 1])
def test_offset_box_and_uneven_thresholds(stk, orc, wl, prec):
    # projected coordinates far from the origin stress the FP32 frames
    box = (512_345.5, 517_345.5, 3_301_000.0, 3_305_000.0, 7300.0, 7665.0)
    x, y, t = wl.csr(3000, box, 21)
    s = np.array([3.0, 17.5, 40.0, 41.0, 200.0, 333.3, 900.0, 1999.0])
    tt = np.array([0.01, 0.5, 2.0, 7.25, 30.0])
    want = oracle_k(orc, x, y, t, box, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        assert_grids(p.k(s, tt, prec=prec), want, prec, "offset box")


@pytest.mark.parametrize("prec", [0, 1])
def test_degenerate_patterns(stk, orc, prec):
    box = (0.0, 10.0, 0.0, 10.0, 0.0, 10.0)
    s, tt = np.array([0.5, 2.0]), np.array([1.0, 3.0])
    # n = 2, coincident
    x, y, t = np.array([3.0, 3.0]), np.array([4.0, 4.0]), np.array([5.0, 5.0])
    with stk.Pattern(x, y, t, box) as p:
        got = p.k(s, tt, prec=prec)
    assert (got["C"] == 2).all()
    assert_grids(got, oracle_k(orc, x, y, t, box, s, tt), prec, "n=2")
    # every point at one location on a corner (one cell holds everything)
    n = 700
    x, y, t = np.zeros(n), np.zeros(n), np.zeros(n)
    with stk.Pattern(x, y, t, box) as p:
        got = p.k(s, tt, prec=prec)
    assert (got["C"] == n * (n - 1)).all()
    assert_grids(got, oracle_k(orc, x, y, t, box, s, tt), prec, "coincident corner")
    # no qualifying pair at all
    x, y, t = np.array([0.0, 10.0, 0.0]), np.array([0.0, 10.0, 10.0]), np.array([0.0, 10.0, 5.0])
    with stk.Pattern(x, y, t, box) as p:
        got = p.k(s, tt, prec=prec)
    assert (got["C"] == 0).all() and (got["K"] == 0).all()
    np.testing.assert_allclose(got["L"], -np.repeat(s[:, None], 2, axis=1), rtol=0, atol=0)


_REFINE_CASE = {}


def _refine_case(orc, wl):
    # clustered data near the edges and the period's end, computed once for all refinements
    if not _REFINE_CASE:
        rng = np.random.default_rng(31)
        box = (0.0, 6000.0, 0.0, 5000.0, 0.0, 300.0)
        x, y, t = wl.thomas(12000, box, 30, 150.0, 8.0, rng)
        s = wl.even_thresholds(450.0, 9)
        tt = wl.even_thresholds(24.0, 8)
        _REFINE_CASE.update(x=x, y=y, t=t, box=box, s=s, tt=tt,
                            want=oracle_k(orc, x, y, t, box, s, tt))
    return _REFINE_CASE


@pytest.mark.parametrize("fs,ft", [(1, 1), (2, 2), (3, 3), (2, 3), (3, 1), (1, 2)])
@pytest.mark.parametrize("prec", [0, 1])
def test_every_grid_refinement(stk, orc, wl, prec, fs, ft, monkeypatch):
    # cells of s_max/fs x t_max/ft: each refinement walks a different neighbourhood in a
    # different cell frame and must give the same grids
    monkeypatch.setenv("STK_GRID_F", str(fs))
    monkeypatch.setenv("STK_GRID_FT", str(ft))
    c = _refine_case(orc, wl)
    with stk.Pattern(c["x"], c["y"], c["t"], c["box"]) as p:
        assert_grids(p.k(c["s"], c["tt"], prec=prec), c["want"], prec, f"f={fs},{ft}")
        st = p.stats()
        assert (st["grid_refinement"], st["grid_refinement_t"]) == (fs, ft)
        assert st["internal_errors"] == 0


@pytest.mark.parametrize("tile,bps", [(8, 2), (32, 2), (64, 2), (1, 2), (16, 3), (64, 3)])
def test_every_launch_shape(stk, orc, wl, tile, bps, monkeypatch):
    # the FP32 kernel's launch shape (units per tile claim, blocks per SM with the matching
    # register allocation) changes only the schedule: the accumulators are exact integers, so
    # every shape gives the default shape's grids bit for bit, and the oracle's
    c = _refine_case(orc, wl)
    with stk.Pattern(c["x"], c["y"], c["t"], c["box"]) as p:
        monkeypatch.setenv("STK_GRID_F", "2")
        ref = p.run(c["s"], c["tt"], n_sims=3, seed=11, prec=1, want_sims=True)
        st0 = p.stats()
        assert (st0["tile_units"], st0["blocks_per_sm"]) == (16, 2)
        monkeypatch.setenv("STK_TILE_UNITS", str(tile))
        monkeypatch.setenv("STK_BLOCKS_PER_SM", str(bps))
        got = p.run(c["s"], c["tt"], n_sims=3, seed=11, prec=1, want_sims=True)
        st = p.stats()
    assert st["tile_units"] == tile
    assert st["blocks_per_sm"] in ((3,) if bps == 3 else (2,))
    assert st["internal_errors"] == 0
    for key in ("K", "L", "S", "C", "K_sims", "C_sims", "K_lo", "K_hi"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    assert_grids(got, c["want"], 1, f"tile={tile}, bps={bps}")


def test_tuned_refinement_gives_the_same_job(stk, wl, monkeypatch):
    # a batched job large enough to be tuned: the tuner's choice (1..3) must not change counts,
    # and K stays within the FP32 tolerance of the planner's grid
    rng = np.random.default_rng(8)
    box = (0.0, 20000.0, 0.0, 20000.0, 0.0, 365.0)
    x, y, t = wl.thomas(300000, box, 300, 150.0, 10.0, rng)
    s, tt = wl.even_thresholds(600.0, 10), wl.even_thresholds(30.0, 10)
    with stk.Pattern(x, y, t, box) as p:
        monkeypatch.setenv("STK_TUNE", "0")
        ref = p.run(s, tt, n_sims=80, seed=5, want_sims=True)
        f_plan = p.stats()["grid_refinement"]
        monkeypatch.setenv("STK_TUNE", "1")
        got = p.run(s, tt, n_sims=80, seed=5, want_sims=True)
        st = p.stats()
        # a job of the same shape too small to be tuned takes the tuned launch shape
        p.run(s, tt, n_sims=2, seed=6)
        st_small = p.stats()
    assert st["grid_refinement"] in (1, 2, 3) and st["grid_refinement_t"] in (1, 2, 3)
    assert st["tile_units"] in (8, 16, 32, 64) and st["blocks_per_sm"] in (2, 3)
    shape = ("grid_refinement", "grid_refinement_t", "tile_units", "blocks_per_sm")
    assert [st_small[k] for k in shape] == [st[k] for k in shape]
    assert f_plan in (1, 2)
    np.testing.assert_array_equal(got["C"], ref["C"])
    np.testing.assert_array_equal(got["C_sims"], ref["C_sims"])
    assert rel_err(got["K_sims"], ref["K_sims"]).max() <= 1e-6
    assert rel_err(got["K"], ref["K"]).max() <= 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_shapes_and_modes(stk, orc, wl, prec):
    w = wl.config_csr_small(seed=4, n=1500)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        # one threshold per axis
        s1, t1 = np.array([60.0]), np.array([12.0])
        assert_grids(p.k(s1, t1, prec=prec), oracle_k(orc, w.x, w.y, w.t, w.box, s1, t1), prec,
                     "1x1")
        # the maximum grid, 64 x 64
        s64 = wl.even_thresholds(120.0, 64)
        t64 = wl.even_thresholds(40.0, 64)
        assert_grids(p.k(s64, t64, prec=prec), oracle_k(orc, w.x, w.y, w.t, w.box, s64, t64),
                     prec, "64x64")
        # no edge correction: S equals C exactly
        got = p.k(w.s, w.tt, prec=prec, edge_mode=0)
        np.testing.assert_array_equal(got["S"], got["C"].astype(np.float64))
        assert_grids(got, oracle_k(orc, w.x, w.y, w.t, w.box, w.s, w.tt, edge=0), prec, "none")
        # A*D/n^2 normalisation
        assert_grids(p.k(w.s, w.tt, prec=prec, norm=1),
                     oracle_k(orc, w.x, w.y, w.t, w.box, w.s, w.tt, norm=1), prec, "n^2")


@pytest.mark.parametrize("prec", [0, 1])
def test_sampled_centre_mode(stk, orc, wl, prec):
    w = wl.config_csr_small(seed=8, n=3000)
    mask = np.zeros(w.n, np.uint8)
    mask[np.random.default_rng(1).choice(w.n, 211, replace=False)] = 1
    cnt, wsum, _ = orc.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, centre_mask=mask)
    C, S, K, L = orc.finalize(w.n, w.box, w.s, w.tt, cnt, wsum)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        got = p.run(w.s, w.tt, centre_mask=mask, prec=prec)
    assert_grids(got, {"C": C, "S": S, "K": K, "L": L, "s": w.s}, prec, "masked")


# ------------------------------------------------------------------------------ envelopes


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("exec_mode", [0, 1])
def test_envelope_config1(stk, orc, wl, prec, exec_mode):
    w = wl.config_csr_small(seed=0)
    seed = 2024
    env = orc.envelope(w.n, w.box, w.s, w.tt, w.n_sims, seed, keep_all=True)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        got = p.run(w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=prec, exec_mode=exec_mode,
                    want_sims=True)
    tol = TOL[prec]
    for k in range(w.n_sims):
        x, y, t = orc.csr_points(w.n, w.box, seed, k)
        want = orc.k_function(x, y, t, w.box, w.s, w.tt)
        np.testing.assert_array_equal(got["C_sims"][k], want["C"], err_msg=f"sim {k}")
        assert rel_err(got["K_sims"][k], env["K_all"][k]).max() <= tol
    for key in ("K_lo", "K_hi"):
        assert rel_err(got[key], env[key]).max() <= tol
    for key in ("L_lo", "L_hi"):
        assert rel_err(got[key] + w.s[:, None], env[key] + w.s[:, None]).max() <= tol


def test_envelope_entry_point_and_batched_equals_plain(stk, wl):
    w = wl.config_csr_small(seed=1, n=2500)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        a = p.run(w.s, w.tt, n_sims=9, seed=5, exec_mode=0, want_sims=True)
        b = p.run(w.s, w.tt, n_sims=9, seed=5, exec_mode=1, want_sims=True)
        e = p.envelope(w.s, w.tt, 9, 5)
    # integer accumulation: batched and per-realization launches agree bit for bit
    for key in ("C", "S", "K", "C_sims", "K_sims", "K_lo", "K_hi"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    for key in ("K_lo", "K_hi", "L_lo", "L_hi"):
        np.testing.assert_array_equal(e[key], a[key], err_msg=key)


def test_fp32_and_fp64_paths_agree_on_thomas(stk, wl):
    w = wl.config_thomas(seed=2, n=60_000)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        a = p.run(w.s, w.tt, n_sims=3, seed=9, prec=1, want_sims=True)
        sa = p.stats()
        b = p.run(w.s, w.tt, n_sims=3, seed=9, prec=0, want_sims=True)
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["C_sims"], b["C_sims"])
    assert rel_err(a["K"], b["K"]).max() <= 1e-6
    assert rel_err(a["K_sims"], b["K_sims"]).max() <= 1e-6
    assert sa["fp64_recomputed"] < 1e-2 * sa["qualifying_pairs"]


# ------------------------------------------------------------------------------ errors


def test_invalid_requests_are_rejected(stk, wl):
    w = wl.config_csr_small(seed=0, n=200)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        bad = [
            (np.array([10.0, 5.0]), w.tt),  # not increasing
            (np.array([0.0, 5.0]), w.tt),  # zero threshold
            (np.array([600.0]), w.tt),  # > half the box side
            (wl.even_thresholds(100.0, 65), w.tt),  # too many
            (w.s, np.array([np.nan])),
        ]
        for s, tt in bad:
            with pytest.raises(stk.StkError) as e:
                p.k(s, tt)
            assert e.value.code == 1
        # the handle still works afterwards
        assert p.k(w.s, w.tt)["C"].shape == (10, 10)
