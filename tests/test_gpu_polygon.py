"""Polygon study areas (Sections 3 and 6: the paper's experiments use an 85-vertex outline):
CSR realizations in the polygon bit-identical to the oracle's, and K grids and envelopes over
a polygon within the parity bar (counts exact; K relative 1e-9 in FP64, 1e-6 in FP32)."""
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


def _star(nv, r0, r1, cx, cy, seed):
    rng = np.random.default_rng(seed)
    th = np.sort(rng.uniform(0, 2 * np.pi, nv))
    rad = np.where(np.arange(nv) % 2 == 0, r0, r1) * rng.uniform(0.85, 1.0, nv)
    return cx + rad * np.cos(th), cy + rad * np.sin(th)


def _pattern(orc, box, vx, vy, n, seed):
    # clustered points inside the polygon: CSR in it plus jittered copies, kept if inside
    x, y, t = orc.csr_polygon_points(n, box, vx, vy, seed, 0)
    rng = np.random.default_rng(seed)
    k = n // 3
    jx = x[:k] + rng.normal(0, 25.0, k)
    jy = y[:k] + rng.normal(0, 25.0, k)
    keep = np.array([orc.point_in_polygon(a, b, vx, vy) for a, b in zip(jx, jy)])
    x = np.r_[x, jx[keep]]
    y = np.r_[y, jy[keep]]
    t = np.r_[t, np.clip(t[:k][keep] + rng.normal(0, 2.0, keep.sum()), box[4], box[5])]
    return x, y, t


def test_csr_in_polygon_bit_exact(stk, orc):
    vx, vy = _star(85, 1000.0, 600.0, 1200.0, 1100.0, 1)
    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    for n, seed, sim in ((1, 0, 0), (5000, 3, 1), (120000, 2**50 + 1, 9)):
        got = stk.stk_sim_points_polygon(box, vx, vy, n, seed, sim)
        want = orc.csr_polygon_points(n, box, vx, vy, seed, sim)
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("nv", [24, 85])
@pytest.mark.parametrize("prec", [0, 1])
def test_observed_k_in_polygon(stk, orc, nv, prec):
    vx, vy = _star(nv, 1000.0, 600.0, 1200.0, 1100.0, nv)
    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    x, y, t = _pattern(orc, box, vx, vy, 3000, 7 + nv)
    s, tt = np.linspace(40.0, 320.0, 8), np.linspace(5.0, 40.0, 6)
    want = orc.k_function_polygon(x, y, t, box, vx, vy, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        p.set_polygon(vx, vy)
        got = p.k(s, tt, prec=prec)
        assert p.stats()["internal_errors"] == 0
        np.testing.assert_array_equal(got["C"], want["C"])
        assert _rel(got["S"], want["S"]).max() <= TOL[prec]
        assert _rel(got["K"], want["K"]).max() <= TOL[prec]
        # back to the box: the rectangle's estimator again
        p.set_polygon(None)
        box_k = orc.k_function(x, y, t, box, s, tt)
        assert _rel(p.k(s, tt, prec=prec)["K"], box_k["K"]).max() <= TOL[prec]


@pytest.mark.parametrize("method", [0, 1])
def test_envelope_in_polygon(stk, orc, method):
    vx, vy = _star(40, 1000.0, 650.0, 1200.0, 1100.0, 3)
    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    x, y, t = _pattern(orc, box, vx, vy, 2000, 11)
    s, tt = np.linspace(50.0, 250.0, 5), np.linspace(6.0, 36.0, 6)
    sims, seed = 5, 17
    want = orc.envelope_of(method, x, y, t, box, s, tt, sims, seed, polygon=(vx, vy))
    with stk.Pattern(x, y, t, box) as p:
        p.set_polygon(vx, vy)
        got = p.run(s, tt, n_sims=sims, seed=seed, sim_method=method, want_sims=True)
    for k in range(sims):
        assert _rel(got["K_sims"][k], want["K_all"][k]).max() <= TOL[1]
    for key in ("K_lo", "K_hi"):
        assert _rel(got[key], want[key]).max() <= TOL[1], key
    for key in ("L_lo", "L_hi"):  # L through L + s = sqrt(K / (2 pi t)), as K
        assert _rel(got[key] + s[:, None], want[key] + s[:, None]).max() <= TOL[1], key


def test_polygon_arguments_checked(stk, orc):
    box = (0.0, 100.0, 0.0, 100.0, 0.0, 10.0)
    x, y, t = np.array([10.0, 90.0, 50.0]), np.array([10.0, 90.0, 50.0]), np.array([1.0, 2, 3])
    with stk.Pattern(x, y, t, box) as p:
        with pytest.raises(stk.StkError) as e:  # (90, 90) is outside this triangle
            p.set_polygon([0.0, 100.0, 0.0], [0.0, 0.0, 100.0])
        assert e.value.code == stk.STK_EDOMAIN
        with pytest.raises(stk.StkError) as e:  # too small a share of the box
            p.set_polygon([0.0, 10.0, 0.0], [0.0, 0.0, 10.0])
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:  # a vertex outside the box
            p.set_polygon([0.0, 200.0, 100.0, 0.0], [0.0, 0.0, 100.0, 100.0])
        assert e.value.code == stk.STK_EINVAL
        p.set_polygon([0.0, 100.0, 100.0, 0.0], [0.0, 0.0, 100.0, 100.0])  # the box itself
        assert p.k(np.array([30.0]), np.array([5.0]))["C"][0, 0] >= 0
        with pytest.raises(stk.StkError) as e:  # cross K takes the rectangle only
            p.run(np.array([30.0]), np.array([5.0]), labels=np.zeros(3, np.uint8), cross=(0, 0))
        assert e.value.code == stk.STK_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_k_and_envelope_in_smooth_outline(stk, orc, prec):
    """An outline without spikes (about two boundary crossings per circle), where the FP32
    kernel takes its FP32-guarded polygon weights (poly_share_f32) rather than FP64 ones."""
    from paper_1912_04753_gb300 import workloads as wl

    vx, vy = wl.smooth_polygon(60, 800.0, 1200.0, 1100.0, 4)
    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    x, y, t = _pattern(orc, box, vx, vy, 3000, 21)
    s, tt = np.linspace(40.0, 320.0, 8), np.linspace(5.0, 40.0, 6)
    want = orc.k_function_polygon(x, y, t, box, vx, vy, s, tt)
    sims, seed = 4, 29
    env = orc.envelope_of(0, x, y, t, box, s, tt, sims, seed, polygon=(vx, vy))
    with stk.Pattern(x, y, t, box) as p:
        p.set_polygon(vx, vy)
        got = p.run(s, tt, n_sims=sims, seed=seed, prec=prec, want_sims=True)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], want["C"])
    assert _rel(got["S"], want["S"]).max() <= TOL[prec]
    assert _rel(got["K"], want["K"]).max() <= TOL[prec]
    for k in range(sims):
        assert _rel(got["K_sims"][k], env["K_all"][k]).max() <= TOL[prec]


def test_largest_threshold_grid_in_polygon(stk, orc):
    """The largest threshold grid (64 x 64 bins) in a polygon, FP32-guarded, with simulations:
    the polygon kernel keeps a second histogram set in shared memory (realizations of either
    parity have their own), which at this grid takes it to one block per SM; every
    realization's K at the parity bar against the oracle, the observed counts exact."""
    vx, vy = _star(85, 1000.0, 600.0, 1200.0, 1100.0, 85)
    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    x, y, t = _pattern(orc, box, vx, vy, 1500, 5)
    s, tt = np.linspace(5.0, 320.0, 64), np.linspace(0.7, 45.0, 64)
    sims, seed = 5, 23
    want = orc.envelope_of(0, x, y, t, box, s, tt, sims, seed, polygon=(vx, vy))
    obs = orc.k_function_polygon(x, y, t, box, vx, vy, s, tt)
    with stk.Pattern(x, y, t, box) as p:
        p.set_polygon(vx, vy)
        got = p.run(s, tt, n_sims=sims, seed=seed, want_sims=True)
        assert p.stats()["internal_errors"] == 0
    np.testing.assert_array_equal(got["C"], obs["C"])
    assert _rel(got["K"], obs["K"]).max() <= TOL[1]
    for k in range(sims):
        assert _rel(got["K_sims"][k], want["K_all"][k]).max() <= TOL[1]
