"""Serving loop (include/stk.h, stk_server_*): results through the server equal the same job
run alone through stk_run, whether the job ran alone, merged with other jobs into one batch,
beside jobs on other point sets, or in memory-limited waves; served grids match the oracle;
admission refuses what can never fit and keeps serving the rest."""
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


def _sets():
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(5)
    box_a = (0.0, 1000.0, 0.0, 1000.0, 0.0, 365.0)
    a = wl.csr(3000, box_a, 11) + (box_a,)
    box_b = (0.0, 4000.0, 0.0, 4000.0, 0.0, 365.0)
    b = wl.thomas(20000, box_b, 40, 120.0, 8.0, rng) + (box_b,)
    box_c = (0.0, 6000.0, 0.0, 6000.0, 0.0, 365.0 * 86400.0)
    c = wl.poi_mixture(40000, box_c, 60, rng, sigma_s=150.0, sigma_t_s=10.0 * 86400.0)
    c = tuple(np.floor(v) if k == 2 else v for k, v in enumerate(c)) + (box_c,)
    return [a, b, c]


def _alone(stk, pts, job):
    x, y, t, box = pts
    with stk.Pattern(x, y, t, box) as p:
        return p.run(job["s"], job["tt"], n_sims=job["n_sims"], seed=job["seed"],
                     prec=job.get("prec", stk.STK_PREC_FP32_GUARDED), want_sims=True)


def _same(got, want, what):
    for k in want:
        if k == "L":  # NaN-free here; compare bitwise like the rest
            pass
        np.testing.assert_array_equal(got[k], want[k], err_msg=f"{what}: {k}")


def test_served_equals_alone_merged_and_mixed(stk):
    from paper_1912_04753_gb300 import workloads as wl

    sets = _sets()
    sa, ta = wl.even_thresholds(80.0, 8), wl.even_thresholds(20.0, 6)
    sb, tb = wl.even_thresholds(400.0, 12), wl.even_thresholds(30.0, 9)
    sc, tc = wl.even_thresholds(500.0, 10), wl.even_thresholds(30.0 * 86400.0, 10)
    jobs = [
        # a blocker on A with its own grid, so the next three queue up and merge
        dict(d=0, s=wl.even_thresholds(100.0, 5), tt=tb[:5], n_sims=40, seed=1),
        dict(d=0, s=sa, tt=ta, n_sims=7, seed=101),
        dict(d=0, s=sa, tt=ta, n_sims=0, seed=0),
        dict(d=0, s=sa, tt=ta, n_sims=12, seed=(7 << 40) + 3),
        dict(d=1, s=sb, tt=tb, n_sims=5, seed=5),
        dict(d=1, s=sb, tt=tb, n_sims=9, seed=6),
        dict(d=2, s=sc, tt=tc, n_sims=4, seed=77),
        dict(d=2, s=sc, tt=tc, n_sims=3, seed=77, prec=stk.STK_PREC_FP64),
        dict(d=1, s=sb[:4], tt=tb, n_sims=2, seed=9),
    ]
    with stk.Server(slots=3) as sv:
        ids = [sv.register(*p) for p in sets]
        tickets = []
        for j in jobs:
            tickets.append(sv.submit(ids[j["d"]], j["s"], j["tt"], n_sims=j["n_sims"],
                                     seed=j["seed"], want_sims=True,
                                     prec=j.get("prec", stk.STK_PREC_FP32_GUARDED)))
        served = [sv.poll(tk, wait_ms=120000) for tk in tickets]
        st = sv.stats()
    assert all(r is not None for r in served)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["merged_jobs"] >= 2, st
    assert st["batches"] < len(jobs)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for k, (j, (got, lat)) in enumerate(zip(jobs, served)):
        assert lat > 0
        want = _alone(stk, sets[j["d"]], j)
        _same(got, want, f"job {k}")


def test_served_matches_oracle(stk, orc):
    from paper_1912_04753_gb300 import workloads as wl

    x, y, t, box = _sets()[1]
    s, tt = wl.even_thresholds(300.0, 7), wl.even_thresholds(25.0, 5)
    with stk.Server(slots=2) as sv:
        d = sv.register(x, y, t, box)
        t32 = sv.submit(d, s, tt)
        t64 = sv.submit(d, s, tt, prec=stk.STK_PREC_FP64)
        g32, _ = sv.poll(t32)
        g64, _ = sv.poll(t64)
    want = orc.k_function(x, y, t, box, s, tt)
    for got, tol in ((g32, 1e-6), (g64, 1e-9)):
        np.testing.assert_array_equal(got["C"], want["C"])
        for k in ("S", "K"):
            den = np.where(want[k] == 0, 1.0, np.abs(want[k]))
            assert (np.abs(got[k] - want[k]) / den).max() <= tol


def test_admission_by_memory(stk):
    from paper_1912_04753_gb300 import workloads as wl

    box = (0.0, 1000.0, 0.0, 1000.0, 0.0, 365.0)
    small = wl.csr(2000, box, 3)
    big_box = (0.0, 20000.0, 0.0, 20000.0, 0.0, 365.0)
    big = wl.csr(200000, big_box, 4)
    s, tt = wl.even_thresholds(50.0, 6), wl.even_thresholds(10.0, 4)
    # point sets + about 6 MB: the small job runs in waves, the big one can never start
    budget = 24 * (2000 + 200000) + (6 << 20)
    with stk.Server(slots=2, mem_budget_bytes=budget) as sv:
        ds = sv.register(*small, box)
        db = sv.register(*big, big_box)
        tb = sv.submit(db, wl.even_thresholds(500.0, 6), tt, n_sims=3, seed=1)
        t1 = sv.submit(ds, s, tt, n_sims=60, seed=42, want_sims=True)
        with pytest.raises(stk.StkError) as e:
            sv.poll(tb)
        assert e.value.code == stk.STK_ENOMEM
        got, _ = sv.poll(t1)
        st = sv.stats()
        assert st["peak_bytes"] <= budget
        # the queue keeps working after the refusal
        t2 = sv.submit(ds, s, tt, n_sims=2, seed=43)
        assert sv.poll(t2) is not None
    want = _alone(stk, small + (box,), dict(s=s, tt=tt, n_sims=60, seed=42))
    _same(got, want, "memory-limited job")


def test_request_errors(stk):
    from paper_1912_04753_gb300 import workloads as wl

    box = (0.0, 1000.0, 0.0, 1000.0, 0.0, 365.0)
    x, y, t = wl.csr(500, box, 1)
    with stk.Server(slots=1) as sv:
        d = sv.register(x, y, t, box)
        with pytest.raises(stk.StkError) as e:
            sv.submit(d + 100, [10.0], [1.0])
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            sv.submit(d, [10.0, 5.0], [1.0])  # not increasing
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            sv.submit(d, [600.0], [1.0])  # beyond half the side
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            stk.stk_poll(sv.sv, 123456, 1, 1)
        assert e.value.code == stk.STK_EINVAL
        tk = sv.submit(d, [10.0, 20.0], [1.0, 2.0], n_sims=30, seed=3)
        r = sv.poll(tk, wait_ms=0)  # usually still running; a finished job is fine too
        if r is None:
            r = sv.poll(tk, wait_ms=60000)
        assert r is not None
        sv.unregister(d)
        with pytest.raises(stk.StkError):
            sv.submit(d, [10.0], [1.0])


def test_served_polygon_and_intensity(stk, orc):
    # a registered point set with a polygon study area, another with an intensity: the served
    # grids equal the handle's own
    from paper_1912_04753_gb300 import workloads as wl

    box = (0.0, 2400.0, 0.0, 2200.0, 0.0, 365.0)
    vx, vy = wl.star_polygon(24, 1000.0, 650.0, 1200.0, 1100.0, 3)
    x, y, t = orc.csr_polygon_points(1500, box, vx, vy, 4, 0)
    s, tt = wl.even_thresholds(200.0, 5), wl.even_thresholds(30.0, 4)
    rho = wl.histogram_intensity(x, y, t, box, (2, 3, 3))
    with stk.Server(slots=2) as sv:
        dp = sv.register(x, y, t, box)
        di = sv.register(x, y, t, box)
        sv.set_polygon(dp, vx, vy)
        sv.set_intensity(di, rho)
        gp, _ = sv.poll(sv.submit(dp, s, tt, n_sims=2, seed=3))
        gi, _ = sv.poll(sv.submit(di, s, tt, n_sims=2, seed=3))
        with pytest.raises(stk.StkError) as e:
            sv.set_polygon(999, vx, vy)
        assert e.value.code == stk.STK_EINVAL
    with stk.Pattern(x, y, t, box) as p:
        p.set_polygon(vx, vy)
        wp = p.run(s, tt, n_sims=2, seed=3)
        p.set_polygon(None)
        p.set_intensity(rho)
        wi = p.run(s, tt, n_sims=2, seed=3)
    for got, want in ((gp, wp), (gi, wi)):
        for k in ("C", "K", "K_lo", "K_hi"):
            np.testing.assert_array_equal(got[k], want[k])
