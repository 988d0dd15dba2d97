"""Several jobs on different point sets with one persistent pair launch (stk_run_fused,
include/stk.h): every job equals the same job run alone through stk_run bit for bit (the sums
are exact fixed-point integers and a job takes its problem shape's grid either way), the
observed grids match the FP64 oracle at the FP32-guarded bar, jobs of one kernel class share
one pair launch, jobs that cannot share it run alone with the same results, and bad arguments
are refused with the handles still usable."""
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
    """Point sets of different sizes, shapes and boxes (CSR, clusters on an offset box, a
    POI-like mixture in whole seconds)."""
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(17)
    box_a = (0.0, 1000.0, 0.0, 1000.0, 0.0, 365.0)
    a = wl.csr(2500, box_a, 3) + (box_a,)
    box_b = (5.0e5, 5.04e5, 3.3e6, 3.303e6, 0.0, 200.0)
    xb, yb, tb = wl.thomas(9000, (0.0, 4000.0, 0.0, 3000.0, 0.0, 200.0), 25, 100.0, 6.0, rng)
    b = (xb + 5.0e5, yb + 3.3e6, tb, box_b)
    box_c = (0.0, 6000.0, 0.0, 6000.0, 0.0, 365.0 * 86400.0)
    c = wl.poi_mixture(15000, box_c, 40, rng, sigma_s=150.0, sigma_t_s=10.0 * 86400.0)
    c = tuple(np.floor(v) if k == 2 else v for k, v in enumerate(c)) + (box_c,)
    box_d = (0.0, 2000.0, 0.0, 500.0, 0.0, 100.0)
    d = wl.csr(1200, box_d, 9) + (box_d,)
    return [a, b, c, d]


def _jobs(stk):
    from paper_1912_04753_gb300 import workloads as wl

    return [
        dict(s=wl.even_thresholds(80.0, 8), tt=wl.even_thresholds(20.0, 6), n_sims=7, seed=1,
             want_sims=True),
        dict(s=wl.even_thresholds(300.0, 12), tt=wl.even_thresholds(25.0, 9), n_sims=0, seed=2),
        dict(s=wl.even_thresholds(500.0, 10), tt=wl.even_thresholds(30.0 * 86400.0, 10),
             n_sims=4, seed=3, want_sims=True),
        dict(s=wl.even_thresholds(120.0, 5), tt=wl.even_thresholds(10.0, 5), n_sims=12, seed=4,
             edge_mode=stk.STK_EDGE_NONE, want_sims=True),
    ]


def _same(got, want, what):
    assert sorted(got) == sorted(want), what
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=f"{what}: {k}")


def _alone(stk, pts, job):
    x, y, t, box = pts
    with stk.Pattern(x, y, t, box) as p:
        out = p.run(**job)
        return out, p.stats()


def test_fused_jobs_equal_jobs_alone_and_the_oracle(stk, orc):
    sets, jobs = _sets(), _jobs(stk)
    alone = [_alone(stk, pts, job) for pts, job in zip(sets, jobs)]
    pats = [stk.Pattern(*pts) for pts in sets]
    try:
        for rep in range(2):  # the second run reuses every handle's workspace
            res, launches = stk.stk_run_fused([p.h for p in pats], jobs)
            # one kernel class (even thresholds; edge correction or not is a class of its own)
            assert launches == 2, launches
            for i, (got, (want, st_alone)) in enumerate(zip(res, alone)):
                _same(got, want, f"job {i} run {rep}")
                st = pats[i].stats()
                assert st["qualifying_pairs"] == st_alone["qualifying_pairs"]
                assert st["candidate_pairs"] == st_alone["candidate_pairs"]
                assert st["internal_errors"] == 0
    finally:
        for p in pats:
            p.close()
    # the observed grids against the FP64 oracle (counts exact, the rest at 1e-6)
    for i in (0, 1, 3):
        x, y, t, box = sets[i]
        job = jobs[i]
        want = orc.k_function(x, y, t, box, job["s"], job["tt"],
                              edge_mode=job.get("edge_mode", stk.STK_EDGE_ISOTROPIC))
        got = alone[i][0]
        np.testing.assert_array_equal(got["C"], want["C"])
        for key in ("K", "S"):
            rel = np.abs(got[key] - want[key]) / np.maximum(np.abs(want[key]), 1e-300)
            assert rel.max() <= 1e-6, (i, key, rel.max())


def test_one_kernel_class_takes_one_launch(stk):
    sets, jobs = _sets(), _jobs(stk)
    keep = [0, 1, 2]  # even thresholds, isotropic correction
    pats = [stk.Pattern(*sets[i]) for i in keep]
    try:
        res, launches = stk.stk_run_fused([p.h for p in pats], [jobs[i] for i in keep])
        assert launches == 1
        st = [p.stats() for p in pats]
        # the fused pair launch is counted once, with the first job
        alone_launches = []
        for i in keep:
            _, s_alone = _alone(stk, sets[i], jobs[i])
            alone_launches.append(s_alone["kernel_launches"])
        assert st[0]["kernel_launches"] == alone_launches[0]
        assert [s["kernel_launches"] for s in st[1:]] == [a - 1 for a in alone_launches[1:]]
        for k, i in enumerate(keep):
            _same(res[k], _alone(stk, sets[i], jobs[i])[0], f"job {i}")
    finally:
        for p in pats:
            p.close()


def test_jobs_that_cannot_share_the_launch_run_alone(stk):
    from paper_1912_04753_gb300 import workloads as wl

    sets, jobs = _sets(), _jobs(stk)
    # FP64, uneven thresholds (their own class), the directional K: FP64 and sectors run alone
    odd = [
        dict(jobs[0], prec=stk.STK_PREC_FP64),
        dict(jobs[1], s=np.array([37.0, 90.0, 300.0]), tt=np.array([3.0, 11.0, 25.0])),
        dict(jobs[2], edge_mode=stk.STK_EDGE_TRANSLATION, n_sectors=4, want_sims=False,
             tt=wl.even_thresholds(30.0 * 86400.0, 5)),
        jobs[3],
    ]
    alone = [_alone(stk, pts, job)[0] for pts, job in zip(sets, odd)]
    pats = [stk.Pattern(*pts) for pts in sets]
    try:
        res, launches = stk.stk_run_fused([p.h for p in pats], odd)
        assert launches == 2  # uneven isotropic job 1; no edge correction job 3
        for i, (got, want) in enumerate(zip(res, alone)):
            _same(got, want, f"job {i}")
    finally:
        for p in pats:
            p.close()


def test_fused_arguments_checked(stk):
    sets, jobs = _sets(), _jobs(stk)
    with stk.Pattern(*sets[0]) as p, stk.Pattern(*sets[1]) as q:
        with pytest.raises(stk.StkError) as e:
            stk.stk_run_fused([p.h, p.h], [jobs[0], jobs[1]])  # one handle twice
        assert e.value.code == stk.STK_EINVAL
        with pytest.raises(stk.StkError) as e:
            stk.stk_run_fused([p.h, q.h], [jobs[0], dict(jobs[1], s=np.array([-1.0]))])
        assert e.value.code == stk.STK_EINVAL
        # both handles still compute correctly
        res, _ = stk.stk_run_fused([p.h, q.h], [jobs[0], jobs[1]])
        _same(res[0], _alone(stk, sets[0], jobs[0])[0], "after errors")


@pytest.mark.parametrize("fuse", [True, False])
def test_served_jobs_on_several_point_sets_share_a_launch(stk, fuse):
    """One slot: while an FP64 job (never fused) holds it, small jobs on four point sets queue;
    the slot then takes them as one group with shared pair launches.  Every served result
    equals the job alone, and the statistics count the fused jobs (none without fuse)."""
    from paper_1912_04753_gb300 import workloads as wl

    sets, jobs = _sets(), _jobs(stk)
    alone = [_alone(stk, pts, job)[0] for pts, job in zip(sets, jobs)]
    with stk.Server(slots=1, fuse=fuse) as sv:
        ids = [sv.register(*p) for p in sets]
        blocker = sv.submit(ids[2], wl.even_thresholds(500.0, 10),
                            wl.even_thresholds(30.0 * 86400.0, 10), n_sims=60, seed=5,
                            prec=stk.STK_PREC_FP64)
        tickets = []
        for i, j in enumerate(jobs):
            kw = {k: v for k, v in j.items() if k not in ("s", "tt", "n_sims", "seed")}
            tickets.append(sv.submit(ids[i], j["s"], j["tt"], n_sims=j["n_sims"],
                                     seed=j["seed"], **kw))
        served = [sv.poll(tk, wait_ms=120000) for tk in tickets]
        assert sv.poll(blocker, wait_ms=120000) is not None
        st = sv.stats()
    assert st["completed"] == 5 and st["failed"] == 0
    if not fuse:
        assert st["fused_jobs"] == 0
    else:
        assert st["fused_jobs"] >= 2, st
    for i, (got, _lat) in enumerate(served):
        want = {k: v for k, v in alone[i].items() if k in got}
        _same(got, want, f"served job {i}")
