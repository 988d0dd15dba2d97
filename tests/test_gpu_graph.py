"""CUDA-graph replay of batched jobs (one graph per wave): a job whose shape, constants and
buffers match the last captured one is replayed from its graphs (new simulation seeds reach them
through the pinned staging copies) and gives exactly the grids of the same job issued launch by
launch, for single-wave and multi-wave jobs; the pair kernel is timed inside the graph."""
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


def test_graph_replay_equals_direct_issue(stk, monkeypatch):
    from paper_1912_04753_gb300 import workloads as wl

    rng = np.random.default_rng(2)
    box = (0.0, 3000.0, 0.0, 3000.0, 0.0, 365.0)
    x, y, t = wl.thomas(6000, box, 20, 100.0, 6.0, rng)
    s, tt = wl.even_thresholds(200.0, 8), wl.even_thresholds(20.0, 6)
    for prec in (stk.STK_PREC_FP32_GUARDED, stk.STK_PREC_FP64):
        with stk.Pattern(x, y, t, box) as p:
            monkeypatch.setenv("STK_GRAPHS", "1")
            first = p.run(s, tt, n_sims=7, seed=11, prec=prec, want_sims=True)
            assert p.stats()["graph_replays"] == 0  # captured, launched once
            # the observed index is resident from now on: another graph, captured once more
            p.run(s, tt, n_sims=7, seed=11, prec=prec, want_sims=True)
            assert p.stats()["obs_index_reused"] == 1 and p.stats()["graph_replays"] == 0
            runs = {}
            for seed in (11, 12, 13):
                runs[seed] = p.run(s, tt, n_sims=7, seed=seed, prec=prec, want_sims=True)
                assert p.stats()["graph_replays"] == 1
            monkeypatch.setenv("STK_GRAPHS", "0")
            for seed in (11, 12, 13):
                direct = p.run(s, tt, n_sims=7, seed=seed, prec=prec, want_sims=True)
                assert p.stats()["graph_replays"] == 0
                for k in direct:
                    np.testing.assert_array_equal(runs[seed][k], direct[k], err_msg=k)
            for k in first:
                np.testing.assert_array_equal(first[k], runs[11][k], err_msg=k)
            # a different shape is captured anew, never replayed from the old graph
            monkeypatch.setenv("STK_GRAPHS", "1")
            p.run(s, tt, n_sims=5, seed=1, prec=prec)
            assert p.stats()["graph_replays"] == 0


def test_multi_wave_graph_replay_equals_direct_issue(stk, monkeypatch):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_thomas(seed=3, n=20_000)
    monkeypatch.setenv("STK_MEM_BUDGET_MB", "9")  # a few realizations per wave
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        monkeypatch.setenv("STK_GRAPHS", "0")
        direct = p.run(w.s, w.tt, n_sims=9, seed=4, want_sims=True)
        st = p.stats()
        assert st["waves"] >= 3 and st["graph_replays"] == 0
        monkeypatch.delenv("STK_GRAPHS")
        p.run(w.s, w.tt, n_sims=9, seed=4, want_sims=True)  # a first occurrence: issued directly
        assert p.stats()["graph_replays"] == 0
        p.run(w.s, w.tt, n_sims=9, seed=4, want_sims=True)  # the shape repeats: captured
        assert p.stats()["graph_replays"] == 0
        got = p.run(w.s, w.tt, n_sims=9, seed=4, want_sims=True)  # replayed
        sg = p.stats()
    assert sg["graph_replays"] == sg["waves"] == st["waves"]
    assert 0.0 < sg["ms_pair"] <= sg["ms_total"]
    for k in direct:
        np.testing.assert_array_equal(got[k], direct[k], err_msg=k)


def test_job_log_lines(stk, orc, tmp_path):
    # STK_JOB_LOG: one JSON line per job with the job's statistics
    import json
    import os

    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=2, n=1500)
    path = tmp_path / "jobs.jsonl"
    os.environ["STK_JOB_LOG"] = str(path)
    try:
        with stk.Pattern(w.x, w.y, w.t, w.box) as p:
            p.run(w.s, w.tt, n_sims=3, seed=1)
            st = p.stats()
            p.run(w.s, w.tt, n_sectors=2, edge_mode=stk.STK_EDGE_TRANSLATION)
    finally:
        del os.environ["STK_JOB_LOG"]
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert len(lines) == 2
    a, b = lines
    assert a["n"] == 1500 and a["realizations"] == 4 and a["cs"] == len(w.s)
    assert a["qualifying_pairs"] == st["qualifying_pairs"]
    assert a["internal_errors"] == 0 and b["n_sectors"] == 2 and b["edge_mode"] == 2
