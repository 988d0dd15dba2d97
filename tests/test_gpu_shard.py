"""One job split into shards (the multi-GPU split of the method), run one after another on one
GPU and merged on the host exactly as the ranks' all-reduce would: the merged grids equal the
single-process job bit for bit (observed K, L, S, C through stk_merge_grids; the envelope
through stk_envelope_merge), in both precisions and for the directional K.  No shard waits on
another."""
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


def _combine(parts):
    """What reduce_shards computes across ranks: accumulators summed, K_lo / K_hi min / max."""
    acc = parts[0]["acc"].copy()
    for p in parts[1:]:
        acc = acc + p["acc"]
    lo = np.min(np.stack([p["K_lo"] for p in parts]), axis=0)
    hi = np.max(np.stack([p["K_hi"] for p in parts]), axis=0)
    return {"acc": acc, "K_lo": lo, "K_hi": hi,
            "qualifying_pairs": sum(p["qualifying_pairs"] for p in parts)}


CASES = [
    ("csr_fp32", dict(prec=1)),
    ("csr_fp64", dict(prec=0)),
    ("dir_fp32", dict(prec=1, n_sectors=4, edge_mode=2)),
    ("none_n2", dict(prec=1, edge_mode=0, norm=1)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_job_equals_single_job(stk, name, kw, world):
    from paper_1912_04753_gb300 import shard, workloads as wl

    w = wl.config_thomas(seed=5, n=30_000)
    n_sims, seed = 7, 23
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        whole = p.run(w.s, w.tt, n_sims=n_sims, seed=seed, **kw)
        qual_whole = p.stats()["qualifying_pairs"]
        parts = [shard.run_shard(p, w.s, w.tt, n_sims, seed, world, r, **kw)
                 for r in range(world)]
        assert sum(pt["n_local"] for pt in parts) == n_sims
        merged = _combine(parts)
        got = shard.merge(p, w.s, w.tt, merged, n_sims, **kw)
    for k in ("C", "K", "L", "S", "K_lo", "K_hi", "L_lo", "L_hi"):
        np.testing.assert_array_equal(got[k], whole[k], err_msg=k)
    assert merged["qualifying_pairs"] == qual_whole
    # every shard did a share of the observed pattern's pairs
    assert all(int(pt["acc"][0, 0].sum()) > 0 for pt in parts)


def test_merge_of_unsharded_accumulators_is_the_job(stk):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=8, n=4000)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        r = p.run(w.s, w.tt, n_sims=3, seed=2, want_sims=True)
        acc = stk.stk_last_accumulators(p.h, 0, 4, cs=len(w.s), ct=len(w.tt))
        g = stk.stk_merge_grids(p.h, acc, w.s, w.tt)
        with pytest.raises(stk.StkError):
            stk.stk_last_accumulators(p.h, 2, 3, cs=len(w.s), ct=len(w.tt))
    np.testing.assert_array_equal(g["K"][0], r["K"])
    np.testing.assert_array_equal(g["C"][1:], r["C_sims"])
    np.testing.assert_array_equal(g["K"][1:], r["K_sims"])
    env = stk.stk_envelope_merge(r["K_sims"], w.s, w.tt)
    for k in ("K_lo", "K_hi", "L_lo", "L_hi"):
        np.testing.assert_array_equal(env[k], r[k], err_msg=k)


def test_shard_arguments_checked(stk):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.config_csr_small(seed=8, n=500)
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        for bad in ((2, 2), (3, -1), (70000, 0)):
            with pytest.raises(stk.StkError) as e:
                p.run(w.s, w.tt, shard=bad)
            assert e.value.code == stk.STK_EINVAL
        p.run(w.s, w.tt)  # still usable
