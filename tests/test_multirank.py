"""Multi-rank logic on CPU ranks (gloo, world size 2): bench.py reports the maximum time over
ranks and the summed work; one job split across ranks (realization blocks, observed-pattern
shards) reduces exactly; under torchrun the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t, q = bench.reduce_over_ranks([12.5, 30.0][rank], [1000, 234][rank], "cpu")
    out.put((rank, t, q))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, qual in res:
        assert t == 30.0 and qual == 1234.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(5.0, 7, "cpu") == (5.0, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.build_parser().parse_args(["--impl", "reference"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def _shard_rank_main(rank, ws, port, out):
    """A rank of a split job on CPU: the oracle stands in for the library on this rank's share
    (observed pairs of its centres, K of its block of realizations); reduce_shards combines
    the shares over gloo."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_1912_04753_gb300 import shard, workloads as wl

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = wl.config_csr_small(seed=31, n=300)
    n_sims, seed = 5, 4
    # observed: this rank's centres (a partition of the points), counts in the accumulator's
    # count row (bins not cumulative)
    mask = (np.arange(w.n) % ws == rank).astype(np.uint8)
    cnt, _, _ = oracle.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=1,
                                 centre_mask=mask)
    acc = np.zeros((1, 4, cnt.size), np.uint64)
    acc[0, 0] = np.asarray(cnt, np.int64).reshape(-1).astype(np.uint64)
    first, count = shard.sim_block(n_sims, ws, rank)
    env = oracle.envelope_of(oracle.SIM_CSR, w.x, w.y, w.t, w.box, w.s, w.tt, n_sims, seed)
    mine = env["K_all"][first:first + count]
    part = {"acc": acc,
            "K_lo": mine.min(axis=0) if count else np.full(env["K_lo"].shape, np.inf),
            "K_hi": mine.max(axis=0) if count else np.full(env["K_hi"].shape, -np.inf),
            "qualifying_pairs": rank + 1}
    m = shard.reduce_shards(part)
    full, _, _ = oracle.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=1)
    ok = (np.array_equal(m["acc"][0, 0].astype(np.int64), np.asarray(full).reshape(-1))
          and np.array_equal(m["K_lo"], env["K_lo"]) and np.array_equal(m["K_hi"], env["K_hi"])
          and m["qualifying_pairs"] == ws * (ws + 1) // 2 and not m["acc"][0, 1:].any())
    out.put((rank, bool(ok), first, count))
    dist.barrier()
    dist.destroy_process_group()


def test_split_job_reduces_exactly_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in res)
    assert [(f, c) for _, _, f, c in res] == [(0, 3), (3, 2)]


def test_sim_blocks_partition_the_realizations():
    sys.path.insert(0, ROOT)
    from paper_1912_04753_gb300 import shard

    for n_sims in (0, 1, 5, 99, 100):
        for world in (1, 2, 3, 8):
            blocks = [shard.sim_block(n_sims, world, r) for r in range(world)]
            covered = [k for f, c in blocks for k in range(f, f + c)]
            assert covered == list(range(n_sims))
            assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1
    with pytest.raises(ValueError):
        shard.sim_block(10, 2, 2)
