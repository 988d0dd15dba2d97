"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): each rank runs its own job
with its own seed (weak scaling, no data-path collective); the reported time is the maximum
over ranks and the work the sum; under torchrun the reference arm runs on rank 0 only."""
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
    out.put((rank, t, q, bench.rank_seed(99, rank)))
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
    for rank, t, qual, seed in res:
        assert t == 30.0 and qual == 1234.0
    assert res[0][3] != res[1][3]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(5.0, 7, "cpu") == (5.0, 7.0)
    assert bench.rank_seed(3, 0) == 3


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.build_parser().parse_args(["--impl", "reference"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
