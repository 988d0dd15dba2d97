"""One job split across processes, one GPU each (the data-parallel split of the method).

The paper spreads the pair work of one K estimation over Spark workers by partitioning the
points (Section 4.4) and runs the simulations of the envelope (Section 3) as independent tasks.
Here the same job is split in two ways that need no exchange during the computation:

  * simulations: realization k of the job belongs to one rank (contiguous blocks of the
    counter-based generator's realizations, ``sim_block``), so every rank generates, indexes
    and evaluates only its own realizations;
  * the observed pattern: its work units are split into ``world`` contiguous shards
    (``stk_request.shard_count / shard_index``), each unordered pair in exactly one shard.

After the computation each rank holds (a) the observed pattern's raw integer accumulators of
its shard, which add exactly, and (b) the element-wise min / max of K over its realizations,
which reduce exactly and in any order.  ``reduce_shards`` combines them with three
torch.distributed all-reduces (SUM over int64, MIN and MAX over float64: a few tens of KB), and
``merge`` has the library turn the sums into K, L, S, C (``stk_merge_grids``, 128-bit fixed
point on the device) and the envelope into L (``stk_envelope_merge``).  The result equals the
single-process job bit for bit.  Host logic only: every number is computed by the library.
"""
from __future__ import annotations

import numpy as np

from . import _lib


def sim_block(n_sims: int, world: int, rank: int):
    """(first_sim, count) of `rank`'s contiguous block of realizations 0 .. n_sims - 1 (block
    sizes differ by at most one; the first n_sims % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n_sims), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def run_shard(pattern, s, tt, n_sims, seed, world, rank, **kw):
    """This rank's part of the job: its shard of the observed pattern and its block of
    realizations.  Returns {"acc": uint64 [1, 4, nbins] observed accumulators of the shard,
    "K_lo", "K_hi": min / max of K over the rank's realizations (+inf / -inf where it has
    none), "first_sim", "n_local", "qualifying_pairs"}."""
    first, cnt = sim_block(n_sims, world, rank)
    nsec = kw.get("n_sectors", 0)
    r = _lib.stk_run(pattern.h, s, tt, n_sims=cnt, seed=seed, first_sim=first,
                     shard=(world, rank) if world > 1 else (0, 0), **kw)
    acc = _lib.stk_last_accumulators(pattern.h, 0, 1, n_sectors=nsec, cs=len(s), ct=len(tt))
    st = _lib.stk_last_stats(pattern.h)
    if cnt > 0:
        lo, hi = r["K_lo"], r["K_hi"]
    else:
        lo = np.full_like(r["K"], np.inf)
        hi = np.full_like(r["K"], -np.inf)
    return {"acc": acc, "K_lo": lo, "K_hi": hi, "first_sim": first, "n_local": cnt,
            "qualifying_pairs": st["qualifying_pairs"]}


def reduce_shards(part, group=None, device=None):
    """All-reduce of the partial results of every rank (torch.distributed, any backend):
    accumulators summed (int64, exact), K_lo / K_hi reduced by MIN / MAX (exact).  `device`:
    where the collective's tensors live (a CUDA device for NCCL; CPU for gloo)."""
    import torch
    import torch.distributed as dist

    if device is None:
        device = (torch.device("cuda", torch.cuda.current_device())
                  if dist.get_backend(group) == "nccl" else torch.device("cpu"))
    acc = np.ascontiguousarray(part["acc"], dtype=np.uint64)
    if int(acc.max(initial=0)) >= 2**63:
        raise OverflowError("accumulator beyond int64")
    a = torch.from_numpy(acc.view(np.int64).copy()).to(device)
    lo = torch.from_numpy(np.ascontiguousarray(part["K_lo"], np.float64)).to(device)
    hi = torch.from_numpy(np.ascontiguousarray(part["K_hi"], np.float64)).to(device)
    q = torch.tensor([int(part.get("qualifying_pairs", 0))], dtype=torch.int64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return {"acc": a.cpu().numpy().view(np.uint64), "K_lo": lo.cpu().numpy(),
            "K_hi": hi.cpu().numpy(), "qualifying_pairs": int(q.item())}


def merge(pattern, s, tt, merged, n_sims, **kw):
    """Final grids of the job from the reduced partial results: observed K, L, S, C (through
    stk_merge_grids) and the envelope K_lo, K_hi, L_lo, L_hi (through stk_envelope_merge)."""
    nsec = kw.get("n_sectors", 0)
    g = _lib.stk_merge_grids(pattern.h, merged["acc"], s, tt, **kw)
    out = {k: v[0] for k, v in g.items()}
    if n_sims > 0:
        rows = np.stack([merged["K_lo"], merged["K_hi"]])
        out.update(_lib.stk_envelope_merge(rows, s, tt, n_sectors=nsec))
    return out


def run_sharded(pattern, s, tt, n_sims, seed, world, rank, group=None, device=None, **kw):
    """The whole job split over `world` ranks (this process is `rank`): run_shard, then
    reduce_shards, then merge.  Every rank returns the same final grids."""
    part = run_shard(pattern, s, tt, n_sims, seed, world, rank, **kw)
    merged = reduce_shards(part, group=group, device=device) if world > 1 else part
    out = merge(pattern, s, tt, merged, n_sims, **kw)
    out["qualifying_pairs"] = merged.get("qualifying_pairs", part["qualifying_pairs"])
    return out
