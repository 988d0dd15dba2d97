"""Benchmark: observed space-time K + 99-simulation CSR envelope on the n=2,000,000 POI-shaped
mixture (50 km x 50 km x 1095 days, timestamps in whole seconds, 25 x 25 thresholds to 2 km /
90 days), batched FP32-guarded path, on one GB300.

One step = one whole job (the observed pattern and 99 CSR realizations through generation,
grid index, pair kernel, finalize and envelope).  The headline unit is qualifying ordered pairs
per second (pairs with d <= s_max and u <= t_max, summed over all 100 realizations).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Besides the headline it carries the end-to-end time through the C ABI
from host arrays (`e2e`), the plain FP64 comparison (`plain_fp64`), the CPU oracle on a bounded
sample (`cpu_baseline`), the serving loop (`serve`), permutation and bootstrap simulations
(`sim_methods`), a polygon study area (`polygon`), the inhomogeneous and the directional K
(`inhomogeneous`, `directional`), the pair kernel's roofline and the clocks seen.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload (random
centres of the observed pattern against all n points).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("pair evals/s & K+99-sim envelope time at n=2M (batched FP32 vs plain FP64); "
          "serve p50/p99")
UNIT = "qualifying ordered pairs/s"
# per-unit instruction counts of the pair kernel's algorithm (candidate test; qualifying-pair
# binning + histogram update), used for the ALU roofline
OPS_PER_CANDIDATE = 8
OPS_PER_QUALIFYING = 12
# DRAM bytes (read + write) of the pair kernel per realization of the 2M-point mixture, from
# one ncu capture of the kernel as built (a launch of 2 CSR realizations; the clustered observed
# realization is one of the job's hundred)
PAIR_DRAM_BYTES_PER_REALIZATION = {"poi_n2M": 124.1e6}


def _workload(name, sims=None):
    from paper_1912_04753_gb300 import workloads as wl

    w = wl.CONFIGS[name]()
    if sims is not None:
        w.n_sims = sims
    return w


def reduce_over_ranks(elapsed_ms: float, qual: float, device):
    """(max elapsed over ranks, sum of qualifying pairs over ranks); identity on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return float(elapsed_ms), float(qual)
    tmax = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(qual)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


def cpu_baseline(w, target_s=15.0, seed=123):
    """Time the FP64 oracle on random centres of the observed pattern against all n points."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    n = w.n
    # calibrate on a few centres, then size the sample for ~target_s of CPU work
    R = min(8, n)
    total_pairs, total_t, used = 0, 0.0, 0
    while total_t < target_s:
        mask = np.zeros(n, np.uint8)
        mask[rng.choice(n, R, replace=False)] = 1
        t0 = time.perf_counter()
        _, _, q = oracle.pair_hist(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=1,
                                   centre_mask=mask)
        dt = time.perf_counter() - t0
        total_pairs += q
        total_t += dt
        used += R
        per = dt / R
        R = int(max(8, min(4096, (target_s - total_t) / max(per, 1e-6))))
        R = min(R, n)  # small patterns: at most every point once per draw
        if target_s - total_t < 0.5:
            break
    what = (f"{used} random centres of the observed n={n} pattern" if used < n else
            f"{used / n:.1f} passes over all n={n} centres of the observed pattern")
    return {"value": total_pairs / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{what} x all n points, FP64 single thread, {total_t:.1f} s",
            "seconds": total_t}


def host_info():
    """CPU model and the number of host cores (the CPU baselines' machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name") and ":" in ln:
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    key = ln.split(":")[0].strip().lower()
                    if key in ("model name", "cpu model", "hardware", "cpu part") and ":" in ln:
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpu_grid_baseline(w, target_s=10.0, seed=321):
    """Time the oracle's grid restatement (FP64, the same per-pair arithmetic, pairs restricted
    to adjacent cells of a grid wider than the thresholds) on all host cores, on random
    centres of the observed pattern against all n points."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    n, cores = w.n, os.cpu_count() or 1
    R = min(256, n)
    total_pairs, total_t, used = 0, 0.0, 0
    while total_t < target_s:
        mask = np.zeros(n, np.uint8)
        mask[rng.choice(n, R, replace=False)] = 1
        t0 = time.perf_counter()
        _, _, q = oracle.pair_hist_grid(w.x, w.y, w.t, w.box, w.s, w.tt, edge_mode=1,
                                        centre_mask=mask, threads=cores)
        dt = time.perf_counter() - t0
        total_pairs += q
        total_t += dt
        used += R
        per = dt / R
        R = int(max(256, min(n, (target_s - total_t) / max(per, 1e-7))))
        if target_s - total_t < 0.5:
            break
    return {"value": total_pairs / total_t, "unit": UNIT, "cores": cores,
            "kind": "oracle grid restatement, all host cores",
            "sample": f"{used} random centres of the observed n={n} pattern x all n points "
                      f"(grid of cells wider than the thresholds, FP64, {cores} threads, "
                      f"{total_t:.1f} s; includes the grid build per draw)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.config, args.sims)
    steps = []
    total_pairs, total_t = 0, 0.0
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, target_s=args.ref_seconds, seed=1000 + i)
        if i >= args.warmup:
            steps.append(cb)
            total_pairs += cb["value"] * cb["seconds"]
            total_t += cb["seconds"]
    value = total_pairs / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / max(1, args.steps), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "sims": w.n_sims,
                       "thresholds": [len(w.s), len(w.tt)]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": steps[-1]["sample"] if steps else ""},
            "host": host_info(),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _serve_stream(sv, ids, reqs, rate):
    """Submits `reqs` at their arrival times from another thread, waits for every result;
    returns (the rate's row of statistics, the served results)."""
    sv.reset_stats()
    tickets = [None] * len(reqs)

    def submit_all():
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            dt = r["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets[i] = sv.submit(ids[r["dataset"]], r["s"], r["tt"],
                                   n_sims=r["n_sims"], seed=r["seed"], want_sims=False)

    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    served = [sv.poll(tk) for tk in tickets]
    st = sv.stats()
    done = max(1, st["completed"])
    row = {
        "rate_hz": rate, "offered_s": reqs[-1]["arrival_s"],
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
        "mean_ms": st["mean_ms"], "jobs_per_s": st["jobs_per_s"],
        "sims_per_s": st["sims_per_s"], "completed": st["completed"],
        "failed": st["failed"], "batches": st["batches"],
        "merged_fraction": st["merged_jobs"] / done,
        "fused_fraction": st["fused_jobs"] / done,
        "launches_per_job": st["kernel_launches"] / done,
        "max_queue_depth": st["max_queue_depth"], "peak_device_bytes": st["peak_bytes"]}
    return row, served


def serve_bench(args, stk, seed=0):
    """Serving loop on synthetic request streams (Poisson arrivals, n log-uniform in [1e3, 1e6],
    CSR / Thomas / POI-mixture point sets kept resident, 5-50 thresholds per axis, 0-199
    simulations, own seed per request), swept over arrival rates from light load to overload:
    per rate p50 / p99 / max latency from submission to result, jobs/s, the share of jobs merged
    into another job's batch and kernel launches per job.  Then: a sample of served results
    against the same jobs run alone (must be identical), and the first requests of the lightest
    stream through a single FIFO queue running each job as the plain FP64 path (one launch per
    realization), the comparison the FP32-guarded continuous batching is measured against."""
    from paper_1912_04753_gb300 import workloads as wl

    rates = [float(r) for r in str(args.serve_rates).split(",") if r]
    count = args.serve_requests
    datasets, _ = wl.serving_stream(1, seed=seed, rate_hz=rates[0])
    out = {"requests_per_rate": count, "datasets": len(datasets),
           "n_range": [min(d.n for d in datasets), max(d.n for d in datasets)], "sweep": []}
    served_sample = []
    with stk.Server(slots=args.serve_slots) as sv:
        ids = [sv.register(d.x, d.y, d.t, d.box) for d in datasets]
        # warm-up: one small job per point set (workspaces, kernel attributes)
        for k, d in enumerate(datasets):
            sv.poll(sv.submit(ids[k], d.s, d.tt, n_sims=1, seed=1))
        for ri, rate in enumerate(rates):
            ds2, reqs = wl.serving_stream(count, seed=seed, rate_hz=rate)
            assert len(ds2) == len(datasets) and all(a.n == b.n for a, b in zip(ds2, datasets))
            row, served = _serve_stream(sv, ids, reqs, rate)
            out["sweep"].append(row)
            if ri == len(rates) - 1:  # results of the heaviest stream, to check against alone
                served_sample = [(reqs[i], served[i][0])
                                 for i in range(0, len(reqs), max(1, len(reqs) // 20))][:20]
        out["slots"] = args.serve_slots
    # small jobs on different point sets sharing pair launches (cfg.fuse): the heaviest stream
    # again, and a stream of tiny jobs (n in [1e3, 1e4], at most 20 simulations) with and
    # without it
    def fused_vs_not(dsets, reqs, rate):
        rows = {}
        for fuse in (True, False):
            with stk.Server(slots=args.serve_slots, fuse=fuse) as sv:
                ids = [sv.register(d.x, d.y, d.t, d.box) for d in dsets]
                for k, d in enumerate(dsets):
                    sv.poll(sv.submit(ids[k], d.s, d.tt, n_sims=1, seed=1))
                rows["fused" if fuse else "not_fused"], _ = _serve_stream(sv, ids, reqs, rate)
        return rows

    _, reqs = wl.serving_stream(count, seed=seed, rate_hz=rates[-1])
    out["heaviest_with_fusing"] = fused_vs_not(datasets, reqs, rates[-1])["fused"]
    tiny_rate = 2000.0
    tiny_sets, tiny_reqs = wl.serving_stream(3 * count, seed=seed + 1, rate_hz=tiny_rate,
                                             n_lo=1000, n_hi=10000, max_sims=20)
    out["tiny_jobs"] = {"requests": len(tiny_reqs), "rate_hz": tiny_rate,
                        "n_range": [min(d.n for d in tiny_sets), max(d.n for d in tiny_sets)],
                        **fused_vs_not(tiny_sets, tiny_reqs, tiny_rate)}
    # the fused launch itself, one thread: 12 tiny jobs (one per point set, 20 simulations
    # each) in one stk_run_fused call against the same jobs through stk_run one after another
    pats = [stk.Pattern(d.x, d.y, d.t, d.box) for d in tiny_sets]
    jobs = [dict(s=d.s, tt=d.tt, n_sims=20, seed=7 + k) for k, d in enumerate(tiny_sets)]
    for p_, j in zip(pats, jobs):  # warm-up (tuning, workspaces)
        p_.run(**j)
    stk.stk_run_fused([p_.h for p_ in pats], jobs)
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        for p_, j in zip(pats, jobs):
            p_.run(**j)
    t_seq = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        _, fl = stk.stk_run_fused([p_.h for p_ in pats], jobs)
    t_fused = (time.perf_counter() - t0) / reps
    for p_ in pats:
        p_.close()
    out["fused_call"] = {"jobs": len(jobs), "sims_each": 20, "ms_one_by_one": 1e3 * t_seq,
                         "ms_fused": 1e3 * t_fused, "pair_launches_fused": fl}
    # served = alone, bit for bit, on a sample of the heaviest stream's requests
    same, counts, checked, worst = True, True, 0, 0.0
    for r, got in served_sample:
        d = datasets[r["dataset"]]
        with stk.Pattern(d.x, d.y, d.t, d.box) as p:
            alone = p.run(r["s"], r["tt"], n_sims=r["n_sims"], seed=r["seed"])
        same = same and all(np.array_equal(got[k], alone[k]) for k in alone)
        counts = counts and np.array_equal(got["C"], alone["C"])
        for k in ("K", "K_lo", "K_hi"):
            if k in alone:
                den = np.where(alone[k] == 0, 1.0, np.abs(alone[k]))
                worst = max(worst, float((np.abs(got[k] - alone[k]) / den).max()))
        checked += 1
    out["served_equals_alone"] = {"checked": checked, "identical": same,
                                  "counts_identical": counts, "max_rel_diff_K": worst}
    if args.serve_fp64 > 0:
        _, reqs = wl.serving_stream(args.serve_fp64, seed=seed, rate_hz=rates[0])
        handles = [stk.Pattern(d.x, d.y, d.t, d.box) for d in datasets]
        for k, d in enumerate(datasets):  # warm-up as above
            handles[k].run(d.s, d.tt, n_sims=1, seed=1, prec=stk.STK_PREC_FP64,
                           exec_mode=stk.STK_EXEC_PLAIN)
        lat = []
        t0 = time.perf_counter()
        for r in reqs:
            wait = r["arrival_s"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            handles[r["dataset"]].run(r["s"], r["tt"], n_sims=r["n_sims"], seed=r["seed"],
                                      prec=stk.STK_PREC_FP64, exec_mode=stk.STK_EXEC_PLAIN)
            lat.append(1e3 * (time.perf_counter() - t0 - r["arrival_s"]))
        wall = time.perf_counter() - t0 - reqs[0]["arrival_s"]
        for hd in handles:
            hd.close()
        lat = np.sort(np.array(lat))
        q = lambda p: float(lat[max(0, int(np.ceil(p / 100 * len(lat))) - 1)])
        out["fp64_plain_fifo"] = {"requests": len(reqs), "rate_hz": rates[0], "p50_ms": q(50),
                                  "p99_ms": q(99), "max_ms": float(lat[-1]),
                                  "jobs_per_s": len(reqs) / wall,
                                  "sims_per_s": int(sum(r["n_sims"] for r in reqs)) / wall}
    return out


def run_ours(args):
    import torch

    import paper_1912_04753_gb300 as stk
    from paper_1912_04753_gb300 import build as _b

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _b.build()
    stk.load()
    w = _workload(args.config, args.sims)
    prec = stk.STK_PREC_FP32_GUARDED if args.prec == "fp32" else stk.STK_PREC_FP64
    exec_mode = stk.STK_EXEC_BATCHED if args.exec == "batched" else stk.STK_EXEC_PLAIN
    seed = w.sim_seed
    stream = torch.cuda.Stream()
    h = stk.stk_create(w.x, w.y, w.t, w.box)
    stk.stk_set_stream(h, stream)
    dev = torch.device("cuda", local)

    def run_on(handle):
        """One whole job; with N ranks each runs its share (a block of the realizations and a
        shard of the observed pattern's pairs) and the partial results are all-reduced."""
        if ws == 1:
            return stk.stk_run(handle, w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=prec,
                               exec_mode=exec_mode)
        from types import SimpleNamespace

        from paper_1912_04753_gb300 import shard

        return shard.run_sharded(SimpleNamespace(h=handle), w.s, w.tt, w.n_sims, seed, ws, rank,
                                 device=dev, prec=prec, exec_mode=exec_mode)

    def job():
        return run_on(h)

    for _ in range(args.warmup):
        job()
    st = stk.stk_last_stats(h)
    sampler = ClockSampler(local)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pair_ms, qual, cand, launches = 0.0, 0, 0, 0
    ev0.record(stream)
    for _ in range(args.steps):
        out = job()
        s = stk.stk_last_stats(h)
        pair_ms += s["ms_pair"]
        qual += s["qualifying_pairs"]
        cand += s["candidate_pairs"]
        launches += s["kernel_launches"]
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms, qual_all = reduce_over_ranks(elapsed_ms, qual, torch.device("cuda", local))
    value = qual_all / (elapsed_ms / 1e3)

    # end to end through the C ABI from host buffers: create (H2D of the points), job, D2H of
    # the result grids, every step
    e2e_ms = 0.0
    nb = len(w.s) * len(w.tt)
    h2d = 3 * 8 * w.n
    d2h = nb * (8 * 4 + 8) + 4 * nb * 8
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        barrier()
        t0 = time.perf_counter()
        h2 = stk.stk_create(w.x, w.y, w.t, w.box)
        run_on(h2)
        stk.stk_destroy(h2)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
    e2e_ms /= e2e_steps
    e2e_value = (qual_all / args.steps) / (e2e_ms / 1e3)

    # plain FP64 comparison (spec pairing): one job, one launch per realization, and the
    # per-cell error of the FP32-guarded grids against it on the same realizations
    plain = None
    if args.compare_fp64 and rank == 0:
        stk.stk_run(h, w.s, w.tt, n_sims=1, seed=seed, prec=stk.STK_PREC_FP64,
                    exec_mode=stk.STK_EXEC_PLAIN)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ref = stk.stk_run(h, w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=stk.STK_PREC_FP64,
                          exec_mode=stk.STK_EXEC_PLAIN, want_sims=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ps = stk.stk_last_stats(h)
        pms = e0.elapsed_time(e1)
        f32 = stk.stk_run(h, w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=prec,
                          exec_mode=exec_mode, want_sims=True)
        ka = np.concatenate([f32["K"][None], f32["K_sims"]])
        kb = np.concatenate([ref["K"][None], ref["K_sims"]])
        rel = np.abs(ka - kb) / np.where(kb == 0, 1.0, np.abs(kb))
        same_counts = bool(np.array_equal(f32["C"], ref["C"]) and
                           np.array_equal(f32["C_sims"], ref["C_sims"]))
        plain = {"job_s": pms / 1e3, "value": ps["qualifying_pairs"] / (pms / 1e3),
                 "unit": UNIT, "sims_per_s": w.n_sims / (pms / 1e3),
                 "speedup_batched_fp32": pms / (elapsed_ms / args.steps),
                 "fp32_vs_fp64": {"cells": int(rel.size), "counts_identical": same_counts,
                                  "max_rel_err_K": float(rel.max()),
                                  "p99_rel_err_K": float(np.quantile(rel, 0.99)),
                                  "median_rel_err_K": float(np.median(rel))}}

    serve = serve_bench(args, stk) if (args.serve_requests > 0 and rank == 0) else None

    # the other two simulation methods of Section 3 on the same job shape
    methods = None
    if args.methods and rank == 0:
        methods = {}
        for name, mth in (("permutation", stk.STK_SIM_PERMUTATION),
                          ("bootstrap", stk.STK_SIM_BOOTSTRAP)):
            stk.stk_run(h, w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=prec,
                        exec_mode=exec_mode, sim_method=mth)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stk.stk_run(h, w.s, w.tt, n_sims=w.n_sims, seed=seed, prec=prec,
                        exec_mode=exec_mode, sim_method=mth)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_m = e0.elapsed_time(e1)
            sm = stk.stk_last_stats(h)
            methods[name] = {"job_s": ms_m / 1e3, "sims_per_s": w.n_sims / (ms_m / 1e3),
                             "value": sm["qualifying_pairs"] / (ms_m / 1e3), "unit": UNIT,
                             "qualifying_pairs": sm["qualifying_pairs"]}

    # polygon study areas (85-vertex outlines, Thomas process, CSR simulations in them): a
    # spiky star, whose circles cross the boundary six times on average and keep FP64 weights,
    # and a smooth outline, which takes the FP32-guarded ones; 9 simulations each
    def polygon_job(name):
        wp = _workload(name, sims=9)
        with stk.Pattern(wp.x, wp.y, wp.t, wp.box) as pp:
            pp.set_polygon(*wp.meta["polygon"])
            stk.stk_set_stream(pp.h, stream)
            pp.run(wp.s, wp.tt, n_sims=wp.n_sims, seed=seed, prec=prec, exec_mode=exec_mode)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pp.run(wp.s, wp.tt, n_sims=wp.n_sims, seed=seed, prec=prec, exec_mode=exec_mode)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_p = e0.elapsed_time(e1)
            sp = pp.stats()
        return {"workload": wp.name, "n": wp.n, "vertices": len(wp.meta["polygon"][0]),
                "sims": wp.n_sims, "job_s": ms_p / 1e3,
                "sims_per_s": wp.n_sims / (ms_p / 1e3),
                "value": sp["qualifying_pairs"] / (ms_p / 1e3), "unit": UNIT,
                "pair_kernel_s": sp["ms_pair"] / 1e3,
                "fp64_queue_share": sp["fp64_recomputed"] / max(1, sp["qualifying_pairs"])}

    polygon = polygon_smooth = None
    if args.polygon and rank == 0:
        polygon = polygon_job("thomas_polygon85_n200k")
        polygon_smooth = polygon_job("thomas_smooth85_n200k")

    # the inhomogeneous K (intensity-weighted pairs; FP32-guarded and FP64) on the Thomas
    # pattern with a histogram intensity, observed + 99 intensity-weighted simulations
    inhom = None
    if args.inhom and rank == 0:
        wi = _workload("thomas_inhom_n200k")
        times = {}
        with stk.Pattern(wi.x, wi.y, wi.t, wi.box) as pi_:
            pi_.set_intensity(wi.meta["rho"])
            stk.stk_set_stream(pi_.h, stream)
            for pname, pv in (("fp32", stk.STK_PREC_FP32_GUARDED), ("fp64", stk.STK_PREC_FP64)):
                kw = dict(n_sims=wi.n_sims, seed=seed, exec_mode=exec_mode, prec=pv)
                pi_.run(wi.s, wi.tt, **kw)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pi_.run(wi.s, wi.tt, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                times[pname] = (e0.elapsed_time(e1), pi_.stats())
        ms_i, si = times["fp32"]
        inhom = {"workload": wi.name, "n": wi.n, "intensity_cells": list(wi.meta["rho"].shape),
                 "sims": wi.n_sims, "dtype": "f32 (guarded, f64 ties)", "job_s": ms_i / 1e3,
                 "sims_per_s": wi.n_sims / (ms_i / 1e3),
                 "value": si["qualifying_pairs"] / (ms_i / 1e3), "unit": UNIT,
                 "pair_kernel_s": si["ms_pair"] / 1e3,
                 "fp64_recomputed": si["fp64_recomputed"],
                 "fp64_job_s": times["fp64"][0] / 1e3}

    # the directional K (8 axial sectors, translation correction; FP32-guarded and FP64) on the
    # Thomas pattern, observed + 99 CSR simulations
    directional = None
    if args.directional and rank == 0:
        wd = _workload("thomas_n200k")
        times = {}
        with stk.Pattern(wd.x, wd.y, wd.t, wd.box) as pd:
            stk.stk_set_stream(pd.h, stream)
            for pname, pv in (("fp32", stk.STK_PREC_FP32_GUARDED), ("fp64", stk.STK_PREC_FP64)):
                kw = dict(n_sims=wd.n_sims, seed=seed, exec_mode=exec_mode, prec=pv,
                          edge_mode=stk.STK_EDGE_TRANSLATION, n_sectors=8)
                pd.run(wd.s, wd.tt, **kw)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pd.run(wd.s, wd.tt, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                times[pname] = (e0.elapsed_time(e1), pd.stats())
        ms_d, sd = times["fp32"]
        directional = {"workload": wd.name, "n": wd.n, "sectors": 8, "edge": "translation",
                       "sims": wd.n_sims, "dtype": "f32 (guarded, f64 ties)",
                       "job_s": ms_d / 1e3, "sims_per_s": wd.n_sims / (ms_d / 1e3),
                       "value": sd["qualifying_pairs"] / (ms_d / 1e3), "unit": UNIT,
                       "pair_kernel_s": sd["ms_pair"] / 1e3,
                       "fp64_recomputed": sd["fp64_recomputed"],
                       "fp64_job_s": times["fp64"][0] / 1e3}

    if rank != 0:
        stk.stk_destroy(h)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    peaks, src = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak_ops = n_sm * 128 * mhz * 1e6  # FP32 lanes x clock = thread-instruction issue rate
    achieved = (OPS_PER_CANDIDATE * cand + OPS_PER_QUALIFYING * qual) / (pair_ms / 1e3)
    per_real = PAIR_DRAM_BYTES_PER_REALIZATION.get(w.name)
    waves = max(1, st.get("waves", 1))
    # bytes per pair launch (a job of R realizations runs in `waves` launches)
    fp32_job = prec == stk.STK_PREC_FP32_GUARDED
    traffic = per_real * st["realizations"] / waves if (per_real and fp32_job) else None
    cb = cpu_baseline(w, target_s=args.cpu_seconds) if args.cpu_seconds > 0 else None
    if cb:
        cb.pop("seconds", None)
    cbg = cpu_grid_baseline(w, target_s=args.cpu_seconds) if args.cpu_seconds > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32 (guarded, f64 ties)"
        if prec == stk.STK_PREC_FP32_GUARDED else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "sims": w.n_sims,
                   "thresholds": [len(w.s), len(w.tt)], "s_max_m": float(w.s[-1]),
                   "t_max_s": float(w.tt[-1]), "exec": args.exec, "prec": args.prec,
                   "l2": "inputs larger than L2 (100 realizations x 2M points resident)",
                   "parallelism": (f"one job split over {ws} ranks: realization blocks + "
                                   "observed-pattern shards, exact all-reduce"
                                   if ws > 1 else "one job, one GPU")},
        "job_s": elapsed_ms / args.steps / 1e3,
        "sims_per_s": w.n_sims * args.steps / (elapsed_ms / 1e3),
        "candidate_pairs_per_step": cand // args.steps,
        "qualifying_pairs_per_step": qual // args.steps,
        "fp64_recomputed_per_step": st["fp64_recomputed"],
        "pair_kernel_ms_per_step": pair_ms / args.steps,
        "launch_shape": {"grid_refinement": [st["grid_refinement"], st["grid_refinement_t"]],
                         "tile_units": st["tile_units"], "blocks_per_sm": st["blocks_per_sm"],
                         "chosen_by": ("environment" if any(
                             os.environ.get(v) for v in ("STK_GRID_F", "STK_TILE_UNITS",
                                                         "STK_BLOCKS_PER_SM"))
                             else "launch-shape tuner (process-wide, per job shape)")},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {mhz:.0f} MHz ({src})"},
        "cpu_baseline": cb,
        "cpu_baseline_grid": cbg,
        "host": host_info(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "plain_fp64": plain,
        "serve": serve,
        "sim_methods": methods,
        "polygon": polygon,
        "polygon_smooth": polygon_smooth,
        "inhomogeneous": inhom,
        "directional": directional,
    }
    print(json.dumps(line), flush=True)
    stk.stk_destroy(h)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="poi_n2M")
    ap.add_argument("--sims", type=int, default=None, help="override the simulation count")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--exec", choices=["batched", "plain"], default="batched")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--compare-fp64", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests per arrival rate in the serving-loop sweep (0: skip it)")
    ap.add_argument("--serve-rates", default="15,30,60",
                    help="mean arrivals per second of the sweep, comma-separated")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-fp64", type=int, default=48,
                    help="requests of the lightest stream also run through a FIFO of plain "
                         "FP64 jobs (0: skip)")
    ap.add_argument("--methods", type=int, default=1,
                    help="also time the job with permutation and bootstrap simulations")
    ap.add_argument("--polygon", type=int, default=1,
                    help="also time a job over an 85-vertex polygon study area")
    ap.add_argument("--inhom", type=int, default=1,
                    help="also time an inhomogeneous-K job (intensity-weighted, FP64)")
    ap.add_argument("--directional", type=int, default=1,
                    help="also time a directional-K job (8 sectors, translation correction)")
    return ap


def main():
    args = build_parser().parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
