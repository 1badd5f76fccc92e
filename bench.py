"""Benchmark: ADMM iterations/s of the component-decomposed ACOPF solver on a
synthetic 70,000-bus grid (88,207 branches, 10,390 generators, Table 1 shape).

A step is one inner ADMM iteration of Algorithm 1 over the whole grid:
branch_tron (every branch subproblem) then bus_dual (generator, bus, z and y
updates, residual reduction, loop control).  The grid state (~80 MB) fits in
L2, so L2 is flushed (256 MiB write) between timed steps.

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# kernels of this library launched per timed step (admm_profile_iterations of
# one iteration): slot_begin, run_begin, branch_tron, bus_dual, control,
# flush_lambda, clear_pending
LAUNCHES_PER_STEP = 7
METRIC = "ADMM iterations/s, 70k-bus synthetic grid (plus time to 1e-3 and p50/p99 tracking latency)"
C_RESIDUALS_BYTES = 72   # sizeof(admm_residuals): 4 int32 + 7 double
UNIT = "iter/s"

# Algorithmic FP64 operations of the branch subproblem solver, counted by
# hand from the operations the method specifies (an FMA counts 2; add, mul,
# div, sqrt, sin and cos 1 each; comparisons, min/max and projections 0).
# Multiplied by the counters the kernel reports for one launch.
FLOPS = dict(
    fgh=392,        # f, gradient and Hessian of eq. branch: flows and their
                    # derivatives (80), coupling/AL accumulation (180), h-terms (54), rest
    f=74,           # f alone at a trial point (flows, residuals, AL terms)
    cauchy=103,     # one Cauchy trial: projected step (18), |s|^2 (12), q(s) (60), g's (12)
    tron_iter=461,  # per TRON iteration besides trials/CG/search/evaluations: projected
                    # gradient, breakpoints, g + H sc, scaled Cholesky, PCG set-up, ratio test
    cg=254,         # one PCG iteration: H p (72), curvature, TR test, updates, M^-1 r (84)
    ps=100,         # one projected-search trial: step (24), q(s) (60), descent test
    al=13,          # one AL pass: h of both ends, multiplier and penalty update
)


def algorithmic_flops(stats: dict) -> float:
    return (FLOPS["fgh"] * stats["fgh_evals"] + FLOPS["f"] * stats["f_evals"]
            + FLOPS["cauchy"] * stats["cauchy_trials"] + FLOPS["tron_iter"] * stats["tron_iters"]
            + FLOPS["cg"] * stats["cg_iters"] + FLOPS["ps"] * stats["ps_trials"]
            + FLOPS["al"] * stats["al_passes"])


# DRAM bytes (read + write) of one branch_tron launch of the default workload
# (70,000 buses, seed 1) from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum).  Reported only while the kernel's code (comments
# aside) is the one the counters were taken on; any change to it makes the
# figure stale (null).
TRAFFIC_CAPTURE = {"nbus": 70000, "seed": 1,
                   "source_digest": "6b67b7ddfa9cda687518f1edbbe25247fd1098a368d904035744fc370060021b",
                   "bytes_per_launch": 22.235648e6 + 0.447744e6}


def kernel_source_digest(path):
    """SHA-256 of a CUDA source with comments and whitespace removed, so that
    only changes to the code itself count."""
    import hashlib
    import re
    with open(path, encoding="utf-8") as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256("".join(text.split()).encode()).hexdigest()


def branch_tron_traffic(args):
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2110_06879_gb300",
                       "csrc", "branch_tron.cu")
    try:
        digest = kernel_source_digest(src)
    except OSError:
        return None
    c = TRAFFIC_CAPTURE
    if digest != c["source_digest"] or args.nbus != c["nbus"] or args.seed != c["seed"]:
        return None
    return c["bytes_per_launch"]


def fp64_peak_gflops(fma_per_clk_smsp=0.5, sm_mhz=2070.0, sms=152):
    """FP64 peak from unit counts and clock: SMs x 4 sub-partitions x FP64 FMAs
    per clock per sub-partition (0.5 on GB300: one warp instruction per 64
    cycles; measured live by admm_fp64_peak) x 2 flops x the SM clock
    (152 x 4 x 0.5 x 2 x 2.07 GHz = 1,258.6 GFLOP/s)."""
    return sms * 4 * fma_per_clk_smsp * 2 * sm_mhz / 1e3


def bus_dual_work(grid):
    """Algorithmic work of one bus_dual launch (one inner iteration's
    generator, bus, z and y updates and residual sums), from the closed forms:
    FP64 flops (an FMA counts 2) and compulsory DRAM bytes.
      per branch-end coupling 36 flops: target u + z + y/rho (3), bus sums
        (2.5), bus copy (2.5), dual residual (2), u - xbar (1), z (4), y (3),
        seven squared norms (15), branch target xbar - z - y/rho (3);
      per generator coupling 41 (the closed-form generator update instead of
        the branch target); per bus 30 (pooled w, 2x2 solve, theta);
      bytes per branch end 228 (reads u, z, y 4 each, sx 2, col; writes z, y 4
        each, sx 2, targets 4), per generator 164, per bus 68."""
    nb, nl, ng = grid.nbus, grid.nbranch, grid.ngen
    flops = 36 * 8 * nl + 41 * 2 * ng + 30 * nb
    nbytes = 228 * 2 * nl + 164 * ng + 68 * nb
    return flops, nbytes


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json, driver-written),
    else the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json"), encoding="utf-8") as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


class ClockSampler:
    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # let the sampler produce its first line before the timed region starts
        t0 = time.perf_counter()
        while self.p and time.perf_counter() - t0 < 2.0 and os.path.getsize(self.f.name) == 0:
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                for n, v in zip(names, r[3:7]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job_rate(t_local_s, steps, device=None):
    """Replicas: every rank times its own `steps`; the whole job's rate is the
    steps all ranks processed over the slowest rank's time (max over ranks,
    the one collective of the bench, outside the timed region).  Returns
    (rate, max time)."""
    import torch
    import torch.distributed as dist
    ws, t = 1, float(t_local_s)
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return ws * steps / t, t


def make_workload(nbus, seed):
    from paper_2110_06879_gb300 import synth
    grid = synth.sized_grid(nbus, seed=seed)
    rp, rv, so = synth.penalties_for(nbus)
    return grid, dict(rho_pq=rp, rho_va=rv, obj_scale=so)


def cpu_baseline(grid, opts, seconds=15.0):
    """The oracle as it stands on the host cores: iterations after a one-
    iteration cold start, until about `seconds` of CPU time are spent."""
    import oracle
    o = oracle.Oracle(grid, **opts)
    o.solve(tol=0.0, max_iter=1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.solve(tol=0.0, max_iter=1, warm_start=True)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{n} warm iterations (iterations 2..{n + 1} of a cold solve) of the "
                      f"{grid.nbus}-bus grid, single-threaded C oracle"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    grid, opts = make_workload(args.nbus, args.seed)
    import oracle
    o = oracle.Oracle(grid, **opts)
    o.solve(tol=0.0, max_iter=1)
    for _ in range(args.warmup):
        o.solve(tol=0.0, max_iter=1, warm_start=True)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.solve(tol=0.0, max_iter=1, warm_start=True)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(grid, opts, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1,
                             "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} warm ADMM iterations of the {grid.nbus}-bus "
                                       "grid after a cold start and warm-up, single-threaded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(grid, opts, args):
    return {"workload": f"synthetic {grid.nbus}-bus grid ({grid.nbranch} branches, {grid.ngen} "
                        f"generators), one inner ADMM iteration per step after a cold start",
            "nbus": grid.nbus, "nbranch": grid.nbranch, "ngen": grid.ngen, "seed": args.seed,
            "rho_pq": opts["rho_pq"], "rho_va": opts["rho_va"], "obj_scale": opts["obj_scale"],
            "l2": "flushed (256 MiB write) between timed steps", "parallelism": "replicas"}


STOP_RULE = ("standard ADMM test (Boyd et al. 2011, Sec. 3.3.1), absolute and relative tolerance "
             "both tol: ||u - xbar||_2 <= sqrt(m) tol + tol max(||u||_2, ||xbar||_2), "
             "||rho (xbar - xbar_prev)||_2 <= sqrt(m) tol + tol ||y||_2, and ||z||_2 <= the "
             "first bound (two-level); m couplings")


def solve_timed(s, stream, tol, max_iter, warm):
    """One admm_solve (a single graph launch) timed with CUDA events on the
    handle's stream, with the residual norms, the objective and ||c(x)||_inf of
    the point it returns."""
    import torch
    from paper_2110_06879_gb300 import admm
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.solve_async(tol=tol, max_iter=max_iter, warm_start=warm)
    ev1.record(stream)
    torch.cuda.synchronize()
    r = s.residuals()
    sol = s.solution()
    secs = ev0.elapsed_time(ev1) / 1e3
    return {"tol": tol, "warm_start": bool(warm), "seconds": secs, "iters": r["iters"],
            "iters_per_s": r["iters"] / secs if secs > 0 else None,
            "outer_iters": r["outer_iters"],
            "status": admm.lib().admm_status_string(r["status"]).decode(),
            "primal": r["primal"], "eps_pri": r["eps_pri"], "dual": r["dual"],
            "eps_dual": r["eps_dual"], "z_norm": r["z_norm"], "objective": sol["objective"],
            "max_viol": sol["max_viol"], "stop_rule": STOP_RULE}


def time_to_violation(s, stream, target, max_iter, chunk):
    """Cold start, then `chunk` iterations at a time (one graph launch each)
    until ||c(x)||_inf of the current point (flows recomputed from the bus
    voltages; power balance, line limits at the full rating, voltage bounds)
    is at most `target`, or max_iter iterations.  The timed region includes the
    evaluation of ||c(x)||_inf after every chunk."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    s.slot_begin(0, tol=0.0, max_iter=max_iter, warm_start=False)
    it, sol, best = 0, None, None
    while it < max_iter:
        s.run(chunk)
        sol = s.solution()
        it = int(s.slot_status()[1][0])
        if best is None or sol["max_viol"] < best[1]:
            best = (it, sol["max_viol"])
        if sol["max_viol"] <= target:
            break
    ev1.record(stream)
    torch.cuda.synchronize()
    secs = ev0.elapsed_time(ev1) / 1e3
    reached = sol["max_viol"] <= target
    return {"target_max_viol": target, "reached": bool(reached), "seconds": secs, "iters": it,
            "max_viol": sol["max_viol"], "objective": sol["objective"],
            "best_max_viol": best[1], "best_at_iter": best[0], "check_every": chunk,
            "max_iter": max_iter}


def shard_scenarios(sizes, ws, rank):
    """Indices of the scenarios rank `rank` of `ws` solves: longest first onto
    the least-loaded rank (load = buses), ties to the lower rank; disjoint,
    covering, identical on every rank."""
    load = [0] * ws
    mine = []
    for k in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(ws), key=lambda q: (load[q], q))
        load[r] += sizes[k]
        if r == rank:
            mine.append(k)
    return sorted(mine)


def reduce_over_ranks(seconds, counts, device=None):
    """Max of `seconds` and sums of `counts` (a dict of numbers) over ranks;
    identity without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, dict(counts)
    keys = sorted(counts)
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([float(counts[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), {k: float(v) for k, v in zip(keys, c.tolist())}


def run_batched(args, admm, stream, device=None):
    """Scenarios of uneven size in one batched handle (one persistent launch
    per iteration over the flattened component index, per-scenario stopping),
    autotuned; against a loop of plain one-grid solves on a sample.  With
    several ranks the scenarios are sharded (longest first, balanced by bus
    count) with no collective on the data path; the job's rate is all
    scenarios over the slowest rank's time."""
    import numpy as np
    import torch
    from paper_2110_06879_gb300 import synth
    ws, rank, _ = dist_env()
    grids_all = synth.batch_grids(args.batched, lo=500, hi=20000, seed=args.seed)
    mine = shard_scenarios([g.nbus for g in grids_all], ws, rank)
    grids = [grids_all[k] for k in mine]
    kw = dict(rho_pq=3e3, rho_va=3e4)
    b = admm.Solver(grids, stream=stream, **kw)
    blocks, body, _, lanes = b.autotune(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.solve(tol=1e-3, max_iter=3000)        # cold start of every scenario
    dt_local = time.perf_counter() - t0
    st, it = b.slot_status()
    b.close()
    dt, tot = reduce_over_ranks(dt_local, {"scenarios": len(grids), "converged": int((st == 0).sum())},
                                device=device)
    rng = np.random.default_rng(args.seed)
    sample = rng.choice(len(grids_all), min(args.batch_sample, len(grids_all)), replace=False)
    tloop = 0.0
    if rank == 0:
        for k in sample:
            s = admm.Solver(grids_all[int(k)], stream=stream, **kw)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s.solve(tol=1e-3, max_iter=3000)
            tloop += time.perf_counter() - t1
            s.close()
    n_all = int(tot["scenarios"])
    return {"scenarios": n_all, "buses": int(sum(g.nbus for g in grids_all)),
            "branches": int(sum(g.nbranch for g in grids_all)), "seconds": dt,
            "scenarios_per_s": n_all / dt, "converged": int(tot["converged"]),
            "ranks": ws, "sharding": "longest first by buses, no collective on the data path",
            "iters_p50": int(np.median(it)), "iters_max": int(it.max()),   # rank 0's scenarios
            "autotuned_branch_blocks": blocks, "autotuned_graph_body_iters": body,
            "autotuned_lanes_per_branch": lanes,
            "plain_loop_sample": len(sample),
            "plain_loop_scenarios_per_s": len(sample) / tloop if tloop > 0 else None,
            "speedup_vs_plain_loop": (n_all / dt) / (len(sample) / tloop) if tloop > 0 else None,
            "tol": 1e-3, "max_iter": 3000, "rho_pq": kw["rho_pq"], "rho_va": kw["rho_va"]}


def gather_objects(obj):
    """Every rank's `obj`, in rank order (just [obj] without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def run_served(args, admm, stream):
    """Continuous batching over a resident pool (log-uniform 1k-70k buses, one
    grid pinned at 70k) under Poisson load-snapshot requests at each rate of
    --rates, against the same streams served by serial plain solves.  With
    several ranks the pool is sharded like the batched scenarios and each rank
    serves the requests for its own grids; the records are gathered once per
    rate at the end."""
    import dataclasses
    import numpy as np
    from paper_2110_06879_gb300 import serve, synth
    ws, rank, _ = dist_env()
    rng = np.random.Generator(np.random.PCG64(args.seed + 5))
    sizes = list(np.exp(rng.uniform(np.log(1000), np.log(70000), args.pool - 1)).astype(int))
    sizes.append(70000)
    grids = [synth.sized_grid(int(n), seed=500 + k) for k, n in enumerate(sizes)]
    mine = shard_scenarios(sizes, ws, rank)
    local = {k: i for i, k in enumerate(mine)}
    my_grids = [grids[k] for k in mine]
    srv = serve.Server(my_grids, mem_budget=args.mem_budget_gb << 30, tick_iters=8, max_iter=500,
                       stream=stream)
    warm = srv.warm_up()
    serial_solvers = {}
    per_rate = []
    for q, rate in enumerate(args.rates):
        duration = min(args.serve_seconds, args.max_requests / rate)
        deadline = duration + args.grace_seconds
        reqs = serve.poisson_requests(grids, rate=rate, duration=duration,
                                      seed=args.seed + 9 + 101 * q)
        my_reqs = [dataclasses.replace(r, grid=local[r.grid]) for r in reqs if r.grid in local]
        recs, rejected, wall = srv.run(my_reqs, deadline=deadline)
        recs2, wall2 = serve.serial_baseline(my_grids, my_reqs, max_iter=500, stream=stream,
                                             deadline=deadline, solvers=serial_solvers)
        parts = gather_objects(dict(recs=recs, rejected=len(rejected), wall=wall, recs2=recs2,
                                    wall2=wall2))
        all_recs = [r for p in parts for r in p["recs"]]
        all_recs2 = [r for p in parts for r in p["recs2"]]
        per_rate.append({"rate_per_s": rate, "arrival_seconds": duration,
                         "no_admission_after_s": deadline,
                         "served": serve.summarize(all_recs, max(p["wall"] for p in parts)),
                         "rejected": sum(p["rejected"] for p in parts),
                         "serial": serve.summarize(all_recs2, max(p["wall2"] for p in parts))})
    # the same pool under a device-memory budget that holds about half of it:
    # grids are swapped in as requests for them arrive (idle ones evicted,
    # least recently used first, their states kept on the host)
    limited = None
    if args.limited_share > 0:
        states = srv.saved_states()
        budget = int(args.limited_share * serve.state_bytes(my_grids))
        srv2 = serve.Server(my_grids, mem_budget=budget, tick_iters=8, max_iter=500, stream=stream,
                            states=states, tuned=srv.tuned)
        rate = args.rates[0]
        duration = min(args.serve_seconds, args.max_requests / rate)
        reqs = serve.poisson_requests(grids, rate=rate, duration=duration, seed=args.seed + 77)
        my_reqs = [dataclasses.replace(r, grid=local[r.grid]) for r in reqs if r.grid in local]
        resident0 = len(srv2.grid_ids)
        recs, rejected, wall = srv2.run(my_reqs, deadline=duration + args.grace_seconds)
        parts = gather_objects(dict(recs=recs, rejected=len(rejected), wall=wall,
                                    swaps=srv2.swaps, evictions=srv2.evictions, budget=budget,
                                    resident0=resident0))
        limited = {"rate_per_s": rate, "arrival_seconds": duration,
                   "budget_bytes": sum(p["budget"] for p in parts),
                   "budget_share_of_pool": args.limited_share,
                   "initially_resident": sum(p["resident0"] for p in parts),
                   "swaps": sum(p["swaps"] for p in parts),
                   "evictions": sum(p["evictions"] for p in parts),
                   "served": serve.summarize([r for p in parts for r in p["recs"]],
                                             max(p["wall"] for p in parts)),
                   "rejected": sum(p["rejected"] for p in parts)}
        srv2.solver.close()
    srv.solver.close()
    for sv in serial_solvers.values():
        sv.close()
    info = gather_objects(dict(resident=len(srv.grid_ids), bytes=srv.bytes, warm=warm,
                               tuned=srv.tuned))
    tuned = info[0]["tuned"]
    return {"pool": len(grids), "ranks": ws,
            "resident": sum(p["resident"] for p in info),
            "resident_bytes": sum(p["bytes"] for p in info),
            "pool_buses": int(sum(sizes)),
            "autotuned_branch_blocks": tuned[0] if tuned else None,
            "autotuned_graph_body_iters": tuned[1] if tuned else None,
            "autotuned_lanes_per_branch": tuned[3] if tuned else None,
            "pool_cold_solve_s": max(p["warm"] for p in info),
            "rates": per_rate, "memory_limited": limited,
            "tol": 1e-3, "max_iter_per_request": 500, "tick_iters": 8}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_2110_06879_gb300 import admm

    grid, opts = make_workload(args.nbus, args.seed + rank)
    stream = torch.cuda.current_stream()
    s = admm.Solver(grid, stream=stream, **opts)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # warm-up: cold start + W iterations; the state after them is kept so that
    # the end-to-end leg times exactly the same iterations
    s.solve(tol=0.0, max_iter=max(args.warmup, 3))
    torch.cuda.synchronize()
    checkpoint = s.get_state()
    st0 = s.stats()
    stats_acc = {k: 0 for k in st0}
    branch_ms, iter_ms, bus_ms = [], [], []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            p = s.profile_iterations(1)
            st = s.stats()
            for k in stats_acc:
                stats_acc[k] += st[k]
            branch_ms.append(p["branch_ms"])
            bus_ms.append(p["bus_ms"])
            iter_ms.append(p["iter_ms"])
        torch.cuda.synchronize()
    clocks = clk.summary()
    value, t_total = whole_job_rate(sum(iter_ms) / 1e3, args.steps, device=dev)

    # dominant kernel roofline (FP64 ALU bound): the peak from the FP64 rate
    # per clock measured live by the calibration kernel, at the SM clock the
    # timed region ran at
    cal = admm.fp64_peak(20000, stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = fp64_peak_gflops(cal["fma_per_clk_smsp"], mhz, sms)
    b_mean = sum(branch_ms) / len(branch_ms)
    flops_per_launch = algorithmic_flops(stats_acc) / args.steps
    achieved = flops_per_launch / (b_mean * 1e-3) / 1e9
    u_mean = sum(bus_ms) / len(bus_ms)
    bd_flops, bd_bytes = bus_dual_work(grid)
    bd_achieved = bd_flops / (u_mean * 1e-3) / 1e9
    hbm_peak = measured_hbm_gbs()

    # end to end through the public API with host buffers, over the same
    # iterations (state restored to the end of the warm-up)
    pd = torch.tensor(grid.pd, dtype=torch.float64).pin_memory().numpy()
    qd = torch.tensor(grid.qd, dtype=torch.float64).pin_memory().numpy()
    s.set_state(checkpoint)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_loads(pd, qd)
        s.solve_async(tol=0.0, max_iter=1, warm_start=True)
        s.residuals()               # device -> host read of the step's result
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": args.steps / e2e_dt * ws, "unit": UNIT,
           "h2d_bytes_per_step": int(pd.nbytes + qd.nbytes),
           "d2h_bytes_per_step": C_RESIDUALS_BYTES}

    # time to residual 1e-3 from a cold start (whole solve, one graph launch),
    # then warm after one AR(1) load step (Section IV-C)
    tt = tt_warm = None
    if args.time_to_tol:
        tt = solve_timed(s, stream, 1e-3, args.tol_max_iter, False)
        tt["graph_launches"] = 1
        from paper_2110_06879_gb300 import synth
        pd1, qd1 = synth.ar1_loads(grid, 1, seed=args.seed + 400 + rank)
        s.set_loads(pd1[0], qd1[0])
        tt_warm = solve_timed(s, stream, 1e-3, args.tol_max_iter, True)
        tt_warm["load_step"] = "one AR(1) step, phi 0.9, 1% noise per bus"
        s.set_loads(grid.pd, grid.qd)

    # time to a usable point: ||c(x)||_inf <= 1.5e-2 (Table 2's level at 70k)
    feas = None
    if args.feasible:
        fs = admm.Solver(grid, stream=stream, **dict(opts, rho_pq=args.feas_rho[0],
                                                     rho_va=args.feas_rho[1]))
        feas = time_to_violation(fs, stream, args.feas_target, args.feas_max_iter, 100)
        feas.update({"rho_pq": args.feas_rho[0], "rho_va": args.feas_rho[1]})
        fs.close()

    # the one-level variant (z = 0, Mhanna et al.) on the same grid, as a speed
    # comparison: time to the same tolerance from a cold start; and the
    # two-level method with the adaptive outer penalty (beta_rule 1)
    tt1 = tta = None
    if args.time_to_tol and args.one_level:
        s1 = admm.Solver(grid, stream=stream, two_level=0, **opts)
        tt1 = solve_timed(s1, stream, 1e-3, args.tol_max_iter, False)
        s1.close()
        sa = admm.Solver(grid, stream=stream, beta_rule=1, **opts)
        tta = solve_timed(sa, stream, 1e-3, args.tol_max_iter, False)
        sa.close()

    # smaller grids of the same kind (2k, 10k): time to 1e-3 and to the
    # violation target, and the 2k objective against the oracle's own solve
    sizes = None
    if args.sizes:
        from paper_2110_06879_gb300 import synth
        sizes = []
        for nb in args.sizes:
            g2 = synth.sized_grid(nb, seed=args.seed + rank)
            o2 = dict(rho_pq=args.size_rho[0], rho_va=args.size_rho[1], obj_scale=1.0)
            # launch shape from the library's tuner (on a separate handle, a few
            # iterations into a cold solve); every leg of this grid uses it
            tp = admm.Solver(g2, stream=stream, **o2)
            tp.solve(tol=0.0, max_iter=5)
            tb, tbody, _, tl = tp.autotune(4)
            tp.close()
            shape = dict(branch_blocks=tb, graph_body_iters=tbody, lanes_per_branch=tl)
            s2 = admm.Solver(g2, stream=stream, **o2, **shape)
            rec = {"nbus": nb, "nbranch": g2.nbranch, "ngen": g2.ngen,
                   "rho_pq": o2["rho_pq"], "rho_va": o2["rho_va"],
                   "launch_shape": {"branch_blocks": tb, "graph_body_iters": tbody,
                                    "lanes_per_branch": tl},
                   "time_to_tol": solve_timed(s2, stream, 1e-3, args.tol_max_iter, False)}
            s2.close()
            # the adaptive outer penalty (beta_rule 1), same grid and penalties
            s5 = admm.Solver(g2, stream=stream, beta_rule=1, **o2, **shape)
            rec["time_to_tol_adaptive_beta"] = solve_timed(s5, stream, 1e-3, args.tol_max_iter,
                                                           False)
            s5.close()
            if args.feasible:
                s3 = admm.Solver(g2, stream=stream, **shape, **dict(o2, rho_pq=args.feas_rho[0],
                                                                   rho_va=args.feas_rho[1]))
                rec["time_to_max_viol"] = time_to_violation(s3, stream, args.feas_target,
                                                            args.feas_max_iter, 100)
                rec["time_to_max_viol"].update({"rho_pq": args.feas_rho[0],
                                                "rho_va": args.feas_rho[1]})
                s3.close()
                s6 = admm.Solver(g2, stream=stream, beta_rule=1, **shape,
                                 **dict(o2, rho_pq=args.feas_rho[0], rho_va=args.feas_rho[1]))
                rec["time_to_max_viol_adaptive_beta"] = time_to_violation(
                    s6, stream, args.feas_target, args.feas_max_iter, 100)
                s6.close()
                # the one-level variant (z = 0) at its own penalties
                s4 = admm.Solver(g2, stream=stream, two_level=0, **shape,
                                 **dict(o2, rho_pq=args.feas_rho1[0], rho_va=args.feas_rho1[1]))
                rec["time_to_max_viol_one_level"] = time_to_violation(
                    s4, stream, args.feas_target, args.feas_max_iter, 100)
                rec["time_to_max_viol_one_level"].update({"rho_pq": args.feas_rho1[0],
                                                          "rho_va": args.feas_rho1[1]})
                s4.close()
            if nb == args.lanes_nbus:
                # one lane against two lanes per branch on the same iterations
                # (iterations 6-25 of a cold solve), and the autotuner's pick
                lc = {}
                for lanes in (1, 2):
                    sl = admm.Solver(g2, stream=stream, lanes_per_branch=lanes, **o2)
                    sl.solve(tol=0.0, max_iter=5)
                    pr = [sl.profile_iterations(1) for _ in range(20)]
                    lc[f"lanes_{lanes}_branch_ms"] = sum(p["branch_ms"] for p in pr) / len(pr)
                    sl.close()
                st_ = admm.Solver(g2, stream=stream, **o2)
                st_.solve(tol=0.0, max_iter=5)
                tb, tbody, tms, tl = st_.autotune(4)
                st_.close()
                lc.update({"autotuned_lanes_per_branch": tl, "autotuned_branch_blocks": tb,
                           "autotuned_branch_ms": tms})
                rec["lanes_per_branch"] = lc
            gpu_iters = rec["time_to_tol"]["iters"]
            if rank == 0 and nb <= args.gap_max_nbus and gpu_iters > args.gap_max_iter:
                rec["oracle"] = {"skipped": f"the GPU solve took {gpu_iters} iterations; the "
                                            f"oracle leg runs at most {args.gap_max_iter}"}
            elif rank == 0 and nb <= args.gap_max_nbus:
                # the oracle's own solve of the same problem, at most as many
                # iterations as the GPU took (the trajectories agree, so both
                # stop on the same iteration)
                import oracle
                oo = oracle.Oracle(g2, **o2)
                t0 = time.perf_counter()
                st = oo.solve(tol=1e-3, max_iter=gpu_iters)
                osec = time.perf_counter() - t0
                of = oo.finalize()
                og = rec["time_to_tol"]["objective"]
                rec["oracle"] = {"status": int(st), "iters": oo.residuals()["iters"],
                                 "seconds_1core": osec, "objective": of["objective"],
                                 "max_viol": of["max_viol"],
                                 "objective_gap_rel": abs(og - of["objective"]) / abs(of["objective"])}
            sizes.append(rec)

    # warm-start tracking: 10k-bus grid, AR(1) load snapshots, renewable ramps,
    # 2% ramp limit, each snapshot warm-started (Section IV-C)
    track = None
    if args.tracking:
        from paper_2110_06879_gb300 import synth, tracking
        tgrid = synth.sized_grid(10000, seed=args.seed + 100 + rank)
        topts = dict(rho_pq=3e3, rho_va=3e4, obj_scale=1.0)
        ts = admm.Solver(tgrid, stream=stream, **topts)
        tuned_t = ts.autotune(4)        # launch shape for this grid (state put back)
        pds, qds = synth.ar1_loads(tgrid, args.track_steps, seed=args.seed + 200 + rank)
        pmaxs = tracking.renewable_pmax(tgrid, args.track_steps, seed=args.seed + 300 + rank)
        cold, recs = tracking.run_tracking(ts, tgrid, pds, qds, pmaxs, tol=1e-3, max_iter=5000,
                                           sync=torch.cuda.synchronize)
        track = tracking.summarize(cold, recs)
        track.update({"workload": f"synthetic {tgrid.nbus}-bus grid ({tgrid.nbranch} branches, "
                                  f"{tgrid.ngen} generators), AR(1) loads phi 0.9 noise 1%, 20% "
                                  "renewable p_max ramps +-3%, ramp limit 2% p_max, warm starts",
                      "rho_pq": topts["rho_pq"], "rho_va": topts["rho_va"], "tol": 1e-3,
                      "stop_rule": STOP_RULE, "autotuned_branch_blocks": tuned_t[0],
                      "autotuned_graph_body_iters": tuned_t[1],
                      "autotuned_lanes_per_branch": tuned_t[3]})
        ts.close()

    batched = run_batched(args, admm, stream, device=dev) if args.batched > 0 else None
    served = run_served(args, admm, stream) if args.served else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sum(iter_ms) / len(iter_ms),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(grid, opts, args),
                "roofline": {"kernel": "branch_tron", "bound": "alu", "achieved": achieved,
                             "peak": peak, "unit": "GFLOP/s (FP64)", "frac": achieved / peak,
                             "traffic": branch_tron_traffic(args), "traffic_unit": "bytes",
                             "ms_per_launch": b_mean,
                             "flops_per_launch": flops_per_launch,
                             "peak_source": "SMs x 4 x measured FP64 FMA/clk per sub-partition "
                                            "x 2 x max SM clock sampled in the timed region"},
                "roofline_bus_dual": {"kernel": "bus_dual", "bound": "alu", "achieved": bd_achieved,
                                      "peak": peak, "unit": "GFLOP/s (FP64)",
                                      "frac": bd_achieved / peak, "ms_per_launch": u_mean,
                                      "flops_per_launch": bd_flops,
                                      "bytes_per_launch": bd_bytes,
                                      "achieved_gbs": bd_bytes / (u_mean * 1e-3) / 1e9,
                                      "hbm_peak_gbs": hbm_peak,
                                      "hbm_frac": (bd_bytes / (u_mean * 1e-3) / 1e9 / hbm_peak)
                                      if hbm_peak else None},
                "fp64_calibration": cal,
                "bus_dual_ms": u_mean,
                "branch_solves_per_s": value * grid.nbranch,
                "e2e": e2e, "clocks": clocks, "gpu_launches": LAUNCHES_PER_STEP * args.steps * ws,
                "tron_stats_per_step": {k: v / args.steps for k, v in stats_acc.items()}}
        if tt is not None:
            line["time_to_tol"] = tt
        if tt_warm is not None:
            line["time_to_tol_warm"] = tt_warm
        if feas is not None:
            line["time_to_max_viol"] = feas
        if tt1 is not None:
            line["time_to_tol_one_level"] = tt1
        if tta is not None:
            line["time_to_tol_adaptive_beta"] = tta
        if sizes is not None:
            line["grids"] = sizes
        if track is not None:
            line["tracking"] = track
        if batched is not None:
            line["batched"] = batched
        if served is not None:
            line["served"] = served
        if args.cpu_baseline and ws >= 1:
            line["cpu_baseline"] = cpu_baseline(grid, opts, args.cpu_seconds)
        print(json.dumps(line))
    s.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nbus", type=int, default=70000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-time-to-tol", dest="time_to_tol", action="store_false")
    ap.add_argument("--tol-max-iter", type=int, default=5000)
    ap.add_argument("--no-feasible", dest="feasible", action="store_false",
                    help="skip the time-to-||c(x)||_inf legs")
    ap.add_argument("--feas-target", type=float, default=1.5e-2)
    ap.add_argument("--feas-max-iter", type=int, default=12000)
    ap.add_argument("--feas-rho", type=float, nargs=2, default=[3e4, 3e6])
    ap.add_argument("--feas-rho1", type=float, nargs=2, default=[1e4, 1e6],
                    help="penalties of the one-level time-to-violation leg on the smaller grids")
    ap.add_argument("--sizes", type=int, nargs="*", default=[2000, 10000],
                    help="smaller grids timed to 1e-3 and to the violation target")
    ap.add_argument("--size-rho", type=float, nargs=2, default=[3e3, 3e4])
    ap.add_argument("--gap-max-nbus", type=int, default=10000,
                    help="largest grid whose objective is compared with an oracle solve")
    ap.add_argument("--lanes-nbus", type=int, default=10000,
                    help="grid of --sizes on which one and two lanes per branch are compared")
    ap.add_argument("--gap-max-iter", type=int, default=1500,
                    help="longest GPU solve (iterations) the oracle comparison repeats")
    ap.add_argument("--no-tracking", dest="tracking", action="store_false")
    ap.add_argument("--no-one-level", dest="one_level", action="store_false",
                    help="skip the one-level (z = 0) time-to-tolerance comparison")
    ap.add_argument("--batched", type=int, default=256,
                    help="scenarios of the batched leg (0 skips it)")
    ap.add_argument("--batch-sample", type=int, default=8)
    ap.add_argument("--no-served", dest="served", action="store_false",
                    help="skip the continuous-batching leg")
    ap.add_argument("--pool", type=int, default=32)
    ap.add_argument("--rates", type=float, nargs="+", default=[50.0, 200.0, 2000.0])
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="longest arrival window per rate")
    ap.add_argument("--max-requests", type=int, default=300,
                    help="arrival window per rate is at most this many mean arrivals")
    ap.add_argument("--grace-seconds", type=float, default=3.0,
                    help="admission closes this long after the last arrival")
    ap.add_argument("--mem-budget-gb", type=int, default=16)
    ap.add_argument("--limited-share", type=float, default=0.5,
                    help="served pool again under this share of its device bytes (0 skips)")
    ap.add_argument("--track-steps", type=int, default=60)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
