"""Warm-start tracking of a load-snapshot sequence (Section IV-C).

Each snapshot changes the bus loads (and, for renewable-tagged generators, the
real-power upper bound) and is solved warm from the previous primal, dual and
penalty state, with the generator ramp limit |p_{t+1} - p_t| <= 2% of p_max of
Section IV-C applied on the device around the previous dispatch.  The loop
only sequences calls of the C ABI; every computation runs in the library.
"""
from __future__ import annotations

import time

import numpy as np


def renewable_pmax(grid, steps: int, seed: int, share: float = 0.2, ramp: float = 0.03):
    """Upper bounds per snapshot: a seeded `share` of the generators is tagged
    renewable and its p_max moves linearly to (1 +- ramp) p_max over the
    horizon (sign drawn per generator); the others keep p_max."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    tagged = rng.random(grid.ngen) < share
    sign = np.where(rng.random(grid.ngen) < 0.5, -1.0, 1.0)
    t = np.arange(1, steps + 1)[:, None] / steps
    return grid.pmax[None, :] * (1.0 + tagged[None, :] * sign[None, :] * ramp * t)


def run_tracking(solver, grid, pds, qds, pmaxs, tol=1e-3, max_iter=5000, ramp_frac=0.02,
                 sync=None):
    """Solve snapshot 0 cold at the grid's own loads, then every snapshot t
    (rows of pds, qds, pmaxs) warm.  Returns the cold record and one record per
    snapshot: iterations, status and latency (host wall time from the first
    input call to the solve's return, which blocks until the device is done)."""
    def _sync():
        if sync is not None:
            sync()

    _sync()
    t0 = time.perf_counter()
    st = solver.solve(tol=tol, max_iter=max_iter, warm_start=False)
    cold_s = time.perf_counter() - t0
    r = solver.residuals()
    cold = dict(status=st, iters=r["iters"], seconds=cold_s)
    out = []
    for t in range(len(pds)):
        _sync()
        t0 = time.perf_counter()
        solver.set_gen_bounds(grid.pmin, pmaxs[t])
        solver.set_ramp_limit(ramp_frac)
        solver.set_loads(pds[t], qds[t])
        st = solver.solve(tol=tol, max_iter=max_iter, warm_start=True)
        dt = time.perf_counter() - t0
        r = solver.residuals()
        out.append(dict(snapshot=t + 1, status=st, iters=r["iters"], latency_s=dt,
                        primal=r["primal"], dual=r["dual"], z_norm=r["z_norm"]))
    return cold, out


def summarize(cold, recs):
    lat = np.array([r["latency_s"] for r in recs]) * 1e3
    its = np.array([r["iters"] for r in recs])
    return {"snapshots": len(recs), "cold_iters": cold["iters"], "cold_s": cold["seconds"],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "mean_iters": float(its.mean()),
            "max_iters": int(its.max()),
            "converged": int(sum(1 for r in recs if r["status"] == 0))}
