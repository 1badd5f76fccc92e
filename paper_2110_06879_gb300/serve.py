"""Continuous-batching request loop for load-snapshot solves (tracking under
load fluctuation, Section IV-C, served).

A pool of grids stays resident in one batched handle, each grid a slot whose
primal, dual and penalty state persists between requests (warm starts).
Requests carry a new load snapshot for one grid.  The loop admits a waiting
request as soon as its grid's slot is free, even while other slots are being
iterated, runs the batched iteration graph for a few iterations at a time
(`tick_iters`), and retires every slot whose solve has stopped.  Grids enter
the pool while their device state fits the memory budget.  All computation
runs in the library; this loop only sequences C-ABI calls.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import admm

# device bytes of one grid's state, per component (the handle's layout rounded up)
_BYTES_PER_BUS = 8 * 10 + 4
_BYTES_PER_BRANCH = 8 * 43 + 4 * 3 + 2 * 4 * 20 + 8 * 12 * 2
_BYTES_PER_GEN = 8 * 11 + 4 + 8 * 12


def state_bytes(grid) -> int:
    """Approximate device memory one grid occupies in a handle."""
    return (grid.nbus * _BYTES_PER_BUS + grid.nbranch * _BYTES_PER_BRANCH
            + grid.ngen * _BYTES_PER_GEN)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    grid: int               # index into the server's grid list
    pd: np.ndarray
    qd: np.ndarray


class Server:
    def __init__(self, grids, mem_budget: int, rho_pq=3e3, rho_va=3e4, tol=1e-3, max_iter=2000,
                 tick_iters=8, stream=None, **opts):
        admitted, used = [], 0
        for k, g in enumerate(grids):
            b = state_bytes(g)
            if used + b <= mem_budget:
                admitted.append(k)
                used += b
        if not admitted:
            raise ValueError("no grid fits the memory budget")
        self.grid_ids = admitted
        self.slot_of = {k: s for s, k in enumerate(admitted)}
        self.grids = [grids[k] for k in admitted]
        self.bytes = used
        self.tol, self.max_iter, self.tick = tol, max_iter, tick_iters
        self.rho = (rho_pq, rho_va)
        self.solver = admm.Solver(self.grids, stream=stream, rho_pq=rho_pq, rho_va=rho_va, **opts)
        self.tuned = None

    def warm_up(self, max_iter=5000, tune=True):
        """Cold-solve every resident grid once, all together, then (tune) pick
        the launch shape for the pool on replayed iterations (the tuner puts
        the state back, so no result changes); returns seconds."""
        t0 = time.perf_counter()
        self.solver.solve(tol=self.tol, max_iter=max_iter)
        self.tuned = self.solver.autotune(2) if tune else None
        return time.perf_counter() - t0

    def run(self, requests, deadline: float = float("inf")):
        """Serve `requests` (sorted by arrival) in real time; returns one record
        per request (latency = completion - arrival, iterations, status), the
        requests for grids that are not resident, and the wall time.  After
        `deadline` seconds no request is admitted any more: solves in flight
        finish, waiting ones are returned with status "dropped"."""
        s = self.solver
        pending = collections.deque(r for r in requests if r.grid in self.slot_of)
        rejected = [r for r in requests if r.grid not in self.slot_of]
        waiting = collections.defaultdict(collections.deque)   # slot -> queued requests
        busy = {}                                             # slot -> request in flight
        out = []
        t0 = time.perf_counter()
        total = len(pending)
        while len(out) < total:
            now = time.perf_counter() - t0
            if now > deadline and not busy:
                for q in waiting.values():
                    out.extend(dict(rid=r.rid, grid=r.grid, latency_s=float("nan"), iters=0,
                                    status="dropped") for r in q)
                    q.clear()
                out.extend(dict(rid=r.rid, grid=r.grid, latency_s=float("nan"), iters=0,
                                status="dropped") for r in pending)
                pending.clear()
                break
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                waiting[self.slot_of[r.grid]].append(r)
            # admit: every free slot with a waiting request joins the batch
            for slot, q in waiting.items():
                if q and slot not in busy and now <= deadline:
                    r = q.popleft()
                    s.select(slot)
                    s.set_loads(r.pd, r.qd)
                    s.slot_begin(slot, tol=self.tol, max_iter=self.max_iter, warm_start=True,
                                 rho_pq=self.rho[0], rho_va=self.rho[1])
                    busy[slot] = r
            if not busy:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
                continue
            s.run(self.tick)
            status, iters = s.slot_status()       # waits for the tick
            done_t = time.perf_counter() - t0
            for slot in list(busy):
                if status[slot] != 2:
                    r = busy.pop(slot)
                    out.append(dict(rid=r.rid, grid=r.grid, latency_s=done_t - r.arrival,
                                    iters=int(iters[slot]), status=int(status[slot])))
        wall = time.perf_counter() - t0
        return out, rejected, wall


def serial_baseline(grids, requests, rho_pq=3e3, rho_va=3e4, tol=1e-3, max_iter=2000,
                    stream=None, deadline: float = float("inf"), **opts):
    """The same request stream through plain one-grid handles, one solve at a
    time in arrival order (each grid warm from its previous solve); requests
    not started by `deadline` seconds are dropped."""
    solvers = {}
    for k in sorted({r.grid for r in requests}):
        sv = admm.Solver(grids[k], stream=stream, rho_pq=rho_pq, rho_va=rho_va, **opts)
        sv.solve(tol=tol, max_iter=5000)
        solvers[k] = sv
    out = []
    t0 = time.perf_counter()
    for r in requests:
        now = time.perf_counter() - t0
        if now > deadline:
            out.append(dict(rid=r.rid, grid=r.grid, latency_s=float("nan"), iters=0,
                            status="dropped"))
            continue
        if r.arrival > now:
            time.sleep(r.arrival - now)
        sv = solvers[r.grid]
        sv.set_loads(r.pd, r.qd)
        st = sv.solve(tol=tol, max_iter=max_iter, warm_start=True)
        done_t = time.perf_counter() - t0
        out.append(dict(rid=r.rid, grid=r.grid, latency_s=done_t - r.arrival,
                        iters=sv.residuals()["iters"], status=st))
    wall = time.perf_counter() - t0
    for sv in solvers.values():
        sv.close()
    return out, wall


def poisson_requests(grids, rate: float, duration: float, seed: int, phi=0.9, sigma=0.01):
    """Poisson arrivals at `rate` per second over `duration` seconds, each for a
    uniformly drawn grid with that grid's next AR(1) load snapshot."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out, state = 0.0, [], {}
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        k = int(rng.integers(len(grids)))
        g = grids[k]
        a = state.get(k, np.zeros(g.nbus))
        a = phi * a + sigma * rng.standard_normal(g.nbus)
        state[k] = a
        out.append(Request(len(out), t, k, g.pd * (1.0 + a), g.qd * (1.0 + a)))
    return out


def summarize(records, wall):
    done = [r for r in records if r["status"] != "dropped"]
    lat = np.array([r["latency_s"] for r in done]) * 1e3 if done else np.array([np.nan])
    return {"requests": len(records), "completed": len(done),
            "dropped": len(records) - len(done),
            "solves_per_s": len(done) / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_iters": float(np.mean([r["iters"] for r in done])) if done else 0.0,
            "converged": int(sum(1 for r in done if r["status"] == 0))}
