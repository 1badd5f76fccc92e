"""Continuous-batching request loop for load-snapshot solves (tracking under
load fluctuation, Section IV-C, served).

A pool of grids stays resident in one batched handle, each grid a slot whose
primal, dual and penalty state persists between requests (warm starts).
Requests carry a new load snapshot for one grid.  The loop admits a waiting
request as soon as its grid's slot is free, even while other slots are being
iterated, runs the batched iteration graph for a few iterations at a time
(`tick_iters`), and retires every slot whose solve has stopped.

Residency follows a device-memory budget, counted in the bytes the library
reports for a handle over the resident grids (admm_device_bytes).  Grids that
do not fit wait outside.  When requests arrive for a grid that is not
resident, the loop stops admitting new work, lets the solves in flight
finish, and swaps: it saves every resident grid's state to the host
(admm_get_scenario_state), evicts idle grids least recently used until the
newcomer fits, rebuilds the handle over the new resident set and puts the
saved states back (admm_set_scenario_state).  A grid that returns continues
from its saved state bitwise; a grid seen for the first time is cold-solved at
its own loads on admission, as the initial pool is in warm_up.  All
computation runs in the library; this loop only sequences C-ABI calls.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import admm


def state_bytes(grids) -> int:
    """Device bytes of a handle over `grids` (one grid or a list)."""
    return admm.device_bytes(grids)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    grid: int               # index into the server's grid list
    pd: np.ndarray
    qd: np.ndarray


class Server:
    """`states` (grid index -> scenario state blob, e.g. another server's
    `saved_states()`) seeds the pool with solved grids: their states are put
    back whenever they are resident, and none of them is cold-solved on entry
    (`warm_iters` sets the cold-solve length for the others).  `tuned` is a
    launch shape (branch blocks, iterations per graph body, ms, lanes per
    branch), as Solver.autotune returns it, used for every rebuilt handle."""

    def __init__(self, grids, mem_budget: int, rho_pq=3e3, rho_va=3e4, tol=1e-3, max_iter=2000,
                 tick_iters=8, stream=None, states=None, tuned=None, warm_iters=None, **opts):
        self.all = list(grids)
        self.budget = int(mem_budget)
        self.tol, self.max_iter, self.tick = tol, max_iter, tick_iters
        self.rho = (rho_pq, rho_va)
        self.stream, self.opts = stream, dict(opts)
        admitted = []
        for k, g in enumerate(self.all):
            if state_bytes([self.all[j] for j in admitted + [k]]) <= self.budget:
                admitted.append(k)
        if not admitted:
            raise ValueError("no grid fits the memory budget")
        self.saved = dict(states or {})     # grid -> scenario state blob (host)
        self.warm_iters = warm_iters        # cold-solve length on first entry (None: none)
        self.last_used = collections.defaultdict(lambda: -1.0)
        self.swaps = self.evictions = 0
        self.solver = None
        self.tuned = tuned
        self._build(admitted)

    def _build(self, ids):
        """Handle over the grids `ids` (kept sorted), their saved states put back."""
        if self.solver is not None:
            self.solver.close()
        self.grid_ids = sorted(ids)
        self.slot_of = {k: s for s, k in enumerate(self.grid_ids)}
        self.grids = [self.all[k] for k in self.grid_ids]
        self.bytes = state_bytes(self.grids)
        extra = {}
        if self.tuned:
            extra = dict(branch_blocks=self.tuned[0], graph_body_iters=self.tuned[1],
                         lanes_per_branch=self.tuned[3])
        self.solver = admm.Solver(self.grids, stream=self.stream, rho_pq=self.rho[0],
                                  rho_va=self.rho[1], **dict(self.opts, **extra))
        for k in self.grid_ids:
            if k in self.saved:
                self.solver.set_scenario_state(self.slot_of[k], self.saved[k])

    def warm_up(self, max_iter=5000, tune=True):
        """Cold-solve every resident grid once, all together, then (tune) pick
        the launch shape for the pool on replayed iterations (the tuner puts
        the state back, so no result changes); returns seconds.  Grids
        admitted later are cold-solved the same way (at most max_iter
        iterations) when they enter."""
        self.warm_iters = max_iter
        t0 = time.perf_counter()
        self.solver.solve(tol=self.tol, max_iter=max_iter)
        self.tuned = self.solver.autotune(2) if tune else None
        return time.perf_counter() - t0

    def saved_states(self):
        """Every grid's latest state blob: resident ones read now, the others
        as saved at their eviction."""
        out = dict(self.saved)
        for k in self.grid_ids:
            out[k] = self.solver.get_scenario_state(self.slot_of[k])
        return out

    def _swap_in(self, k, protect):
        """Make grid k resident (every slot idle): evict idle grids least
        recently used, except those in `protect`, until the set fits.  Returns
        False when k cannot fit even alone."""
        if state_bytes([self.all[k]]) > self.budget:
            return False
        for j in self.grid_ids:                     # save every resident state
            self.saved[j] = self.solver.get_scenario_state(self.slot_of[j])
        keep = list(self.grid_ids)
        order = sorted(keep, key=lambda j: (j in protect, self.last_used[j], j))
        while keep and state_bytes([self.all[j] for j in keep + [k]]) > self.budget:
            keep.remove(order.pop(0))
            self.evictions += 1
        fresh = k not in self.saved
        self._build(keep + [k])
        self.swaps += 1
        if fresh and self.warm_iters:               # first entry: cold solve at its loads
            slot = self.slot_of[k]
            self.solver.slot_begin(slot, tol=self.tol, max_iter=self.warm_iters,
                                   warm_start=False, rho_pq=self.rho[0], rho_va=self.rho[1])
            while self.solver.slot_status()[0][slot] == 2:
                self.solver.run(max(self.tick, 64))
        return True

    def run(self, requests, deadline: float = float("inf")):
        """Serve `requests` (sorted by arrival) in real time; returns one record
        per request (latency = completion - arrival, iterations, status), the
        requests for grids that cannot fit the budget even alone, and the wall
        time.  After `deadline` seconds no request is admitted any more: solves
        in flight finish, waiting ones are returned with status "dropped"."""
        fits = {k for k in {r.grid for r in requests} if state_bytes([self.all[k]]) <= self.budget}
        pending = collections.deque(r for r in requests if r.grid in fits)
        rejected = [r for r in requests if r.grid not in fits]
        waiting = collections.defaultdict(collections.deque)   # grid -> queued requests
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
                waiting[r.grid].append(r)
            # first come, first served: when the oldest waiting request is for a
            # grid that is not resident, admit nothing new until the solves in
            # flight are done, then swap that grid in (it is served next)
            heads = [(q[0].arrival, k) for k, q in waiting.items() if q]
            oldest = min(heads)[1] if heads else None
            if oldest is not None and oldest not in self.slot_of and now <= deadline:
                if not busy:
                    protect = {j for j, q in waiting.items() if q}
                    self._swap_in(oldest, protect)
                    continue
            else:
                # admit: every free slot with a waiting request joins the batch
                for k, q in waiting.items():
                    slot = self.slot_of.get(k)
                    if q and slot is not None and slot not in busy and now <= deadline:
                        r = q.popleft()
                        s = self.solver
                        s.select(slot)
                        s.set_loads(r.pd, r.qd)
                        s.slot_begin(slot, tol=self.tol, max_iter=self.max_iter, warm_start=True,
                                     rho_pq=self.rho[0], rho_va=self.rho[1])
                        busy[slot] = r
                        self.last_used[k] = now
            if not busy:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
                continue
            self.solver.run(self.tick)
            status, iters = self.solver.slot_status()       # waits for the tick
            done_t = time.perf_counter() - t0
            for slot in list(busy):
                if status[slot] != 2:
                    r = busy.pop(slot)
                    out.append(dict(rid=r.rid, grid=r.grid, latency_s=done_t - r.arrival,
                                    iters=int(iters[slot]), status=int(status[slot])))
        wall = time.perf_counter() - t0
        return out, rejected, wall


def serial_baseline(grids, requests, rho_pq=3e3, rho_va=3e4, tol=1e-3, max_iter=2000,
                    stream=None, deadline: float = float("inf"), solvers=None, **opts):
    """The same request stream through plain one-grid handles, one solve at a
    time in arrival order (each grid warm from its previous solve); requests
    not started by `deadline` seconds are dropped.  `solvers` (a dict grid
    index -> Solver) keeps the handles, already cold-solved, across calls; the
    caller then closes them."""
    own = solvers is None
    solvers = {} if own else solvers
    for k in sorted({r.grid for r in requests}):
        if k not in solvers:
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
    if own:
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
