"""Host logic of the continuous-batching server without a GPU: admission by a
device-memory budget, draining, eviction (least recently used, idle grids
first), swap-in with saved states put back, first come first served.  The
library is replaced by a fake with the same calls that records what the
server asks of it."""
import types

import numpy as np
import pytest

from paper_2110_06879_gb300 import serve


class FakeGrid:
    def __init__(self, gid, size):
        self.gid, self.size = gid, size
        self.nbus, self.pd, self.qd = 1, np.zeros(1), np.zeros(1)


class FakeSolver:
    """Scenario s runs `iters_per_solve` iterations per slot_begin; its
    'state' is the number of solves it has completed, and a blob carries
    (grid id, solves)."""
    log = []

    def __init__(self, grids, stream=None, iters_per_solve=5, **opts):
        self.grids = list(grids)
        self.left = [0] * len(grids)
        self.solves = [0] * len(grids)
        self.iters = [0] * len(grids)
        self.k = iters_per_solve
        FakeSolver.log.append(("build", tuple(g.gid for g in grids)))

    def select(self, s):
        self.sel = s

    def set_loads(self, pd, qd):
        pass

    def slot_begin(self, s, tol, max_iter, warm_start, rho_pq=None, rho_va=None):
        self.left[s] = self.k
        self.iters[s] = 0

    def run(self, n):
        for s in range(len(self.left)):
            d = min(n, self.left[s])
            self.left[s] -= d
            self.iters[s] += d
            if d and self.left[s] == 0:
                self.solves[s] += 1

    def slot_status(self):
        st = np.array([2 if x > 0 else 1 for x in self.left], dtype=np.int32)
        return st, np.array(self.iters, dtype=np.int32)

    def solve(self, tol, max_iter):
        pass

    def autotune(self, iters):
        return (1, 1, 0.1, 1)

    def get_scenario_state(self, s):
        return (self.grids[s].gid, self.solves[s])

    def set_scenario_state(self, s, blob):
        assert blob[0] == self.grids[s].gid        # a grid's state goes back to that grid
        self.solves[s] = blob[1]

    def close(self):
        pass


@pytest.fixture
def fake_admm(monkeypatch):
    fake = types.SimpleNamespace(Solver=FakeSolver,
                                 device_bytes=lambda gs: 10 + sum(g.size for g in gs))
    monkeypatch.setattr(serve, "admm", fake)
    FakeSolver.log = []
    return fake


def _reqs(order, spacing=0.0):
    return [serve.Request(rid=i, arrival=i * spacing, grid=g, pd=np.zeros(1), qd=np.zeros(1))
            for i, g in enumerate(order)]


def test_all_requests_served_with_swaps_and_states_kept(fake_admm):
    grids = [FakeGrid(k, 100) for k in range(4)]
    srv = serve.Server(grids, mem_budget=10 + 200, tick_iters=2)     # two grids fit
    assert srv.grid_ids == [0, 1]
    order = [2, 0, 3, 1, 2, 2, 0, 3, 3, 1, 0]
    recs, rejected, _ = srv.run(_reqs(order))
    assert not rejected and len(recs) == len(order)
    assert all(r["status"] == 1 for r in recs)
    assert srv.swaps >= 2 and srv.evictions >= 2
    # every grid completed exactly its own requests' solves, across evictions
    states = srv.saved_states()
    for k in range(4):
        assert states[k] == (k, order.count(k))
    # first come, first served: completion order follows arrival order per grid
    done = [r["rid"] for r in recs]
    for k in range(4):
        mine = [i for i, g in enumerate(order) if g == k]
        assert [d for d in done if d in mine] == mine
    # resident sets never exceed the budget
    for kind, ids in FakeSolver.log:
        assert 10 + 100 * len(ids) <= 210


def test_grid_larger_than_budget_is_rejected(fake_admm):
    grids = [FakeGrid(0, 50), FakeGrid(1, 500), FakeGrid(2, 50)]
    srv = serve.Server(grids, mem_budget=200)
    recs, rejected, _ = srv.run(_reqs([1, 0, 2, 1]))
    assert [r.grid for r in rejected] == [1, 1]
    assert len(recs) == 2


def test_deadline_drops_waiting_requests(fake_admm):
    grids = [FakeGrid(k, 100) for k in range(3)]
    srv = serve.Server(grids, mem_budget=10 + 100, tick_iters=1)
    recs, rejected, _ = srv.run(_reqs([0, 1, 2, 0, 1, 2]), deadline=0.0)
    assert len(recs) == 6
    assert any(r["status"] == "dropped" for r in recs)
