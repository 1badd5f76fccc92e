"""Served continuous batching: every request's result equals replaying that
grid's requests alone through a plain one-grid handle (bitwise), and the
memory budget decides which grids are resident."""
import numpy as np
import pytest

import oracle
from paper_2110_06879_gb300 import admm, serve, synth
from parity import compare_state

pytestmark = pytest.mark.gpu

KW = dict(rho_pq=1e3, rho_va=1e4, beta0=1e5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_served_results_equal_solo_replay():
    grids = [synth.tiny_grid(20), synth.tiny_grid(21), synth.sized_grid(300, seed=22)]
    reqs = serve.poisson_requests(grids, rate=400.0, duration=0.05, seed=3)
    assert len(reqs) >= 6
    srv = serve.Server(grids, mem_budget=1 << 30, tol=1e-4, max_iter=300, tick_iters=4, **KW)
    srv.warm_up(max_iter=300, tune=False)   # bitwise replay: the same launch shape as solo
    recs, rejected, wall = srv.run(reqs)
    assert not rejected and len(recs) == len(reqs)
    for k, g in enumerate(grids):
        solo = admm.Solver(g, **KW)
        solo.solve(tol=1e-4, max_iter=300)
        mine = [r for r in reqs if r.grid == k]
        for r in mine:
            solo.set_loads(r.pd, r.qd)
            solo.solve(tol=1e-4, max_iter=300, warm_start=True)
        srv.solver.select(k)
        for w in (admm.ADMM_VEC_U, admm.ADMM_VEC_XBAR, admm.ADMM_VEC_Z, admm.ADMM_VEC_Y,
                  admm.ADMM_VEC_LAMBDA, admm.ADMM_VEC_BRANCH_X):
            assert np.array_equal(srv.solver.vector(w), solo.vector(w)), (k, w)
        by_id = {rec["rid"]: rec for rec in recs}
        if mine:
            assert by_id[mine[-1].rid]["iters"] == solo.residuals()["iters"]


def test_served_results_match_oracle():
    """Served requests against the oracle at 1e-9: each grid's state after
    its last request equals an oracle run that replays the same inputs --
    a cold start, then per request that grid's loads and a warm solve of the
    same length (tol 0: every solve runs exactly max_iter iterations)."""
    grids = [synth.tiny_grid(20), synth.tiny_grid(21, devices=True),
             synth.sized_grid(300, seed=22)]
    reqs = serve.poisson_requests(grids, rate=400.0, duration=0.02, seed=3)
    assert len(reqs) >= 4
    n = 6
    srv = serve.Server(grids, mem_budget=1 << 30, tol=0.0, max_iter=n, tick_iters=4, **KW)
    srv.warm_up(max_iter=n)
    recs, rejected, _ = srv.run(reqs)
    assert not rejected and len(recs) == len(reqs)
    assert all(r["iters"] == n for r in recs)
    for k, g in enumerate(grids):
        o = oracle.Oracle(g, **KW)
        o.solve(tol=0.0, max_iter=n)
        for r in (r for r in reqs if r.grid == k):
            o.set_loads(r.pd, r.qd)
            o.solve(tol=0.0, max_iter=n, warm_start=True)
        srv.solver.select(k)
        compare_state(srv.solver, o, 1e-9, f"grid {k}")


def test_memory_budget_swaps_grids_in_and_out():
    """Admission by device memory as it frees up: the budget holds two of the
    three grids (counted in the library's own allocation size).  Requests for
    the third make the server drain, save the resident states, evict the
    least recently used idle grid and rebuild; an evicted grid that returns
    continues from its saved state.  Every grid's final state is bitwise its
    solo replay: a cold solve at its own loads, then each of its requests warm."""
    grids = [synth.tiny_grid(23), synth.sized_grid(2000, seed=24), synth.tiny_grid(25)]
    budget = serve.state_bytes([grids[0], grids[1]])
    assert serve.state_bytes(grids) > budget >= serve.state_bytes([grids[1], grids[2]])
    srv = serve.Server(grids, mem_budget=budget, tol=1e-4, max_iter=200, tick_iters=4, **KW)
    assert srv.grid_ids == [0, 1]
    srv.warm_up(max_iter=300, tune=False)   # bitwise replay: the same launch shape as solo
    reqs = serve.poisson_requests(grids, rate=300.0, duration=0.06, seed=4)
    assert {r.grid for r in reqs} == {0, 1, 2}
    recs, rejected, _ = srv.run(reqs)
    assert not rejected and len(recs) == len(reqs)
    assert all(r["status"] != "dropped" for r in recs)
    assert srv.swaps >= 1 and srv.evictions >= 1
    by_id = {rec["rid"]: rec for rec in recs}
    for k, g in enumerate(grids):
        solo = admm.Solver(g, **KW)
        solo.solve(tol=1e-4, max_iter=300)
        mine = [r for r in reqs if r.grid == k]
        for r in mine:
            solo.set_loads(r.pd, r.qd)
            solo.solve(tol=1e-4, max_iter=200, warm_start=True)
        if k in srv.slot_of:
            srv.solver.select(srv.slot_of[k])
            mineh = srv.solver
        else:
            mineh = admm.Solver(g, **KW)
            mineh.set_scenario_state(0, srv.saved[k])
        for w in (admm.ADMM_VEC_U, admm.ADMM_VEC_XBAR, admm.ADMM_VEC_Z, admm.ADMM_VEC_Y,
                  admm.ADMM_VEC_LAMBDA, admm.ADMM_VEC_BRANCH_X, admm.ADMM_VEC_BRANCH_LT):
            assert np.array_equal(mineh.vector(w), solo.vector(w)), (k, w)
        assert by_id[mine[-1].rid]["iters"] == solo.residuals()["iters"]
    srv.solver.close()


def test_scenario_state_moves_between_handles():
    """admm_get_scenario_state / admm_set_scenario_state: a scenario's state
    taken out of a batch and put into a one-grid handle continues bitwise like
    the batch would; a blob of another shape or a running scenario is refused."""
    grids = [synth.tiny_grid(26), synth.sized_grid(400, seed=27)]
    b = admm.Solver(grids, **KW)
    b.solve(tol=0.0, max_iter=9)
    blob = b.get_scenario_state(1)
    one = admm.Solver(grids[1], **KW)
    one.set_scenario_state(0, blob)
    b.slot_begin(1, tol=0.0, max_iter=5, warm_start=True)
    b.run(20)
    one.solve(tol=0.0, max_iter=5, warm_start=True)
    b.select(1)
    for w in (admm.ADMM_VEC_U, admm.ADMM_VEC_XBAR, admm.ADMM_VEC_Z, admm.ADMM_VEC_Y,
              admm.ADMM_VEC_LAMBDA, admm.ADMM_VEC_BRANCH_X, admm.ADMM_VEC_BRANCH_LT):
        assert np.array_equal(b.vector(w), one.vector(w)), w
    with pytest.raises(admm.AdmmError):
        b.set_scenario_state(0, blob)                 # scenario 0 has another shape
    b.slot_begin(1, tol=0.0, max_iter=3, warm_start=True)
    with pytest.raises(admm.AdmmError):
        b.set_scenario_state(1, blob)                 # scenario 1 is running
    b.run(10)
    b.close()
    one.close()
