"""Served continuous batching: every request's result equals replaying that
grid's requests alone through a plain one-grid handle (bitwise), and the
memory budget decides which grids are resident."""
import numpy as np
import pytest

from paper_2110_06879_gb300 import admm, serve, synth

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
    srv.warm_up(max_iter=300)
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


def test_memory_budget_admission():
    grids = [synth.tiny_grid(23), synth.sized_grid(2000, seed=24), synth.tiny_grid(25)]
    budget = serve.state_bytes(grids[0]) + serve.state_bytes(grids[2]) + 1
    srv = serve.Server(grids, mem_budget=budget, **KW)
    assert srv.grid_ids == [0, 2]
    reqs = serve.poisson_requests(grids, rate=300.0, duration=0.03, seed=4)
    srv.warm_up(max_iter=100)
    recs, rejected, _ = srv.run(reqs)
    assert all(r.grid == 1 for r in rejected)
    assert len(recs) + len(rejected) == len(reqs)
