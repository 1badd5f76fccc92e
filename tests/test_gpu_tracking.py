"""Warm-start tracking (Section IV-C) through the C ABI: load snapshots,
renewable upper-bound ramps and the 2% ramp limit applied on the device
follow the oracle iterate by iterate."""
import numpy as np
import pytest

import oracle
from paper_2110_06879_gb300 import admm, synth, tracking

pytestmark = pytest.mark.gpu

TINY = dict(rho_pq=1e3, rho_va=1e4, beta0=1e5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def relerr(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / s if s > 0 else np.abs(a).max()


def test_tracking_sequence_matches_oracle():
    grid = synth.tiny_grid(8)
    steps = 4
    pds, qds = synth.ar1_loads(grid, steps, seed=5)
    pmaxs = tracking.renewable_pmax(grid, steps, seed=5)
    s = admm.Solver(grid, **TINY)
    o = oracle.Oracle(grid, **TINY)
    s.solve(tol=0.0, max_iter=30)
    o.solve(tol=0.0, max_iter=30)
    for t in range(steps):
        pg_prev = s.vector(admm.ADMM_VEC_U)[0:2 * grid.ngen:2]
        for side in (s, o):
            side.set_gen_bounds(grid.pmin, pmaxs[t])
            side.set_ramp_limit(0.02)
            side.set_loads(pds[t], qds[t])
            side.solve(tol=0.0, max_iter=20, warm_start=True)
        for wg, wo in ((admm.ADMM_VEC_U, oracle.U), (admm.ADMM_VEC_XBAR, oracle.XBAR),
                       (admm.ADMM_VEC_Z, oracle.Z), (admm.ADMM_VEC_Y, oracle.Y),
                       (admm.ADMM_VEC_LAMBDA, oracle.LAMBDA), (admm.ADMM_VEC_BUS, oracle.BUS)):
            assert relerr(s.vector(wg), o.get(wo)) <= 1e-9, (t, wg)
        # the ramp limit holds for the new dispatch
        pg = s.vector(admm.ADMM_VEC_U)[0:2 * grid.ngen:2]
        assert np.all(np.abs(pg - pg_prev) <= 0.02 * grid.pmax + 1e-12)
        assert np.all(pg <= pmaxs[t] + 1e-12)


def test_tracking_loop_converges_warm():
    grid = synth.tiny_grid(9)
    steps = 5
    pds, qds = synth.ar1_loads(grid, steps, seed=9)
    pmaxs = tracking.renewable_pmax(grid, steps, seed=9)
    s = admm.Solver(grid, **TINY)
    cold, recs = tracking.run_tracking(s, grid, pds, qds, pmaxs, tol=1e-4, max_iter=20000)
    summ = tracking.summarize(cold, recs)
    assert summ["snapshots"] == steps
    assert summ["converged"] == steps
    # warm solves need far fewer iterations than the cold start
    assert summ["mean_iters"] < cold["iters"]
