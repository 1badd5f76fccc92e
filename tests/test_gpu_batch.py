"""Batched scenarios in one handle: each scenario's iterates are bitwise the
same alone and in the mix (segment-local reductions, per-scenario stopping),
and scenarios begun at different times (continuous batching) follow their own
solo trajectories."""
import numpy as np
import pytest

import oracle
from paper_2110_06879_gb300 import admm, synth
from parity import compare_state

pytestmark = pytest.mark.gpu

TINY = dict(rho_pq=1e3, rho_va=1e4, beta0=1e5)
VECS = (admm.ADMM_VEC_U, admm.ADMM_VEC_XBAR, admm.ADMM_VEC_Z, admm.ADMM_VEC_Y,
        admm.ADMM_VEC_LAMBDA, admm.ADMM_VEC_BRANCH_X, admm.ADMM_VEC_BRANCH_LT, admm.ADMM_VEC_BUS)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def snapshot(s):
    return [s.vector(w) for w in VECS] + [np.array([s.residuals()["iters"]])]


def solo(grid, tol, max_iter, **kw):
    s = admm.Solver(grid, **kw)
    s.solve(tol=tol, max_iter=max_iter)
    out = snapshot(s)
    s.close()
    return out


def test_batch_equals_solo_bitwise():
    grids = [synth.tiny_grid(10), synth.sized_grid(600, seed=3), synth.tiny_grid(11),
             synth.sized_grid(300, seed=4)]
    b = admm.Solver(grids, **TINY)
    st = b.solve(tol=1e-4, max_iter=400)
    assert st in (admm.ADMM_OK, admm.ADMM_NOT_CONVERGED)
    iters = []
    for k, g in enumerate(grids):
        b.select(k)
        mine = snapshot(b)
        ref = solo(g, 1e-4, 400, **TINY)
        for a, r in zip(mine, ref):
            assert np.array_equal(a, r), k
        iters.append(int(mine[-1][0]))
    # scenarios stopped independently (per-scenario convergence mask)
    st_all, it_all = b.slot_status()
    assert list(it_all) == iters


def test_batched_scenarios_match_oracle():
    """Each scenario of a mixed batch against an oracle run of the same grid
    and inputs at 1e-9: scenarios of different sizes (one with shunts and
    transformers) begun at different times -- two join while others are
    iterating -- and one restarted warm with new loads after it stopped."""
    grids = [synth.tiny_grid(10), synth.sized_grid(600, seed=3),
             synth.tiny_grid(11, devices=True), synth.sized_grid(300, seed=4)]
    b = admm.Solver(grids, **TINY)
    b.slot_begin(0, tol=0.0, max_iter=10)
    b.slot_begin(1, tol=0.0, max_iter=8)
    b.run(4)
    b.slot_begin(2, tol=0.0, max_iter=6)              # joins mid-run
    b.run(3)
    b.slot_begin(3, tol=0.0, max_iter=9)              # joins later still
    b.run(100)
    pd1, qd1 = grids[1].pd * 1.03, grids[1].qd * 0.98
    b.select(1)
    b.set_loads(pd1, qd1)
    b.slot_begin(1, tol=0.0, max_iter=5, warm_start=True)   # warm restart, new loads
    b.run(50)
    st, it = b.slot_status()
    assert list(it) == [10, 5, 6, 9]
    for k, (g, n) in enumerate(zip(grids, (10, 8, 6, 9))):
        o = oracle.Oracle(g, **TINY)
        o.solve(tol=0.0, max_iter=n)
        if k == 1:
            o.set_loads(pd1, qd1)
            o.solve(tol=0.0, max_iter=5, warm_start=True)
        b.select(k)
        compare_state(b, o, 1e-9, f"scenario {k}")
    b.close()


def test_large_batch_with_trip_barrier_matches_oracle():
    """A batch with more branches than one block per SM holds (four 10k-bus
    grids, ~50,000 branches): the default launch then runs two blocks per SM
    whose warps meet every loop trip.  Every scenario against the oracle at
    1e-9 after four iterations, one of them begun two iterations late."""
    grids = [synth.sized_grid(10000, seed=21 + k, devices=(k == 1)) for k in range(4)]
    kw = dict(rho_pq=3e3, rho_va=3e4)
    b = admm.Solver(grids, **kw)
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert sum(g.nbranch for g in grids) >= 2 * sms * 128   # two blocks per SM by default
    for k in (0, 1, 2):
        b.slot_begin(k, tol=0.0, max_iter=4)
    b.run(2)
    b.slot_begin(3, tol=0.0, max_iter=4)               # joins two iterations late
    b.run(100)
    st, it = b.slot_status()
    assert list(it) == [4, 4, 4, 4]
    for k, g in enumerate(grids):
        o = oracle.Oracle(g, **kw)
        o.solve(tol=0.0, max_iter=4)
        b.select(k)
        compare_state(b, o, 1e-9, f"scenario {k}")
    b.close()


def test_continuous_batching_slots_follow_solo_trajectories():
    grids = [synth.tiny_grid(12), synth.tiny_grid(13), synth.sized_grid(400, seed=5)]
    b = admm.Solver(grids, **TINY)
    b.slot_begin(0, tol=0.0, max_iter=30)
    b.run(10)
    b.slot_begin(2, tol=0.0, max_iter=15)            # joins while slot 0 is running
    b.run(5)
    b.slot_begin(1, tol=0.0, max_iter=20)
    b.run(100)                                       # ends when every slot is done
    st, it = b.slot_status()
    assert list(it) == [30, 20, 15]
    assert all(x == admm.ADMM_NOT_CONVERGED for x in st)
    for k, n in ((0, 30), (1, 20), (2, 15)):
        b.select(k)
        mine = snapshot(b)
        ref = solo(grids[k], 0.0, n, **TINY)
        for a, r in zip(mine, ref):
            assert np.array_equal(a, r), k


def test_warm_slot_restart_matches_solo_warm_start():
    grids = [synth.tiny_grid(14), synth.tiny_grid(15)]
    b = admm.Solver(grids, **TINY)
    b.solve(tol=0.0, max_iter=12)
    b.select(1)
    b.set_loads(grids[1].pd * 1.03, grids[1].qd * 1.03)
    b.slot_begin(1, tol=0.0, max_iter=7, warm_start=True)
    b.run(50)
    mine = snapshot(b)
    s = admm.Solver(grids[1], **TINY)
    s.solve(tol=0.0, max_iter=12)
    s.set_loads(grids[1].pd * 1.03, grids[1].qd * 1.03)
    s.solve(tol=0.0, max_iter=7, warm_start=True)
    for a, r in zip(mine, snapshot(s)):
        assert np.array_equal(a, r)


def test_autotune_changes_no_result():
    """The tuner replays iterations from a saved copy and puts the state back:
    the tuned handle's solve is bitwise the untuned one's."""
    grids = [synth.tiny_grid(14), synth.sized_grid(800, seed=6)]
    tuned = admm.Solver(grids, **TINY)
    tuned.solve(tol=0.0, max_iter=4)
    before = tuned.get_state()
    blocks, body, ms, lanes = tuned.autotune(2)
    assert blocks >= 1 and body in (1, 2, 4) and ms > 0.0 and lanes in (1, 2)
    assert tuned.get_state() == before
    tuned.solve(tol=0.0, max_iter=3, warm_start=True)
    # the reference continues the same saved state with the tuned lane count
    # (one and two lanes agree to rounding, not bitwise); blocks and graph
    # shape change no bit
    ref2 = admm.Solver(grids, lanes_per_branch=lanes, **TINY)
    ref2.set_state(before)
    ref2.solve(tol=0.0, max_iter=3, warm_start=True)
    for k in range(len(grids)):
        tuned.select(k)
        ref2.select(k)
        for a, r in zip(snapshot(tuned), snapshot(ref2)):
            assert np.array_equal(a, r), k
    for s in (tuned, ref2):
        s.close()


@pytest.mark.parametrize("blocks", [1, 3, 40])
def test_branch_block_count_changes_no_result(blocks):
    """The branch queue order (longest first, first fill dealt across warps)
    and the number of resident blocks decide only which lane solves which
    branch, never a value: iterates are bitwise the same."""
    grid = synth.sized_grid(2000, seed=7)
    ref = admm.Solver(grid, rho_pq=3e3, rho_va=3e4)
    ref.solve(tol=0.0, max_iter=6)
    s = admm.Solver(grid, rho_pq=3e3, rho_va=3e4, branch_blocks=blocks)
    s.solve(tol=0.0, max_iter=6)
    for a, r in zip(snapshot(s), snapshot(ref)):
        assert np.array_equal(a, r)
    s.close()
    ref.close()


@pytest.mark.parametrize("body", [2, 3])
def test_graph_body_iterations_change_no_result(body):
    """Several iterations per WHILE body stop after exactly the same iteration
    (by the iteration cap mid-body, and by convergence), bitwise."""
    grid = synth.tiny_grid(15)
    for tol, cap in ((0.0, 7), (1e-4, 400)):
        ref = admm.Solver(grid, **TINY)
        st_ref = ref.solve(tol=tol, max_iter=cap)
        s = admm.Solver(grid, graph_body_iters=body, **TINY)
        st = s.solve(tol=tol, max_iter=cap)
        assert st == st_ref
        for a, r in zip(snapshot(s), snapshot(ref)):
            assert np.array_equal(a, r)
        assert np.array_equal(s.history(), ref.history())
        s.close()
        ref.close()


def test_api_error_paths():
    """Calls with arguments the handle cannot serve fail with an error, leave
    the handle usable, and change no state."""
    grids = [synth.tiny_grid(16), synth.tiny_grid(17)]
    b = admm.Solver(grids, **TINY)
    b.solve(tol=0.0, max_iter=3)
    before = b.get_state()
    with pytest.raises(admm.AdmmError):
        b.select(2)                                   # no such scenario
    with pytest.raises(admm.AdmmError):
        b.set_state(before[:-8])                      # truncated blob
    other = admm.Solver(synth.tiny_grid(18), **TINY)
    with pytest.raises(admm.AdmmError):
        other.set_state(before)                       # blob of another handle
    with pytest.raises(admm.AdmmError):
        b.slot_begin(5, tol=0.0, max_iter=3)          # no such slot
    assert b.get_state() == before
    b.select(1)
    assert b.solve(tol=0.0, max_iter=2, warm_start=True) == admm.ADMM_NOT_CONVERGED
    other.close()
    b.close()
