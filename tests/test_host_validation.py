"""Host-side validation of the C ABI: invalid grids and options are rejected
with ADMM_ERR_INVALID_ARG and a message before any device work, so these run
without a GPU."""
import copy

import numpy as np
import pytest

from paper_2110_06879_gb300 import admm, synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def rejected(grid, match, **opts):
    with pytest.raises(admm.AdmmError) as e:
        admm.Solver(grid, **opts)
    msg = str(e.value)
    assert "ADMM_ERR_INVALID_ARG" in msg and match in msg, msg


def mutated(field, fn):
    g = copy.deepcopy(synth.tiny_grid(0))
    a = np.array(getattr(g, field), copy=True)
    fn(a)
    setattr(g, field, a)
    return g


def test_invalid_grids_are_rejected():
    g = synth.tiny_grid(0)
    rejected(mutated("t_bus", lambda a: a.__setitem__(0, g.f_bus[0])), "")          # self loop
    rejected(mutated("f_bus", lambda a: a.__setitem__(0, g.nbus)), "")              # bus index
    rejected(mutated("gen_bus", lambda a: a.__setitem__(0, -1)), "generator 0")
    rejected(mutated("pmin", lambda a: a.__setitem__(0, 1e9)), "generator 0")       # empty bounds
    rejected(mutated("c2", lambda a: a.__setitem__(0, -1.0)), "generator 0")
    rejected(mutated("vmin", lambda a: a.__setitem__(0, 0.0)), "bus 0")
    rejected(mutated("pd", lambda a: a.__setitem__(0, np.nan)), "")


def test_invalid_options_are_rejected():
    g = synth.tiny_grid(0)
    rejected(g, "penalties", rho_pq=0.0)
    rejected(g, "penalties", rho_va=-1.0)
    rejected(g, "branch_blocks", branch_blocks=-1)
    rejected(g, "graph_body_iters", graph_body_iters=0)
    rejected(g, "graph_body_iters", graph_body_iters=17)
    rejected(g, "iteration caps", max_outer=0)
    rejected(g, "iteration caps", tron_max_iter=0)


def test_batch_error_names_the_scenario():
    bad = mutated("f_bus", lambda a: a.__setitem__(0, 10**6))
    with pytest.raises(admm.AdmmError, match="scenario 1"):
        admm.Solver([synth.tiny_grid(1), bad])
