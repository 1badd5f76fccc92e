"""The allocation-free entry point admm_dual_update_noalloc, called through
the C ABI, reproduces the z / y update and residual norms that admm_solve
computes (with its own allocated scratch) for the same iteration, on two calls
in a row.  Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_2110_06879_gb300 import admm, synth

pytestmark = pytest.mark.gpu

TOL = 1e-9   # normwise relative, as in the other parity tests


def relerr(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / s if s > 0 else np.abs(a).max()


def test_noalloc_dual_update_matches_solver():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    grid = synth.sized_grid(5000, seed=2)
    kw = dict(rho_pq=5e1, rho_va=5e3)
    s = admm.Solver(grid, **kw)
    s.solve(tol=0.0, max_iter=3)
    stream = torch.cuda.current_stream()
    g = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    for call in range(2):
        xbar_prev = s.vector(admm.ADMM_VEC_XBAR)
        z_prev, y_prev = s.vector(admm.ADMM_VEC_Z), s.vector(admm.ADMM_VEC_Y)
        lam, rho = s.vector(admm.ADMM_VEC_LAMBDA), s.vector(admm.ADMM_VEC_RHO)
        beta = s.residuals()["beta"]
        # the existing entry point: one more iteration of the solver
        s.solve(tol=0.0, max_iter=1, warm_start=True)
        r = s.residuals()
        u, xbar = s.vector(admm.ADMM_VEC_U), s.vector(admm.ADMM_VEC_XBAR)
        z_exp, y_exp = s.vector(admm.ADMM_VEC_Z), s.vector(admm.ADMM_VEC_Y)
        # the allocation-free entry point on caller-owned device buffers
        du, dx, dxp, dr, dl = g(u), g(xbar), g(xbar_prev), g(rho), g(lam)
        dz, dy = g(z_prev), g(y_prev)
        dn = torch.zeros(4, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = admm.lib().admm_dual_update_noalloc(
            C.c_int64(s.m), C.c_void_p(du.data_ptr()), C.c_void_p(dx.data_ptr()),
            C.c_void_p(dxp.data_ptr()), C.c_void_p(dr.data_ptr()), C.c_void_p(dl.data_ptr()),
            beta, 1, C.c_void_p(dz.data_ptr()), C.c_void_p(dy.data_ptr()),
            C.c_void_p(dn.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == admm.ADMM_OK
        torch.cuda.synchronize()
        assert relerr(dz.cpu().numpy(), z_exp) <= TOL, call
        assert relerr(dy.cpu().numpy(), y_exp) <= TOL, call
        n = dn.cpu().numpy()
        exp = np.array([r["primal"], r["primal_z"], r["dual"], r["z_norm"]])
        assert np.all(np.abs(n - exp) <= TOL * np.maximum(np.abs(exp), 1e-300)), (call, n, exp)
    # sizes beyond the stated maximum are rejected without touching the GPU
    rc = admm.lib().admm_dual_update_noalloc(C.c_int64(16777217), C.c_void_p(du.data_ptr()),
                                             C.c_void_p(dx.data_ptr()), C.c_void_p(dxp.data_ptr()),
                                             C.c_void_p(dr.data_ptr()), C.c_void_p(dl.data_ptr()),
                                             beta, 1, C.c_void_p(dz.data_ptr()),
                                             C.c_void_p(dy.data_ptr()), C.c_void_p(dn.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
    assert rc == admm.ADMM_ERR_INVALID_ARG
    s.close()
