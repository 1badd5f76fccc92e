"""ctypes binding of libadmm.so (include/admm.h), argument marshalling only.

Every function of the C ABI is exposed under the same name; ``Solver`` wraps a
handle for convenience.  All computation happens in the CUDA library: when the
library is missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadmm.so")

ADMM_OK, ADMM_NOT_CONVERGED = 0, 1
ADMM_ERR_INVALID_ARG, ADMM_ERR_CUDA, ADMM_ERR_NUMERICAL, ADMM_ERR_OOM = -1, -2, -3, -4
(ADMM_VEC_U, ADMM_VEC_XBAR, ADMM_VEC_Z, ADMM_VEC_Y, ADMM_VEC_LAMBDA, ADMM_VEC_BRANCH_X,
 ADMM_VEC_BRANCH_LT, ADMM_VEC_BUS, ADMM_VEC_RHO, ADMM_VEC_ADMITTANCE) = range(10)
STAT_NAMES = ("tron_calls", "tron_iters", "fgh_evals", "f_evals", "cauchy_trials", "cg_iters",
              "ps_trials", "al_passes", "tron_maxiter_hits")


class admm_grid(C.Structure):
    _fields_ = [("nbus", C.c_int32), ("nbranch", C.c_int32), ("ngen", C.c_int32),
                ("ref_bus", C.c_int32), ("base_mva", C.c_double)] + [
        (n, C.c_void_p) for n in ("pd", "qd", "gs", "bs", "vmin", "vmax", "f_bus", "t_bus",
                                  "r", "x", "b", "tap", "shift", "rate_a", "gen_bus", "pmin",
                                  "pmax", "qmin", "qmax", "c2", "c1", "c0")]


_OPT_D = ("rho_pq", "rho_va", "obj_scale", "line_limit_frac", "beta0", "beta_factor", "z_decay",
          "beta_max", "lambda_max", "tol_in0", "tol_in_decay", "al_rho0", "al_tol", "al_decay",
          "al_rho_factor", "al_rho_max", "tron_gtol", "tron_ftol", "tron_xtol")
_OPT_I = ("two_level", "max_outer", "max_inner", "al_max_iter", "tron_max_iter", "use_graph",
          "branch_blocks", "graph_body_iters", "beta_rule", "lanes_per_branch")


class admm_options(C.Structure):
    _fields_ = [(n, C.c_double) for n in _OPT_D] + [(n, C.c_int32) for n in _OPT_I]


class admm_residuals(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer_iters", C.c_int32), ("status", C.c_int32),
                ("tron_failures", C.c_int32), ("primal_res", C.c_double),
                ("dual_res", C.c_double), ("z_norm", C.c_double), ("primal_z", C.c_double),
                ("beta", C.c_double), ("eps_pri", C.c_double), ("eps_dual", C.c_double),
                ("objective", C.c_double), ("max_viol", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def lib():
    """Load libadmm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, d = C.c_void_p, C.c_int32, C.c_double
        sig = {
            "admm_default_options": (None, [C.POINTER(admm_options)]),
            "admm_create": (C.c_int, [C.POINTER(admm_grid), C.POINTER(admm_options), C.POINTER(vp)]),
            "admm_create_batch": (C.c_int, [C.POINTER(admm_grid), i32, C.POINTER(admm_options),
                                            C.POINTER(vp)]),
            "admm_scenario_count": (i32, [vp]),
            "admm_select_scenario": (C.c_int, [vp, i32]),
            "admm_slot_begin": (C.c_int, [vp, i32, d, d, d, i32, i32]),
            "admm_run": (C.c_int, [vp, i32]),
            "admm_slot_status": (C.c_int, [vp, vp, vp]),
            "admm_destroy": (None, [vp]),
            "admm_set_stream": (C.c_int, [vp, vp]),
            "admm_set_loads": (C.c_int, [vp, vp, vp]),
            "admm_set_loads_device": (C.c_int, [vp, vp, vp]),
            "admm_set_gen_bounds": (C.c_int, [vp, vp, vp]),
            "admm_set_ramp_limit": (C.c_int, [vp, d]),
            "admm_solve": (C.c_int, [vp, d, d, d, i32, i32]),
            "admm_solve_async": (C.c_int, [vp, d, d, d, i32, i32]),
            "admm_get_solution": (C.c_int, [vp] + [vp] * 8),
            "admm_get_residuals": (C.c_int, [vp, C.POINTER(admm_residuals)]),
            "admm_get_history": (i32, [vp, vp, i32]),
            "admm_get_vector": (C.c_int, [vp, i32, vp]),
            "admm_get_csr": (C.c_int, [vp, vp, vp]),
            "admm_get_stats": (C.c_int, [vp, vp]),
            "admm_get_state": (C.c_int, [vp, vp, C.POINTER(C.c_size_t)]),
            "admm_set_state": (C.c_int, [vp, vp, C.c_size_t]),
            "admm_profile_iterations": (C.c_int, [vp, i32, vp]),
            "admm_autotune": (C.c_int, [vp, i32, vp, vp, vp, vp]),
            "admm_dual_update_noalloc": (C.c_int, [C.c_int64, vp, vp, vp, vp, vp, d, i32, vp, vp,
                                                   vp, vp]),
            "admm_fp64_peak": (C.c_int, [i32, vp, vp]),
            "admm_get_scenario_state": (C.c_int, [vp, i32, vp, C.POINTER(C.c_size_t)]),
            "admm_set_scenario_state": (C.c_int, [vp, i32, vp, C.c_size_t]),
            "admm_device_bytes": (C.c_int, [C.POINTER(admm_grid), i32, C.POINTER(C.c_size_t)]),
            "admm_status_string": (C.c_char_p, [C.c_int]),
            "admm_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def fp64_peak(iters=20000, stream=None) -> dict:
    """FP64 FMA-only calibration launch (admm_fp64_peak): achieved GFLOP/s,
    the SM clock in MHz during it, FMAs per clock per SM sub-partition."""
    out = np.zeros(3)
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().admm_fp64_peak(iters, C.c_void_p(raw or 0), _ptr(out)), "admm_fp64_peak")
    return dict(gflops=float(out[0]), sm_mhz=float(out[1]), fma_per_clk_smsp=float(out[2]))


def device_bytes(grids) -> int:
    """Device bytes a handle over `grids` (one grid or a list) allocates for
    its state (admm_device_bytes)."""
    grids = list(grids) if isinstance(grids, (list, tuple)) else [grids]
    keep = []
    arr = (admm_grid * len(grids))(*[_grid_struct(g, keep) for g in grids])
    n = C.c_size_t(0)
    _check(lib().admm_device_bytes(arr, len(grids), C.byref(n)), "admm_device_bytes")
    return int(n.value)


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class AdmmError(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        raise AdmmError(f"{what}: {lib().admm_status_string(rc).decode()} "
                        f"({lib().admm_last_error().decode()})")
    return rc


def default_options(**kw) -> admm_options:
    o = admm_options()
    lib().admm_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _grid_struct(grid, keep: list) -> admm_grid:
    g = admm_grid()
    g.nbus, g.nbranch, g.ngen, g.ref_bus = grid.nbus, grid.nbranch, grid.ngen, grid.ref_bus
    g.base_mva = grid.base_mva
    for name in ("pd", "qd", "gs", "bs", "vmin", "vmax", "r", "x", "b", "tap", "shift",
                 "rate_a", "pmin", "pmax", "qmin", "qmax", "c2", "c1", "c0"):
        a = np.ascontiguousarray(getattr(grid, name), dtype=np.float64)
        keep.append(a)
        setattr(g, name, a.ctypes.data)
    for name in ("f_bus", "t_bus", "gen_bus"):
        a = np.ascontiguousarray(getattr(grid, name), dtype=np.int32)
        keep.append(a)
        setattr(g, name, a.ctypes.data)
    return g


class Solver:
    """One grid, or a batch of grids, resident on the current CUDA device
    (``admm_create`` / ``admm_create_batch``).  Per-scenario methods address the
    scenario chosen with ``select``."""

    def __init__(self, grid, stream=None, **opts):
        grids = list(grid) if isinstance(grid, (list, tuple)) else [grid]
        self.grids = grids
        self.opts = default_options(**opts)
        keep = []
        arr = (admm_grid * len(grids))(*[_grid_struct(g, keep) for g in grids])
        h = C.c_void_p()
        _check(lib().admm_create_batch(arr, len(grids), C.byref(self.opts), C.byref(h)),
               "admm_create_batch")
        self.h = h
        self.nscen = len(grids)
        self.select(0)
        if stream is not None:
            self.set_stream(stream)

    def select(self, s: int):
        _check(lib().admm_select_scenario(self.h, s), "admm_select_scenario")
        g = self.grids[s]
        self.grid = g
        self.nb, self.nl, self.ng = g.nbus, g.nbranch, g.ngen
        self.m = 2 * self.ng + 8 * self.nl

    def slot_begin(self, s, tol=1e-4, max_iter=5000, warm_start=False, rho_pq=None, rho_va=None):
        rp = self.opts.rho_pq if rho_pq is None else rho_pq
        rv = self.opts.rho_va if rho_va is None else rho_va
        _check(lib().admm_slot_begin(self.h, s, rp, rv, tol, max_iter, 1 if warm_start else 0),
               "admm_slot_begin")

    def run(self, max_iters):
        _check(lib().admm_run(self.h, max_iters), "admm_run")

    def slot_status(self):
        st = np.zeros(self.nscen, dtype=np.int32)
        it = np.zeros(self.nscen, dtype=np.int32)
        _check(lib().admm_slot_status(self.h, _ptr(st), _ptr(it)), "admm_slot_status")
        return st, it

    def close(self):
        if getattr(self, "h", None):
            lib().admm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().admm_set_stream(self.h, C.c_void_p(raw or 0)), "admm_set_stream")

    def set_loads(self, pd, qd):
        pd = np.ascontiguousarray(pd, dtype=np.float64)
        qd = np.ascontiguousarray(qd, dtype=np.float64)
        _check(lib().admm_set_loads(self.h, _ptr(pd), _ptr(qd)), "admm_set_loads")

    def set_loads_device(self, d_pd, d_qd):
        """Device pointers (ints) or contiguous float64 CUDA tensors of nbus
        entries (those are checked here; raw pointers are the caller's)."""
        for t in (d_pd, d_qd):
            if hasattr(t, "data_ptr"):
                ok = (str(t.dtype) == "torch.float64" and t.is_cuda and t.is_contiguous()
                      and t.numel() == self.nb)
                if not ok:
                    raise AdmmError("set_loads_device: need contiguous float64 CUDA tensors "
                                    f"of {self.nb} entries")
        p = getattr(d_pd, "data_ptr", lambda: d_pd)()
        q = getattr(d_qd, "data_ptr", lambda: d_qd)()
        _check(lib().admm_set_loads_device(self.h, C.c_void_p(p), C.c_void_p(q)),
               "admm_set_loads_device")

    def set_gen_bounds(self, pmin, pmax):
        pmin = np.ascontiguousarray(pmin, dtype=np.float64)
        pmax = np.ascontiguousarray(pmax, dtype=np.float64)
        _check(lib().admm_set_gen_bounds(self.h, _ptr(pmin), _ptr(pmax)), "admm_set_gen_bounds")

    def set_ramp_limit(self, frac=0.02):
        _check(lib().admm_set_ramp_limit(self.h, frac), "admm_set_ramp_limit")

    def solve(self, tol=1e-4, max_iter=5000, warm_start=False, rho_pq=None, rho_va=None) -> int:
        rp = self.opts.rho_pq if rho_pq is None else rho_pq
        rv = self.opts.rho_va if rho_va is None else rho_va
        return _check(lib().admm_solve(self.h, rp, rv, tol, max_iter, 1 if warm_start else 0),
                      "admm_solve")

    def solve_async(self, tol=1e-4, max_iter=5000, warm_start=False, rho_pq=None, rho_va=None):
        rp = self.opts.rho_pq if rho_pq is None else rho_pq
        rv = self.opts.rho_va if rho_va is None else rho_va
        return _check(lib().admm_solve_async(self.h, rp, rv, tol, max_iter,
                                             1 if warm_start else 0), "admm_solve_async")

    def residuals(self) -> dict:
        r = admm_residuals()
        _check(lib().admm_get_residuals(self.h, C.byref(r)), "admm_get_residuals")
        d = r.as_dict()
        return dict(primal=d["primal_res"], dual=d["dual_res"], z_norm=d["z_norm"],
                    primal_z=d["primal_z"], beta=d["beta"], eps_pri=d["eps_pri"],
                    eps_dual=d["eps_dual"], iters=d["iters"],
                    outer_iters=d["outer_iters"], status=d["status"],
                    tron_failures=d["tron_failures"], objective=d["objective"],
                    max_viol=d["max_viol"])

    def solution(self) -> dict:
        nb, nl, ng = self.nb, self.nl, self.ng
        out = dict(pg=np.zeros(ng), qg=np.zeros(ng), vm=np.zeros(nb), va=np.zeros(nb),
                   pf=np.zeros(nl), qf=np.zeros(nl), pt=np.zeros(nl), qt=np.zeros(nl))
        _check(lib().admm_get_solution(self.h, *[_ptr(out[k]) for k in
                                                 ("pg", "qg", "vm", "va", "pf", "qf", "pt", "qt")]),
               "admm_get_solution")
        r = self.residuals()
        out["objective"] = r["objective"]
        out["max_viol"] = r["max_viol"]
        return out

    def history(self, cap=65536) -> np.ndarray:
        out = np.zeros((cap, 4))
        n = _check(lib().admm_get_history(self.h, _ptr(out), cap), "admm_get_history")
        return out[:n]

    def vector(self, which: int) -> np.ndarray:
        n = {ADMM_VEC_BRANCH_X: 6 * self.nl, ADMM_VEC_BRANCH_LT: 2 * self.nl,
             ADMM_VEC_BUS: 2 * self.nb, ADMM_VEC_ADMITTANCE: 8 * self.nl}.get(which, self.m)
        out = np.zeros(n)
        _check(lib().admm_get_vector(self.h, which, _ptr(out)), "admm_get_vector")
        return out

    def csr(self):
        row = np.zeros(self.nb + 1, dtype=np.int32)
        col = np.zeros(2 * self.nl + self.ng, dtype=np.int32)
        _check(lib().admm_get_csr(self.h, _ptr(row), _ptr(col)), "admm_get_csr")
        return row, col

    def stats(self) -> dict:
        out = np.zeros(9, dtype=np.int64)
        _check(lib().admm_get_stats(self.h, _ptr(out)), "admm_get_stats")
        return dict(zip(STAT_NAMES, (int(v) for v in out)))

    def profile_iterations(self, iters=1) -> dict:
        out = np.zeros(3)
        _check(lib().admm_profile_iterations(self.h, iters, _ptr(out)), "admm_profile_iterations")
        return dict(branch_ms=out[0], bus_ms=out[1], iter_ms=out[2])

    def autotune(self, iters=3):
        """Tune the launch shape; returns (branch blocks, iterations per graph
        body, fastest mean branch_tron ms, lanes per branch)."""
        n = C.c_int32(0)
        body = C.c_int32(0)
        ms = C.c_double(0.0)
        lanes = C.c_int32(0)
        _check(lib().admm_autotune(self.h, iters, C.byref(n), C.byref(body), C.byref(ms),
                                   C.byref(lanes)), "admm_autotune")
        return int(n.value), int(body.value), float(ms.value), int(lanes.value)

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().admm_get_state(self.h, None, C.byref(n)), "admm_get_state")
        buf = C.create_string_buffer(n.value)
        _check(lib().admm_get_state(self.h, buf, C.byref(n)), "admm_get_state")
        return buf.raw[: n.value]

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().admm_set_state(self.h, buf, len(blob)), "admm_set_state")

    def get_scenario_state(self, s: int) -> bytes:
        n = C.c_size_t(0)
        _check(lib().admm_get_scenario_state(self.h, s, None, C.byref(n)), "admm_get_scenario_state")
        buf = C.create_string_buffer(n.value)
        _check(lib().admm_get_scenario_state(self.h, s, buf, C.byref(n)), "admm_get_scenario_state")
        return buf.raw[: n.value]

    def set_scenario_state(self, s: int, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().admm_set_scenario_state(self.h, s, buf, len(blob)), "admm_set_scenario_state")
