"""ctypes binding of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the bench load this module; the library under ``paper_2110_06879_gb300``
never does.  ``build()`` compiles ``liboracle.so`` with gcc (no FMA contraction).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
LIB = os.path.join(HERE, "liboracle.so")

U, XBAR, Z, Y, LAMBDA, BRANCH_X, BRANCH_LT, BUS, RHO = range(9)


def build(force: bool = False) -> str:
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(LIB) for s in (SRC, HDR))
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class OraGrid(C.Structure):
    _fields_ = [("nbus", C.c_int32), ("nbranch", C.c_int32), ("ngen", C.c_int32),
                ("ref_bus", C.c_int32), ("base_mva", C.c_double)] + [
        (n, C.c_void_p) for n in ("pd", "qd", "gs", "bs", "vmin", "vmax", "f_bus", "t_bus",
                                  "r", "x", "b", "tap", "shift", "rate_a", "gen_bus", "pmin",
                                  "pmax", "qmin", "qmax", "c2", "c1", "c0")]


OPT_DOUBLES = ("rho_pq", "rho_va", "obj_scale", "line_limit_frac", "beta0", "beta_factor",
               "z_decay", "beta_max", "lambda_max", "tol_in0", "tol_in_decay", "al_rho0",
               "al_tol", "al_decay", "al_rho_factor", "al_rho_max", "tron_gtol", "tron_ftol",
               "tron_xtol")
OPT_INTS = ("two_level", "max_outer", "max_inner", "al_max_iter", "tron_max_iter", "beta_rule")


class OraOptions(C.Structure):
    _fields_ = [(n, C.c_double) for n in OPT_DOUBLES] + [(n, C.c_int32) for n in OPT_INTS]


class OraBranchProb(C.Structure):
    _fields_ = [("Y", C.c_double * 8), ("lo", C.c_double * 6), ("hi", C.c_double * 6),
                ("xbar", C.c_double * 8), ("z", C.c_double * 8), ("y", C.c_double * 8),
                ("rho", C.c_double * 8), ("lt", C.c_double * 2), ("rt", C.c_double),
                ("alpha", C.c_double)]


class OraStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("tron_calls", "tron_iters", "fgh_evals", "f_evals",
                                         "cauchy_trials", "cg_iters", "ps_trials", "al_passes",
                                         "tron_maxiter_hits")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def default_options(**kw) -> dict:
    """The method's parameters (Table 1 penalties for grids up to ~3k buses,
    Section IV-A iteration caps) and this implementation's readings of the
    parameters the paper leaves open."""
    o = dict(rho_pq=10.0, rho_va=1000.0, obj_scale=1.0, line_limit_frac=0.99,
             beta0=0.0, beta_factor=6.0, z_decay=0.8, beta_max=1e12, lambda_max=1e12,
             tol_in0=1e-2, tol_in_decay=0.5, al_rho0=0.0, al_tol=1e-6, al_decay=0.1,
             al_rho_factor=100.0, al_rho_max=1e12, tron_gtol=1e-10, tron_ftol=1e-12, tron_xtol=1e-13,
             two_level=1, max_outer=20, max_inner=1000, al_max_iter=20, tron_max_iter=200,
             beta_rule=0)
    for k, v in kw.items():
        if k not in o:
            raise KeyError(k)
        o[k] = v
    return o


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i32, d = C.c_void_p, C.c_int32, C.c_double
        L.ora_create.restype = vp
        L.ora_create.argtypes = [C.POINTER(OraGrid), C.POINTER(OraOptions)]
        L.ora_destroy.argtypes = [vp]
        L.ora_cold_start.argtypes = [vp]
        L.ora_set_loads.argtypes = [vp, vp, vp]
        L.ora_set_gen_bounds.argtypes = [vp, vp, vp]
        L.ora_set_ramp_limit.argtypes = [vp, d]
        L.ora_solve.argtypes = [vp, d, i32, i32]
        L.ora_solve.restype = C.c_int
        L.ora_get.argtypes = [vp, i32, vp]
        L.ora_get_residuals.argtypes = [vp, vp, vp]
        L.ora_get_history.argtypes = [vp, vp, i32]
        L.ora_get_history.restype = i32
        L.ora_get_stats.argtypes = [vp, C.POINTER(OraStats)]
        L.ora_get_csr.argtypes = [vp, vp, vp]
        L.ora_get_admittance.argtypes = [vp, vp]
        L.ora_finalize.argtypes = [vp] + [vp] * 9
        L.ora_admittance.argtypes = [d, d, d, d, d, vp]
        L.ora_branch_fgh.argtypes = [C.POINTER(OraBranchProb), vp, vp, vp, vp]
        L.ora_branch_flows.argtypes = [vp, vp, vp]
        L.ora_tron.argtypes = [C.POINTER(OraBranchProb), vp, C.POINTER(OraOptions),
                               C.POINTER(OraStats)]
        L.ora_tron.restype = C.c_int
        L.ora_branch_solve.argtypes = [C.POINTER(OraBranchProb), vp, C.POINTER(OraOptions),
                                       C.POINTER(OraStats)]
        L.ora_gen_solve.argtypes = [d] * 8
        L.ora_gen_solve.restype = d
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def make_options(opts: dict) -> OraOptions:
    o = OraOptions()
    for k, v in opts.items():
        setattr(o, k, v)
    return o


class Oracle:
    """Whole-problem oracle: ``Oracle(grid, **options)``."""

    def __init__(self, grid, **opts):
        self.grid = grid
        self.opts = default_options(**opts)
        self._keep = {}
        g = OraGrid()
        g.nbus, g.nbranch, g.ngen, g.ref_bus = grid.nbus, grid.nbranch, grid.ngen, grid.ref_bus
        g.base_mva = grid.base_mva
        for name in ("pd", "qd", "gs", "bs", "vmin", "vmax", "r", "x", "b", "tap", "shift",
                     "rate_a", "pmin", "pmax", "qmin", "qmax", "c2", "c1", "c0"):
            a = np.ascontiguousarray(getattr(grid, name), dtype=np.float64)
            self._keep[name] = a
            setattr(g, name, _ptr(a))
        for name in ("f_bus", "t_bus", "gen_bus"):
            a = np.ascontiguousarray(getattr(grid, name), dtype=np.int32)
            self._keep[name] = a
            setattr(g, name, _ptr(a))
        self._o = make_options(self.opts)
        self.h = lib().ora_create(C.byref(g), C.byref(self._o))
        self.nb, self.nl, self.ng = grid.nbus, grid.nbranch, grid.ngen
        self.m = 2 * self.ng + 8 * self.nl

    def __del__(self):
        if getattr(self, "h", None):
            lib().ora_destroy(self.h)
            self.h = None

    def solve(self, tol=1e-4, max_iter=5000, warm_start=False) -> int:
        return lib().ora_solve(self.h, tol, max_iter, 1 if warm_start else 0)

    def set_loads(self, pd, qd):
        pd = np.ascontiguousarray(pd, dtype=np.float64)
        qd = np.ascontiguousarray(qd, dtype=np.float64)
        lib().ora_set_loads(self.h, _ptr(pd), _ptr(qd))

    def set_gen_bounds(self, pmin, pmax):
        pmin = np.ascontiguousarray(pmin, dtype=np.float64)
        pmax = np.ascontiguousarray(pmax, dtype=np.float64)
        lib().ora_set_gen_bounds(self.h, _ptr(pmin), _ptr(pmax))

    def set_ramp_limit(self, frac=0.02):
        lib().ora_set_ramp_limit(self.h, frac)

    def get(self, which: int) -> np.ndarray:
        n = {BRANCH_X: 6 * self.nl, BRANCH_LT: 2 * self.nl, BUS: 2 * self.nb}.get(which, self.m)
        out = np.empty(n)
        lib().ora_get(self.h, which, _ptr(out))
        return out

    def residuals(self) -> dict:
        d = np.zeros(9)
        i = np.zeros(4, dtype=np.int32)
        lib().ora_get_residuals(self.h, _ptr(d), _ptr(i))
        return dict(primal=d[0], dual=d[1], z_norm=d[2], primal_z=d[3], beta=d[4], tol_in=d[5],
                    u_norm=d[6], xbar_norm=d[7], y_norm=d[8],
                    iters=int(i[0]), outer_iters=int(i[1]), status=int(i[2]),
                    total_iters=int(i[3]))

    def history(self, cap=200000) -> np.ndarray:
        out = np.zeros((cap, 4))
        n = lib().ora_get_history(self.h, _ptr(out), cap)
        return out[:n]

    def stats(self) -> dict:
        s = OraStats()
        lib().ora_get_stats(self.h, C.byref(s))
        return s.as_dict()

    def csr(self):
        row = np.zeros(self.nb + 1, dtype=np.int32)
        col = np.zeros(2 * self.nl + self.ng, dtype=np.int32)
        lib().ora_get_csr(self.h, _ptr(row), _ptr(col))
        return row, col

    def admittance(self) -> np.ndarray:
        out = np.zeros(8 * self.nl)
        lib().ora_get_admittance(self.h, _ptr(out))
        return out.reshape(self.nl, 8)

    def finalize(self) -> dict:
        nb, nl, ng = self.nb, self.nl, self.ng
        arrs = dict(pg=np.zeros(ng), qg=np.zeros(ng), vm=np.zeros(nb), va=np.zeros(nb),
                    pf=np.zeros(nl), qf=np.zeros(nl), pt=np.zeros(nl), qt=np.zeros(nl))
        om = np.zeros(2)
        lib().ora_finalize(self.h, *[_ptr(arrs[k]) for k in
                                     ("pg", "qg", "vm", "va", "pf", "qf", "pt", "qt")], _ptr(om))
        arrs["objective"] = float(om[0])
        arrs["max_viol"] = float(om[1])
        return arrs


def admittance(r, x, b, tap=1.0, shift=0.0) -> np.ndarray:
    out = np.zeros(8)
    lib().ora_admittance(r, x, b, tap, shift, _ptr(out))
    return out


def branch_prob(Y, lo, hi, xbar, z, y, rho, lt, rt) -> OraBranchProb:
    p = OraBranchProb()
    for name, val in (("Y", Y), ("lo", lo), ("hi", hi), ("xbar", xbar), ("z", z), ("y", y),
                      ("rho", rho), ("lt", lt)):
        arr = getattr(p, name)
        for i, v in enumerate(val):
            arr[i] = float(v)
    p.rt = float(rt)
    p.alpha = 1.0
    return p


def branch_fgh(bp: OraBranchProb, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros(1)
    g = np.zeros(6)
    H = np.zeros(36)
    lib().ora_branch_fgh(C.byref(bp), _ptr(x), _ptr(f), _ptr(g), _ptr(H))
    return f[0], g, H.reshape(6, 6)


def branch_flows(Y, x) -> np.ndarray:
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(4)
    lib().ora_branch_flows(_ptr(Y), _ptr(x), _ptr(out))
    return out


def tron(bp: OraBranchProb, x0, **opts):
    x = np.array(x0, dtype=np.float64)
    o = make_options(default_options(**opts))
    st = OraStats()
    status = lib().ora_tron(C.byref(bp), _ptr(x), C.byref(o), C.byref(st))
    return x, status, st.as_dict()


def branch_solve(bp: OraBranchProb, x0, **opts):
    x = np.array(x0, dtype=np.float64)
    o = make_options(default_options(**opts))
    st = OraStats()
    lib().ora_branch_solve(C.byref(bp), _ptr(x), C.byref(o), C.byref(st))
    return x, np.array(bp.lt[:]), float(bp.rt), st.as_dict()


def gen_solve(cost2, cost1, rho, xbar, z, y, lo, hi) -> float:
    return lib().ora_gen_solve(cost2, cost1, rho, xbar, z, y, lo, hi)
