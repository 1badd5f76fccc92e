"""Independent reference solve of the whole ACOPF (eq. acopf, Section II-A).

Used only by the tests to pin the oracle: the problem is written in polar
voltages with branch currents from the pi-model circuit (an ideal transformer
of ratio a = tap e^{j shift} at the from end, series impedance r + jx, half the
line charging at each end of the series element), and solved by SciPy's SLSQP.
Nothing here comes from the oracle or the library.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize


def branch_currents(V, grid):
    f, t = grid.f_bus, grid.t_bus
    tap = np.where(grid.tap == 0.0, 1.0, grid.tap)
    a = tap * np.exp(1j * grid.shift)
    z = grid.r + 1j * grid.x
    Vf_sec = V[f] / a                       # voltage behind the ideal transformer
    i_ser = (Vf_sec - V[t]) / z
    i_f_sec = i_ser + 0.5j * grid.b * Vf_sec
    i_f = i_f_sec / np.conj(a)              # lossless transformer: S conserved
    i_t = -i_ser + 0.5j * grid.b * V[t]
    return i_f, i_t


def branch_power(V, grid):
    i_f, i_t = branch_currents(V, grid)
    return V[grid.f_bus] * np.conj(i_f), V[grid.t_bus] * np.conj(i_t)


def mismatch(vm, va, pg, qg, grid):
    """Complex power balance residual per bus: generation - load - shunt - flows out."""
    V = vm * np.exp(1j * va)
    sf, st = branch_power(V, grid)
    out = np.zeros(grid.nbus, dtype=complex)
    np.add.at(out, grid.f_bus, sf)
    np.add.at(out, grid.t_bus, st)
    gen = np.zeros(grid.nbus, dtype=complex)
    np.add.at(gen, grid.gen_bus, pg + 1j * qg)
    shunt = (grid.gs - 1j * grid.bs) * vm ** 2
    return gen - (grid.pd + 1j * grid.qd) - shunt - out


def cost(pg, grid):
    base = grid.base_mva
    P = pg * base
    return float(np.sum(grid.c2 * P ** 2 + grid.c1 * P + grid.c0))


def solve_acopf(grid, line_limit_frac=0.99, x0=None, maxiter=500):
    nb, ng = grid.nbus, grid.ngen
    nv = 2 * nb + 2 * ng
    sl = lambda v: (v[:nb], v[nb:2 * nb], v[2 * nb:2 * nb + ng], v[2 * nb + ng:])
    scale = 1.0 / max(1.0, cost(grid.pg0, grid))

    def obj(v):
        return cost(sl(v)[2], grid) * scale

    def eq(v):
        vm, va, pg, qg = sl(v)
        m = mismatch(vm, va, pg, qg, grid)
        return np.concatenate([m.real, m.imag, [va[grid.ref_bus]]])

    lim = (line_limit_frac * grid.rate_a) ** 2

    def ineq(v):
        vm, va, _, _ = sl(v)
        sf, st = branch_power(vm * np.exp(1j * va), grid)
        return np.concatenate([lim - np.abs(sf) ** 2, lim - np.abs(st) ** 2])

    bounds = ([(grid.vmin[i], grid.vmax[i]) for i in range(nb)]
              + [(-2 * np.pi, 2 * np.pi)] * nb
              + [(grid.pmin[k], grid.pmax[k]) for k in range(ng)]
              + [(grid.qmin[k], grid.qmax[k]) for k in range(ng)])
    if x0 is None:
        x0 = np.concatenate([grid.vm0, grid.va0, grid.pg0, grid.qg0])
    res = minimize(obj, x0, method="SLSQP", bounds=bounds,
                   constraints=[{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}],
                   options={"maxiter": maxiter, "ftol": 1e-12})
    vm, va, pg, qg = sl(res.x)
    return dict(success=bool(res.success), objective=cost(pg, grid), vm=vm, va=va, pg=pg, qg=qg,
                eq_viol=float(np.abs(eq(res.x)).max()), ineq_viol=float(max(0.0, -ineq(res.x).min())),
                message=res.message)
