"""Seeded synthetic power grids shaped like the grids of the paper's Table 1.

The paper's experiments use MATPOWER cases (pegase, ACTIVSg) and an ISO-NE load
profile; none of those data are available here, so every workload is a seeded
synthetic grid with the same proportions (branches ~1.26 x buses, generators
~0.15 x buses for the 70k case, Table 1) and a feasible operating point built
in by construction.

This module only *creates inputs*.  It holds none of the ADMM method's
arithmetic: the operating point that makes each grid feasible is computed from
circuit laws (branch currents of the pi model behind an ideal transformer,
Section II-A), not from the solver's admittance or flow routines, and both the
CPU oracle and the CUDA library receive the arrays built here.

Recipe (all draws from one ``numpy.random.Generator(PCG64(seed))``):

* Topology: buses uniform in the unit square; a random spanning tree is the
  minimum spanning tree of the Delaunay graph under edge weights
  ``length * U[1, 2]``; mesh edges are random remaining Delaunay edges until the
  branch count is reached.  Each branch gets a random orientation.
* Lines: ``r ~ U[0.002, 0.03]``, ``x = r * U[3, 10]``, ``b ~ U[0, 0.05]`` (pu), tap 1,
  shift 0; bus shunts ``gs = bs = 0``; voltage bounds ``[0.94, 1.06]``.
* Optional devices (``devices=True``; off for the benchmark grids, on in the
  tests that pin the shunt and transformer terms): 10% of the buses get a shunt
  ``gs ~ U[0, 0.03]``, ``bs ~ U[-0.1, 0.3]`` (pu at 1 pu voltage), 10% of the
  branches become transformers with ``tap ~ U[0.95, 1.05]``, and a fifth of
  those phase shifters with ``shift ~ U[-0.1, 0.1]`` rad.  The feasible point
  below then accounts for both: flows through an ideal transformer of ratio
  ``tap e^{j shift}`` at the from end, shunt power ``(gs - j bs) |V|^2`` drawn
  at the bus.
* Generators: ``ngen`` distinct random buses; costs ``c2 ~ U[0.01, 0.1]`` $/MW^2h,
  ``c1 ~ U[10, 40]`` $/MWh, ``c0 = 0``.
* Feasible point: base loads ``pd0 ~ LogNormal(0, 0.8)`` scaled to mean 0.3 pu;
  dispatch ``pg0`` = the load of each generator's nearest-bus region times
  ``U[0.9, 1.1]``, normalised to ``sum pg0 = sum pd0``; angles from a DC power flow
  of ``pg0 - pd0``, the reference bus being the generator bus nearest the middle
  of the angle range, scaled by ``k <= 1`` so that the 99th percentile of line
  angle differences is at most 0.3 rad and no bus angle exceeds ``theta_max``
  (scaling moves a share ``1 - k`` of each load onto the generator buses); magnitudes
  a smooth field ``1 + 0.03 sin(2 pi (a px + b py) + phi)``; ``qg0 = 0.2 pg0 U[-1, 1]``.
  Loads are then reset to generation minus the AC injection of that point, so
  the point satisfies the AC power balance exactly.
* Limits: ``pmax = pg0 / U[0.6, 0.8]`` (total load ~70% of capacity), ``pmin = 0``,
  ``q`` bounds ``qg0 -+ (|qg0| + 0.5)``, line rating
  ``rate_a = max(1.3 max(|S_ij|, |S_ji|), 0.05)`` so the point is strictly inside
  the 99%-tightened limit the method uses (Section IV-A).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

BRANCH_RATIO_70K = 88207.0 / 70000.0   # Table 1, ACTIVSg70k
GEN_RATIO_70K = 10390.0 / 70000.0      # Table 1, ACTIVSg70k


@dataclass
class Grid:
    """Plain arrays describing one grid (0-based indices, per unit except costs)."""
    nbus: int
    nbranch: int
    ngen: int
    ref_bus: int
    base_mva: float
    pd: np.ndarray
    qd: np.ndarray
    gs: np.ndarray
    bs: np.ndarray
    vmin: np.ndarray
    vmax: np.ndarray
    f_bus: np.ndarray
    t_bus: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    tap: np.ndarray
    shift: np.ndarray
    rate_a: np.ndarray
    gen_bus: np.ndarray
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray
    c0: np.ndarray
    # the built-in feasible operating point (used by tests only)
    vm0: np.ndarray = field(default=None, repr=False)
    va0: np.ndarray = field(default=None, repr=False)
    pg0: np.ndarray = field(default=None, repr=False)
    qg0: np.ndarray = field(default=None, repr=False)
    seed: int = 0

    def with_loads(self, pd: np.ndarray, qd: np.ndarray) -> "Grid":
        return replace(self, pd=np.ascontiguousarray(pd, dtype=np.float64),
                       qd=np.ascontiguousarray(qd, dtype=np.float64))


def _topology(rng: np.random.Generator, nbus: int, nbranch: int):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    from scipy.spatial import Delaunay

    pos = rng.random((nbus, 2))
    tri = Delaunay(pos)
    simp = tri.simplices
    e = np.concatenate([simp[:, [0, 1]], simp[:, [1, 2]], simp[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    length = np.linalg.norm(pos[e[:, 0]] - pos[e[:, 1]], axis=1)
    if nbranch < nbus - 1:
        raise ValueError("nbranch must be at least nbus - 1")
    if nbranch > len(e):
        raise ValueError(f"nbranch {nbranch} exceeds the {len(e)} Delaunay edges")
    w = length * rng.uniform(1.0, 2.0, len(e))
    g = coo_matrix((w, (e[:, 0], e[:, 1])), shape=(nbus, nbus)).tocsr()
    mst = minimum_spanning_tree(g).tocoo()
    tree = np.stack([np.minimum(mst.row, mst.col), np.maximum(mst.row, mst.col)], axis=1)
    if len(tree) != nbus - 1:
        raise RuntimeError("Delaunay graph is not connected")
    key_all = e[:, 0].astype(np.int64) * nbus + e[:, 1]
    key_tree = tree[:, 0].astype(np.int64) * nbus + tree[:, 1]
    in_tree = np.isin(key_all, key_tree)
    rest = rng.permutation(np.flatnonzero(~in_tree))
    mesh = e[rest[: nbranch - (nbus - 1)]]
    edges = np.concatenate([tree, mesh]).astype(np.int64)
    # random order and orientation
    edges = edges[rng.permutation(len(edges))]
    flip = rng.random(len(edges)) < 0.5
    edges[flip] = edges[flip][:, ::-1]
    return pos, edges


def _dc_angles(nbus, f, t, x, pinj, ref):
    from scipy.sparse import coo_matrix
    from scipy.sparse.linalg import spsolve
    bser = 1.0 / x
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([bser, bser, -bser, -bser])
    B = coo_matrix((vals, (rows, cols)), shape=(nbus, nbus)).tocsr()
    keep = np.ones(nbus, dtype=bool)
    keep[ref] = False
    idx = np.flatnonzero(keep)
    Bred = B[idx][:, idx].tocsc()
    th = np.zeros(nbus)
    th[idx] = spsolve(Bred, pinj[idx])
    return th


def _branch_power(V, f, t, r, x, b, tap=None, shift=None):
    """Complex power entering each branch at its two ends, from branch currents
    of the pi model (series impedance r + jx, half of b at each end of the
    series element) behind an ideal transformer of ratio tap e^{j shift} at the
    from end (tap 1, shift 0 when not given)."""
    a = np.ones(len(f), dtype=np.complex128)
    if tap is not None:
        a = np.where(tap == 0.0, 1.0, tap) * np.exp(1j * (shift if shift is not None else 0.0))
    z = r + 1j * x
    vf = V[f] / a                           # from-end voltage behind the transformer
    i_series = (vf - V[t]) / z
    i_f = (i_series + 0.5j * b * vf) / np.conj(a)   # the ideal transformer passes S through
    i_t = -i_series + 0.5j * b * V[t]
    return V[f] * np.conj(i_f), V[t] * np.conj(i_t)


def make_grid(nbus: int, nbranch: int, ngen: int, seed: int = 0,
              theta_max: float = 2.0, base_mva: float = 100.0, devices: bool = False) -> Grid:
    """Build one seeded synthetic grid with a built-in AC-feasible point
    (``devices``: add bus shunts, transformers and phase shifters)."""
    if not (nbus >= 2 and ngen >= 1 and ngen <= nbus):
        raise ValueError("need nbus >= 2 and 1 <= ngen <= nbus")
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, edges = _topology(rng, nbus, nbranch)
    f = edges[:, 0].astype(np.int32)
    t = edges[:, 1].astype(np.int32)
    nl = len(edges)
    r = rng.uniform(0.002, 0.03, nl)
    x = r * rng.uniform(3.0, 10.0, nl)
    b = rng.uniform(0.0, 0.05, nl)

    gen_bus = np.sort(rng.choice(nbus, size=ngen, replace=False)).astype(np.int32)
    c2 = rng.uniform(0.01, 0.1, ngen)
    c1 = rng.uniform(10.0, 40.0, ngen)
    c0 = np.zeros(ngen)

    from scipy.spatial import cKDTree
    pd0 = rng.lognormal(0.0, 0.8, nbus)
    pd0 *= 0.3 / pd0.mean()
    _, region = cKDTree(pos[gen_bus]).query(pos)
    pg0 = np.bincount(region, weights=pd0, minlength=ngen) * rng.uniform(0.9, 1.1, ngen)
    pg0 *= pd0.sum() / pg0.sum()

    pinj = -pd0.copy()
    np.add.at(pinj, gen_bus, pg0)
    th = _dc_angles(nbus, f, t, x, pinj, int(gen_bus[0]))
    mid = 0.5 * (th.max() + th.min())
    ref = int(gen_bus[np.argmin(np.abs(th[gen_bus] - mid))])
    th -= th[ref]
    d99 = np.percentile(np.abs(th[f] - th[t]), 99)
    amax = np.max(np.abs(th))
    k = 1.0
    if d99 > 0.3:
        k = 0.3 / d99
    if amax * k > theta_max:
        k = theta_max / amax
    th *= k

    a, bb = rng.uniform(0.5, 1.5, 2)
    phi = rng.uniform(0.0, 2.0 * np.pi)
    vm = 1.0 + 0.03 * np.sin(2.0 * np.pi * (a * pos[:, 0] + bb * pos[:, 1]) + phi)
    V = vm * np.exp(1j * th)
    qg0 = 0.2 * pg0 * rng.uniform(-1.0, 1.0, ngen)

    tap, shift = np.ones(nl), np.zeros(nl)
    gs, bs = np.zeros(nbus), np.zeros(nbus)
    if devices:
        # drawn after every draw of the plain recipe, so the plain grid of a
        # seed is the same with and without devices up to these
        d_rng = np.random.Generator(np.random.PCG64(seed + 0x5eed))
        sh = d_rng.random(nbus) < 0.1
        gs[sh] = d_rng.uniform(0.0, 0.03, sh.sum())
        bs[sh] = d_rng.uniform(-0.1, 0.3, sh.sum())
        tx = d_rng.random(nl) < 0.1
        tap[tx] = d_rng.uniform(0.95, 1.05, tx.sum())
        ps = tx & (d_rng.random(nl) < 0.2)
        shift[ps] = d_rng.uniform(-0.1, 0.1, ps.sum())

    s_f, s_t = _branch_power(V, f, t, r, x, b, tap, shift)
    inj = np.zeros(nbus, dtype=np.complex128)
    np.add.at(inj, f, s_f)
    np.add.at(inj, t, s_t)
    gen_p = np.zeros(nbus)
    gen_q = np.zeros(nbus)
    np.add.at(gen_p, gen_bus, pg0)
    np.add.at(gen_q, gen_bus, qg0)
    # balance: generation - load - shunt (gs - j bs)|V|^2 = power into the branches
    pd = gen_p - inj.real - gs * vm ** 2
    qd = gen_q - inj.imag + bs * vm ** 2

    pmax = pg0 / rng.uniform(0.6, 0.8, ngen)
    pmin = np.zeros(ngen)
    qmin = qg0 - (np.abs(qg0) + 0.5)
    qmax = qg0 + (np.abs(qg0) + 0.5)
    rate_a = np.maximum(1.3 * np.maximum(np.abs(s_f), np.abs(s_t)), 0.05)

    f64 = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    return Grid(
        nbus=nbus, nbranch=nl, ngen=ngen, ref_bus=ref, base_mva=base_mva,
        pd=f64(pd), qd=f64(qd), gs=f64(gs), bs=f64(bs),
        vmin=np.full(nbus, 0.94), vmax=np.full(nbus, 1.06),
        f_bus=np.ascontiguousarray(f), t_bus=np.ascontiguousarray(t),
        r=f64(r), x=f64(x), b=f64(b), tap=f64(tap), shift=f64(shift),
        rate_a=f64(rate_a), gen_bus=np.ascontiguousarray(gen_bus),
        pmin=f64(pmin), pmax=f64(pmax), qmin=f64(qmin), qmax=f64(qmax),
        c2=f64(c2), c1=f64(c1), c0=f64(c0),
        vm0=f64(vm), va0=f64(th), pg0=f64(pg0), qg0=f64(qg0), seed=seed)


def tiny_grid(seed: int = 0, devices: bool = False) -> Grid:
    """30 buses, 41 branches (29 tree + 12 mesh edges), 6 generators."""
    return make_grid(30, 41, 6, seed=seed, theta_max=0.2, devices=devices)


def sized_grid(nbus: int, seed: int = 0, devices: bool = False) -> Grid:
    """A grid with the ACTIVSg70k proportions of Table 1 (2k, 10k, 70k buses...)."""
    nl = int(round(BRANCH_RATIO_70K * nbus))
    ng = max(1, int(round(GEN_RATIO_70K * nbus)))
    return make_grid(nbus, nl, ng, seed=seed, theta_max=2.0, devices=devices)


def penalties_for(nbus: int):
    """(rho_pq, rho_va, obj_scale) by grid size, following Table 1 and Section IV-A."""
    if nbus <= 5000:
        return 1e1, 1e3, 1.0
    if nbus <= 20000:
        return 5e1, 5e3, 1.0
    if nbus <= 40000:
        return 3e3, 3e4, 1.0
    return 3e4, 3e5, 2.0


def ar1_loads(grid: Grid, steps: int, seed: int, phi: float = 0.9, sigma: float = 0.01):
    """AR(1) relative load multipliers a_t = phi a_{t-1} + sigma N(0,1) per bus;
    returns arrays (steps, nbus) of pd_t = pd_0 (1 + a_t) and qd_t likewise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.zeros(grid.nbus)
    pds, qds = [], []
    for _ in range(steps):
        a = phi * a + sigma * rng.standard_normal(grid.nbus)
        pds.append(grid.pd * (1.0 + a))
        qds.append(grid.qd * (1.0 + a))
    return np.array(pds), np.array(qds)


def batch_grids(n: int, lo: int = 500, hi: int = 20000, seed: int = 0, load_noise: float = 0.02):
    """`n` independent grids with bus counts log-uniform in [lo, hi] (branches
    and generators in the ACTIVSg70k ratios of Table 1), each with its own
    seeded load perturbation pd (1 + load_noise N(0,1)) (qd likewise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(int)
    out = []
    for k, nb in enumerate(sizes):
        g = sized_grid(int(nb), seed=seed * 100003 + k)
        r = np.random.Generator(np.random.PCG64(seed * 7919 + k)).standard_normal(g.nbus)
        out.append(g.with_loads(g.pd * (1.0 + load_noise * r), g.qd * (1.0 + load_noise * r)))
    return out
