"""Comparison of the CUDA path's state with the oracle's (shared by the GPU
parity tests).

The bar is relative to the size of each quantity, taken per kind of entry so
that small entries are not hidden behind large ones of another kind: the
coupling vectors (u, xbar, z, y, lambda) are split into generator p, generator
q and the eight branch couplings p_ij, q_ij, p_ji, q_ji, w_i, theta_i, w_j,
theta_j; the branch variables into their six columns; the bus values into w
and theta.  Each group must satisfy
    max |gpu - oracle| <= tol * max(max |oracle| over the group,
                                    1e-4 max |oracle| over the whole vector)
so that a group of rounding noise (z and y of a bus's only w coupling, for
instance, are zero up to rounding) is measured against the vector's scale
(absolute when the vector is identically zero).  lambda-tilde, the line-limit
multiplier, is compared relative to max(|lambda-tilde|, 1) per end, within
LT_TOL = 1e-7: it accumulates rho-tilde h over the AL passes, and on a binding
line rho-tilde grows to 1e8-1e12 while h is only as accurate as the TRON stop
(so rounding differences in h reach lambda-tilde multiplied by rho-tilde; the
worst difference measured on the first-ten-iteration grids is 2.3e-9); on a
line whose limit never binds lambda-tilde is rounding noise around zero,
which has no scale of its own.  The multipliers enter the iterates only
through the branch solutions, which are held to the 1e-9 bar.
"""
import numpy as np

import oracle
from paper_2110_06879_gb300 import admm

VEC_PAIRS = ((admm.ADMM_VEC_U, oracle.U), (admm.ADMM_VEC_XBAR, oracle.XBAR),
             (admm.ADMM_VEC_Z, oracle.Z), (admm.ADMM_VEC_Y, oracle.Y),
             (admm.ADMM_VEC_LAMBDA, oracle.LAMBDA), (admm.ADMM_VEC_BRANCH_X, oracle.BRANCH_X),
             (admm.ADMM_VEC_BRANCH_LT, oracle.BRANCH_LT), (admm.ADMM_VEC_BUS, oracle.BUS))
NAMES = {admm.ADMM_VEC_U: "u", admm.ADMM_VEC_XBAR: "xbar", admm.ADMM_VEC_Z: "z",
         admm.ADMM_VEC_Y: "y", admm.ADMM_VEC_LAMBDA: "lambda", admm.ADMM_VEC_BRANCH_X: "x",
         admm.ADMM_VEC_BRANCH_LT: "lt", admm.ADMM_VEC_BUS: "bus"}
COUPLING_KINDS = ("p_ij", "q_ij", "p_ji", "q_ji", "w_i", "th_i", "w_j", "th_j")
LT_TOL = 1e-7


GROUP_FLOOR = 1e-4


def relerr(a, b, floor=0.0):
    """Normwise relative error max|a - b| / max(max|b|, floor) (absolute if
    both are zero)."""
    if not a.size:
        return 0.0
    scale = max(np.abs(b).max() if b.size else 0.0, floor)
    if scale == 0.0:
        return np.abs(a).max()
    return np.abs(a - b).max() / scale


def groups(which, a, b, ngen):
    """(name, gpu part, oracle part) per kind of entry of one state vector."""
    if which in (admm.ADMM_VEC_U, admm.ADMM_VEC_XBAR, admm.ADMM_VEC_Z, admm.ADMM_VEC_Y,
                 admm.ADMM_VEC_LAMBDA):
        out = [("gen p", a[0:2 * ngen:2], b[0:2 * ngen:2]),
               ("gen q", a[1:2 * ngen:2], b[1:2 * ngen:2])]
        ab, bb = a[2 * ngen:].reshape(-1, 8), b[2 * ngen:].reshape(-1, 8)
        return out + [(COUPLING_KINDS[k], ab[:, k], bb[:, k]) for k in range(8)]
    if which == admm.ADMM_VEC_BRANCH_X:
        ab, bb = a.reshape(-1, 6), b.reshape(-1, 6)
        return [(n, ab[:, k], bb[:, k]) for k, n in enumerate(("v_i", "v_j", "th_i", "th_j",
                                                               "s_ij", "s_ji"))]
    if which == admm.ADMM_VEC_BUS:
        ab, bb = a.reshape(-1, 2), b.reshape(-1, 2)
        return [("w", ab[:, 0], bb[:, 0]), ("theta", ab[:, 1], bb[:, 1])]
    return [("all", a, b)]


def state_errors(s, o, ngen):
    """{(vector, group): error} of the GPU handle s (its selected scenario)
    against the oracle o."""
    errs = {}
    for w_gpu, w_ora in VEC_PAIRS:
        a, b = s.vector(w_gpu), o.get(w_ora)
        assert a.shape == b.shape
        if w_gpu == admm.ADMM_VEC_BRANCH_LT:
            ab, bb = a.reshape(-1, 2), b.reshape(-1, 2)
            for e, n in enumerate(("ij", "ji")):
                d = np.abs(ab[:, e] - bb[:, e])
                errs[("lt", n)] = (d.max() / max(np.abs(bb[:, e]).max(), 1.0)) if d.size else 0.0
            continue
        floor = GROUP_FLOOR * (np.abs(b).max() if b.size else 0.0)
        for name, ga, gb in groups(w_gpu, a, b, ngen):
            errs[(NAMES[w_gpu], name)] = relerr(ga, gb, floor)
    return errs


def compare_state(s, o, tol, label=""):
    """Assert every group of the state within tol of the oracle; returns the errors."""
    errs = state_errors(s, o, s.ng)
    bad = {k: v for k, v in errs.items() if not v <= (max(tol, LT_TOL) if k[0] == "lt" else tol)}
    assert not bad, (label, bad, max(errs.values()))
    return errs
