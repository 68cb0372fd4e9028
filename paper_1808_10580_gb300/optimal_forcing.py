"""The optimal-forcing example of Section 4 (Eq. bvp:ex1, Eq. bvp:ex1:cost):
find source strengths F = (F_1, ..., F_n) such that the solution theta of the
boundary-value problem in the unit square matches data y at a few points,
with a Nelder-Mead search as in the paper.

By Theorem 3.2 the particle map is affine in F:
    theta(x_i; F) = E[g(X_tau)] - sum_q F_q E[int_0^tau phi_q(X_s) ds],
so one call of pm_forward_square_bvp (per observation, the n + 1 functionals
on one set of paths) serves every evaluation of G(F) the search makes; each
evaluation is then a small matrix-vector product.  The search itself is the
Nelder-Mead simplex method (Nelder & Mead 1965, with the standard
coefficients: reflection 1, expansion 2, contraction 1/2, shrink 1/2; the
ordering and tie rules of Lagarias, Reeds, Wright & Wright 1998)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import _lib as pm
from . import inputs


def functionals(ctx, w: inputs.SquareBVPWorkload, flags=pm.PM_FP32, M=None, x=None):
    """E [n_obs, n_src + 1] and its Monte Carlo standard errors: column 0 is
    E[g(X_tau)], column q + 1 is E[int phi_q]."""
    M = w.M if M is None else M
    x = np.ascontiguousarray(w.x if x is None else x, dtype=np.float64)
    prob = pm.SquareBVP(w.prob.b, w.prob.kappa, w.prob.c, w.prob.w, w.prob.g_cos, w.prob.g_quad)
    n_f = len(w.prob.c) + 1
    mean = np.empty(len(x) * n_f)
    var = np.empty(len(x) * n_f)
    pm.pm_forward_square_bvp(ctx, prob, x, len(x), M, w.dt, w.max_steps, w.seed, flags, mean, var)
    E = mean.reshape(len(x), n_f)
    return E, np.sqrt(var.reshape(len(x), n_f) / M)


def G(E: np.ndarray, F: np.ndarray) -> np.ndarray:
    """theta at the observation points for source strengths F."""
    return E[:, 0] - E[:, 1:] @ np.asarray(F, dtype=np.float64)


def cost(E: np.ndarray, y: np.ndarray, F: np.ndarray) -> float:
    """|| y - G(F) || (Eq. bvp:ex1:cost)."""
    return float(np.linalg.norm(np.asarray(y, dtype=np.float64) - G(E, F)))


@dataclass
class NMResult:
    x: np.ndarray
    fun: float
    evaluations: int
    iterations: int


def nelder_mead(f, x0, step=1.0, xtol=1e-10, ftol=1e-12, max_evals=20000) -> NMResult:
    """Minimise f from x0 with the Nelder-Mead simplex method."""
    x0 = np.asarray(x0, dtype=np.float64)
    n = x0.size
    simplex = [x0.copy()]
    for k in range(n):
        v = x0.copy()
        v[k] += step
        simplex.append(v)
    values = [f(v) for v in simplex]
    evals = n + 1
    it = 0
    while evals < max_evals:
        order = np.argsort(values, kind="stable")
        simplex = [simplex[k] for k in order]
        values = [values[k] for k in order]
        spread_x = max(np.max(np.abs(v - simplex[0])) for v in simplex[1:])
        if spread_x <= xtol and values[-1] - values[0] <= ftol:
            break
        it += 1
        centroid = np.mean(simplex[:-1], axis=0)
        worst = simplex[-1]
        xr = centroid + (centroid - worst)
        fr = f(xr)
        evals += 1
        if values[0] <= fr < values[-2]:
            simplex[-1], values[-1] = xr, fr
            continue
        if fr < values[0]:
            xe = centroid + 2.0 * (centroid - worst)
            fe = f(xe)
            evals += 1
            if fe < fr:
                simplex[-1], values[-1] = xe, fe
            else:
                simplex[-1], values[-1] = xr, fr
            continue
        if fr < values[-1]:  # outside contraction
            xc = centroid + 0.5 * (xr - centroid)
            fc = f(xc)
            evals += 1
            if fc <= fr:
                simplex[-1], values[-1] = xc, fc
                continue
        else:  # inside contraction
            xc = centroid + 0.5 * (worst - centroid)
            fc = f(xc)
            evals += 1
            if fc < values[-1]:
                simplex[-1], values[-1] = xc, fc
                continue
        best = simplex[0]
        for k in range(1, n + 1):  # shrink towards the best vertex
            simplex[k] = best + 0.5 * (simplex[k] - best)
            values[k] = f(simplex[k])
        evals += n
    k = int(np.argmin(values))
    return NMResult(simplex[k], float(values[k]), evals, it)


def solve(E: np.ndarray, y: np.ndarray, F0=None, **kw) -> NMResult:
    """The optimal forcing by Nelder-Mead on the particle map's functionals."""
    F0 = np.zeros(E.shape[1] - 1) if F0 is None else F0
    return nelder_mead(lambda F: cost(E, y, F), F0, **kw)
