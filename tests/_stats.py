"""Statistical comparisons for the parity tests of the Monte Carlo estimators.

Algorithms 1 and 2 return sample means of per-path values, so two correct
implementations agree only up to Monte Carlo error unless they draw identical
paths, and on a chaotic flow even paths driven by identical Brownian
increments separate under rounding (float against double).  These helpers turn
per-observation comparisons into tests whose false-alarm rate is stated:

* ``zcheck``: per-observation z-scores must (a) exceed 3 in absolute value no
  more often than a binomial allowance for n independent N(0, 1) scores at a
  family-wise false-alarm rate alpha, and (b) have a sum of squares below the
  (1 - alpha) quantile of chi-square with n degrees of freedom.  (a) catches a
  few badly wrong observations, (b) a small bias shared by many.
* ``two_sample_z``: the z-score of the difference of two independent means,
  3 standard errors = 3 sqrt(SE_1^2 + SE_2^2).
* ``paired_z``: the z-score of the mean of per-path differences of two
  estimators driven by the same streams (path i of observation j on both
  sides); it is far more sensitive than the two-sample score while the paths
  stay close.
* ``ks_positions``: two-sample Kolmogorov-Smirnov tests on end positions on
  the unit torus (both coordinates and the two diagonals, modulo 1), with a
  Bonferroni correction over observations and projections.
"""
from __future__ import annotations

import numpy as np
from scipy import stats as st

ALPHA = 1e-4


def allowed_exceedances(n: int, z: float = 3.0, alpha: float = ALPHA) -> int:
    """Largest count k of |z_j| > z among n independent N(0,1) scores with
    P(count > k) <= alpha."""
    p = 2.0 * st.norm.sf(z)
    k = 0
    while st.binom.sf(k, n, p) > alpha:
        k += 1
    return k


def zcheck(z, alpha: float = ALPHA) -> dict:
    z = np.asarray(z, dtype=np.float64).ravel()
    n = z.size
    k = allowed_exceedances(n, 3.0, alpha)
    chi2 = float((z ** 2).sum())
    chi2_max = float(st.chi2.isf(alpha, n))
    exceed = int((np.abs(z) > 3.0).sum())
    return dict(n=n, exceed_3=exceed, allowed=k, chi2=chi2, chi2_max=chi2_max, max_abs_z=float(np.abs(z).max()),
                ok=bool(exceed <= k and chi2 <= chi2_max))


def two_sample_z(m1, se1, m2, se2):
    m1, se1, m2, se2 = (np.asarray(a, dtype=np.float64) for a in (m1, se1, m2, se2))
    return (m1 - m2) / np.sqrt(se1 ** 2 + se2 ** 2)


def paired_z(a, b):
    """a, b: [n_obs, M] per-path values on the same streams -> z of mean(a - b)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    M = d.shape[1]
    se = d.std(axis=1, ddof=1) / np.sqrt(M)
    mean = d.mean(axis=1)
    # identical paths: difference exactly 0 is no evidence either way
    return np.where(se > 0, mean / np.where(se > 0, se, 1.0), np.where(mean == 0, 0.0, np.inf))


def ks_positions(xa, xb, alpha: float = 1e-3) -> dict:
    """xa [n_obs, Ma, 2], xb [n_obs, Mb, 2] end positions in [0,1)^2 from
    independent streams -> smallest p-value over observations and the
    projections x1, x2, x1 + x2, x1 - x2 (mod 1), and the Bonferroni verdict."""
    xa = np.asarray(xa, dtype=np.float64)
    xb = np.asarray(xb, dtype=np.float64)
    projections = [lambda x: x[..., 0], lambda x: x[..., 1], lambda x: np.mod(x[..., 0] + x[..., 1], 1.0),
                   lambda x: np.mod(x[..., 0] - x[..., 1], 1.0)]
    pmin = 1.0
    for j in range(xa.shape[0]):
        for f in projections:
            pmin = min(pmin, float(st.ks_2samp(f(xa[j]), f(xb[j])).pvalue))
    n_tests = xa.shape[0] * len(projections)
    return dict(n_tests=n_tests, p_min=pmin, p_bonferroni=min(1.0, pmin * n_tests), ok=bool(pmin * n_tests > alpha))


def paired_position_z(xa, xb):
    """Per-observation z-scores of the mean displacement between end positions
    on the same streams (torus difference wrapped to [-1/2, 1/2)), both
    coordinates -> [n_obs, 2]."""
    d = np.asarray(xa, dtype=np.float64) - np.asarray(xb, dtype=np.float64)
    d -= np.round(d)
    M = d.shape[1]
    se = d.std(axis=1, ddof=1) / np.sqrt(M)
    return d.mean(axis=1) / np.where(se > 0, se, np.inf)
