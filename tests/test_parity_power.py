"""What the statistical parity tests of the time-dependent map can and cannot
see, shown on the FP64 oracle alone (no GPU): the same checks that
tests/test_gpu_oracle_sample_parity.py applies to the CUDA path, applied to two
oracle runs that differ in a known way.

* Short horizon (t = 0.02, 20 Euler steps on the 440-mode field, 100 grid
  points, 1000 paths): a one-ulp change of the start points (the size of float
  rounding) passes the pathwise bound (median observation <= 1e-5, every one
  <= 2e-4); a 1 % change of the largest stream-function coefficient fails it by
  two orders of magnitude.
* The workload's own time t = 0.25 (20 observations, 1000 paths each side,
  independent streams): a second correct run passes the two-sample check, and
  a sign error in one coefficient (a plausible coding mistake: a flipped term)
  fails it.  A 1 % change of one coefficient moves the means by less than the
  Monte Carlo error of 1000 paths at t >= 0.25, which is why the short-horizon
  test carries that sensitivity."""
import dataclasses

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _stats as S

pytestmark = pytest.mark.slow

MO = 1000


def short_horizon_ok(d):
    d = np.abs(np.asarray(d))
    return bool(np.median(d) <= 1e-5 and d.max() <= 2e-4)


def test_short_horizon_bound_separates_rounding_from_a_one_percent_change(orc):
    w = inputs.timedep_k10()
    x = inputs.grid_points(10)
    t = np.full(len(x), 0.02)
    run = lambda u, xx: orc.timedep_paths(w.K, u, w.kappa, w.theta0, xx, t, w.dt, w.seed, npaths=MO).mean(axis=1)
    base = run(w.u, x)
    ulp = run(w.u, x * (1 + 2.0 ** -23))
    u1 = w.u.copy()
    u1[int(np.argmax(np.abs(u1)))] *= 1.01
    one_percent = run(u1, x)
    assert short_horizon_ok(ulp - base)
    assert not short_horizon_ok(one_percent - base)
    assert np.median(np.abs(one_percent - base)) > 100 * 1e-5


def test_two_sample_check_size_and_a_sign_error(orc):
    w = inputs.timedep_k10()
    obs = np.arange(0, 100, 5)  # t = 0.25
    est = lambda u, seed: orc.estimate(orc.timedep_paths(w.K, u, w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, seed,
                                                         npaths=MO, obs_id=obs))
    m0, _, se0 = est(w.u, w.seed)
    m1, _, se1 = est(w.u, w.seed + 7919)
    assert S.zcheck(S.two_sample_z(m1, se1, m0, se0))["ok"]
    flipped = w.u.copy()
    h = int(np.argmax(np.abs(flipped)))
    flipped[h] = -flipped[h]
    m2, _, se2 = est(flipped, w.seed + 7919)
    assert not S.zcheck(S.two_sample_z(m2, se2, m0, se0))["ok"]


def test_multiplicity_allowance_matches_the_binomial_tail():
    # n independent N(0,1) scores: the count beyond 3 is Binomial(n, 0.0027).
    assert S.allowed_exceedances(20) == 2
    assert S.allowed_exceedances(60) == 3
    rng = np.random.default_rng(5)
    fails = sum(not S.zcheck(rng.standard_normal(60))["ok"] for _ in range(2000))
    assert fails <= 3  # expected about 2000 * 2e-4 = 0.4
