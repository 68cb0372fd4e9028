"""Pins of the oracle's Algorithm 2 (Dirichlet problem in a disk)."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _bruteforce as bf

BGK = 0.5826  # -zeta(1/2)/sqrt(2 pi): Broadie-Glasserman-Kou discrete-monitoring shift


def test_exit_time_in_disk(orc):
    # v = 0, g = 0, f = -1: theta(x) = E[tau] = (R^2 - |x|^2) / (4 kappa) (Theorem 3.2).
    # Discrete monitoring exits late; the BGK shift R + 0.5826 sigma sqrt(dt) corrects it.
    kappa, dt, R = 0.25, 1e-3, 1.0
    gd = inputs.DirichletData(R=R, quad=0.0, f_const=-1.0, a=np.zeros(0), b=np.zeros(0))
    x = np.array([[0.0, 0.0], [0.5, 0.2], [-0.1, -0.7]])
    g, st = orc.dirichlet_paths(0, np.zeros(0), 1.0, kappa, gd, x, dt, 10**6, 31, npaths=20_000)
    assert np.all(st > 0)
    assert np.allclose(g, st * dt, rtol=1e-12)
    mean, var, se = orc.estimate(g)
    reff = R + BGK * np.sqrt(2 * kappa * dt)
    exact = (reff ** 2 - (x ** 2).sum(1)) / (4 * kappa)
    naive = (R ** 2 - (x ** 2).sum(1)) / (4 * kappa)
    assert np.all(np.abs(mean - exact) < 4.5 * se + 2e-3 * exact), (mean, exact, se)
    # and the continuity correction matters at this dt (the naive value is rejected)
    assert np.any(np.abs(mean - naive) > 4.5 * se)


def test_harmonic_boundary_data_is_reproduced(orc):
    # v = 0, f = 0, g = y1^2 - y2^2 (harmonic): theta(x) = x1^2 - x2^2.
    kappa, dt = 0.25, 2e-4
    gd = inputs.DirichletData(R=1.0, quad=1.0, f_const=0.0, a=np.zeros(0), b=np.zeros(0))
    x = np.array([[0.5, 0.1], [-0.2, 0.6], [0.3, -0.3]])
    g, st = orc.dirichlet_paths(0, np.zeros(0), 1.0, kappa, gd, x, dt, 10**6, 37, npaths=20_000)
    mean, var, se = orc.estimate(g)
    exact = x[:, 0] ** 2 - x[:, 1] ** 2
    assert np.all(np.abs(mean - exact) < 4.5 * se + 0.5 * np.sqrt(2 * kappa * dt)), (mean, exact, se)


def test_angular_boundary_data(orc):
    # g = cos(phi) + 0.5 sin(2 phi) on the unit circle is the trace of the harmonic
    # function x1 + x1 x2, which the estimator must reproduce at interior points.
    kappa, dt = 0.25, 2e-4
    gd = inputs.DirichletData(R=1.0, quad=0.0, f_const=0.0, a=np.array([1.0, 0.0]), b=np.array([0.0, 0.5]))
    x = np.array([[0.4, 0.3], [-0.5, -0.1]])
    g, st = orc.dirichlet_paths(0, np.zeros(0), 1.0, kappa, gd, x, dt, 10**6, 41, npaths=20_000)
    mean, var, se = orc.estimate(g)
    exact = x[:, 0] + x[:, 0] * x[:, 1]
    assert np.all(np.abs(mean - exact) < 4.5 * se + 0.5 * np.sqrt(2 * kappa * dt)), (mean, exact, se)


def test_start_outside_domain_exits_at_step_zero(orc):
    gd = inputs.DirichletData(R=1.0, quad=1.0, f_const=2.0, a=np.zeros(0), b=np.zeros(0))
    x = np.array([[1.2, 0.0], [0.0, -1.0]])
    g, st = orc.dirichlet_paths(2, inputs.prior_field(2, 3), 1.0, 0.1, gd, x, 1e-3, 100, 5, npaths=2)
    assert np.all(st == 0)
    assert np.allclose(g[0], 1.0) and np.allclose(g[1], -1.0)


def test_step_cap_marks_unexited_paths(orc):
    gd = inputs.DirichletData(R=1.0, quad=1.0, f_const=1.0, a=np.zeros(0), b=np.zeros(0))
    x = np.array([[0.0, 0.0]])
    g, st = orc.dirichlet_paths(0, np.zeros(0), 1.0, 0.01, gd, x, 1e-4, 50, 5, npaths=8)
    assert np.all(st == -1) and np.all(g == 0.0)


@pytest.mark.parametrize("drift", [0.0, 0.5])
def test_brute_force_tiny(orc, drift):
    K = 2
    u = inputs.prior_field(K, 44)
    gd = inputs.DirichletData(R=0.3, quad=1.0, f_const=0.5, a=np.array([0.1]), b=np.array([0.2]))
    x = np.array([[0.1, 0.05], [-0.2, 0.1]])
    seed = 991
    dt = 2e-3
    g, st, xe = orc.dirichlet_paths(K, u, drift, 0.5, gd, x, dt, 400, seed, i0=1, npaths=3, want_x=True)
    for j in range(2):
        for p in range(3):
            X, n = bf.dirichlet_path(K, u, drift, 0.5, 0.3, x[j], dt, 400, seed, j, 1 + p)
            assert n == st[j, p]
            assert np.allclose(xe[j, p], X, rtol=0, atol=1e-14)
            if n > 0:
                r = np.hypot(*X)
                y = 0.3 * np.asarray(X) / r
                phi = np.arctan2(y[1], y[0])
                want = y[0] ** 2 - y[1] ** 2 + 0.1 * np.cos(phi) + 0.2 * np.sin(phi) - 0.5 * n * dt
                assert abs(g[j, p] - want) < 1e-13
