"""Pins of the oracle's Algorithm 1 (time-dependent problem)."""
import math

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _bruteforce as bf


def heat_closed_form(th, x, kappa, t):
    """Kolmogorov backward equation with v = 0 (Theorem 3.1): each Fourier mode
    of theta0 decays as exp(-4 pi^2 kappa |k|^2 t)."""
    k = th.k.astype(float)
    ph = 2 * np.pi * (x @ k.T)
    dec = np.exp(-4 * np.pi ** 2 * kappa * (k ** 2).sum(1) * t)
    return (np.cos(ph) * th.a * dec + np.sin(ph) * th.b * dec).sum(1)


def test_num_steps_reading(orc):
    assert orc.num_steps(1.0, 0.01) == 100
    assert orc.num_steps(0.25, 1e-3) == 250
    assert orc.num_steps(0.0, 0.1) == 0
    assert orc.num_steps(0.105, 0.01) == 11


def test_zero_horizon_returns_theta0(orc):
    th = inputs.Fourier(np.array([[1, 2], [0, 1]], dtype=np.int32), np.array([0.3, -1.0]), np.array([0.5, 0.2]))
    x = np.array([[0.1, 0.7], [0.9, 0.3]])
    g = orc.timedep_paths(2, inputs.prior_field(2, 1), 0.1, th, x, np.zeros(2), 0.01, 5, npaths=3)
    assert np.allclose(g, orc.theta0(th, x)[:, None], atol=0, rtol=0)


def test_heat_kernel_closed_form(orc):
    # v = 0 (K = 0): Euler-Maruyama is exact in law, so only Monte Carlo error remains.
    th = inputs.Fourier(np.array([[1, 0], [1, 1], [0, 2]], dtype=np.int32),
                        np.array([0.8, -0.5, 0.3]), np.array([0.2, 0.4, -0.6]))
    x = np.array([[0.1, 0.2], [0.5, 0.5], [0.73, 0.11]])
    kappa, t = 0.02, 0.5
    g = orc.timedep_paths(0, np.zeros(0), kappa, th, x, np.full(3, t), 0.05, 11, npaths=100_000)
    mean, var, se = orc.estimate(g)
    exact = heat_closed_form(th, x, kappa, t)
    assert np.all(np.abs(mean - exact) < 4.5 * se), (mean, exact, se)
    # the decay is visible: the exact values differ clearly from theta0(x)
    assert np.abs(exact - orc.theta0(th, x)).max() > 20 * se.max()


def test_drift_along_wave_fronts_is_invisible(orc):
    # One stream mode k and theta0 a function of k.x only: v is perpendicular to k,
    # so k.X is a Brownian motion and the heat closed form holds despite the drift.
    K = 2
    modes = orc.half_modes(K)
    h = [tuple(m) for m in modes].index((1, 2))
    u = np.zeros(2 * len(modes))
    u[2 * h], u[2 * h + 1] = 0.3, 0.2        # |v| ~ 2 pi |k| |u| ~ 5
    th = inputs.Fourier(np.array([[1, 2]], dtype=np.int32), np.array([1.0]), np.array([0.0]))
    x = np.array([[0.3, 0.4], [0.05, 0.9]])
    kappa, t = 0.01, 0.5
    g = orc.timedep_paths(K, u, kappa, th, x, np.full(2, t), 0.01, 13, npaths=40_000)
    mean, var, se = orc.estimate(g)
    exact = heat_closed_form(th, x, kappa, t)
    assert np.all(np.abs(mean - exact) < 4.5 * se), (mean, exact, se)


def test_single_mode_pure_advection_is_exact(orc):
    # kappa = 0, one mode: v is constant along its own streamline, so every Euler step
    # moves by the same -v(x) dt and X_t = x - t v(x) (mod 1) for any dt.
    K = 3
    modes = orc.half_modes(K)
    h = [tuple(m) for m in modes].index((2, -1))
    u = np.zeros(2 * len(modes))
    u[2 * h], u[2 * h + 1] = 0.05, -0.03
    x = np.array([[0.12, 0.34], [0.6, 0.8]])
    t = 0.7
    th = inputs.Fourier(np.array([[1, 0]], dtype=np.int32), np.array([1.0]), np.array([0.0]))
    g, xe = orc.timedep_paths(K, u, 0.0, th, x, np.full(2, t), 0.013, 3, npaths=2, want_x=True)
    want = x - t * orc.velocity(K, u, x)
    want -= np.floor(want)
    for p in range(2):
        d = xe[:, p, :] - want
        d -= np.round(d)
        assert np.abs(d).max() < 1e-12


@pytest.mark.parametrize("K,kappa,dt,t", [(1, 0.05, 0.1, 0.35), (2, 0.01, 0.02, 0.1)])
def test_brute_force_tiny(orc, K, kappa, dt, t):
    u = inputs.prior_field(K, 21 + K)
    th = inputs.Fourier(np.array([[1, 1], [2, -1]], dtype=np.int32), np.array([0.4, 0.1]), np.array([-0.2, 0.3]))
    x = np.array([[0.2, 0.9], [0.55, 0.45]])
    seed = (3 << 32) + 17
    g, xe = orc.timedep_paths(K, u, kappa, th, x, np.full(2, t), dt, seed, i0=2, npaths=4, want_x=True)
    for j in range(2):
        for p in range(4):
            X = bf.timedep_path(K, u, kappa, x[j], t, dt, seed, j, 2 + p)
            assert np.allclose(xe[j, p], X, rtol=0, atol=1e-14)
    assert np.allclose(g, orc.theta0(th, xe.reshape(-1, 2)).reshape(2, 4), atol=0)


def test_observation_ids_select_rng_stream(orc):
    w = inputs.plain_fp64_k2()
    full = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=3)
    sub = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x[[4, 7]], w.t[[4, 7]], w.dt, w.seed,
                            npaths=3, obs_id=[4, 7])
    assert np.array_equal(sub, full[[4, 7]])
    part = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, i0=1, npaths=2)
    assert np.array_equal(part, full[:, 1:3])


def test_estimator_matches_exact_sums(orc):
    rng = np.random.default_rng(4)
    g = rng.normal(0.3, 1.0, size=(3, 1001))
    mean, var, se = orc.estimate(g)
    for j in range(3):
        n = g.shape[1]
        m = math.fsum(g[j]) / n
        v = math.fsum((gi - m) ** 2 for gi in g[j]) / (n - 1)
        assert abs(mean[j] - m) < 1e-15 and abs(var[j] - v) < 1e-14
        assert abs(se[j] - math.sqrt(v / n)) < 1e-15
