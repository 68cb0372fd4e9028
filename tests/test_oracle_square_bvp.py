"""Pins of the oracle for the optimal-forcing boundary-value problem in the
unit square (Section 4, Eq. bvp:ex1; Algorithm 2, Theorem 3.2): closed forms
that do not come from the oracle.

* kappa = 0: the paths are the straight lines x - b t, so the exit point, the
  boundary value there and the time integral of each Gaussian source profile
  along the line (an error-function integral) are known exactly, up to the
  left-point rule's O(dt).
* zero drift, a constant source (w = 0, profile 1): the integral is the exit
  time, whose mean solves kappa Laplace u = -1 in the square (the torsion
  problem, a double sine series).  Discrete monitoring of the exit lets paths
  leave and return between steps; the continuity correction of Broadie,
  Glasserman & Kou (1997) accounts for it by moving the boundary out by
  0.5826 sigma sqrt(dt), sigma = sqrt(2 kappa)."""
import math

import numpy as np
import pytest

import oracle
from paper_1808_10580_gb300 import inputs


def line_integral(p0, b, c, w, T):
    """int_0^T exp(-w |p0 - b t - c|^2) dt."""
    p = np.asarray(p0, float) - np.asarray(c, float)
    b = np.asarray(b, float)
    bb = b @ b
    t0 = (p @ b) / bb
    d2 = p @ p - (p @ b) ** 2 / bb
    a = math.sqrt(w * bb)
    return math.exp(-w * d2) * math.sqrt(math.pi) / (2 * a) * (math.erf(a * (T - t0)) - math.erf(-a * t0))


def torsion(x, y, kappa, L=1.0, shift=0.0, terms=199):
    """Mean exit time of sqrt(2 kappa) W from the square [-shift, L - shift]^2."""
    xs, ys = x + shift, y + shift
    s = 0.0
    for m in range(1, terms + 1, 2):
        sm = math.sin(m * math.pi * xs / L) / m
        for n in range(1, terms + 1, 2):
            s += sm * math.sin(n * math.pi * ys / L) / (n * (m * m + n * n))
    return 16 * L * L / (kappa * math.pi ** 4) * s


def test_zero_diffusion_exit_point_boundary_value_and_source_integrals():
    prob = inputs.SquareBVP(b=np.array([1.0, 0.5]), kappa=0.0,
                            c=np.array([[0.2, 0.3], [0.7, 0.6]]), w=4.0)
    x = np.array([[0.35, 0.8], [0.9, 0.2]])
    dt = 1e-4
    out, st = oracle.square_bvp_paths(prob, x, dt, 10 ** 6, seed=7, npaths=3)
    for j in range(2):
        T = min(x[j, 0] / prob.b[0], x[j, 1] / prob.b[1])        # first coordinate to reach 0
        y = np.clip(x[j] - prob.b * T, 0.0, 1.0)
        g = 0.5 * (math.cos(math.pi * y[0] / 2) + math.cos(math.pi * y[1] / 2))
        assert np.all(np.abs(st[j] - T / dt) <= 1.5)    # the step that crosses 0
        assert np.all(np.abs(out[j, 0] - g) <= 2e-4)
        for q in range(2):
            exact = line_integral(x[j], prob.b, prob.c[q], prob.w, T)
            assert np.all(np.abs(out[j, q + 1] - exact) <= 5e-4 * max(exact, 1e-3) + 2 * dt)


@pytest.mark.parametrize("point", [(0.5, 0.5), (0.2, 0.7)])
def test_mean_exit_time_is_the_torsion_function(point):
    kappa, dt = 0.282, 1e-4
    prob = inputs.SquareBVP(b=np.zeros(2), kappa=kappa, c=np.array([[0.5, 0.5]]), w=0.0, g_cos=0.0)
    out, st = oracle.square_bvp_paths(prob, np.array([point]), dt, 10 ** 7, seed=11, npaths=20000)
    tau = out[0, 1]
    assert np.allclose(tau, st[0] * dt)                      # the constant profile integrates to the exit time
    se = tau.std(ddof=1) / math.sqrt(tau.size)
    delta = 0.5826 * math.sqrt(2 * kappa * dt)
    exact = torsion(point[0], point[1], kappa, L=1 + 2 * delta, shift=delta)
    assert abs(tau.mean() - exact) <= 3 * se + 2e-3 * exact, (tau.mean(), exact, se)
    # without the correction the continuous-time value is measurably below
    assert torsion(point[0], point[1], kappa) < exact
