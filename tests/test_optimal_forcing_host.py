"""Host logic of the optimal-forcing search (no GPU): the Nelder-Mead method
against known minima, and the affine structure of G(F)."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import optimal_forcing as of


def test_nelder_mead_finds_the_rosenbrock_minimum():
    f = lambda v: (1 - v[0]) ** 2 + 100 * (v[1] - v[0] ** 2) ** 2
    r = of.nelder_mead(f, [-1.2, 1.0], step=0.5, xtol=1e-10, ftol=1e-16)
    assert np.allclose(r.x, [1.0, 1.0], atol=1e-6) and r.fun < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_nelder_mead_on_the_forcing_cost_matches_the_linear_solve(seed):
    rng = np.random.default_rng(seed)
    E = np.column_stack([rng.random(3), 0.05 + 0.2 * rng.random((3, 3))])
    y = np.zeros(3)
    r = of.solve(E, y, xtol=1e-12, ftol=1e-16)
    exact = np.linalg.solve(E[:, 1:], E[:, 0] - y)        # G(F) = y exactly (3 sources, 3 points)
    assert np.allclose(r.x, exact, rtol=1e-6, atol=1e-8), (r.x, exact)
    assert of.cost(E, y, r.x) < 1e-8


def test_G_is_affine_in_the_source_strengths():
    E = np.array([[0.8, 0.1, 0.2], [0.7, 0.3, 0.1]])
    F1, F2 = np.array([1.0, -2.0]), np.array([0.5, 3.0])
    a = 0.3
    assert np.allclose(of.G(E, a * F1 + (1 - a) * F2), a * of.G(E, F1) + (1 - a) * of.G(E, F2))
    assert np.allclose(of.G(E, np.zeros(2)), E[:, 0])
