"""Pins of the oracle's mode enumerator and velocity (Eq. v_expand)."""
import os

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "mode_counts.txt")


def _counts():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        kind, r, n = line.split()
        yield kind, int(r), int(n)


@pytest.mark.parametrize("kind,r,n", list(_counts()))
def test_mode_counts_match_paper(orc, kind, r, n):
    if kind == "euclid":
        assert orc.count_disk_modes(r) == n
    else:
        assert len(orc.half_modes(r)) == n
        assert len(inputs.half_mode_list(r)) == n


def test_half_modes_cover_lattice_once(orc):
    K = 4
    hm = [tuple(v) for v in orc.half_modes(K)]
    assert hm == [tuple(v) for v in inputs.half_mode_list(K)]
    full = set(hm) | {(-m, -n) for m, n in hm}
    assert len(full) == 2 * len(hm)
    assert full == {(m, n) for m in range(-K, K + 1) for n in range(-K, K + 1)} - {(0, 0)}


def test_single_coefficient_is_single_mode(orc):
    K = 3
    modes = orc.half_modes(K)
    rng = np.random.default_rng(0)
    x = rng.random((20, 2))
    for h in (0, 5, len(modes) - 1):
        for part in (0, 1):
            u = np.zeros(2 * len(modes))
            u[2 * h + part] = 1.0
            th = 2 * np.pi * (x @ modes[h].astype(float))
            want = np.cos(th) if part == 0 else np.sin(th)
            assert np.allclose(orc.stream_function(K, u, x), want, atol=1e-13)


def test_velocity_is_perp_gradient_of_stream_function(orc):
    # v = (-d psi/dx2, d psi/dx1) by 4th-order central differences of psi.
    K = 3
    u = inputs.prior_field(K, 5)
    rng = np.random.default_rng(1)
    x = rng.random((50, 2))
    h = 1e-4
    e1, e2 = np.array([h, 0.0]), np.array([0.0, h])

    def d(e):
        f = lambda y: orc.stream_function(K, u, y)
        return (-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * h)

    v = orc.velocity(K, u, x)
    assert np.allclose(v[:, 0], -d(e2), atol=1e-7)
    assert np.allclose(v[:, 1], d(e1), atol=1e-7)


def test_velocity_is_divergence_free_and_periodic(orc):
    K = 4
    u = inputs.prior_field(K, 6)
    rng = np.random.default_rng(2)
    x = rng.random((40, 2))
    h = 1e-5
    d11 = (orc.velocity(K, u, x + [h, 0])[:, 0] - orc.velocity(K, u, x - [h, 0])[:, 0]) / (2 * h)
    d22 = (orc.velocity(K, u, x + [0, h])[:, 1] - orc.velocity(K, u, x - [0, h])[:, 1]) / (2 * h)
    # each term is O(10-100); their sum vanishes up to the O(h^2) difference error
    assert np.abs(d11 + d22).max() < 1e-7 * np.abs(d11).max()
    assert np.abs(d11).max() > 1.0
    assert np.allclose(orc.velocity(K, u, x + [1, -2]), orc.velocity(K, u, x), atol=1e-11)


def test_velocity_is_perpendicular_to_single_wave_vector(orc):
    K = 3
    modes = orc.half_modes(K)
    rng = np.random.default_rng(3)
    x = rng.random((30, 2))
    for h in (2, 9, 17):
        u = np.zeros(2 * len(modes))
        u[2 * h] = 0.7
        u[2 * h + 1] = -0.4
        v = orc.velocity(K, u, x)
        assert np.abs(v @ modes[h].astype(float)).max() < 1e-12
        assert np.abs(v).max() > 0.1


@pytest.mark.parametrize("K", [24, 40, 64])
def test_wide_bounds_enumerate_the_box_once(orc, K):
    # |H_K| = ((2K+1)^2 - 1) / 2 half-modes, and with their negatives every nonzero
    # lattice point of the box exactly once.
    hm = orc.half_modes(K)
    assert len(hm) == ((2 * K + 1) ** 2 - 1) // 2
    assert np.array_equal(hm, inputs.half_mode_list(K))
    full = {tuple(v) for v in hm} | {(-m, -n) for m, n in hm}
    assert len(full) == 2 * len(hm) == (2 * K + 1) ** 2 - 1


@pytest.mark.parametrize("K", [24, 64])
def test_single_high_mode_velocity_closed_form(orc, K):
    # psi = a cos(2 pi k.x) + b sin(2 pi k.x)  =>  v = (-d2 psi, d1 psi)
    #     = 2 pi (-k2, k1) (b cos(2 pi k.x) - a sin(2 pi k.x)), written out here
    # for modes at the corners and edges of the box.
    modes = orc.half_modes(K)
    rng = np.random.default_rng(K)
    x = rng.random((25, 2))
    picks = [(K, K), (K, -K), (0, K), (1, -K), (K - 1, 3)]
    index = {tuple(v): h for h, v in enumerate(modes)}
    for k in picks:
        h = index[k]
        a, b = 0.3, -0.8
        u = np.zeros(2 * len(modes))
        u[2 * h], u[2 * h + 1] = a, b
        th = 2 * np.pi * (x @ np.array(k, dtype=float))
        amp = 2 * np.pi * (b * np.cos(th) - a * np.sin(th))
        want = np.stack([-k[1] * amp, k[0] * amp], axis=1)
        assert np.allclose(orc.velocity(K, u, x), want, rtol=0, atol=1e-9 * K), k
