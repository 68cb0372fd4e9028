"""Evidence for reading the parity bound per observation rather than per path
(float and double paths separate on the 440-mode field), from the oracle alone: on
the 440-mode field a rounding-size change of a path's start grows to macroscopic
size within the observation horizon (chaotic advection), while on the fields used
for pathwise parity (zero drift, one stream mode) it does not."""
import numpy as np

from paper_1808_10580_gb300 import inputs


def separation(orc, K, u, kappa, t, dt, npaths=8, eps=1e-12):
    th = inputs.Fourier(np.array([[1, 0]], dtype=np.int32), np.array([1.0]), np.array([0.0]))
    x = np.array([[0.35, 0.55], [0.35 + eps, 0.55]])
    # same observation id for both rows: identical Brownian increments
    g, xe = orc.timedep_paths(K, u, kappa, th, x, np.full(2, t), dt, 4001, npaths=npaths, want_x=True,
                              obs_id=[7, 7])
    d = xe[1] - xe[0]
    d -= np.round(d)
    return np.abs(d).max(axis=1)


def test_440_mode_field_amplifies_rounding_beyond_1e5(orc):
    w = inputs.timedep_k10()
    s = separation(orc, 10, w.u, w.kappa, 1.0, w.dt)
    assert np.median(s) > 1e-12 * 1e6


def test_shear_and_zero_drift_do_not(orc):
    w = inputs.timedep_k10()
    modes = orc.half_modes(10)
    h = [tuple(m) for m in modes].index((2, 3))
    u = np.zeros_like(w.u)
    u[2 * h], u[2 * h + 1] = 0.05, 0.02
    assert separation(orc, 10, u, w.kappa, 1.0, w.dt).max() < 1e-12 * 1e3
    assert separation(orc, 0, np.zeros(0), w.kappa, 1.0, w.dt).max() < 1e-12 * 10
