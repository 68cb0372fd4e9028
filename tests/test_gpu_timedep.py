"""GPU parity of Algorithm 1 (time-dependent map) against the FP64 oracle."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def rounding_sensitivity(orc, w, M):
    """How far the oracle's own estimate moves when every field coefficient is
    perturbed by 4 ulps: the scale on which two correct double-precision
    implementations (different but equally exact summation orders) can differ
    once the flow has amplified their roundings."""
    (m0, _, _), _ = orc.timedep_estimate(w, npaths=M)
    u = w.u
    w.u = u * (1.0 + 2.0 ** -50)
    (m1, _, _), _ = orc.timedep_estimate(w, npaths=M)
    w.u = u
    return np.abs(m1 - m0).max()


def test_plain_fp64_workload_matches_oracle(c, orc):
    # K=2, 3x3 grid, t=1, M=1000, dt=0.01: the whole estimate, same stream, FP64 paths.
    w = inputs.plain_fp64_k2()
    mean, var, g, xe = _gpu.timedep(c, w, pm.PM_FP64, g_out=True, x_out=True)
    (rm, rv, rse), rg = orc.timedep_estimate(w)
    sens = rounding_sensitivity(orc, w, w.M)
    d = np.abs(g - rg).reshape(-1)
    print(f"C0 fp64: max|dmean| {np.abs(mean - rm).max():.3e} sens {sens:.3e} "
          f"path |dg| quantiles 50/90/99/max {np.quantile(d, [0.5, 0.9, 0.99]).tolist()} {d.max():.3e}")
    assert np.abs(mean - rm).max() <= max(1e-12, 100 * sens)
    assert np.abs(mean - rm).max() <= 1e-5
    assert np.allclose(var, rv, rtol=1e-4, atol=1e-12)
    assert np.median(d) <= 1e-10          # most paths agree to near rounding level


@pytest.mark.parametrize("fp64", [False, True])
def test_zero_drift_matches_oracle_pathwise(c, orc, fp64):
    # v = 0: no amplification of rounding, so paths agree to rounding level.
    w = inputs.plain_fp64_k2()
    w.u = np.zeros_like(w.u)
    mean, var, g, xe = _gpu.timedep(c, w, pm.PM_FP64 if fp64 else pm.PM_FP32, g_out=True, x_out=True)
    rg, rx = orc.timedep_paths(0, np.zeros(0), w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M, want_x=True)
    dx = xe - rx
    dx -= np.round(dx)
    # float: the normals themselves carry ~2e-7 relative error (logf, sqrtf, sincospif),
    # 100 increments of size 0.03 random-walk to ~1e-7; the sum itself is compensated.
    assert np.abs(dx).max() <= (1e-13 if fp64 else 5e-7)
    assert np.abs(g - rg).max() <= (1e-13 if fp64 else 5e-6)
    rm, rv, rse = orc.estimate(rg)
    assert np.abs(mean - rm).max() <= (1e-14 if fp64 else 5e-7)


@pytest.mark.parametrize("device", [True, False])
def test_fp64_host_and_device_pointers_agree(c, device):
    w = inputs.plain_fp64_k2()
    a = _gpu.timedep(c, w, pm.PM_FP64, M=300, device=device)
    b = _gpu.timedep(c, w, pm.PM_FP64, M=300, device=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_zero_drift_fp32_matches_oracle_at_full_size(c, orc):
    # K=10 kernel with u = 0 (v = 0) at the 300-observation, M=1e4 shape: no chaos,
    # so the float paths track the FP64 paths and the estimate agrees to 1e-5.
    w = inputs.timedep_k10()
    w.u = np.zeros_like(w.u)
    mean, var = _gpu.timedep(c, w, pm.PM_FP32)
    obs = np.array([0, 37, 99, 100, 151, 199, 200, 263, 299])
    g = orc.timedep_paths(0, np.zeros(0), w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, w.seed, npaths=w.M,
                          obs_id=obs)
    rm, rv, rse = orc.estimate(g)
    assert np.abs(mean[obs] - rm).max() <= 1e-5


@pytest.mark.parametrize("fp64", [False, True])
def test_single_mode_shear_matches_oracle(c, orc, fp64):
    # One stream mode (a laminar shear flow): paths separate at most linearly in
    # time, so float paths stay within 1e-5 of the FP64 estimate.
    w = inputs.timedep_k10(M=4000)
    modes = orc.half_modes(10)
    h = [tuple(m) for m in modes].index((2, 3))
    u = np.zeros_like(w.u)
    u[2 * h], u[2 * h + 1] = 0.05, 0.02
    w.u = u
    obs = np.array([5, 120, 250])
    mean, var, gg = _gpu.timedep(c, w, pm.PM_FP64 if fp64 else pm.PM_FP32, obs=obs, g_out=True)
    g = orc.timedep_paths(10, u, w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, w.seed, npaths=w.M, obs_id=np.arange(3))
    rm, rv, rse = orc.estimate(g)
    print(f"shear fp64={fp64}: max|dmean| {np.abs(mean - rm).max():.3e} max|dg| {np.abs(gg - g).max():.3e}")
    assert np.abs(mean - rm).max() <= (1e-11 if fp64 else 1e-5)


def test_repeated_calls_are_bit_identical(c):
    w = inputs.timedep_k10(M=1000)
    a = _gpu.timedep(c, w, pm.PM_FP32, obs=np.arange(0, 300, 7))
    b = _gpu.timedep(c, w, pm.PM_FP32, obs=np.arange(0, 300, 7))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_zero_horizon_and_tiny_M(c, orc):
    w = inputs.plain_fp64_k2()
    w.t = np.zeros_like(w.t)
    mean, var = _gpu.timedep(c, w, pm.PM_FP64, M=1)
    assert np.allclose(mean, orc.theta0(w.theta0, w.x), rtol=0, atol=1e-15)
    assert np.all(var == 0)


def test_invalid_arguments_raise(c):
    w = inputs.plain_fp64_k2()
    with pytest.raises(pm.PMError):
        w2 = inputs.plain_fp64_k2(); w2.dt = 0.0
        _gpu.timedep(c, w2)
    with pytest.raises(pm.PMError):
        w2 = inputs.plain_fp64_k2(); w2.K = 7; w2.u = np.zeros(224)
        _gpu.timedep(c, w2)
    with pytest.raises(pm.PMError):
        w2 = inputs.plain_fp64_k2(); w2.u = w2.u.copy(); w2.u[3] = np.nan
        _gpu.timedep(c, w2)
    with pytest.raises(pm.PMError):
        w2 = inputs.plain_fp64_k2(); w2.t = w2.t.copy(); w2.t[2] = -1.0
        _gpu.timedep(c, w2)
