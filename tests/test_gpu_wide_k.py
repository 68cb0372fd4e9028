"""The time-dependent map at the wide wave-number bounds K = 24 ... 64
(N_u = 2400 ... 16640 real coefficients; Section 4's larger Fourier bases):
the FP32-pipe kernel with its velocity table in shared memory and the
tensor-core kernel with 256 accumulator columns, each against the FP64 oracle,
against each other, and with shared paths against single-observation calls;
and at K = 80 (N_u = 25920) on the FP32 pipes alone."""
import copy

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch
TC = pm.PM_FP32 | pm.PM_TENSOR
WIDE = [24, 32, 40, 48, 56, 64]


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def wide_workload(K, M, n_pts=64, seed=0):
    w = inputs.timedep_k10(M=M)
    w.K = K
    w.u = inputs.prior_field(K, 500 + K)
    rng = np.random.default_rng(seed + K)
    w.x = rng.random((n_pts, 2))
    return w


@pytest.mark.parametrize("K", WIDE)
@pytest.mark.parametrize("tensor", [False, True])
def test_one_step_positions_match_oracle(c, orc, K, tensor):
    # One Euler step: X1 - x = -v(x) dt + noise exposes the velocity each kernel evaluated.
    w = wide_workload(K, 128)
    w.dt = 0.01
    w.t = np.full(len(w.x), w.dt)
    _, _, xe = _gpu.timedep(c, w, TC if tensor else pm.PM_FP32, x_out=True)
    _, xo = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=128, want_x=True)
    modes = orc.half_modes(K).astype(float)
    scale = float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(w.u.reshape(-1, 2)).sum(1)).sum())
    d = xe - xo
    d -= np.round(d)
    assert np.abs(d).max() <= w.dt * 4e-6 * scale + 1e-7, np.abs(d).max()


@pytest.mark.parametrize("K", WIDE)
def test_shear_at_the_highest_modes_matches_oracle(c, orc, K):
    # A single mode near the corner of the wave-number box, 50 steps: both float
    # kernels against the FP64 oracle on the same stream.
    w = wide_workload(K, 1000, n_pts=3)
    modes = [tuple(m) for m in orc.half_modes(K)]
    h = modes.index((K - 1, -(K - 3)))
    w.u = np.zeros_like(w.u)
    w.u[2 * h], w.u[2 * h + 1] = 2e-4, -1e-4
    w.t = np.full(3, 0.05)
    g = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M, obs_id=np.arange(3))
    rm, _, _ = orc.estimate(g)
    for flags in (pm.PM_FP32, TC):
        mean, _ = _gpu.timedep(c, w, flags)
        assert np.abs(mean - rm).max() <= 1e-5, (flags, np.abs(mean - rm).max())


@pytest.mark.parametrize("K", WIDE)
def test_tensor_and_pipes_agree_on_a_prior_field(c, K):
    # A prior draw, 8 points x 2000 paths (a ragged last tile).  Over a few steps the
    # two float kernels' paths stay together; over 100 steps the flow's stretching
    # (the velocity gradient of a prior draw grows like the square root of the
    # number of modes) separates paths that differ by rounding, so the estimates
    # agree in distribution only.
    w = wide_workload(K, 2000, n_pts=8)
    w.t = np.full(8, 0.003)
    _, _, g_tc = _gpu.timedep(c, w, TC, g_out=True)
    _, _, g_sm = _gpu.timedep(c, w, pm.PM_FP32, g_out=True)
    assert np.median(np.abs(g_tc - g_sm)) <= 1e-4, np.median(np.abs(g_tc - g_sm))
    w.t = np.full(8, 0.1)
    m_tc, v_tc, g_tc = _gpu.timedep(c, w, TC, g_out=True)
    m_sm, v_sm, g_sm = _gpu.timedep(c, w, pm.PM_FP32, g_out=True)
    assert np.all(np.isfinite(g_tc)) and np.all(np.isfinite(g_sm))
    se = np.sqrt((v_tc + v_sm) / w.M)
    assert np.all(np.abs(m_tc - m_sm) <= 5 * se + 1e-6), (m_tc - m_sm) / se


@pytest.mark.parametrize("tensor", [False, True])
def test_shared_paths_equal_single_observation_calls_bitwise(c, tensor):
    K = 32
    flags = TC if tensor else pm.PM_FP32
    w = wide_workload(K, 200, n_pts=2)
    w.dt = 0.01
    layout = [(0, 0.05), (1, 0.03), (0, 0.1234), (1, 0.0), (0, 0.05)]
    w.x = np.array([w.x[k] for k, _ in layout])
    w.t = np.array([tt for _, tt in layout])
    mean, var, g = _gpu.timedep(c, w, flags | pm.PM_SHARE_PATHS, g_out=True)
    _, stream_of, _, _ = pm.pm_path_groups(w.x, w.t, w.dt)
    for j in range(len(w.t)):
        s = int(stream_of[j])
        v = copy.copy(w)
        v.x = np.repeat(w.x[j:j + 1], s + 1, axis=0)
        v.t = np.full(s + 1, 0.02)
        v.t[s] = w.t[j]
        m1, v1, g1 = _gpu.timedep(c, v, flags, g_out=True)
        assert np.array_equal(g1[s], g[j]), j
        assert m1[s] == mean[j] and v1[s] == var[j], j


def test_host_pointers_and_repeatability(c):
    w = wide_workload(24, 300, n_pts=5)
    w.t = np.full(5, 0.02)
    a = _gpu.timedep(c, w, TC)
    b = _gpu.timedep(c, w, TC, device=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_wide_bounds_are_float_only(c):
    # FP64 paths stop at K = 16; the batched map and the general disk map
    # (forcing and diffusion) take the wide bounds on the tensor cores only.
    w = wide_workload(24, 128, n_pts=2)
    w.t = np.full(2, 0.01)
    with pytest.raises(pm.PMError):
        _gpu.timedep(c, w, pm.PM_FP64)
    d = inputs.dirichlet_disk_k10(M=16)
    d.K = 24
    d.u = inputs.prior_field(24, 7)
    with pytest.raises(pm.PMError):
        _gpu.dirichlet(c, d, pm.PM_FP64, obs=np.array([0]))
    ws = [w, d]
    d.x = d.x[:2]
    with pytest.raises(pm.PMError):
        _gpu.batched(c, ws, flags=pm.PM_FP32)
    gw, df = inputs.dirichlet_general_disk(M=16)
    gw.K, gw.u = 24, inputs.prior_field(24, 7)
    x = np.ascontiguousarray(gw.x[:1])
    with pytest.raises(pm.PMError):
        pm.pm_forward_dirichlet_general(c, pm.Field(gw.K, gw.u), gw.drift_scale,
                                        pm.DirichletData(gw.g.R, gw.g.quad, gw.g.f_const, gw.g.a, gw.g.b),
                                        pm.DiffusionForcing(df.s0, df.s1, df.milstein, df.c, df.F, df.w),
                                        x, 1, 16, gw.dt, 100, gw.seed, pm.PM_FP32, np.empty(1))


# The widest bound, K = 80 (N_u = 25,920: the |k|_2 <= 80 basis of the paper's
# third example fits in it): the time-dependent map with float paths on the
# FP32 pipes only.
def test_k80_one_step_positions_match_oracle(c, orc):
    K = 80
    w = wide_workload(K, 128, n_pts=16)
    w.dt = 0.01
    w.t = np.full(len(w.x), w.dt)
    _, _, xe = _gpu.timedep(c, w, pm.PM_FP32, x_out=True)
    _, xo = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=128, want_x=True)
    modes = orc.half_modes(K).astype(float)
    scale = float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(w.u.reshape(-1, 2)).sum(1)).sum())
    d = xe - xo
    d -= np.round(d)
    assert np.abs(d).max() <= w.dt * 4e-6 * scale + 1e-7, np.abs(d).max()


def test_k80_shear_at_the_highest_modes_matches_oracle(c, orc):
    K = 80
    w = wide_workload(K, 256, n_pts=3)
    modes = [tuple(m) for m in orc.half_modes(K)]
    h = modes.index((K - 1, -(K - 3)))
    w.u = np.zeros_like(w.u)
    w.u[2 * h], w.u[2 * h + 1] = 2e-4, -1e-4
    w.t = np.full(3, 0.05)
    g = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M, obs_id=np.arange(3))
    rm, _, _ = orc.estimate(g)
    mean, _ = _gpu.timedep(c, w, pm.PM_FP32)
    assert np.abs(mean - rm).max() <= 1e-5, np.abs(mean - rm).max()


def test_k80_tensor_flag_runs_the_fp32_pipes_and_other_maps_refuse_it(c):
    K = 80
    w = wide_workload(K, 300, n_pts=4)
    w.t = np.full(4, 0.02)
    a = _gpu.timedep(c, w, pm.PM_FP32, g_out=True)
    b = _gpu.timedep(c, w, TC, g_out=True)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert pm.pm_last_grid(c) == 4 * 2  # 256 paths per CTA: two CTAs per observation
    with pytest.raises(pm.PMError):
        _gpu.timedep(c, w, pm.PM_FP64)
    d = inputs.dirichlet_disk_k10(M=16)
    d.K = K
    d.u = inputs.prior_field(K, 7)
    for flags in (pm.PM_FP32, TC):
        with pytest.raises(pm.PMError):
            _gpu.dirichlet(c, d, flags, obs=np.array([0]))
    d.x = d.x[:2]
    with pytest.raises(pm.PMError):
        _gpu.batched(c, [w, d], flags=TC)
