"""Shared paths (PM_SHARE_PATHS, tensor-core and FP32/FP64-pipe kernels): observations at one
point x share their paths, each member stopping at its own time.  Checked
against single-observation calls on the same RNG stream (bit for bit: the same
arithmetic), against the FP64 oracle with the same stream map on fields where
float paths stay close to FP64 paths, and for the step count."""
import copy

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch
TC = pm.PM_FP32 | pm.PM_TENSOR


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def mixed_workload(M=300, dt=0.01):
    w = inputs.timedep_k10(M=M)
    rng = np.random.default_rng(11)
    p = rng.random((3, 2))
    # points p0, p1, p2; times include a partial last step (0.1234), a zero time
    # and two equal times at one point
    layout = [(0, 0.25), (1, 0.3), (0, 0.5), (0, 0.1234), (2, 0.0), (1, 0.7), (0, 0.5), (2, 0.05)]
    w.x = np.array([p[k] for k, _ in layout])
    w.t = np.array([tt for _, tt in layout])
    w.dt = dt
    return w


def test_members_equal_single_observation_calls_bitwise(c):
    w = mixed_workload()
    mean, var, g, xe = _gpu.timedep(c, w, TC | pm.PM_SHARE_PATHS, g_out=True, x_out=True)
    _, stream_of, _, _ = pm.pm_path_groups(w.x, w.t, w.dt)
    for j in range(len(w.t)):
        s = int(stream_of[j])
        # observation j alone at index s (so its RNG stream is s); dummies before it
        v = copy.copy(w)
        v.x = np.repeat(w.x[j:j + 1], s + 1, axis=0)
        v.t = np.full(s + 1, 0.02)
        v.t[s] = w.t[j]
        m1, v1, g1, x1 = _gpu.timedep(c, v, TC, g_out=True, x_out=True)
        assert np.array_equal(g1[s], g[j]), j
        assert np.array_equal(x1[s], xe[j]), j
        assert m1[s] == mean[j] and v1[s] == var[j], j


def test_step_count_and_grid(c):
    w = mixed_workload()
    _gpu.timedep(c, w, TC | pm.PM_SHARE_PATHS, device=False)
    _, _, ng, sp = pm.pm_path_groups(w.x, w.t, w.dt)
    assert pm.pm_last_step_count(c) == sp * w.M
    assert pm.pm_last_grid(c) == ng * ((w.M + 127) // 128)
    # headline layout: 1000 instead of 1750 steps per path triple
    h = inputs.timedep_k10(M=256)
    _gpu.timedep(c, h, TC | pm.PM_SHARE_PATHS, device=False)
    assert pm.pm_last_step_count(c) == 100 * 1000 * 256


@pytest.mark.parametrize("field", ["zero", "shear"])
def test_stable_fields_match_oracle_with_the_stream_map(c, orc, field):
    w = mixed_workload(M=512)
    if field == "zero":
        w.u = np.zeros_like(w.u)
    else:
        modes = orc.half_modes(10)
        h = [tuple(m) for m in modes].index((2, 3))
        w.u = np.zeros_like(w.u)
        w.u[2 * h], w.u[2 * h + 1] = 0.05, 0.02
    mean, var, g = _gpu.timedep(c, w, TC | pm.PM_SHARE_PATHS, g_out=True)
    _, stream_of, _, _ = pm.pm_path_groups(w.x, w.t, w.dt)
    go = orc.timedep_paths(10, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M,
                           obs_id=stream_of.astype(np.int64))
    # the estimate to 1e-5 (the parity bound); single float paths of |theta0| ~ 2
    # after up to 70 steps to 5e-5
    rm, rv, rse = orc.estimate(go)
    assert np.abs(mean - rm).max() <= 1e-5
    assert np.abs(g - go).max() <= 5e-5


def test_headline_means_agree_with_unshared_in_distribution(c):
    w = inputs.timedep_k10(M=4096)
    ms, vs = _gpu.timedep(c, w, TC | pm.PM_SHARE_PATHS)
    mu, vu = _gpu.timedep(c, w, TC)
    se = np.sqrt((vs + vu) / w.M)
    # the t = 0.25 observations (index j < 100: their group's stream in both
    # modes) are identical; the others are independent estimates of the same values
    assert np.array_equal(ms[:100], mu[:100])
    assert np.mean(np.abs(ms - mu) <= 5 * se) >= 0.99


@pytest.mark.parametrize("flags", [pm.PM_FP32, pm.PM_FP64])
def test_fp32_and_fp64_pipes_share_paths_too(c, flags):
    # The FP32/FP64-pipe kernels: members equal single-observation calls on the
    # group's stream, bit for bit.
    w = mixed_workload(M=200)
    w.u = inputs.prior_field(4, 77)
    w.K = 4
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


def test_fp64_shared_paths_match_the_oracle_path_by_path(c, orc):
    # Double paths on the 2-mode field: the oracle on the stream map, per path.
    w = mixed_workload(M=128)
    w.K = 2
    w.u = inputs.prior_field(2, 1000)
    mean, var, g = _gpu.timedep(c, w, pm.PM_FP64 | pm.PM_SHARE_PATHS, g_out=True)
    _, stream_of, _, _ = pm.pm_path_groups(w.x, w.t, w.dt)
    go = orc.timedep_paths(2, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M,
                           obs_id=stream_of.astype(np.int64))
    assert np.median(np.abs(g - go)) <= 1e-12 and np.abs(g - go).max() <= 1e-8
