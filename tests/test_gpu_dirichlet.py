"""GPU parity of Algorithm 2 (Dirichlet map, persistent per-lane refill kernel)
against the FP64 oracle."""
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


def zero_drift_workload(M=4000):
    # v = 0 (K=10 kernel with zero coefficients), g = y1^2 - y2^2 + 0.1 sin 3 phi, f = -0.5
    gd = inputs.DirichletData(R=1.0, quad=1.0, f_const=-0.5, a=np.zeros(3), b=np.array([0.0, 0.0, 0.1]))
    return inputs.DirichletWorkload("zero_drift", 10, np.zeros(440), 0.5, 0.25, gd,
                                    inputs.disk_points(12, 0.9, 77), M, 1e-3, 10**6, 99)


@pytest.mark.parametrize("fp64", [False, True])
def test_zero_drift_exit_steps_and_means_match_oracle(c, orc, fp64):
    w = zero_drift_workload()
    r = _gpu.dirichlet(c, w, pm.PM_FP64 if fp64 else pm.PM_FP32, want_paths=True)
    g, st = orc.dirichlet_paths(0, np.zeros(0), 0.0, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=w.M)
    agree = np.mean(r["steps"] == st)
    assert agree >= 0.999, agree
    if fp64:
        assert agree == 1.0
    same = r["steps"] == st
    assert np.abs(r["g"][same] - g[same]).max() < (1e-12 if fp64 else 1e-5)
    rm, rv, rse = orc.estimate(g)
    assert np.all(np.abs(r["mean"] - rm) <= 3 * np.sqrt(2) * rse)
    assert r["unexited"] == 0 and r["rc"] == 0


def test_drift_field_paired_paths(c, orc):
    # The 440-mode field x 0.5 at dt = 1e-3: the flow is chaotic, so float and double paths
    # separate; the estimates must agree in distribution (paired differences within 5 SE).
    w = inputs.dirichlet_disk_k10(M=16)
    w.dt = 1e-3
    r = _gpu.dirichlet(c, w, pm.PM_FP32, want_paths=True)
    g, st = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=w.M)
    d = (r["g"] - g).reshape(-1)
    assert abs(d.mean()) <= 5 * d.std(ddof=1) / np.sqrt(d.size)
    # Early exits happen before the paths decorrelate: those exit steps agree.
    # At dt = 1e-3 float and FP64 paths through this flow stay together to
    # t = 0.2 (200 steps); from there on a few per cent separate each 0.1.
    for lo, hi in ((0, 100), (100, 200), (200, 300), (300, 600)):
        m = (st >= lo) & (st < hi)
        print(f"exit steps [{lo}, {hi}): {int(m.sum())} paths, {int((r['steps'][m] != st[m]).sum())} differ")
    early = st < 200
    assert early.sum() > 20
    assert np.mean(r["steps"][early] == st[early]) >= 0.999


def test_start_outside_and_step_cap(c):
    gd = inputs.DirichletData(R=1.0, quad=1.0, f_const=1.0, a=np.zeros(0), b=np.zeros(0))
    w = inputs.DirichletWorkload("edge", 2, inputs.prior_field(2, 3), 1.0, 0.01, gd,
                                 np.array([[1.5, 0.0], [0.0, 0.0]]), 64, 1e-4, 20, 5)
    r = _gpu.dirichlet(c, w, pm.PM_FP32, want_paths=True)
    assert r["rc"] == pm.PM_WARN_UNEXITED
    assert np.all(r["steps"][0] == 0) and np.allclose(r["g"][0], 1.0)
    assert np.all(r["steps"][1] == -1) and np.all(r["g"][1] == 0.0)
    assert r["unexited"] == 64


def test_repeated_calls_are_bit_identical(c):
    w = inputs.dirichlet_disk_k10(M=200)
    w.dt = 1e-3
    a = _gpu.dirichlet(c, w, pm.PM_FP32)
    b = _gpu.dirichlet(c, w, pm.PM_FP32)
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["var"], b["var"])


@pytest.mark.parametrize("M", [5000, 20000])
def test_reduction_equals_exact_sums_of_the_path_values(c, M):
    # The per-observation mean and variance (one pass, or two passes through
    # chunk partials when M > 8192) against exactly rounded sums (math.fsum)
    # of the same per-path values.
    import math
    w = inputs.dirichlet_disk_k10(M=M)
    w.x = w.x[:4].copy()
    w.max_steps = 20000
    r = _gpu.dirichlet(c, w, pm.PM_FP32, want_paths=True)
    g = r["g"]
    for j in range(g.shape[0]):
        s = math.fsum(g[j])
        m = s / M
        v = (math.fsum(g[j] * g[j]) - s * m) / (M - 1)
        assert abs(r["mean"][j] - m) <= 1e-15 * max(1.0, abs(m))
        assert abs(r["var"][j] - v) <= 1e-12 * max(1.0, v)
