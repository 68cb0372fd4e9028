"""Parity at the full workload sizes, in the launch configurations the benchmark
times.  The FP64 oracle computes a sample of the per-path values one path at a
time; the GPU run is the full one.  On the 440-mode field float and double paths
decorrelate (a chaotic flow: a rounding-size change grows to O(1) by t ~ 0.8),
so the comparison is paired and in distribution:
the mean per-path difference must vanish within 5 standard errors, and paths
that finish early (before the flow separates them) must agree closely."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h, s = _gpu.side_stream_ctx()
    with torch.cuda.stream(s):
        yield h
    pm.pm_destroy(h)


def paired_ok(d):
    d = np.asarray(d).ravel()
    return abs(d.mean()) <= 5 * d.std(ddof=1) / np.sqrt(d.size)


def test_timedep_440_modes_full_size(c, orc):
    w = inputs.timedep_k10()                       # 300 obs x M = 1e4, dt = 1e-3
    mean, var, g = _gpu.timedep(c, w, pm.PM_FP32, g_out=True)
    assert np.all(np.isfinite(mean)) and np.all(var > 0)
    # the estimate is the mean of the per-path values it reports
    np.testing.assert_allclose(mean, g.mean(axis=1), rtol=0, atol=1e-12)
    P = 24
    go = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=P)
    d = g[:, :P] - go
    assert paired_ok(d)
    # (the per-path spread at t = 0.25 is bounded by the oracle's own rounding
    # sensitivity in test_gpu_oracle_sample_parity.py, on 1000 paths)
    # and every estimate lies within 5 SE of the oracle's value on its first P paths
    se = np.sqrt(var / w.M + go.var(axis=1, ddof=1) / P)
    assert np.mean(np.abs(mean - go.mean(axis=1)) <= 5 * se) >= 0.99


def test_dirichlet_disk_full_size(c, orc):
    w = inputs.dirichlet_disk_k10()                # 50 obs x M = 1e5, dt = 1e-4
    r = _gpu.dirichlet(c, w, pm.PM_FP32, want_paths=True)
    assert r["unexited"] == 0 and r["rc"] == 0
    np.testing.assert_allclose(r["mean"], r["g"].mean(axis=1), rtol=0, atol=1e-12)
    P = 3
    go, so = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=P)
    assert paired_ok(r["g"][:, :P] - go)
    early = so < 2000                              # exits before the paths separate
    assert early.sum() >= 10
    assert np.mean(r["steps"][:, :P][early] == so[early]) >= 0.99


def test_batched_256_instances_full_size(c, orc):
    ws = inputs.batched_instances()                # 256 x 100 obs x M = 4096
    rc, mean, var, nu = _gpu.batched(c, ws)
    assert rc == 0 and nu == 0 and np.all(np.isfinite(mean))
    # sampled instances: one of each kind, first paths, through the oracle
    for b in (0, 1):
        w = ws[b]
        rows = slice(100 * b, 100 * b + 100)
        if isinstance(w, inputs.TimedepWorkload):
            go = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=8, inst=b)
        else:
            go, _ = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed,
                                        npaths=4, inst=b)
        # the oracle sample is a few paths: its standard error from the GPU's variance estimate
        se = np.sqrt(var[rows] / w.M + var[rows] / go.shape[1])
        assert np.mean(np.abs(mean[rows] - go.mean(axis=1)) <= 5 * se) >= 0.97
