"""GPU checks of the batched persistent map (many parameter samples, mixed
time-dependent and Dirichlet instances, one launch captured in a CUDA graph)."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h, s = _gpu.side_stream_ctx()   # a capturable stream: the graph path is exercised
    with torch.cuda.stream(s):
        yield h
    pm.pm_destroy(h)


def small_instances(B=6, M=256):
    ws = inputs.batched_instances(B=B, M=M)
    for w in ws:
        if isinstance(w, inputs.DirichletWorkload):
            w.x = w.x[:20].copy()
        else:
            w.x, w.t = w.x[::5].copy(), w.t[::5].copy()
    return ws


def per_instance_reference(c, ws):
    """Each instance through the single-problem entry points with the same RNG instance id."""
    means, vars_ = [], []
    for b, w in enumerate(ws):
        fld = pm.Field(w.K, w.u)
        n = len(w.x)
        mean = np.empty(n)
        var = np.empty(n)
        if isinstance(w, inputs.TimedepWorkload):
            th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
            pm.pm_forward_timedep(c, fld, w.kappa, th, w.x, w.t, n, w.M, w.dt, w.seed, pm.PM_FP32, mean, var,
                                  instance=b)
        else:
            gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
            pm.pm_forward_dirichlet(c, fld, w.drift_scale, w.kappa, gd, w.x, n, w.M, w.dt, w.max_steps, w.seed,
                                    pm.PM_FP32, mean, var, instance=b)
        means.append(mean)
        vars_.append(var)
    return np.concatenate(means), np.concatenate(vars_)


@pytest.mark.parametrize("device", [True, False])
def test_batched_equals_single_instance_calls(c, device):
    # Same coefficient table, same RNG stream, same step code: identical estimates.
    ws = small_instances()
    rc, mean, var, nu = _gpu.batched(c, ws, device=device)
    rm, rv = per_instance_reference(c, ws)
    assert rc == 0 and nu == 0
    np.testing.assert_allclose(mean, rm, rtol=0, atol=1e-12)
    np.testing.assert_allclose(var, rv, rtol=1e-10, atol=1e-12)


def test_graph_replay_picks_up_new_parameters(c):
    ws = small_instances(B=4)
    rc, m1, _, _ = _gpu.batched(c, ws)          # captures the graph
    for k, w in enumerate(ws):                   # same shape, new coefficients and seeds
        w.u = inputs.prior_field(10, 777, counter=k)
        w.seed = w.seed + 1
    rc, m2, v2, _ = _gpu.batched(c, ws)          # replays it
    pm.pm_set_graph_mode(c, 0)
    try:
        rc, m3, v3, _ = _gpu.batched(c, ws)      # direct launches
    finally:
        pm.pm_set_graph_mode(c, 1)
    assert not np.allclose(m1, m2)
    np.testing.assert_array_equal(m2, m3)
    np.testing.assert_array_equal(v2, v3)


def test_batched_timedep_instance_matches_oracle_without_drift(c, orc):
    # v = 0 instances: no amplification of rounding, the float estimate tracks the FP64 oracle.
    ws = small_instances(B=2, M=1000)
    w = ws[0]
    w.u = np.zeros_like(w.u)
    rc, mean, var, nu = _gpu.batched(c, ws)
    g = orc.timedep_paths(0, np.zeros(0), w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=w.M, inst=0)
    rm, rv, rse = orc.estimate(g)
    assert np.abs(mean[:len(w.x)] - rm).max() <= 1e-6


def test_rows_must_tile(c):
    ws = small_instances(B=2)
    b, n_rows = _gpu.batch_from_workloads(ws, device=False)
    b.arr[1].row0 = 3   # overlaps instance 0
    mean = np.empty(n_rows)
    with pytest.raises(pm.PMError, match="tile"):
        pm.pm_forward_batched(c, b, pm.PM_FP32, mean)


def test_full_size_batch_sampled(c, orc):
    # The batched workload as the bench runs it (256 instances x 100 observations x
    # M = 4096, tensor cores): sampled instances equal their single-instance calls bit
    # for bit, and the first 16 paths of every observation of one instance of each kind
    # agree with the FP64 oracle on the same streams in distribution (the 440-mode flow
    # is chaotic, so float and double paths separate; early Dirichlet exits agree).
    ws = inputs.batched_instances()
    flags = pm.PM_FP32 | pm.PM_TENSOR
    rc, mean, var, nu = _gpu.batched(c, ws, flags=flags)
    assert rc == 0 and nu == 0 and np.all(np.isfinite(mean)) and np.all(var >= 0)
    P = 16
    for b in (0, 1, 128, 255):
        w = ws[b]
        n = len(w.x)
        fld = pm.Field(w.K, w.u)
        m = np.empty(n)
        g = np.empty(n * w.M)
        if isinstance(w, inputs.TimedepWorkload):
            th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
            pm.pm_forward_timedep(c, fld, w.kappa, th, w.x, w.t, n, w.M, w.dt, w.seed, flags, m, instance=b, g_out=g)
        else:
            es = np.empty(n * w.M, dtype=np.int32)
            gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
            pm.pm_forward_dirichlet(c, fld, w.drift_scale, w.kappa, gd, w.x, n, w.M, w.dt, w.max_steps, w.seed,
                                    flags, m, None, es, None, instance=b, g_out=g)
        np.testing.assert_allclose(mean[100 * b:100 * (b + 1)], m, rtol=0, atol=1e-12)
        if b > 1:
            continue
        g = g.reshape(n, w.M)[:, :P]
        if isinstance(w, inputs.TimedepWorkload):
            go = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=P, inst=b)
        else:
            go, so = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed,
                                         npaths=P, inst=b)
            st = es.reshape(n, w.M)[:, :P]
            early = so < 100
            assert early.sum() > 20 and np.mean(st[early] == so[early]) >= 0.99
        d = (g - go).ravel()
        assert abs(d.mean()) <= 5 * d.std(ddof=1) / np.sqrt(d.size)
