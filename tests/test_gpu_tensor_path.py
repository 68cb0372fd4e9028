"""Parity of the time-dependent map with the velocity sum on the tensor cores
(PM_TENSOR: tcgen05 with a three-term hi/lo split of TF32 operands for K <= 8
and of FP16 operands from K = 10) against the FP64 oracle
and against the FP32-pipe kernel."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


@pytest.mark.parametrize("K", [4, 5, 6, 8, 10, 12, 16])
def test_one_step_positions_match_oracle(c, orc, K):
    # One Euler step of length dt from 300 points: X1 - x = -v(x) dt + noise, so the
    # end points expose the velocity the tensor-core path evaluated.
    w = inputs.timedep_k10(M=128)
    w.K = K
    w.u = inputs.prior_field(K, 300 + K)
    rng = np.random.default_rng(K)
    w.x = rng.random((64, 2))
    w.dt = 0.01
    w.t = np.full(64, w.dt)
    _, _, xe = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, x_out=True)
    _, _, xs = _gpu.timedep(c, w, pm.PM_FP32, x_out=True)
    _, xo = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=128, want_x=True)
    modes = orc.half_modes(K).astype(float)
    scale = float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(w.u.reshape(-1, 2)).sum(1)).sum())
    d_tc = xe - xo
    d_tc -= np.round(d_tc)
    d_sm = xs - xo
    d_sm -= np.round(d_sm)
    # three products of 11-bit operands keep ~21 bits: velocity error <= ~1e-6 of the term scale
    assert np.abs(d_tc).max() <= w.dt * 4e-6 * scale + 1e-7, (np.abs(d_tc).max(), np.abs(d_sm).max())


@pytest.mark.parametrize("field", ["zero", "shear"])
def test_stable_fields_match_oracle_at_1e5(c, orc, field):
    w = inputs.timedep_k10(M=4000)
    if field == "zero":
        w.u = np.zeros_like(w.u)
    else:
        modes = orc.half_modes(10)
        h = [tuple(m) for m in modes].index((2, 3))
        w.u = np.zeros_like(w.u)
        w.u[2 * h], w.u[2 * h + 1] = 0.05, 0.02
    obs = np.array([5, 120, 250])
    mean, var = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, obs=obs)
    g = orc.timedep_paths(10, w.u, w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, w.seed, npaths=w.M,
                          obs_id=np.arange(3))
    rm, rv, rse = orc.estimate(g)
    assert np.abs(mean - rm).max() <= 1e-5


def test_full_size_440_modes_in_distribution(c, orc):
    w = inputs.timedep_k10()
    mean, var, g = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, g_out=True)
    ms, vs = _gpu.timedep(c, w, pm.PM_FP32)
    P = 16
    go = orc.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=P)
    d = (g[:, :P] - go).ravel()
    assert abs(d.mean()) <= 5 * d.std(ddof=1) / np.sqrt(d.size)
    # the two float kernels are two estimates with correlated early paths: within 5 SE of each other
    se = np.sqrt((var + vs) / w.M)
    assert np.mean(np.abs(mean - ms) <= 5 * se) >= 0.99


def test_repeatable(c):
    w = inputs.timedep_k10(M=512)
    a = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR)
    b = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR)
    assert np.array_equal(a[0], b[0])


def test_dirichlet_zero_drift_exit_steps(c, orc):
    from tests.test_gpu_dirichlet import zero_drift_workload
    w = zero_drift_workload(M=2000)
    r = _gpu.dirichlet(c, w, pm.PM_FP32 | pm.PM_TENSOR, want_paths=True)
    g, st = orc.dirichlet_paths(0, np.zeros(0), 0.0, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=w.M)
    assert np.mean(r["steps"] == st) >= 0.999
    rm, rv, rse = orc.estimate(g)
    assert np.all(np.abs(r["mean"] - rm) <= 3 * np.sqrt(2) * rse)


def test_dirichlet_drift_full_size(c, orc):
    w = inputs.dirichlet_disk_k10()
    r = _gpu.dirichlet(c, w, pm.PM_FP32 | pm.PM_TENSOR, want_paths=True)
    s = _gpu.dirichlet(c, w, pm.PM_FP32)
    assert r["rc"] == 0 and r["unexited"] == 0
    P = 3
    go, so = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=P)
    d = (r["g"][:, :P] - go).ravel()
    assert abs(d.mean()) <= 5 * d.std(ddof=1) / np.sqrt(d.size)
    early = so < 2000
    assert np.mean(r["steps"][:, :P][early] == so[early]) >= 0.99
    se = np.sqrt((r["var"] + s["var"]) / w.M)
    assert np.mean(np.abs(r["mean"] - s["mean"]) <= 5 * se) >= 0.98


def test_batched_tensor_equals_single_instance_tensor_calls():
    from tests.test_gpu_batched import small_instances
    h, s = _gpu.side_stream_ctx()
    try:
        with torch.cuda.stream(s):
            ws = small_instances(B=6, M=256)
            b, n_rows = _gpu.batch_from_workloads(ws, device=True)
            mean = torch.empty(n_rows, dtype=torch.float64, device="cuda")
            var = torch.empty_like(mean)
            rc = pm.pm_forward_batched(h, b, pm.PM_FP32 | pm.PM_TENSOR, mean, var)
            torch.cuda.synchronize()
            got = mean.cpu().numpy()
            ref = []
            for k, w in enumerate(ws):
                n = len(w.x)
                m = np.empty(n)
                if isinstance(w, inputs.TimedepWorkload):
                    pm.pm_forward_timedep(h, pm.Field(w.K, w.u), w.kappa, pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b),
                                          w.x, w.t, n, w.M, w.dt, w.seed, pm.PM_FP32 | pm.PM_TENSOR, m, instance=k)
                else:
                    pm.pm_forward_dirichlet(h, pm.Field(w.K, w.u), w.drift_scale, w.kappa,
                                            pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b), w.x, n, w.M,
                                            w.dt, w.max_steps, w.seed, pm.PM_FP32 | pm.PM_TENSOR, m, instance=k)
                ref.append(m)
        assert rc == 0
        np.testing.assert_allclose(got, np.concatenate(ref), rtol=0, atol=1e-12)
    finally:
        pm.pm_destroy(h)


def test_persistent_tensor_grids_fill_every_sm(c):
    # The persistent tensor-core kernels run several CTAs per SM (registers,
    # shared memory and tensor memory allow 4 at K = 10), not one.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = inputs.dirichlet_disk_k10(M=4096)
    w.max_steps = 2000
    _gpu.dirichlet(c, w, pm.PM_FP32 | pm.PM_TENSOR)
    g_dir = pm.pm_last_grid(c)
    from tests.test_gpu_batched import small_instances
    ws = small_instances(B=8, M=4096)
    _gpu.batched(c, ws, flags=pm.PM_FP32 | pm.PM_TENSOR)
    g_bat = pm.pm_last_grid(c)
    assert g_dir % sms == 0 and g_dir >= 2 * sms, (g_dir, sms)
    assert g_bat % sms == 0 and g_bat >= 2 * sms, (g_bat, sms)


def shear_field(orc, w):
    modes = orc.half_modes(10)
    h = [tuple(m) for m in modes].index((2, 3))
    u = np.zeros_like(w.u)
    u[2 * h], u[2 * h + 1] = 0.05, 0.02
    return u


def test_tensor_path_shards_equal_one_call(c):
    # Paths are keyed by their index, and a tile row's result depends on its
    # own particle only: shards at any path offset reproduce the single call.
    w = inputs.timedep_k10(M=384)
    obs = np.array([3, 150, 299])
    _, _, g = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, obs=obs, g_out=True)
    _, _, g1 = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, obs=obs, M=200, g_out=True)
    _, _, g2 = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, obs=obs, M=184, g_out=True, path_offset=200)
    assert np.array_equal(np.concatenate([g1, g2], axis=1), g)


@pytest.mark.parametrize("M", [1, 129])
def test_tensor_path_zero_horizon_and_ragged_tiles(c, orc, M):
    w = inputs.timedep_k10(M=M)
    w.u = shear_field(orc, w)
    w.x, w.t = w.x[:4].copy(), np.array([0.0, 0.001, 0.0105, 0.3])
    mean, var, g = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, g_out=True)
    go = orc.timedep_paths(10, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=M)
    assert np.abs(g - go).max() <= 5e-5
    # t = 0: every path is theta0 at the observation point
    assert np.ptp(g[0]) == 0.0 and np.abs(g[0] - go[0]).max() <= 1e-6


@pytest.mark.parametrize("device", [False, True])
def test_tensor_path_host_and_device_pointers_agree(c, device):
    w = inputs.timedep_k10(M=256)
    a = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, device=True)
    b = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, device=device)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("K", [10, 16])
@pytest.mark.parametrize("scale", [1e-6, 1e3])
def test_fp16_scale_of_w_at_extreme_field_sizes(c, orc, K, scale):
    # FP16 operands carry W times 2^e with its largest entry in [2^13, 2^14); fields
    # of very small and very large size move e far from 0 (and, folded at K = 16,
    # the n = 0 terms share the scale).  One step from 64 points, as above; the drift
    # of the large field is kept to a fraction of the domain by a short step.
    w = inputs.timedep_k10(M=128)
    w.K = K
    w.u = inputs.prior_field(K, 900 + K) * scale
    rng = np.random.default_rng(K)
    w.x = rng.random((64, 2))
    w.dt = 0.01 / max(1.0, scale)
    w.t = np.full(64, w.dt)
    _, _, xe = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, x_out=True)
    _, xo = orc.timedep_paths(K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=128, want_x=True)
    modes = orc.half_modes(K).astype(float)
    term_scale = float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(w.u.reshape(-1, 2)).sum(1)).sum())
    d = xe - xo
    d -= np.round(d)
    assert np.abs(d).max() <= w.dt * 4e-6 * term_scale + 1e-7, np.abs(d).max()


@pytest.mark.parametrize("K", [4, 8, 16, 24, 40, 64])
def test_batched_tensor_at_other_bounds(K):
    # The batched kernel at other wave-number bounds against single-instance calls:
    # Dirichlet instances share the shape (unfolded up to K = 16, folded like the
    # time-dependent kernel above it), so bit for bit; time-dependent instances
    # equal too where both kernels take the same shape (K = 4, 24 unfolded; 40,
    # 64 folded), and agree within Monte Carlo error where only the
    # single-problem kernel folds the constant column (K = 8, 16).
    from tests.test_gpu_batched import small_instances
    h, s = _gpu.side_stream_ctx()
    try:
        with torch.cuda.stream(s):
            ws = small_instances(B=4, M=256)
            for b, w in enumerate(ws):
                w.K = K
                w.u = inputs.prior_field(K, 1100 + K, counter=b)
            b_, n_rows = _gpu.batch_from_workloads(ws, device=True)
            mean = torch.empty(n_rows, dtype=torch.float64, device="cuda")
            var = torch.empty_like(mean)
            rc = pm.pm_forward_batched(h, b_, pm.PM_FP32 | pm.PM_TENSOR, mean, var)
            torch.cuda.synchronize()
            got, gv = mean.cpu().numpy(), var.cpu().numpy()
            row = 0
            for k, w in enumerate(ws):
                n = len(w.x)
                m = np.empty(n)
                v = np.empty(n)
                if isinstance(w, inputs.TimedepWorkload):
                    pm.pm_forward_timedep(h, pm.Field(w.K, w.u), w.kappa,
                                          pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b), w.x, w.t, n, w.M, w.dt,
                                          w.seed, pm.PM_FP32 | pm.PM_TENSOR, m, v, instance=k)
                    if K > 16 or K % 4 or K < 8:  # the same shape in both kernels
                        np.testing.assert_allclose(got[row:row + n], m, rtol=0, atol=1e-12)
                    else:
                        se = np.sqrt((gv[row:row + n] + v) / w.M)
                        assert np.all(np.abs(got[row:row + n] - m) <= 5 * se + 1e-6)
                else:
                    pm.pm_forward_dirichlet(h, pm.Field(w.K, w.u), w.drift_scale, w.kappa,
                                            pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b), w.x, n,
                                            w.M, w.dt, w.max_steps, w.seed, pm.PM_FP32 | pm.PM_TENSOR, m, v,
                                            instance=k)
                    np.testing.assert_allclose(got[row:row + n], m, rtol=0, atol=1e-12)
                row += n
        assert rc == 0
    finally:
        pm.pm_destroy(h)
