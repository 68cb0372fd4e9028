"""Algorithm 2 (walks to the first exit from the disk) at the wide wave-number
bounds K = 24 ... 64 (N_u = 2400 ... 16640 real coefficients; Section 4's
larger Fourier bases): the FP32-pipe kernel with its velocity table in shared
memory and the tensor-core kernel with its coefficient tiles in global memory
(the folded shape from K = 32), against the FP64 oracle on the same streams."""
import dataclasses
import functools

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu
from tests import _stats as S

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


def wide_disk(K, M, n_pts=8, r_max=0.9, seed=0):
    w = inputs.dirichlet_disk_k10(M=M)
    return dataclasses.replace(w, K=K, u=inputs.prior_field(K, 600 + K),
                               x=inputs.disk_points(n_pts, r_max, 700 + K + seed), dt=1e-3)


def run(c, w, flags, M=None, max_steps=None):
    M = w.M if M is None else M
    n = len(w.x)
    total = n * M
    dx = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    es = torch.empty(total, dtype=torch.int32, device="cuda")
    g = torch.empty(total, dtype=torch.float64, device="cuda")
    xo = torch.empty(2 * total, dtype=torch.float64, device="cuda")
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
    rc = pm.pm_forward_dirichlet(c, pm.Field(w.K, w.u), w.drift_scale, w.kappa, gd, dx, n, M, w.dt,
                                 w.max_steps if max_steps is None else max_steps, w.seed, flags, mean, var, es, nu,
                                 g_out=g, x_out=xo)
    torch.cuda.synchronize()
    return dict(rc=rc, mean=mean.cpu().numpy(), var=var.cpu().numpy(), unexited=int(nu.item()),
                steps=es.cpu().numpy().reshape(n, M), g=g.cpu().numpy().reshape(n, M),
                x=xo.cpu().numpy().reshape(n, M, 2))


def velocity_scale(orc, K, u):
    # sum over the modes of |grad| |psi_h|: a bound on |v| and on its FP32 rounding scale
    modes = orc.half_modes(K).astype(float)
    return float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(u.reshape(-1, 2)).sum(1)).sum())


N_SHORT = 20


@functools.lru_cache(maxsize=None)
def short_horizon_oracle(K):
    """The FP64 paths, and how much each path stretches a small change of its
    start over the horizon (two directions, the larger ratio; the same noise)."""
    import oracle
    # dt = 1e-4: at 1e-3 a step of a K = 64 prior draw already stretches by a
    # factor near 1.5 (dt |grad v| ~ 0.5), and 20 steps by up to 1e5
    ang = 0.3 + np.arange(4) * np.pi / 2
    edge = 0.99 * np.stack([np.cos(ang), np.sin(ang)], 1)  # walks that exit within the horizon
    w = dataclasses.replace(wide_disk(K, 64), x=np.concatenate([inputs.disk_points(6, 0.9, 700 + K), edge]), dt=1e-4)
    base = oracle.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, N_SHORT, w.seed,
                                  npaths=w.M, want_x=True)
    delta = 1e-9
    amp = np.ones((len(w.x), w.M))
    for e in ((delta, 0.0), (0.0, delta)):
        _, s2, x2 = oracle.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x + np.array(e), w.dt, N_SHORT,
                                           w.seed, npaths=w.M, want_x=True)
        a = np.linalg.norm(x2 - base[2], axis=-1) / delta
        amp = np.maximum(amp, np.where(s2 == base[1], a, np.inf))
    return w, base, amp


@pytest.mark.parametrize("K", WIDE)
@pytest.mark.parametrize("tensor", [False, True])
def test_short_horizon_paths_match_oracle(c, orc, K, tensor):
    # 20 steps (t = 0.002) of a prior draw, partly from points near the edge: each float
    # path stays within its velocity rounding (a bound per step, at most
    # 4e-6 of the field's scale) times the stretching the FP64 flow applies
    # to a small change over the horizon, and the walks that exit in that time
    # exit at the same step.  The stretching grows with K (the velocity
    # gradient of a prior draw grows with the number of modes).
    n_steps = N_SHORT
    w, (go, so, xo), amp = short_horizon_oracle(K)
    r = run(c, w, TC if tensor else pm.PM_FP32, max_steps=n_steps)
    assert r["rc"] in (0, pm.PM_WARN_UNEXITED)
    steps = r["steps"].astype(np.int64)
    exited_o = so >= 0
    assert exited_o.sum() > 10 and (~exited_o).sum() > 100
    same = (steps == so) & np.isfinite(amp)
    assert np.mean(same) >= 0.995, np.mean(same)
    step_err = w.dt * w.drift_scale * 4e-6 * velocity_scale(orc, K, w.u)
    tol = 2 * amp * n_steps * step_err + 1e-6
    d = np.linalg.norm(r["x"] - xo, axis=-1)
    ratio = (d / tol)[same]
    print(f"K = {K}, {'tensor cores' if tensor else 'FP32 pipes'}: exit steps identical {np.mean(same):.4f}, "
          f"largest |X - X_oracle| {d[same].max():.2e}, largest stretching {amp[same].max():.1f}, "
          f"largest deviation / bound {ratio.max():.3f}")
    assert ratio.max() <= 1.0
    # the exits' values too (g at the exit point, f = 0)
    both = same & exited_o
    assert np.all(np.abs(r["g"][both] - go[both]) <= 10 * tol[both])


@pytest.mark.parametrize("K", [24, 64])
@pytest.mark.parametrize("tensor", [False, True])
def test_zero_field_exit_steps_match_oracle(c, orc, K, tensor):
    # v = 0 through the wide tables (all-zero W, the FP16 scale at its clamp):
    # the walks are the oracle's Brownian ones, exit step for exit step.
    w = dataclasses.replace(wide_disk(K, 500, r_max=0.8), u=np.zeros((2 * K + 1) ** 2 - 1))
    r = run(c, w, TC if tensor else pm.PM_FP32)
    go, so = orc.dirichlet_paths(0, np.zeros(0), 0.0, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=w.M)
    assert r["rc"] == 0 and r["unexited"] == 0
    same = r["steps"] == so
    assert np.mean(same) >= 0.999
    assert np.abs(r["g"][same] - go[same]).max() < 1e-5


def test_prior_field_in_distribution(c, orc):
    # K = 24, a smaller disk and kappa = 0.2 keep the FP64 oracle to seconds;
    # paired means over 1000 paths per observation on the same streams, and an
    # independent full-size launch against the oracle's estimate.
    MO = 1000
    w = wide_disk(24, 20_000, n_pts=10, r_max=0.4)
    w = dataclasses.replace(w, kappa=0.2, g=dataclasses.replace(w.g, R=0.5))
    go, so = orc.dirichlet_paths(w.K, w.u, w.drift_scale, w.kappa, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=MO)
    mo, _, seo = orc.estimate(go)
    for flags in (TC, pm.PM_FP32):
        same = run(c, w, flags, M=MO)
        ind = run(c, dataclasses.replace(w, seed=w.seed + 7919), flags)
        assert same["unexited"] == 0 and ind["unexited"] == 0
        paired = S.zcheck(S.paired_z(same["g"], go))
        two = S.zcheck(S.two_sample_z(ind["mean"], np.sqrt(ind["var"] / w.M), mo, seo))
        early = so < 100
        agree = float(np.mean(same["steps"][early] == so[early]))
        print("K = 24 disk:", "tensor" if flags & pm.PM_TENSOR else "pipes", "paired", paired, "two-sample", two,
              "exit steps before step 100 identical", agree, "of", int(early.sum()))
        assert paired["ok"] and two["ok"], (paired, two)
        assert agree >= 0.99


def run_general(c, w, df, M=None, max_steps=None, seed=None):
    M = w.M if M is None else M
    n = len(w.x)
    total = n * M
    dx = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    es = torch.empty(total, dtype=torch.int32, device="cuda")
    g = torch.empty(total, dtype=torch.float64, device="cuda")
    xo = torch.empty(2 * total, dtype=torch.float64, device="cuda")
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
    d = pm.DiffusionForcing(df.s0, df.s1, df.milstein, df.c, df.F, df.w)
    rc = pm.pm_forward_dirichlet_general(c, pm.Field(w.K, w.u), w.drift_scale, gd, d, dx, n, M, w.dt,
                                         w.max_steps if max_steps is None else max_steps,
                                         w.seed if seed is None else seed, TC, mean, var, es, nu, g_out=g, x_out=xo)
    torch.cuda.synchronize()
    return dict(rc=rc, mean=mean.cpu().numpy(), var=var.cpu().numpy(), unexited=int(nu.item()),
                steps=es.cpu().numpy().reshape(n, M), g=g.cpu().numpy().reshape(n, M),
                x=xo.cpu().numpy().reshape(n, M, 2))


@pytest.mark.parametrize("K", [24, 64])
def test_general_map_short_horizon_paths_match_oracle(c, orc, K):
    # The general disk map (sigma(x) with the Milstein term, Gaussian sources)
    # on the tensor cores at a wide bound: 20 steps at dt = 1e-4 from interior
    # and edge points, path by path against the FP64 oracle, within the velocity
    # rounding times the FP64 flow's stretching of a small change (as above).
    gw, df = inputs.dirichlet_general_disk(M=64)
    ang = 0.3 + np.arange(4) * np.pi / 2
    edge = 0.99 * np.stack([np.cos(ang), np.sin(ang)], 1)
    w = dataclasses.replace(gw, K=K, u=inputs.prior_field(K, 600 + K), dt=1e-4,
                            x=np.concatenate([inputs.disk_points(6, 0.9, 700 + K), edge]))
    args = (w.K, w.u, w.drift_scale, df, w.g)
    go, so, xo = orc.dirichlet_general_paths(*args, w.x, w.dt, N_SHORT, w.seed, npaths=w.M, want_x=True)
    amp = np.ones((len(w.x), w.M))
    for e in ((1e-9, 0.0), (0.0, 1e-9)):
        _, s2, x2 = orc.dirichlet_general_paths(*args, w.x + np.array(e), w.dt, N_SHORT, w.seed, npaths=w.M,
                                                want_x=True)
        amp = np.maximum(amp, np.where(s2 == so, np.linalg.norm(x2 - xo, axis=-1) / 1e-9, np.inf))
    r = run_general(c, w, df, max_steps=N_SHORT)
    assert r["rc"] in (0, pm.PM_WARN_UNEXITED)
    same = (r["steps"] == so) & np.isfinite(amp)
    assert (so >= 0).sum() > 10 and np.mean(same) >= 0.995
    tol = 2 * amp * N_SHORT * w.dt * w.drift_scale * 4e-6 * velocity_scale(orc, K, w.u) + 1e-6
    ratio = (np.linalg.norm(r["x"] - xo, axis=-1) / tol)[same]
    print(f"general map, K = {K}: exit steps identical {np.mean(same):.4f}, largest deviation / bound {ratio.max():.3f}")
    assert ratio.max() <= 1.0


def test_general_map_wide_in_distribution(c, orc):
    # K = 24, the disk of radius 0.5: paired means on the oracle's streams
    # (1000 paths per observation) and an independent full launch.
    MO = 1000
    gw, df = inputs.dirichlet_general_disk(M=20_000)
    w = dataclasses.replace(gw, K=24, u=inputs.prior_field(24, 624), dt=1e-3,
                            x=inputs.disk_points(10, 0.4, 724), g=dataclasses.replace(gw.g, R=0.5))
    go, so = orc.dirichlet_general_paths(w.K, w.u, w.drift_scale, df, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=MO)
    mo, _, seo = orc.estimate(go)
    same = run_general(c, w, df, M=MO)
    ind = run_general(c, w, df, seed=w.seed + 7919)
    assert same["unexited"] == 0 and ind["unexited"] == 0
    paired = S.zcheck(S.paired_z(same["g"], go))
    two = S.zcheck(S.two_sample_z(ind["mean"], np.sqrt(ind["var"] / w.M), mo, seo))
    print("general map, K = 24 disk: paired", paired, "two-sample", two)
    assert paired["ok"] and two["ok"], (paired, two)
