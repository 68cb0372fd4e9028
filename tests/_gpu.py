"""Helpers for the GPU parity tests: run the CUDA library through the C ABI on
the inputs of a workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1808_10580_gb300 as pm  # noqa: E402
from paper_1808_10580_gb300 import inputs  # noqa: E402


def ctx():
    return pm.pm_create(0, torch.cuda.current_stream().cuda_stream)


def side_stream_ctx():
    s = torch.cuda.Stream()
    return pm.pm_create(0, s.cuda_stream), s


def timedep(c, w, flags=pm.PM_FP32, M=None, obs=None, g_out=False, x_out=False, device=True, path_offset=0):
    M = w.M if M is None else M
    x, t = (w.x, w.t) if obs is None else (w.x[obs], w.t[obs])
    n = len(t)
    fld = pm.Field(w.K, w.u)
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    if device:
        dx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        dt_ = torch.from_numpy(np.ascontiguousarray(t)).cuda()
        mean = torch.empty(n, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        g = torch.empty(n * M, dtype=torch.float64, device="cuda") if g_out else None
        xo = torch.empty(n * M * 2, dtype=torch.float64, device="cuda") if x_out else None
        pm.pm_forward_timedep(c, fld, w.kappa, th, dx, dt_, n, M, w.dt, w.seed, flags, mean, var,
                              path_offset=path_offset, g_out=g, x_out=xo)
        torch.cuda.synchronize()
        out = [mean.cpu().numpy(), var.cpu().numpy()]
        if g_out:
            out.append(g.cpu().numpy().reshape(n, M))
        if x_out:
            out.append(xo.cpu().numpy().reshape(n, M, 2))
        return out
    mean = np.empty(n)
    var = np.empty(n)
    g = np.empty(n * M) if g_out else None
    xo = np.empty(n * M * 2) if x_out else None
    pm.pm_forward_timedep(c, fld, w.kappa, th, np.ascontiguousarray(x), np.ascontiguousarray(t), n, M, w.dt, w.seed,
                          flags, mean, var, path_offset=path_offset, g_out=g, x_out=xo)
    out = [mean, var]
    if g_out:
        out.append(g.reshape(n, M))
    if x_out:
        out.append(xo.reshape(n, M, 2))
    return out


def dirichlet(c, w, flags=pm.PM_FP32, M=None, obs=None, device=True, want_paths=False, path_offset=0):
    M = w.M if M is None else M
    x = w.x if obs is None else w.x[obs]
    n = len(x)
    fld = pm.Field(w.K, w.u)
    gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
    if device:
        dx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        mean = torch.empty(n, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        es = torch.empty(n * M, dtype=torch.int32, device="cuda") if want_paths else None
        g = torch.empty(n * M, dtype=torch.float64, device="cuda") if want_paths else None
        nu = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = pm.pm_forward_dirichlet(c, fld, w.drift_scale, w.kappa, gd, dx, n, M, w.dt, w.max_steps, w.seed, flags,
                                     mean, var, es, nu, path_offset=path_offset, g_out=g)
        torch.cuda.synchronize()
        out = dict(rc=rc, mean=mean.cpu().numpy(), var=var.cpu().numpy(), unexited=int(nu.item()))
        if want_paths:
            out["steps"] = es.cpu().numpy().reshape(n, M)
            out["g"] = g.cpu().numpy().reshape(n, M)
        return out
    mean = np.empty(n)
    var = np.empty(n)
    es = np.empty(n * M, dtype=np.int32) if want_paths else None
    g = np.empty(n * M) if want_paths else None
    nu = np.zeros(1, dtype=np.int64)
    rc = pm.pm_forward_dirichlet(c, fld, w.drift_scale, w.kappa, gd, np.ascontiguousarray(x), n, M, w.dt, w.max_steps,
                                 w.seed, flags, mean, var, es, nu, path_offset=path_offset, g_out=g)
    out = dict(rc=rc, mean=mean, var=var, unexited=int(nu[0]))
    if want_paths:
        out["steps"] = es.reshape(n, M)
        out["g"] = g.reshape(n, M)
    return out


def batch_from_workloads(ws, device=True):
    """pm.Batch over a list of workloads (time-dependent ones share theta0, Dirichlet
    ones share the disk data), rows laid out in list order."""
    xs, ts, inst = [], [], []
    row = 0
    th = disk = None
    for w in ws:
        n = len(w.x)
        xs.append(w.x)
        if isinstance(w, inputs.TimedepWorkload):
            ts.append(w.t)
            th = th or pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
            inst.append(dict(kind=pm.PM_KIND_TIMEDEP, u=w.u, kappa=w.kappa, dt=w.dt, row0=row, n_obs=n, M=w.M,
                             seed=w.seed))
        else:
            ts.append(np.zeros(n))
            disk = disk or pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
            inst.append(dict(kind=pm.PM_KIND_DIRICHLET, u=w.u, kappa=w.kappa, dt=w.dt, row0=row, n_obs=n, M=w.M,
                             seed=w.seed, drift_scale=w.drift_scale, max_steps=w.max_steps))
        row += n
    x = np.ascontiguousarray(np.concatenate(xs))
    t = np.ascontiguousarray(np.concatenate(ts))
    if device:
        x = torch.from_numpy(x).cuda()
        t = torch.from_numpy(t).cuda()
        for d in inst:
            d["u"] = torch.from_numpy(np.ascontiguousarray(d["u"])).cuda()
    K = ws[0].K
    return pm.Batch(K, inst, x, t, th, disk), row


def batched(c, ws, device=True, flags=pm.PM_FP32):
    b, n_rows = batch_from_workloads(ws, device)
    if device:
        mean = torch.empty(n_rows, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        nu = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = pm.pm_forward_batched(c, b, flags, mean, var, nu)
        torch.cuda.synchronize()
        return rc, mean.cpu().numpy(), var.cpu().numpy(), int(nu.item())
    mean = np.empty(n_rows)
    var = np.empty(n_rows)
    nu = np.zeros(1, dtype=np.int64)
    rc = pm.pm_forward_batched(c, b, flags, mean, var, nu)
    return rc, mean, var, int(nu[0])
