"""The disk map with a general forcing and a state-dependent diffusion
(pm_forward_dirichlet_general: Algorithm 2 / Theorem 3.2 with f(x) and
sigma(x), Milstein steps of Eq. millstein), on the FP32 / FP64 pipes and with
the velocity sum on the tensor cores (PM_TENSOR), against the FP64 oracle on
the same streams: path by path where the paths do not separate under rounding
(no drift; straight lines without diffusion), in distribution on the 440-mode
drift field (tests/_stats.py)."""
import dataclasses

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu
from tests import _stats as S
from tests.test_oracle_dirichlet_general import _single_mode_field

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def run(c, w, df, flags, M=None, seed=None):
    M = w.M if M is None else M
    n = len(w.x)
    dx = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    es = torch.empty(n * M, dtype=torch.int32, device="cuda")
    g = torch.empty(n * M, dtype=torch.float64, device="cuda")
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
    d = pm.DiffusionForcing(df.s0, df.s1, df.milstein, df.c, df.F, df.w)
    rc = pm.pm_forward_dirichlet_general(c, pm.Field(w.K, w.u), w.drift_scale, gd, d, dx, n, M, w.dt, w.max_steps,
                                         w.seed if seed is None else seed, flags, mean, var, es, nu, g_out=g)
    torch.cuda.synchronize()
    return dict(rc=rc, mean=mean.cpu().numpy(), var=var.cpu().numpy(), unexited=int(nu.item()),
                steps=es.cpu().numpy().reshape(n, M), g=g.cpu().numpy().reshape(n, M))


def oracle(orc, w, df, M):
    return orc.dirichlet_general_paths(w.K, w.u, w.drift_scale, df, w.g, w.x, w.dt, w.max_steps, w.seed, npaths=M)


def no_drift(M=500):
    w, df = inputs.dirichlet_general_disk(M=M)
    w = dataclasses.replace(w, K=0, u=np.zeros(0), x=w.x[:8], dt=1e-3)
    return w, df


@pytest.mark.parametrize("milstein", [True, False])
def test_double_paths_without_drift_equal_the_oracle_path_by_path(c, orc, milstein):
    w, df = no_drift()
    df = dataclasses.replace(df, milstein=milstein)
    r = run(c, w, df, pm.PM_FP64)
    go, so = oracle(orc, w, df, w.M)
    assert r["rc"] == 0 and r["unexited"] == 0
    assert np.array_equal(r["steps"], so)
    np.testing.assert_allclose(r["g"], go, rtol=0, atol=1e-10)


@pytest.mark.parametrize("tensor", [False, True])
def test_float_paths_without_drift_match_the_oracle(c, orc, tensor):
    # Without drift the float paths stay within rounding of the double ones
    # (nothing amplifies the difference), so the comparison is path by path:
    # a paired test would only measure float rounding against an error bar of
    # that same size.  The tensor-core kernel needs K >= 4: the 440-mode
    # lattice with all coefficients zero.
    w, df = no_drift()
    if tensor:
        w = dataclasses.replace(w, K=10, u=np.zeros(440))
    r = run(c, w, df, pm.PM_FP32 | (pm.PM_TENSOR if tensor else 0))
    go, so = oracle(orc, w, df, w.M)
    same = r["steps"] == so
    assert np.mean(same) >= 0.999
    d = np.abs(r["g"][same] - go[same])
    print("float, no drift: exit steps identical", float(np.mean(same)), "largest |g difference|", d.max())
    assert d.max() <= 1e-5 * max(1.0, np.abs(go).max())


def test_straight_lines_without_diffusion(c, orc):
    # kappa = 0 and one stream-function mode: deterministic straight paths
    w, df = inputs.dirichlet_general_disk(M=4)
    w = dataclasses.replace(w, u=_single_mode_field(10), drift_scale=3.0, dt=1e-3,
                            x=np.array([[0.1, 0.2], [-0.3, 0.4], [0.5, -0.5], [0.0, 0.0]]))
    df = dataclasses.replace(df, s0=np.zeros(2), s1=np.zeros(2))
    go, so = oracle(orc, w, df, w.M)
    for flags, tol in ((pm.PM_FP64, 1e-10), (pm.PM_FP32, 2e-5), (pm.PM_FP32 | pm.PM_TENSOR, 2e-5)):
        r = run(c, w, df, flags)
        assert np.array_equal(r["steps"], so)
        np.testing.assert_allclose(r["g"], go, rtol=0, atol=tol)


def test_constant_sigma_without_sources_reduces_to_the_disk_map(c):
    w, _ = no_drift(M=4000)
    s = np.sqrt(2 * w.kappa)
    df = inputs.DiffusionForcing(s0=np.array([s, s]), s1=np.zeros(2), milstein=True)
    r = run(c, w, df, pm.PM_FP32)
    q = _gpu.dirichlet(c, w, pm.PM_FP32, want_paths=True)
    assert np.mean(r["steps"] == q["steps"]) >= 0.999
    zc = S.zcheck(S.paired_z(r["g"], q["g"]))
    assert zc["ok"], zc


@pytest.mark.parametrize("tensor", [False, True])
def test_drift_field_in_distribution(c, orc, tensor):
    MO = 400
    w, df = inputs.dirichlet_general_disk(M=10_000)
    go, so = oracle(orc, w, df, MO)
    mo, _, seo = orc.estimate(go)
    flags = pm.PM_FP32 | (pm.PM_TENSOR if tensor else 0)
    same = run(c, w, df, flags, M=MO)
    ind = run(c, w, df, flags, seed=w.seed + 7919)
    assert same["unexited"] == 0 and ind["unexited"] == 0
    paired = S.zcheck(S.paired_z(same["g"], go))
    two = S.zcheck(S.two_sample_z(ind["mean"], np.sqrt(ind["var"] / w.M), mo, seo))
    early = so < 1000
    agree = float(np.mean(same["steps"][early] == so[early]))
    print("general disk,", "tensor cores:" if tensor else "FP32 pipes:", "paired", paired, "two-sample", two,
          "early exit agreement", agree, "of", int(early.sum()))
    assert paired["ok"] and two["ok"], (paired, two)
    assert agree >= 0.999
