"""The optimal-forcing boundary-value problem in the unit square on the GPU
(pm_forward_square_bvp) against the FP64 oracle on the same streams: double
paths path by path, float paths by exit steps and within Monte Carlo error;
edge cases; and the optimal forcing found by Nelder-Mead on the GPU's
functionals against the exact linear solve."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from paper_1808_10580_gb300 import optimal_forcing as of
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def run(c, w, flags, M, x=None, max_steps=None, want_paths=True):
    x = np.ascontiguousarray(w.x if x is None else x)
    prob = pm.SquareBVP(w.prob.b, w.prob.kappa, w.prob.c, w.prob.w, w.prob.g_cos, w.prob.g_quad)
    nf = len(w.prob.c) + 1
    mean = np.empty(len(x) * nf)
    var = np.empty(len(x) * nf)
    g = np.empty(len(x) * nf * M) if want_paths else None
    st = np.empty(len(x) * M, dtype=np.int32)
    nu = np.zeros(1, dtype=np.int64)
    rc = pm.pm_forward_square_bvp(c, prob, x, len(x), M, w.dt, max_steps or w.max_steps, w.seed, flags, mean, var,
                                  exit_step=st, n_unexited=nu, g_out=g)
    return dict(rc=rc, mean=mean.reshape(len(x), nf), var=var.reshape(len(x), nf),
                g=g.reshape(len(x), nf, M) if want_paths else None, steps=st.reshape(len(x), M), unexited=int(nu[0]))


def test_double_paths_match_the_oracle_path_by_path(c, orc):
    w = inputs.optimal_forcing(M=2000)
    r = run(c, w, pm.PM_FP64, 2000)
    go, so = orc.square_bvp_paths(w.prob, w.x, w.dt, w.max_steps, w.seed, npaths=2000)
    assert r["rc"] == 0 and r["unexited"] == 0
    assert np.array_equal(r["steps"], so)
    assert np.abs(r["g"] - go).max() <= 1e-10
    m = go.mean(axis=2)
    assert np.abs(r["mean"] - m).max() <= 1e-12


def test_float_paths_exit_steps_and_estimates(c, orc):
    w = inputs.optimal_forcing(M=4096)
    r = run(c, w, pm.PM_FP32, 4096)
    go, so = orc.square_bvp_paths(w.prob, w.x, w.dt, w.max_steps, w.seed, npaths=4096)
    assert np.mean(r["steps"] == so) >= 0.999
    same = r["steps"] == so
    d = np.abs(r["g"] - go)[:, :, :][np.broadcast_to(same[:, None, :], go.shape)]
    assert d.max() <= 1e-4
    rm, rv = go.mean(axis=2), go.var(axis=2, ddof=1)
    se = np.sqrt((rv + r["var"]) / 4096)
    assert np.all(np.abs(r["mean"] - rm) <= 3 * se + 1e-12)


def test_start_on_the_boundary_and_capped_paths(c, orc):
    w = inputs.optimal_forcing(M=64)
    x = np.array([[0.0, 0.5], [0.5, 1.0], [0.5, 0.5]])
    r = run(c, w, pm.PM_FP64, 64, x=x, max_steps=50)
    go, so = orc.square_bvp_paths(w.prob, x, w.dt, 50, w.seed, npaths=64)
    assert np.all(r["steps"][:2] == 0) and np.array_equal(r["steps"], so)
    assert r["rc"] == pm.PM_WARN_UNEXITED and r["unexited"] == 64         # the centre needs >> 50 steps
    assert np.abs(r["g"] - go).max() <= 1e-12


def test_shards_and_repeats_are_identical(c):
    w = inputs.optimal_forcing(M=1000)
    a = run(c, w, pm.PM_FP32, 1000)
    b = run(c, w, pm.PM_FP32, 1000)
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["g"], b["g"])
    prob = pm.SquareBVP(w.prob.b, w.prob.kappa, w.prob.c, w.prob.w)
    g2 = np.empty(3 * 4 * 400)
    m2 = np.empty(12)
    pm.pm_forward_square_bvp(c, prob, w.x, 3, 400, w.dt, w.max_steps, w.seed, pm.PM_FP32, m2, path_offset=600,
                             g_out=g2)
    assert np.array_equal(g2.reshape(3, 4, 400), a["g"][:, :, 600:])


def test_optimal_forcing_by_nelder_mead(c):
    w = inputs.optimal_forcing(M=200_000)
    E, se = of.functionals(c, w)
    r = of.solve(E, w.y, xtol=1e-12, ftol=1e-16)
    exact = np.linalg.solve(E[:, 1:], E[:, 0] - w.y)
    assert np.allclose(r.x, exact, rtol=1e-6, atol=1e-6)
    assert of.cost(E, w.y, r.x) < 1e-8
    # the fitted forcing reproduces the data when the map is re-evaluated on
    # fresh paths: theta(x_i; F*) per path is g - sum_q F*_q int phi_q
    fresh = inputs.optimal_forcing(M=200_000)
    fresh.seed += 1
    p = run(c, fresh, pm.PM_FP32, fresh.M)["g"]
    h = p[:, 0, :] - np.einsum("q,jqm->jm", r.x, p[:, 1:, :])
    resid = h.mean(axis=1) - w.y
    se = h.std(axis=1, ddof=1) / np.sqrt(fresh.M)
    assert np.all(np.abs(resid) <= 5 * se), (resid, se)


def test_invalid_arguments_raise(c):
    w = inputs.optimal_forcing(M=8)
    with pytest.raises(pm.PMError):
        bad = pm.SquareBVP(w.prob.b, -1.0, w.prob.c, w.prob.w)
        pm.pm_forward_square_bvp(c, bad, w.x, 3, 8, w.dt, 100, 1, pm.PM_FP32, np.empty(12))
    with pytest.raises(pm.PMError):
        pm.pm_forward_square_bvp(c, pm.SquareBVP(w.prob.b, 0.1, np.zeros((9, 2)), 1.0), w.x, 3, 8, w.dt, 100, 1,
                                 pm.PM_FP32, np.empty(30))
