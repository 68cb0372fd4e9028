"""GPU pCN chains against the oracle sampler: step-by-step on a linear forward
map, the posterior of delayed acceptance, and a short run over the particle map."""
import numpy as np
import pytest

from oracle import mcmc
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


def toy(sigma=0.5, seed=0, n_obs=6, K=1):
    std = mcmc.prior_std(K)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_obs, len(std)))
    y = A @ (std * rng.standard_normal(len(std))) + sigma * rng.standard_normal(n_obs)
    return A, y, sigma, std


def test_plain_chain_matches_oracle_step_by_step(c):
    A, y, sigma, std = toy()
    u0 = np.zeros((8, len(std)))
    ch = pm.PCN(c, 1, u0, y, sigma, 0.3, seed=123, A=A)
    st = ch.run(300)
    U, phi, s, n = ch.state()
    ch.close()
    U_or, total, ost = mcmc.run(u0, lambda u: A @ u, y, sigma, 0.3, std, 300, seed=123)
    assert st["accepts"] == ost["accepts"] and st["forward_evals"] == 8 * 300
    assert abs(st["sq_jump"] - ost["sq_jump"]) <= 1e-10 * ost["sq_jump"]
    assert np.abs(U - U_or).max() <= 1e-12
    assert np.abs(s - total).max() <= 1e-10 * max(1.0, np.abs(total).max())
    assert n == 8 * 300


def test_delayed_acceptance_reaches_linear_posterior(c):
    A, y, sigma, std = toy()
    m, S = mcmc.linear_gaussian_posterior(A, y, sigma, std)
    # a screen trained briefly on prior draws: close to, not equal to, A u
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((4096, len(std)))
    net = pm.pm_surrogate_create(c, len(std), 128, len(y), 9)
    pm.pm_surrogate_train(c, net, Z.astype(np.float32), ((Z * std) @ A.T).astype(np.float32), epochs=40, batch=256,
                          lr=3e-3)
    ch = pm.PCN(c, 1, np.zeros((8, len(std))), y, sigma, 0.3, seed=77, A=A, screen=net, screen_scale=1.0 / std)
    st = ch.run(6000)
    U, phi, s, n = ch.state()
    ch.close()
    pm.pm_surrogate_destroy(net)
    est = s / n
    assert np.all(np.abs(est - m) <= 0.15 * np.sqrt(np.diag(S))), (est, m)
    assert st["forward_evals"] == st["stage1_accepts"] < st["proposals"]
    assert st["accepts"] <= st["stage1_accepts"]


def test_particle_map_chains_run_and_screen_saves_evaluations(c):
    w = inputs.plain_fp64_k2()
    w.M = 256
    # data from a prior draw through the particle map itself (same stream and seed)
    u_true = inputs.prior_field(2, 55)
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    y = np.empty(len(w.t))
    pm.pm_forward_timedep(c, pm.Field(2, u_true), w.kappa, th, w.x, w.t, len(w.t), w.M, w.dt, 999, pm.PM_FP32, y)
    kw = dict(theta0=th, x=w.x, t=w.t, kappa=w.kappa, dt=w.dt, M=w.M, path_seed=999)
    std = mcmc.prior_std(2)
    u0 = np.zeros((4, 24))
    plain = pm.PCN(c, 2, u0, y, 0.05, 0.2, seed=5, **kw)
    sp = plain.run(20)
    _, phi_p, _, _ = plain.state()
    plain.close()
    assert sp["forward_evals"] == 80 and np.all(np.isfinite(phi_p))
    net = pm.pm_surrogate_create(c, 24, 128, len(y), 2)     # untrained: a poor but valid screen
    da = pm.PCN(c, 2, u0, y, 0.05, 0.2, seed=5, screen=net, screen_scale=1.0 / std, **kw)
    sd = da.run(20)
    da.close()
    pm.pm_surrogate_destroy(net)
    assert sd["forward_evals"] == sd["stage1_accepts"] <= sd["proposals"] == 80


def test_tensor_map_chains_start_from_the_tensor_map_misfit(c):
    # map_flags = PM_TENSOR: the chains' initial misfits are those of the
    # batched tensor-core map on the same stream and seed (stream 0 for all).
    w = inputs.batched_instances(B=1, M=256)[0]
    x, t = w.x[:20].copy(), w.t[:20].copy()
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    u0 = np.stack([inputs.prior_field(10, 70 + k) for k in range(3)])
    y = np.linspace(-0.2, 0.2, len(t))
    sigma = 0.1
    ch = pm.PCN(c, 10, u0, y, sigma, 0.1, seed=3, theta0=th, x=x, t=t, kappa=w.kappa, dt=w.dt, M=256,
                path_seed=w.seed, tensor=True)
    _, phi, _, _ = ch.state()
    ch.close()
    inst = [dict(kind=pm.PM_KIND_TIMEDEP, u=u0[b], kappa=w.kappa, dt=w.dt, row0=b * len(t), n_obs=len(t), M=256,
                 seed=w.seed, stream=0) for b in range(3)]
    batch = pm.Batch(10, inst, np.ascontiguousarray(np.tile(x, (3, 1))), np.ascontiguousarray(np.tile(t, 3)), th, None)
    G = np.empty(3 * len(t))
    pm.pm_forward_batched(c, batch, pm.PM_FP32 | pm.PM_TENSOR, G)
    phi_ref = ((y[None, :] - G.reshape(3, -1)) ** 2).sum(1) / (2 * sigma ** 2)
    np.testing.assert_allclose(phi, phi_ref, rtol=1e-12, atol=0)
    G_simt = np.empty(3 * len(t))
    pm.pm_forward_batched(c, batch, pm.PM_FP32, G_simt)
    assert not np.array_equal(G, G_simt)   # the flag reached the map


def test_screen_shift_zero_equals_no_shift(c):
    A, y, sigma, std = toy(sigma=0.5, seed=3, n_obs=6, K=1)
    net = pm.pm_surrogate_create(c, len(std), 128, len(y), 9)
    runs = []
    for shift in (None, np.zeros(len(std))):
        ch = pm.PCN(c, 1, np.zeros((8, len(std))), y, sigma, 0.3, seed=21, A=A, screen=net, screen_scale=1.0 / std,
                    screen_shift=shift)
        runs.append(ch.run(200))
        ch.close()
    # a shift moves the screen's inputs, so its stage-1 decisions change
    ch = pm.PCN(c, 1, np.zeros((8, len(std))), y, sigma, 0.3, seed=21, A=A, screen=net, screen_scale=1.0 / std,
                screen_shift=np.full(len(std), 3.0))
    shifted = ch.run(200)
    ch.close()
    pm.pm_surrogate_destroy(net)
    keys = ("proposals", "stage1_accepts", "accepts", "forward_evals")
    assert all(runs[0][k] == runs[1][k] for k in keys)
    assert shifted["stage1_accepts"] != runs[0]["stage1_accepts"]


def test_trained_screen_gains_over_plain_pcn(c):
    # What the trained network buys: at a large pCN step most proposals are
    # rejected; the screen rejects them without a forward evaluation, so the
    # chain spends far fewer evaluations per accepted move than plain pCN,
    # and both reach the posterior mean.
    A, y, sigma, std = toy(sigma=0.2, seed=5, n_obs=6, K=1)
    m, S = mcmc.linear_gaussian_posterior(A, y, sigma, std)
    rng = np.random.default_rng(6)
    Z = rng.standard_normal((8192, len(std)))
    net = pm.pm_surrogate_create(c, len(std), 128, len(y), 3)
    pm.pm_surrogate_train(c, net, Z.astype(np.float32), ((Z * std) @ A.T).astype(np.float32), epochs=60, batch=256,
                          lr=3e-3)
    beta, steps = 0.8, 6000
    runs = {}
    for name, screen in (("plain", None), ("da", net)):
        ch = pm.PCN(c, 1, np.tile(m, (32, 1)), y, sigma, beta, seed=31, A=A, screen=screen,
                    screen_scale=(1.0 / std) if screen is not None else None)
        st = ch.run(steps)
        _, _, s, n = ch.state()
        ch.close()
        runs[name] = (st, s / n)
    pm.pm_surrogate_destroy(net)
    (sp, mp), (sd, md) = runs["plain"], runs["da"]
    evals_per_accept_plain = sp["forward_evals"] / sp["accepts"]
    evals_per_accept_da = sd["forward_evals"] / sd["accepts"]
    assert evals_per_accept_da <= 0.5 * evals_per_accept_plain, (evals_per_accept_plain, evals_per_accept_da)
    # both sample the posterior (chains started at its mean, at a step where
    # plain pCN accepts a few percent): within 0.75 posterior standard
    # deviations; the closed-form check of the screened chain from the prior
    # mean is test_delayed_acceptance_reaches_linear_posterior
    for est in (mp, md):
        assert np.all(np.abs(est - m) <= 0.75 * np.sqrt(np.diag(S))), (est, m)
